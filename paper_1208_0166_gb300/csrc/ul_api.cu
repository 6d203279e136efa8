// ul_api.cu — the C ABI declared in include/ul.h: handle life cycle, argument checks,
// device memory, the host-side schedule of sweeps and multilevel levels, and copies of
// results to caller-owned host buffers.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ul.h"
#include "ul_device.cuh"
#include "ul_internal.h"

struct ul_lattice {
    ul::Geo g{};
    int precision = UL_FP64;
    double beta = 0.0;
    uint64_t seed = 0;
    uint64_t metro_pass = 0;
    double width = 1.0;
    int sub_metro = 1;
    int sub_or = 3;
    // bound on the per-sample T/O buffers of the insertion contraction (16 GiB: measured
    // faster than 4 GiB for the 24-frame estimator, 143 MB per sample at 24^4)
    int chunk_mb = 16384;
    bool multihit = false; // correlator at r >= 2 from multihit temporal links
    uint64_t proposed = 0;
    uint64_t launches = 0; // kernels launched on behalf of this handle

    void* theta = nullptr; // R[4][2][Vh]
    void* cs = nullptr;    // (cos, sin) per link, same layout
    double* canon = nullptr;          // 4V doubles, layout conversion staging
    unsigned long long* d_accepted = nullptr;
    double* d_scalar = nullptr;       // small device outputs (plaquette)
    double* plaq_partials = nullptr;

    // multilevel scratch, grown on demand
    void* ml_buf = nullptr;
    size_t ml_bytes = 0;

    // CUDA graphs of recurring launch sequences (compound sweeps, chunks of sub-samples).
    // Update kernels in a graph read their Metropolis pass number relative to *d_pass_base,
    // which a one-thread kernel sets before each replay.
    struct Graph {
        std::vector<long long> key;
        cudaGraphExec_t exec = nullptr;
        long kernels = 0;
    };
    std::vector<Graph> graphs;
    bool use_graphs = true;
    // programmatic dependent launch of consecutive class kernels: 0 never, 1 always, 2 in
    // compound sweeps only (not in the sub-sample passes, which alternate with measurements)
    int use_pdl = 1;
    unsigned long long* d_pass_base = nullptr;
    // persistent cooperative sweeps with a bounded-wait grid barrier
    bool use_persistent = false;
    bool barrier_unreachable = false; // test switch: no barrier can complete
    // slab-resident sub-samples (one thread-block cluster per slab, links in shared memory)
    int slab_mode = 0;    // 0: off, 1: on where the slab fits
    int slab_cluster = 0; // CTAs per slab (0: chosen by slab_plan)
    bool contract_tiled = true; // FP32 insertion contraction in the shared-memory tiled form
    long long copy_wait_cycles = ul::kCopyWaitLimit; // the tiled contraction's copy wait (option "copy_stall_test")
    unsigned long long spin_limit = 1ull << 24;
    unsigned int* d_bar = nullptr;    // [0] arrivals, [1] generation
    int* d_status = nullptr;          // nonzero after a wait gave up
    cudaStream_t cap_stream = nullptr;
    // second stream: the insertion contraction of one chunk of sub-samples runs on it while
    // the next chunk's updates run on the handle's stream; per sample buffer, ev_stored marks
    // the chunk's samples written and ev_contract their contraction done
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_stored[2] = {nullptr, nullptr};
    cudaEvent_t ev_contract[2] = {nullptr, nullptr};
    // a level begun by ul_multilevel_fields_begin: its reduction and result copy run on
    // aux_stream into the pinned staging buffer; ev_result marks their completion
    bool pending = false;
    int pend_r_max = 0, pend_nd = 0;
    size_t pend_n_out = 0;
    bool pend_fields = false;
    double* pinned = nullptr;
    size_t pinned_n = 0;
    cudaEvent_t ev_main = nullptr;
    cudaEvent_t ev_result = nullptr;
    // two-level estimator with insertions: the fold of level-1 iteration k (second stream)
    // has finished with the level-2 accumulators of parity k % 2
    cudaEvent_t ev_fold[2] = {nullptr, nullptr};

    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_init_error;

int fail(ul_lattice* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_init_error = msg;
    return code;
}

int cuda_fail(ul_lattice* h, cudaError_t e, const char* what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? UL_ENOMEM : UL_ECUDA, msg);
}

#define UL_CK(h, call)                                                                                          \
    do {                                                                                                        \
        cudaError_t e_ = (call);                                                                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);                                                \
    } while (0)

size_t real_size(const ul_lattice* h) { return h->precision == UL_FP64 ? sizeof(double) : sizeof(float); }

bool is_f64(const ul_lattice* h) { return h->precision == UL_FP64; }

enum : long long { kGraphSweep = 1, kGraphChunk = 2, kGraphLevel2 = 3, kGraphSym = 4 };

void drop_graphs(ul_lattice* h, long long kind)
{
    std::vector<ul_lattice::Graph> keep;
    for (auto& gr : h->graphs) {
        if (kind == 0 || gr.key[0] == kind) cudaGraphExecDestroy(gr.exec);
        else keep.push_back(gr);
    }
    h->graphs.swap(keep);
}

void release(ul_lattice* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h, 0);
    cudaFree(h->d_pass_base);
    cudaFree(h->d_bar);
    cudaFree(h->d_status);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->aux_stream) cudaStreamSynchronize(h->aux_stream);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_stored[b]) cudaEventDestroy(h->ev_stored[b]);
        if (h->ev_contract[b]) cudaEventDestroy(h->ev_contract[b]);
    }
    if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
    if (h->ev_main) cudaEventDestroy(h->ev_main);
    if (h->ev_result) cudaEventDestroy(h->ev_result);
    for (int b = 0; b < 2; ++b)
        if (h->ev_fold[b]) cudaEventDestroy(h->ev_fold[b]);
    if (h->pinned) cudaFreeHost(h->pinned);
    cudaFree(h->theta);
    cudaFree(h->cs);
    cudaFree(h->canon);
    cudaFree(h->d_accepted);
    cudaFree(h->d_scalar);
    cudaFree(h->plaq_partials);
    cudaFree(h->ml_buf);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

int ensure_ml(ul_lattice* h, size_t bytes)
{
    // work on the multilevel scratch waits for a begun level's reduction and result copy
    // (a no-op when nothing was begun: the event has not been recorded)
    UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_result, 0));
    if (bytes <= h->ml_bytes) return UL_OK;
    UL_CK(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h, kGraphChunk); // they reference the old buffer
    drop_graphs(h, kGraphLevel2);
    drop_graphs(h, kGraphSym);
    cudaFree(h->ml_buf);
    h->ml_buf = nullptr;
    h->ml_bytes = 0;
    cudaError_t e = cudaMalloc(&h->ml_buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, UL_ENOMEM, "multilevel accumulators: cannot allocate " + std::to_string(bytes) + " bytes");
    }
    h->ml_bytes = bytes;
    return UL_OK;
}

long long bits_of(double v)
{
    long long b;
    std::memcpy(&b, &v, sizeof b);
    return b;
}

uint64_t updatable_links(const ul_lattice* h, int slab_t)
{
    long n = 4L * h->g.V;
    if (slab_t > 0) n -= 3L * h->g.L3 * (h->g.Nt / slab_t);
    return static_cast<uint64_t>(n);
}

// Enqueue n_metro Metropolis then n_or overrelaxation passes on st.  The Metropolis passes get
// pass numbers first_pass, first_pass + 1, ... (plus *pass_base when pass_base is set).
// Returns the number of kernels enqueued, or a negative status.
long enqueue_passes(ul_lattice* h, cudaStream_t st, int n_metro, int n_or, int slab_t, uint64_t first_pass,
                    const unsigned long long* pass_base)
{
    long n = 0;
    const bool pdl = h->use_pdl == 1 || (h->use_pdl == 2 && slab_t == 0);
    for (int k = 0; k < n_metro + n_or; ++k) {
        const bool metro = k < n_metro;
        const uint64_t pass = first_pass + (metro ? static_cast<uint64_t>(k) : 0);
        for (int mu = 0; mu < 4; ++mu)
            for (int par = 0; par < 2; ++par) {
                int launched = 0;
                cudaError_t e = is_f64(h)
                    ? ul::launch_update_class<double>(h->g, static_cast<double*>(h->theta), h->cs, mu, par, metro, pass,
                                                      pass_base, h->seed, h->beta, h->width, slab_t, h->d_accepted, st,
                                                      &launched, pdl)
                    : ul::launch_update_class<float>(h->g, static_cast<float*>(h->theta), h->cs, mu, par, metro, pass,
                                                     pass_base, h->seed, h->beta, h->width, slab_t, h->d_accepted, st,
                                                     &launched, pdl);
                if (e != cudaSuccess) return cuda_fail(h, e, "update kernel launch");
                n += launched;
            }
    }
    return n;
}

void account_passes(ul_lattice* h, int n_metro, int slab_t)
{
    h->proposed += static_cast<uint64_t>(n_metro) * updatable_links(h, slab_t);
    h->metro_pass += static_cast<uint64_t>(n_metro);
}

// Run `body(stream, pass_base)` either directly on the handle's stream (pass numbers
// absolute) or as a cached graph keyed by `key` (pass numbers relative to the handle's
// current pass count, supplied through d_pass_base).  body returns kernels enqueued or a
// negative status.
template <class Body>
int run_sequence(ul_lattice* h, const std::vector<long long>& key, Body body)
{
    if (!h->use_graphs) {
        const long n = body(h->stream, h->metro_pass, nullptr);
        if (n < 0) return static_cast<int>(n);
        h->launches += static_cast<uint64_t>(n);
        return UL_OK;
    }
    ul_lattice::Graph* found = nullptr;
    for (auto& gr : h->graphs)
        if (gr.key == key) found = &gr;
    if (!found) {
        UL_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        const long n = body(h->cap_stream, 0, h->d_pass_base);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (n < 0) {
            if (graph) cudaGraphDestroy(graph);
            return static_cast<int>(n);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiation");
        if (h->graphs.size() >= 16) {
            cudaGraphExecDestroy(h->graphs.front().exec);
            h->graphs.erase(h->graphs.begin());
        }
        h->graphs.push_back(ul_lattice::Graph{key, exec, n});
        found = &h->graphs.back();
    }
    cudaError_t e = ul::launch_set_u64(h->d_pass_base, h->metro_pass, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "pass base launch");
    UL_CK(h, cudaGraphLaunch(found->exec, h->stream));
    h->launches += static_cast<uint64_t>(found->kernels) + 1;
    return UL_OK;
}

ul::PersistArgs persist_args(ul_lattice* h, int n_units, int n_metro, int n_or, int slab_t)
{
    ul::PersistArgs a{};
    a.u.parity = 0;
    a.u.metro = 0;
    a.u.slab_t = slab_t;
    a.u.frozen_mask = 0;
    if (slab_t > 0 && h->g.Nt <= 64)
        for (int t = 0; t < h->g.Nt; t += slab_t) a.u.frozen_mask |= 1ull << t;
    a.u.pass = h->metro_pass;
    a.u.pass_base = nullptr;
    a.u.seed = h->seed;
    a.u.beta = h->beta;
    a.u.width = h->width;
    a.u.beta_f = static_cast<float>(h->beta);
    a.u.width_f = static_cast<float>(h->width);
    a.u.accepted = h->d_accepted;
    a.n_units = n_units;
    a.n_metro = n_metro;
    a.n_or = n_or;
    a.bar = h->d_bar;
    a.status = h->d_status;
    a.expected = h->barrier_unreachable ? 0xffffffffu : 0u;
    a.spin_limit = h->spin_limit;
    return a;
}

int launch_persistent(ul_lattice* h, const ul::PersistArgs& a)
{
    UL_CK(h, cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), h->stream));
    cudaError_t e = is_f64(h) ? ul::launch_persistent<double>(h->g, static_cast<double*>(h->theta), h->cs, a, 256, h->stream)
                              : ul::launch_persistent<float>(h->g, static_cast<float*>(h->theta), h->cs, a, 256, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "persistent sweep launch");
    h->launches += 1;
    return UL_OK;
}

// A device-side wait that gave up leaves a nonzero status word: report it once, reset
// the barrier, and keep the handle usable.
int check_device_status(ul_lattice* h)
{
    int st = 0;
    UL_CK(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    if (!st) return UL_OK;
    UL_CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    UL_CK(h, cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned int), h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    if (st == 2)
        return fail(h, UL_ETIMEOUT,
                    "a staging-copy wait of the insertion contraction reached its limit; the field sums of "
                    "this level are incomplete");
    return fail(h, UL_ETIMEOUT,
                "a grid-barrier wait of a persistent sweep reached its limit; the sweep stopped early and "
                "the link state is incomplete");
}

// Sub-samples per insertion contraction: a quarter of the level (so that the contraction of
// one chunk can overlap the next chunk's updates), but at least kMinChunkSamples (a
// contraction launch has a fixed cost, the FP64 read-modify-write of the field sums: with
// fewer samples the overlapped contractions fall behind the slab-resident updates, and a
// level of fewer samples is contracted once), bounded so that two chunk buffers fit into
// the option "insertion_chunk_mb".  FP64 links: the whole level (the double-single
// contraction does not run beside the FP64 updates, which hold the SMs, so chunks would only
// add epilogues and read-modify-writes of the sums), within the same bound.  The same
// chunks in every launch mode, so that the modes give the same sums.
constexpr int kMinChunkSamples = 48;

int chunk_samples(const ul_lattice* h, int n_sub, size_t per_sample)
{
    const size_t cap = (static_cast<size_t>(h->chunk_mb) << 20) / 2;
    const size_t quarter = is_f64(h) ? static_cast<size_t>(n_sub)
                                     : std::max<size_t>((static_cast<size_t>(n_sub) + 3) / 4, kMinChunkSamples);
    return static_cast<int>(std::max<size_t>(1, std::min<size_t>({quarter, static_cast<size_t>(n_sub), cap / per_sample})));
}

int compound_sweep(ul_lattice* h, int n_metro, int n_or)
{
    if (h->use_persistent) {
        int rc = launch_persistent(h, persist_args(h, 1, n_metro, n_or, 0));
        if (rc) return rc;
        account_passes(h, n_metro, 0);
        return UL_OK;
    }
    const std::vector<long long> key = {kGraphSweep, n_metro, n_or, bits_of(h->beta), bits_of(h->width),
                                        static_cast<long long>(h->seed)};
    int rc = run_sequence(h, key, [&](cudaStream_t st, uint64_t first, const unsigned long long* base) {
        return enqueue_passes(h, st, n_metro, n_or, 0, first, base);
    });
    if (rc) return rc;
    account_passes(h, n_metro, 0);
    return UL_OK;
}

// Buffers of one multilevel level: accumulators (sum of T per (s, r, x0); sum of T O per
// (s, r, d, ch, x0); sum of O per (ch, s, x0)), the per-sample T / O storage for two chunks of
// `chunk` sub-samples, and the multihit links (may be null).
struct LevelBufs {
    double2* asum;
    double2* bsum;
    double* osum;
    void* tk;
    void* ok;
    void* ubar;
    int chunk;
};

// n_sub sub-samples of one level (slab thickness slab_t): passes with the slab boundaries
// frozen, a measurement after each, and with fields the insertion contraction of each
// chunk, added into the accumulators of b.  Slab-resident where the slab fits (and neither
// multihit nor persistent mode is on), else persistent or per-class launches.
int run_level(ul_lattice* h, int slab_t, int n_sub, int r_max, int nd, bool fields, const LevelBufs& b,
              bool wait_contraction = true, int buf0 = 0)
{
    const ul::Geo& g = h->g;
    const int S = g.Nt / slab_t;
    const size_t rs = real_size(h);
    const size_t n_a = static_cast<size_t>(S) * r_max * g.L3;
    double2* asum = b.asum;
    double2* bsum = b.bsum;
    double* osum = b.osum;
    void* tk = b.tk;
    void* ok = b.ok;
    void* ubar = b.ubar;
    const int chunk = b.chunk;
    int rc = UL_OK;

    // Slab-resident form: one cluster launch per chunk of sub-samples, where the slab fits
    // into the shared memory of a cluster (multihit values are formed by their own kernel,
    // so that mode keeps the per-class launches).
    int slab_cl = 0, slab_threads = 0;
    if (h->slab_mode && !ubar && !h->use_persistent) {
        cudaError_t e = is_f64(h) ? ul::slab_plan<double>(g, slab_t, h->slab_cluster, &slab_cl, &slab_threads)
                                  : ul::slab_plan<float>(g, slab_t, h->slab_cluster, &slab_cl, &slab_threads);
        if (e != cudaSuccess) return cuda_fail(h, e, "slab plan");
    }

    // Sub-samples in chunks; each chunk (passes + measurement per sample, then the insertion
    // contraction of the chunk) is one launch sequence, replayed as a graph.
    const int seq = fields ? chunk : (slab_cl ? n_sub : std::min(n_sub, 64));
    int chunk_index = 0;
    for (int k = 0; k < n_sub;) {
        const int count = std::min(seq, n_sub - k);
        const int sm = h->sub_metro, so = h->sub_or;
        const bool chunk_first = k == 0; // the first contraction writes the field sums
        if (slab_cl) {
            // chunk c fills buffer c % 2 on the handle's stream; its contraction runs on the
            // auxiliary stream (on the SMs the cluster grid leaves free) while chunk c + 1 runs
            const int buf = (buf0 + chunk_index) % 2;
            void* tkb = static_cast<char*>(tk) + static_cast<size_t>(buf) * n_a * 2 * rs * chunk;
            void* okb = static_cast<char*>(ok) + static_cast<size_t>(buf) * 8ull * S * g.L3 * rs * chunk;
            // the buffer's previous contraction (of this level or an earlier one) has read it
            if (fields) UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_contract[buf], 0));
            ul::SlabArgs a{};
            a.u = persist_args(h, count, sm, so, slab_t).u;
            a.n_units = count;
            a.n_metro = sm;
            a.n_or = so;
            a.cluster = slab_cl;
            a.nz = g.L / slab_cl;
            a.r_max = r_max;
            a.fields = fields ? 1 : 0;
            a.slot0 = 0;
            a.asum = asum;
            a.tk = tkb;
            a.ok = okb;
            a.osum = osum;
            cudaError_t e = is_f64(h)
                ? ul::launch_slab<double>(g, static_cast<double*>(h->theta), h->cs, a, slab_threads, h->stream)
                : ul::launch_slab<float>(g, static_cast<float*>(h->theta), h->cs, a, slab_threads, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "slab-resident launch");
            h->launches += 1;
            if (fields) {
                UL_CK(h, cudaEventRecord(h->ev_stored[buf], h->stream));
                UL_CK(h, cudaStreamWaitEvent(h->aux_stream, h->ev_stored[buf], 0));
                e = is_f64(h) ? ul::launch_insertion_contract<double>(g, slab_t, r_max, nd, count, tkb, okb, bsum,
                                                                      chunk_first, h->aux_stream, h->contract_tiled,
                                                                      h->d_status, h->copy_wait_cycles)
                              : ul::launch_insertion_contract<float>(g, slab_t, r_max, nd, count, tkb, okb, bsum,
                                                                     chunk_first, h->aux_stream, h->contract_tiled,
                                                                     h->d_status, h->copy_wait_cycles);
                if (e != cudaSuccess) return cuda_fail(h, e, "insertion contraction launch");
                UL_CK(h, cudaEventRecord(h->ev_contract[buf], h->aux_stream));
                h->launches += 1;
            }
            account_passes(h, sm * count, slab_t);
            k += count;
            ++chunk_index;
            if (k >= n_sub && fields && wait_contraction)
                UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_contract[buf], 0));
            continue;
        }
        if (h->use_persistent) {
            ul::PersistArgs a = persist_args(h, count, sm, so, slab_t);
            a.measure = 1;
            a.r_max = r_max;
            a.fields = fields ? 1 : 0;
            a.slot0 = 0;
            a.asum = asum;
            a.tk = tk;
            a.ok = ok;
            a.osum = osum;
            a.ubar = ubar;
            if (fields) // sample buffer 0 is free once earlier contractions on the second stream are done
                for (int q = 0; q < 2; ++q) UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_contract[q], 0));
            rc = launch_persistent(h, a);
            if (rc) return rc;
            if (fields) {
                cudaError_t e = is_f64(h)
                    ? ul::launch_insertion_contract<double>(g, slab_t, r_max, nd, count, tk, ok, bsum, chunk_first,
                                                            h->stream, h->contract_tiled, h->d_status, h->copy_wait_cycles)
                    : ul::launch_insertion_contract<float>(g, slab_t, r_max, nd, count, tk, ok, bsum, chunk_first,
                                                           h->stream, h->contract_tiled, h->d_status, h->copy_wait_cycles);
                if (e != cudaSuccess) return cuda_fail(h, e, "insertion contraction launch");
                h->launches += 1;
            }
            account_passes(h, sm * count, slab_t);
            k += count;
            continue;
        }
        // Per-class launches: the chunk's passes and measurements, one launch sequence replayed
        // as a graph, fill sample buffer chunk % 2 on the handle's stream; the chunk's
        // contraction runs on the auxiliary stream beside the next chunk's updates (for FP64
        // links the updates occupy the FP64 pipe and the double-single contraction the FP32
        // pipes), in chunk order, so the sums are those of the serial order.
        const int buf = (buf0 + chunk_index) % 2;
        void* tkb = fields ? static_cast<char*>(tk) + static_cast<size_t>(buf) * n_a * 2 * rs * chunk : tk;
        void* okb = fields ? static_cast<char*>(ok) + static_cast<size_t>(buf) * 8ull * S * g.L3 * rs * chunk : ok;
        if (fields) UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_contract[buf], 0));
        const std::vector<long long> key = {kGraphChunk, slab_t, sm, so, r_max, nd, count,
                                            bits_of(h->beta), bits_of(h->width), static_cast<long long>(h->seed),
                                            reinterpret_cast<long long>(asum), reinterpret_cast<long long>(tkb),
                                            reinterpret_cast<long long>(okb), reinterpret_cast<long long>(osum),
                                            reinterpret_cast<long long>(ubar)};
        rc = run_sequence(h, key, [&](cudaStream_t st, uint64_t first, const unsigned long long* base) -> long {
            long n = 0;
            for (int j = 0; j < count; ++j) {
                const long m = enqueue_passes(h, st, sm, so, slab_t, first + static_cast<uint64_t>(j) * sm, base);
                if (m < 0) return m;
                n += m;
                cudaError_t e;
                if (ubar) {
                    e = is_f64(h) ? ul::launch_multihit<double>(g, h->cs, h->beta, ubar, st)
                                  : ul::launch_multihit<float>(g, h->cs, h->beta, ubar, st);
                    if (e != cudaSuccess) return cuda_fail(h, e, "multihit launch");
                    ++n;
                }
                e = is_f64(h)
                    ? ul::launch_measure_store<double>(g, h->cs, slab_t, r_max, fields, j, asum, tkb, okb, osum, ubar, st)
                    : ul::launch_measure_store<float>(g, h->cs, slab_t, r_max, fields, j, asum, tkb, okb, osum, ubar, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "measurement launch");
                ++n;
            }
            return n;
        });
        if (rc) return rc;
        if (fields) {
            UL_CK(h, cudaEventRecord(h->ev_stored[buf], h->stream));
            UL_CK(h, cudaStreamWaitEvent(h->aux_stream, h->ev_stored[buf], 0));
            cudaError_t e = is_f64(h)
                ? ul::launch_insertion_contract<double>(g, slab_t, r_max, nd, count, tkb, okb, bsum, chunk_first,
                                                        h->aux_stream, h->contract_tiled, h->d_status, h->copy_wait_cycles)
                : ul::launch_insertion_contract<float>(g, slab_t, r_max, nd, count, tkb, okb, bsum, chunk_first,
                                                       h->aux_stream, h->contract_tiled, h->d_status, h->copy_wait_cycles);
            if (e != cudaSuccess) return cuda_fail(h, e, "insertion contraction launch");
            UL_CK(h, cudaEventRecord(h->ev_contract[buf], h->aux_stream));
            h->launches += 1;
        }
        account_passes(h, sm * count, slab_t);
        k += count;
        ++chunk_index;
        if (k >= n_sub && fields && wait_contraction)
            UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_contract[buf], 0));
    }
    return UL_OK;
}

// First half of a level with insertions (everything enqueued; results collected by level_end).
int level_begin(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max, bool fields)
{
    const ul::Geo& g = h->g;
    if (h->pending)
        return fail(h, UL_ESTATE, "ul_multilevel: the results of a begun level have not been collected "
                                  "(ul_multilevel_fields_end)");
    if (slab_t < 1 || g.Nt % slab_t != 0) return fail(h, UL_EINVAL, "ul_multilevel: slab_t must divide Nt");
    if (g.Nt / slab_t > ul::kMaxSlabs) return fail(h, UL_EINVAL, "ul_multilevel: more than 256 slabs");
    if (n_sub < 1) return fail(h, UL_EINVAL, "ul_multilevel: n_sub must be >= 1");
    if (r_max < 1 || r_max > g.L / 2) return fail(h, UL_EINVAL, "ul_multilevel: r_max must be in [1, L/2]");
    if (fields && (d_max < 0 || d_max >= g.L)) return fail(h, UL_EINVAL, "ul_multilevel: d_max must be in [0, L)");
    const int nd = fields ? d_max + 1 : 0;
    const int S = g.Nt / slab_t;

    // Scratch (each region 256-byte aligned): asum | bsum | osum | tk | ok | partials | out.
    // tk / ok hold the T and O of up to `chunk` sub-samples for the deferred insertion
    // contraction; the chunk is bounded by the option "insertion_chunk_mb".
    const size_t rs = real_size(h);
    const size_t n_a = static_cast<size_t>(S) * r_max * g.L3;
    const size_t n_b = n_a * nd * 8;
    const size_t n_o = fields ? 8ull * S * g.L3 : 0;
    const size_t n_p = ul::ml_partials_doubles(g, r_max, nd);
    const size_t n_out = 2ull * r_max + 2ull * r_max * nd * 8 + 8;
    const size_t per_sample = fields ? (n_a * 2 + 8ull * S * g.L3) * rs : 0;
    const int chunk = fields ? chunk_samples(h, n_sub, per_sample) : 0;
    auto al = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
    const size_t off_b = al(n_a * sizeof(double2));
    const size_t off_o = off_b + al(n_b * sizeof(double2));
    const size_t off_t = off_o + al(n_o * sizeof(double));
    const size_t off_k = off_t + al(fields ? n_a * 2 * rs * chunk * 2 : 0); // two chunk buffers
    const size_t off_u = off_k + al(fields ? 8ull * S * g.L3 * rs * chunk * 2 : 0);
    const size_t off_p = off_u + al(h->multihit ? static_cast<size_t>(g.V) * 2 * rs : 0);
    const size_t off_out = off_p + al(n_p * sizeof(double));
    const size_t bytes = off_out + al(n_out * sizeof(double));
    int rc = ensure_ml(h, bytes);
    if (rc) return rc;
    char* base = static_cast<char*>(h->ml_buf);
    double2* asum = reinterpret_cast<double2*>(base);
    double2* bsum = reinterpret_cast<double2*>(base + off_b);
    double* osum = reinterpret_cast<double*>(base + off_o);
    void* tk = base + off_t;
    void* ok = base + off_k;
    void* ubar = h->multihit ? static_cast<void*>(base + off_u) : nullptr;
    double* partials = reinterpret_cast<double*>(base + off_p);
    double* dout = reinterpret_cast<double*>(base + off_out);
    UL_CK(h, cudaMemsetAsync(asum, 0, n_a * sizeof(double2), h->stream));
    if (fields) {
        UL_CK(h, cudaMemsetAsync(osum, 0, n_o * sizeof(double), h->stream));
    }

    rc = run_level(h, slab_t, n_sub, r_max, nd, fields, LevelBufs{asum, bsum, osum, tk, ok, ubar, chunk}, false);
    if (rc) return rc;
    // The reduction and the result copy run on the auxiliary stream after everything the
    // level put on the handle's stream (and after the last contraction, already there), so
    // the handle's stream is free for the next configuration's sweeps meanwhile.
    UL_CK(h, cudaEventRecord(h->ev_main, h->stream));
    UL_CK(h, cudaStreamWaitEvent(h->aux_stream, h->ev_main, 0));
    cudaError_t e = ul::launch_ml_reduce(g, slab_t, n_sub, r_max, nd, asum, bsum, fields ? osum : nullptr, partials,
                                         dout, h->aux_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction launch");
    h->launches += fields ? 3 : 2;
    // pinned staging: the results, then the device status word as of the level's end
    if (h->pinned_n < n_out + 1) {
        if (h->pinned) cudaFreeHost(h->pinned);
        h->pinned = nullptr;
        h->pinned_n = 0;
        UL_CK(h, cudaMallocHost(&h->pinned, (n_out + 1) * sizeof(double)));
        h->pinned_n = n_out + 1;
    }
    UL_CK(h, cudaMemcpyAsync(h->pinned, dout, n_out * sizeof(double), cudaMemcpyDeviceToHost, h->aux_stream));
    UL_CK(h, cudaMemcpyAsync(h->pinned + n_out, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->aux_stream));
    UL_CK(h, cudaEventRecord(h->ev_result, h->aux_stream));
    h->pend_n_out = n_out;
    h->pending = true;
    h->pend_r_max = r_max;
    h->pend_nd = nd;
    h->pend_fields = fields;
    return UL_OK;
}

// Second half: wait for the level's reduction, then copy the results to the caller.
int level_end(ul_lattice* h, double* out_corr, double* out_fields, double* out_vac)
{
    if (!h->pending) return fail(h, UL_ESTATE, "ul_multilevel_fields_end: no level was begun");
    h->pending = false;
    UL_CK(h, cudaEventSynchronize(h->ev_result));
    UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_result, 0));
    int st = 0;
    std::memcpy(&st, h->pinned + h->pend_n_out, sizeof(int));
    if (st) {
        // a persistent sweep of the level gave up at a grid barrier: report it and clear the flag
        const int rc = check_device_status(h);
        if (rc) return rc;
    }
    const int r_max = h->pend_r_max, nd = h->pend_nd;
    const double* host = h->pinned;
    std::memcpy(out_corr, host, 2ull * r_max * sizeof(double));
    if (h->pend_fields) {
        if (out_fields) std::memcpy(out_fields, host + 2 * r_max, 2ull * r_max * nd * 8 * sizeof(double));
        if (out_vac) std::memcpy(out_vac, host + 2 * r_max + 2 * r_max * nd * 8, 8 * sizeof(double));
    }
    return UL_OK;
}

} // namespace

extern "C" {

int ul_init_ex(ul_lattice** out, int L, int Nt, double beta, uint64_t seed, int precision)
{
    if (!out) return fail(nullptr, UL_EINVAL, "ul_init: handle pointer is NULL");
    *out = nullptr;
    if (L < 2 || Nt < 2 || (L & 1) || (Nt & 1))
        return fail(nullptr, UL_EINVAL, "ul_init: L and Nt must be even and >= 2");
    const long long V = static_cast<long long>(L) * L * L * Nt;
    if (V > (1LL << 28)) return fail(nullptr, UL_EINVAL, "ul_init: L^3 Nt must not exceed 2^28");
    if (!(beta >= 0.0)) return fail(nullptr, UL_EINVAL, "ul_init: beta must be >= 0");
    if (precision != UL_FP64 && precision != UL_FP32_ACC64)
        return fail(nullptr, UL_EINVAL, "ul_init: precision must be UL_FP64 or UL_FP32_ACC64");

    ul_lattice* h = new (std::nothrow) ul_lattice();
    if (!h) return fail(nullptr, UL_ENOMEM, "ul_init: host allocation failed");
    h->g.L = L;
    h->g.Nt = Nt;
    h->g.Lh = L / 2;
    h->g.L3 = L * L * L;
    h->g.V = static_cast<int>(V);
    h->g.Vh = static_cast<int>(V / 2);
    h->precision = precision;
    h->beta = beta;
    h->seed = seed;

    auto bail = [&](cudaError_t e, const char* what) {
        std::string msg = std::string("ul_init: ") + what + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        release(h);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? UL_ENOMEM : UL_ECUDA, msg);
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
    h->stream = h->own_stream;
    const size_t nlink = 4ull * static_cast<size_t>(V);
    const size_t rs = real_size(h);
    if ((e = cudaMalloc(&h->theta, nlink * rs)) != cudaSuccess) return bail(e, "link angles");
    if ((e = cudaMalloc(&h->cs, nlink * 2 * rs)) != cudaSuccess) return bail(e, "link phases");
    if ((e = cudaMalloc(&h->canon, nlink * sizeof(double))) != cudaSuccess) return bail(e, "staging buffer");
    if ((e = cudaMalloc(&h->d_accepted, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "counters");
    if ((e = cudaMalloc(&h->d_scalar, 16 * sizeof(double))) != cudaSuccess) return bail(e, "scalars");
    if ((e = cudaMalloc(&h->d_pass_base, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "pass base");
    if ((e = cudaMalloc(&h->d_bar, 2 * sizeof(unsigned int))) != cudaSuccess) return bail(e, "barrier");
    if ((e = cudaMalloc(&h->d_status, sizeof(int))) != cudaSuccess) return bail(e, "status");
    if ((e = cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned int), h->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream)) != cudaSuccess) return bail(e, "memset");
    // graph replay measured faster on GB300 than the persistent kernel with grid barriers
    // (24^4, 100 sweeps: 5.05 against 6.43 us per FP32 class)
    h->use_persistent = false;
    // programmatic dependent launch: measured faster for FP32 classes (4.94 -> 4.60 us at 24^4);
    // for FP64 faster in compound sweeps and slower in the sub-sample passes (which alternate
    // with measurements), so there mode 2 (compound sweeps only)
    h->use_pdl = precision == UL_FP32_ACC64 ? 1 : 2;
    // slab-resident sub-samples: measured faster for FP32 at 24^4 (step 57.4 -> 49.8 ms); the
    // FP64 form is bound by the FP64 pipe and a cluster form leaves a third of the SMs idle
    h->slab_mode = precision == UL_FP32_ACC64 ? 1 : 0;
    if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "capture stream");
    if ((e = cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "auxiliary stream");
    if ((e = cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    if ((e = cudaEventCreateWithFlags(&h->ev_result, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    for (int b = 0; b < 2; ++b)
        if ((e = cudaEventCreateWithFlags(&h->ev_fold[b], cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "event");
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaEventCreateWithFlags(&h->ev_stored[b], cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
        if ((e = cudaEventCreateWithFlags(&h->ev_contract[b], cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "event");
    }
    if ((e = is_f64(h) ? ul::prepare_insertion_contract<double>() : ul::prepare_insertion_contract<float>()) !=
        cudaSuccess)
        return bail(e, "kernel attributes");
    if ((e = ul::prepare_ml_reduce()) != cudaSuccess) return bail(e, "kernel attributes");
    if ((e = cudaMalloc(&h->plaq_partials, ul::plaquette_partials(h->g) * sizeof(double))) != cudaSuccess)
        return bail(e, "plaquette partials");
    if ((e = cudaMemsetAsync(h->d_accepted, 0, sizeof(unsigned long long), h->stream)) != cudaSuccess)
        return bail(e, "memset");
    e = is_f64(h) ? ul::launch_hot_start<double>(h->g, static_cast<double*>(h->theta), h->cs, seed, h->stream)
                  : ul::launch_hot_start<float>(h->g, static_cast<float*>(h->theta), h->cs, seed, h->stream);
    if (e != cudaSuccess) return bail(e, "hot start launch");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(e, "hot start");
    *out = h;
    return UL_OK;
}

int ul_init(ul_lattice** out, int L, int Nt, double beta, uint64_t seed)
{
    return ul_init_ex(out, L, Nt, beta, seed, UL_FP64);
}

int ul_free(ul_lattice* h)
{
    release(h);
    return UL_OK;
}

int ul_sweep(ul_lattice* h, int n_metro, int n_or)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_sweep: NULL handle");
    if (n_metro < 0 || n_or < 0) return fail(h, UL_EINVAL, "ul_sweep: pass counts must be >= 0");
    return compound_sweep(h, n_metro, n_or);
}

int ul_multilevel_fields(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max, double* out_corr,
                         double* out_fields, double* out_vac)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_multilevel: NULL handle");
    if (!out_corr) return fail(h, UL_EINVAL, "ul_multilevel: output pointer is NULL");
    const int rc = level_begin(h, slab_t, n_sub, r_max, d_max, out_fields != nullptr);
    if (rc) return rc;
    return level_end(h, out_corr, out_fields, out_vac);
}

int ul_multilevel_fields_begin(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_multilevel_fields_begin: NULL handle");
    return level_begin(h, slab_t, n_sub, r_max, d_max, d_max >= 0);
}

int ul_multilevel_fields_end(ul_lattice* h, double* out_corr, double* out_fields, double* out_vac)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_multilevel_fields_end: NULL handle");
    if (!out_corr) return fail(h, UL_EINVAL, "ul_multilevel_fields_end: output pointer is NULL");
    return level_end(h, out_corr, out_fields, out_vac);
}

int ul_multilevel_fields_sym(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max, double* out_corr,
                             double* out_fields, double* out_vac)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_multilevel_fields_sym: NULL handle");
    const ul::Geo& g = h->g;
    if (slab_t < 1 || g.Nt % slab_t != 0) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: slab_t must divide Nt");
    if (g.Nt / slab_t > ul::kMaxSlabs) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: more than 256 slabs");
    if (n_sub < 1) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: n_sub must be >= 1");
    if (r_max < 1 || r_max > g.L / 2) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: r_max must be in [1, L/2]");
    if (d_max < 0 || d_max >= g.L) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: d_max must be in [0, L)");
    if (!out_corr || !out_fields) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: output pointer is NULL");
    if (h->multihit) return fail(h, UL_EINVAL, "ul_multilevel_fields_sym: not available with the multihit option");
    const int nd = d_max + 1;
    const int S = g.Nt / slab_t;

    // Scratch: asum3 | bsum3 | osum12 | tk3 (per sample) | csym (per sample) | o12 (one
    // sample) | partials | out3 (three axes) | vac12
    const size_t rs = real_size(h);
    const size_t n_a = static_cast<size_t>(S) * r_max * g.L3;
    const size_t n_b = n_a * nd * 8;
    const size_t n_o = 12ull * S * g.L3;
    const size_t n_c = 3ull * S * nd * 8 * g.L3; // frame sums of one sample
    const size_t n_p = ul::ml_partials_doubles(g, r_max, nd);
    const size_t n_out = 2ull * r_max + 2ull * r_max * nd * 8 + 8;
    const size_t per_sample = (3 * n_a * 2 + n_c) * rs;
    const size_t cap = static_cast<size_t>(h->chunk_mb) << 20;
    const int chunk = static_cast<int>(std::max<size_t>(1, std::min<size_t>(static_cast<size_t>(n_sub), cap / per_sample)));
    auto al = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
    const size_t off_b = al(3 * n_a * sizeof(double2));
    const size_t off_o = off_b + al(3 * n_b * sizeof(double2));
    const size_t off_t = off_o + al(n_o * sizeof(double));
    const size_t off_c = off_t + al(3 * n_a * 2 * rs * chunk);
    const size_t off_k = off_c + al(n_c * rs * chunk);
    const size_t off_p = off_k + al(n_o * rs);
    const size_t off_out = off_p + al(n_p * sizeof(double));
    const size_t bytes = off_out + al((3 * n_out + 12) * sizeof(double));
    int rc = ensure_ml(h, bytes);
    if (rc) return rc;
    char* base = static_cast<char*>(h->ml_buf);
    double2* asum3 = reinterpret_cast<double2*>(base);
    double2* bsum3 = reinterpret_cast<double2*>(base + off_b);
    double* osum12 = reinterpret_cast<double*>(base + off_o);
    void* tk3 = base + off_t;
    void* csym = base + off_c;
    void* o12 = base + off_k;
    double* partials = reinterpret_cast<double*>(base + off_p);
    double* dout = reinterpret_cast<double*>(base + off_out);
    UL_CK(h, cudaMemsetAsync(asum3, 0, 3 * n_a * sizeof(double2), h->stream));
    UL_CK(h, cudaMemsetAsync(osum12, 0, n_o * sizeof(double), h->stream));
    // the sub-sample passes in the slab-resident form where it applies (one cluster launch per
    // sub-sample without its own measurement), else one launch per class
    int slab_cl = 0, slab_threads = 0;
    if (h->slab_mode && !h->use_persistent) {
        cudaError_t e = is_f64(h) ? ul::slab_plan<double>(g, slab_t, h->slab_cluster, &slab_cl, &slab_threads)
                                  : ul::slab_plan<float>(g, slab_t, h->slab_cluster, &slab_cl, &slab_threads);
        if (e != cudaSuccess) return cuda_fail(h, e, "slab plan");
    }

    for (int k = 0; k < n_sub;) {
        const int count = std::min(chunk, n_sub - k);
        const int sm = h->sub_metro, so = h->sub_or;
        const std::vector<long long> key = {kGraphSym, slab_t, sm, so, r_max, nd, count, k == 0 ? 1 : 0, slab_cl,
                                            slab_threads,
                                            bits_of(h->beta), bits_of(h->width), static_cast<long long>(h->seed),
                                            reinterpret_cast<long long>(asum3), reinterpret_cast<long long>(bsum3),
                                            reinterpret_cast<long long>(osum12), reinterpret_cast<long long>(tk3),
                                            reinterpret_cast<long long>(csym), reinterpret_cast<long long>(o12)};
        rc = run_sequence(h, key, [&](cudaStream_t st, uint64_t first, const unsigned long long* pb) -> long {
            long n = 0;
            for (int j = 0; j < count; ++j) {
                if (slab_cl) {
                    ul::SlabArgs a{};
                    a.u = persist_args(h, 1, sm, so, slab_t).u;
                    a.u.pass = first + static_cast<uint64_t>(j) * sm;
                    a.u.pass_base = pb;
                    a.n_units = 1;
                    a.n_metro = sm;
                    a.n_or = so;
                    a.cluster = slab_cl;
                    a.nz = g.L / slab_cl;
                    a.skip_measure = 1;
                    cudaError_t e =
                        is_f64(h)
                            ? ul::launch_slab<double>(g, static_cast<double*>(h->theta), h->cs, a, slab_threads, st)
                            : ul::launch_slab<float>(g, static_cast<float*>(h->theta), h->cs, a, slab_threads, st);
                    if (e != cudaSuccess) return cuda_fail(h, e, "slab-resident launch");
                    n += 1;
                } else {
                    const long m = enqueue_passes(h, st, sm, so, slab_t, first + static_cast<uint64_t>(j) * sm, pb);
                    if (m < 0) return m;
                    n += m;
                }
                cudaError_t e = is_f64(h)
                    ? ul::launch_measure_sym<double>(g, h->cs, slab_t, r_max, nd, j, asum3, tk3, o12, csym, osum12, st)
                    : ul::launch_measure_sym<float>(g, h->cs, slab_t, r_max, nd, j, asum3, tk3, o12, csym, osum12, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "symmetrised measurement launch");
                n += 2;
            }
            cudaError_t e = is_f64(h)
                ? ul::launch_insertion_contract_sym<double>(g, slab_t, r_max, nd, count, tk3, csym, bsum3, k == 0, st,
                                                            h->contract_tiled, h->d_status, h->copy_wait_cycles)
                : ul::launch_insertion_contract_sym<float>(g, slab_t, r_max, nd, count, tk3, csym, bsum3, k == 0, st,
                                                           h->contract_tiled, h->d_status, h->copy_wait_cycles);
            if (e != cudaSuccess) return cuda_fail(h, e, "symmetrised contraction launch");
            return n + 1;
        });
        if (rc) return rc;
        account_passes(h, sm * count, slab_t);
        k += count;
    }
    for (int a = 0; a < 3; ++a) {
        cudaError_t e = ul::launch_ml_reduce(g, slab_t, n_sub, r_max, nd, asum3 + a * n_a, bsum3 + a * n_b, nullptr,
                                             partials, dout + a * n_out, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "reduction launch");
        h->launches += 2;
    }
    cudaError_t e = ul::launch_ml_vacuum(static_cast<int>(S * g.L3), osum12, 12,
                                         static_cast<double>(n_sub) * static_cast<double>(g.V), dout + 3 * n_out,
                                         h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "vacuum launch");
    h->launches += 1;
    std::vector<double> host(3 * n_out + 12);
    UL_CK(h, cudaMemcpyAsync(host.data(), dout, host.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    rc = check_device_status(h);
    if (rc) return rc;
    // correlator: mean over the three axes; fields: the sum over the 24 frames (each axis
    // accumulated its 8 frames) divided by 24
    for (int i = 0; i < 2 * r_max; ++i) out_corr[i] = (host[i] + host[n_out + i] + host[2 * n_out + i]) / 3.0;
    const size_t nf = 2ull * r_max * nd * 8;
    for (size_t i = 0; i < nf; ++i)
        out_fields[i] = (host[2 * r_max + i] + host[n_out + 2 * r_max + i] + host[2 * n_out + 2 * r_max + i]) / 24.0;
    if (out_vac) {
        // vacuum term of each frame channel from the per-plane means (a shifted corner does not
        // change a mean over all sites): channel planes (0,a), (0,b), (0,c), (b,c) with the Im
        // part signed by the frame
        const double* v = host.data() + 3 * n_out; // [plane p][Im, Re], p = (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
        auto plane = [](int mu, int nu) { return mu == 0 ? nu - 1 : (mu == 1 ? (nu == 2 ? 3 : 4) : 5); };
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 1; a <= 3; ++a) {
            const int o1 = a == 1 ? 2 : 1, o2 = a == 3 ? 2 : 3;
            for (int pr = 0; pr < 2; ++pr) {
                const int b = pr == 0 ? o1 : o2, c = pr == 0 ? o2 : o1;
                for (int sb = 1; sb >= -1; sb -= 2)
                    for (int sc = 1; sc >= -1; sc -= 2) {
                        const int pbc = plane(std::min(b, c), std::max(b, c));
                        const double ori = b < c ? 1.0 : -1.0;
                        acc[0] += v[2 * (a - 1)];
                        acc[1] += v[2 * (a - 1) + 1];
                        acc[2] += sb * v[2 * (b - 1)];
                        acc[3] += v[2 * (b - 1) + 1];
                        acc[4] += sc * v[2 * (c - 1)];
                        acc[5] += v[2 * (c - 1) + 1];
                        acc[6] += sb * sc * ori * v[2 * pbc];
                        acc[7] += v[2 * pbc + 1];
                    }
            }
        }
        for (int ch = 0; ch < 8; ++ch) out_vac[ch] = acc[ch] / 24.0;
    }
    return UL_OK;
}

int ul_multilevel(ul_lattice* h, int slab_t, int n_sub, int r_max, double* out)
{
    return ul_multilevel_fields(h, slab_t, n_sub, r_max, -1, out, nullptr, nullptr);
}

int ul_multilevel2(ul_lattice* h, int tau1, int n1, int tau2, int n2, int r_max, double* out)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_multilevel2: NULL handle");
    const ul::Geo& g = h->g;
    if (tau1 < 1 || tau2 < 1 || g.Nt % tau1 != 0 || tau1 % tau2 != 0)
        return fail(h, UL_EINVAL, "ul_multilevel2: tau2 must divide tau1 and tau1 must divide Nt");
    if (g.Nt / tau2 > ul::kMaxSlabs) return fail(h, UL_EINVAL, "ul_multilevel2: more than 256 level-2 slabs");
    if (n1 < 1 || n2 < 1) return fail(h, UL_EINVAL, "ul_multilevel2: n1 and n2 must be >= 1");
    if (r_max < 1 || r_max > g.L / 2 || r_max > 128)
        return fail(h, UL_EINVAL, "ul_multilevel2: r_max must be in [1, min(L/2, 128)]");
    if (!out) return fail(h, UL_EINVAL, "ul_multilevel2: output pointer is NULL");
    const int S1 = g.Nt / tau1, S2 = g.Nt / tau2;
    const size_t rs = real_size(h);
    auto al = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
    const size_t n_a1 = static_cast<size_t>(S1) * r_max * g.L3, n_a2 = static_cast<size_t>(S2) * r_max * g.L3;
    const size_t n_p = ul::ml_partials_doubles(g, r_max, 0);
    const size_t off_2 = al(n_a1 * sizeof(double2));
    const size_t off_u = off_2 + al(n_a2 * sizeof(double2));
    const size_t off_p = off_u + al(h->multihit ? static_cast<size_t>(g.V) * 2 * rs : 0);
    const size_t off_out = off_p + al(n_p * sizeof(double));
    int rc = ensure_ml(h, off_out + al((2ull * r_max + 8) * sizeof(double)));
    if (rc) return rc;
    char* base = static_cast<char*>(h->ml_buf);
    double2* asum1 = reinterpret_cast<double2*>(base);
    double2* asum2 = reinterpret_cast<double2*>(base + off_2);
    void* ubar = h->multihit ? static_cast<void*>(base + off_u) : nullptr;
    double* partials = reinterpret_cast<double*>(base + off_p);
    double* dout = reinterpret_cast<double*>(base + off_out);
    UL_CK(h, cudaMemsetAsync(asum1, 0, n_a1 * sizeof(double2), h->stream));
    const int sm = h->sub_metro, so = h->sub_or;
    const long long kb = bits_of(h->beta), kw = bits_of(h->width), ks = static_cast<long long>(h->seed);

    // level-2 samples of one level-1 iteration: passes with tau2 frozen, measurement into asum2
    auto level2_chunk = [&](int count) -> int {
        if (h->use_persistent) {
            ul::PersistArgs a = persist_args(h, count, sm, so, tau2);
            a.measure = 1;
            a.r_max = r_max;
            a.asum = asum2;
            a.ubar = ubar;
            return launch_persistent(h, a);
        }
        const std::vector<long long> key = {kGraphLevel2, 2, tau2, sm, so, r_max, count, kb, kw, ks,
                                            reinterpret_cast<long long>(asum2), reinterpret_cast<long long>(ubar)};
        return run_sequence(h, key, [&](cudaStream_t st, uint64_t first, const unsigned long long* pb) -> long {
            long n = 0;
            for (int j = 0; j < count; ++j) {
                const long q = enqueue_passes(h, st, sm, so, tau2, first + static_cast<uint64_t>(j) * sm, pb);
                if (q < 0) return q;
                n += q;
                cudaError_t e;
                if (ubar) {
                    e = is_f64(h) ? ul::launch_multihit<double>(g, h->cs, h->beta, ubar, st)
                                  : ul::launch_multihit<float>(g, h->cs, h->beta, ubar, st);
                    if (e != cudaSuccess) return cuda_fail(h, e, "multihit launch");
                    ++n;
                }
                e = is_f64(h) ? ul::launch_measure_store<double>(g, h->cs, tau2, r_max, false, 0, asum2, nullptr, nullptr,
                                                                 nullptr, ubar, st)
                              : ul::launch_measure_store<float>(g, h->cs, tau2, r_max, false, 0, asum2, nullptr, nullptr,
                                                                nullptr, ubar, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "measurement launch");
                ++n;
            }
            return n;
        });
    };

    for (int k1 = 0; k1 < n1; ++k1) {
        // level-1 update: passes with tau1 frozen
        if (h->use_persistent) {
            rc = launch_persistent(h, persist_args(h, 1, sm, so, tau1));
        } else {
            const std::vector<long long> key = {kGraphLevel2, 1, tau1, sm, so, kb, kw, ks};
            rc = run_sequence(h, key, [&](cudaStream_t st, uint64_t first, const unsigned long long* pb) {
                return enqueue_passes(h, st, sm, so, tau1, first, pb);
            });
        }
        if (rc) return rc;
        account_passes(h, sm, tau1);
        UL_CK(h, cudaMemsetAsync(asum2, 0, n_a2 * sizeof(double2), h->stream));
        for (int k2 = 0; k2 < n2;) {
            const int count = std::min(64, n2 - k2);
            rc = level2_chunk(count);
            if (rc) return rc;
            account_passes(h, sm * count, tau2);
            k2 += count;
        }
        cudaError_t e = ul::launch_fold_level2(g, tau1, tau2, r_max, n2, asum2, asum1, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "level-2 fold launch");
        h->launches += 1;
    }
    cudaError_t e = ul::launch_ml_reduce(g, tau1, n1, r_max, 0, asum1, nullptr, nullptr, partials, dout, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction launch");
    h->launches += 2;
    double host[2 * 128];
    UL_CK(h, cudaMemcpyAsync(host, dout, 2ull * r_max * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    rc = check_device_status(h);
    if (rc) return rc;
    std::memcpy(out, host, 2ull * r_max * sizeof(double));
    return UL_OK;
}

int ul_multilevel2_fields(ul_lattice* h, int tau1, int n1, int tau2, int n2, int r_max, int d_max,
                          double* out_corr, double* out_fields, double* out_vac)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_multilevel2_fields: NULL handle");
    const ul::Geo& g = h->g;
    if (tau1 < 1 || tau2 < 1 || g.Nt % tau1 != 0 || tau1 % tau2 != 0)
        return fail(h, UL_EINVAL, "ul_multilevel2_fields: tau2 must divide tau1 and tau1 must divide Nt");
    if (tau1 / tau2 > 16) return fail(h, UL_EINVAL, "ul_multilevel2_fields: tau1 / tau2 must not exceed 16");
    if (g.Nt / tau2 > ul::kMaxSlabs) return fail(h, UL_EINVAL, "ul_multilevel2_fields: more than 256 level-2 slabs");
    if (n1 < 1 || n2 < 1) return fail(h, UL_EINVAL, "ul_multilevel2_fields: n1 and n2 must be >= 1");
    if (r_max < 1 || r_max > g.L / 2) return fail(h, UL_EINVAL, "ul_multilevel2_fields: r_max must be in [1, L/2]");
    if (d_max < 0 || d_max >= g.L) return fail(h, UL_EINVAL, "ul_multilevel2_fields: d_max must be in [0, L)");
    if (!out_corr || !out_fields) return fail(h, UL_EINVAL, "ul_multilevel2_fields: output pointer is NULL");
    if (h->multihit) return fail(h, UL_EINVAL, "ul_multilevel2_fields: not available with the multihit option");
    const int S1 = g.Nt / tau1, S2 = g.Nt / tau2, nd = d_max + 1;

    // Scratch: asum1 | bsum1 | asum2 x 2 | bsum2 x 2 | osum (level-2 layout) | tk | ok | partials | out
    // (the level-2 accumulators are double-buffered by level-1 iteration: the fold of one
    // iteration runs on the second stream while the next iteration updates and measures)
    const size_t rs = real_size(h);
    const size_t n_a1 = static_cast<size_t>(S1) * r_max * g.L3, n_a2 = static_cast<size_t>(S2) * r_max * g.L3;
    const size_t n_b1 = n_a1 * nd * 8, n_b2 = n_a2 * nd * 8;
    const size_t n_o = 8ull * S2 * g.L3;
    const size_t n_p = ul::ml_partials_doubles(g, r_max, nd);
    const size_t n_out = 2ull * r_max + 2ull * r_max * nd * 8 + 8;
    const size_t per_sample = (n_a2 * 2 + 8ull * S2 * g.L3) * rs;
    const int chunk = chunk_samples(h, n2, per_sample);
    auto al = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
    const size_t off_b1 = al(n_a1 * sizeof(double2));
    const size_t off_a2 = off_b1 + al(n_b1 * sizeof(double2));
    const size_t off_b2 = off_a2 + 2 * al(n_a2 * sizeof(double2));
    const size_t off_o = off_b2 + 2 * al(n_b2 * sizeof(double2));
    const size_t off_t = off_o + al(n_o * sizeof(double));
    const size_t off_k = off_t + al(n_a2 * 2 * rs * chunk * 2);
    const size_t off_p = off_k + al(8ull * S2 * g.L3 * rs * chunk * 2);
    const size_t off_out = off_p + al(n_p * sizeof(double));
    int rc = ensure_ml(h, off_out + al(n_out * sizeof(double)));
    if (rc) return rc;
    char* base = static_cast<char*>(h->ml_buf);
    double2* asum1 = reinterpret_cast<double2*>(base);
    double2* bsum1 = reinterpret_cast<double2*>(base + off_b1);
    double2* asum2[2] = {reinterpret_cast<double2*>(base + off_a2),
                         reinterpret_cast<double2*>(base + off_a2 + al(n_a2 * sizeof(double2)))};
    double2* bsum2[2] = {reinterpret_cast<double2*>(base + off_b2),
                         reinterpret_cast<double2*>(base + off_b2 + al(n_b2 * sizeof(double2)))};
    double* osum = reinterpret_cast<double*>(base + off_o);
    void* tk = base + off_t;
    void* ok = base + off_k;
    double* partials = reinterpret_cast<double*>(base + off_p);
    double* dout = reinterpret_cast<double*>(base + off_out);
    UL_CK(h, cudaMemsetAsync(asum1, 0, n_a1 * sizeof(double2), h->stream));
    UL_CK(h, cudaMemsetAsync(bsum1, 0, n_b1 * sizeof(double2), h->stream));
    UL_CK(h, cudaMemsetAsync(osum, 0, n_o * sizeof(double), h->stream));
    const int sm = h->sub_metro, so = h->sub_or;
    const long long kb = bits_of(h->beta), kw = bits_of(h->width), ks = static_cast<long long>(h->seed);
    int buf0 = 0; // sample-buffer parity of the next level-2 chunk

    for (int k1 = 0; k1 < n1; ++k1) {
        // level-1 update: passes with the spatial links on t = 0 mod tau1 frozen
        if (h->use_persistent) {
            rc = launch_persistent(h, persist_args(h, 1, sm, so, tau1));
        } else {
            const std::vector<long long> key = {kGraphLevel2, 1, tau1, sm, so, kb, kw, ks};
            rc = run_sequence(h, key, [&](cudaStream_t st, uint64_t first, const unsigned long long* pb) {
                return enqueue_passes(h, st, sm, so, tau1, first, pb);
            });
        }
        if (rc) return rc;
        account_passes(h, sm, tau1);
        // level 2: n2 sub-samples with t = 0 mod tau2 frozen, measured into fresh accumulators
        // of parity p, once the fold of iteration k1 - 2 has read them
        const int p = k1 & 1;
        UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_fold[p], 0));
        UL_CK(h, cudaMemsetAsync(asum2[p], 0, n_a2 * sizeof(double2), h->stream));
        rc = run_level(h, tau2, n2, r_max, nd, true, LevelBufs{asum2[p], bsum2[p], osum, tk, ok, nullptr, chunk},
                       false, buf0);
        if (rc) return rc;
        buf0 = (buf0 + (n2 + chunk - 1) / chunk) % 2;
        // the fold runs on the second stream after everything the iteration enqueued (in the
        // slab-resident form its last contraction is already there), beside the next
        // iteration; with persistent sweeps (grid barriers that need every block resident) it
        // stays on the handle's stream
        cudaStream_t fs = h->use_persistent ? h->stream : h->aux_stream;
        if (fs != h->stream) {
            UL_CK(h, cudaEventRecord(h->ev_main, h->stream));
            UL_CK(h, cudaStreamWaitEvent(fs, h->ev_main, 0));
        }
        cudaError_t e = ul::launch_fold_level2_fields(g, tau1, tau2, r_max, nd, n2, asum2[p], bsum2[p], asum1, bsum1,
                                                      fs);
        if (e != cudaSuccess) return cuda_fail(h, e, "level-2 fold launch");
        UL_CK(h, cudaEventRecord(h->ev_fold[p], fs));
        h->launches += 1;
    }
    UL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_fold[(n1 - 1) & 1], 0));
    cudaError_t e = ul::launch_ml_reduce(g, tau1, n1, r_max, nd, asum1, bsum1, nullptr, partials, dout, h->stream);
    if (e == cudaSuccess)
        e = ul::launch_ml_vacuum(S2 * g.L3, osum, 8, static_cast<double>(n1) * n2 * static_cast<double>(g.V),
                                 dout + 2 * r_max + 2 * r_max * nd * 8, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction launch");
    h->launches += 3;
    std::vector<double> host(n_out);
    UL_CK(h, cudaMemcpyAsync(host.data(), dout, n_out * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    rc = check_device_status(h);
    if (rc) return rc;
    std::memcpy(out_corr, host.data(), 2ull * r_max * sizeof(double));
    std::memcpy(out_fields, host.data() + 2 * r_max, 2ull * r_max * nd * 8 * sizeof(double));
    if (out_vac) std::memcpy(out_vac, host.data() + 2 * r_max + 2 * r_max * nd * 8, 8 * sizeof(double));
    return UL_OK;
}

int ul_plaquette(ul_lattice* h, double* out)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_plaquette: NULL handle");
    if (!out) return fail(h, UL_EINVAL, "ul_plaquette: output pointer is NULL");
    cudaError_t e = is_f64(h) ? ul::launch_plaquette<double>(h->g, h->cs, h->plaq_partials, h->d_scalar, h->stream)
                              : ul::launch_plaquette<float>(h->g, h->cs, h->plaq_partials, h->d_scalar, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "plaquette launch");
    h->launches += 2;
    double v = 0.0;
    UL_CK(h, cudaMemcpyAsync(&v, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    const int rc = check_device_status(h);
    if (rc) return rc;
    *out = v;
    return UL_OK;
}

int ul_set_option(ul_lattice* h, const char* key, double v)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_set_option: NULL handle");
    if (!key) return fail(h, UL_EINVAL, "ul_set_option: NULL key");
    if (!std::strcmp(key, "metro_width")) {
        if (!(v > 0.0)) return fail(h, UL_EINVAL, "metro_width must be > 0");
        h->width = v;
    } else if (!std::strcmp(key, "sub_metro")) {
        if (!(v >= 0.0) || v != static_cast<int>(v)) return fail(h, UL_EINVAL, "sub_metro must be an integer >= 0");
        h->sub_metro = static_cast<int>(v);
    } else if (!std::strcmp(key, "sub_or")) {
        if (!(v >= 0.0) || v != static_cast<int>(v)) return fail(h, UL_EINVAL, "sub_or must be an integer >= 0");
        h->sub_or = static_cast<int>(v);
    } else if (!std::strcmp(key, "multihit")) {
        if (v != 0.0 && v != 1.0) return fail(h, UL_EINVAL, "multihit must be 0 or 1");
        h->multihit = v != 0.0;
    } else if (!std::strcmp(key, "persistent")) {
        if (v != 0.0 && v != 1.0) return fail(h, UL_EINVAL, "persistent must be 0 or 1");
        h->use_persistent = v != 0.0;
    } else if (!std::strcmp(key, "barrier_spin_limit")) {
        if (!(v >= 1.0) || v > 1e15) return fail(h, UL_EINVAL, "barrier_spin_limit must be in [1, 1e15]");
        h->spin_limit = static_cast<unsigned long long>(v);
    } else if (!std::strcmp(key, "barrier_unreachable")) {
        if (v != 0.0 && v != 1.0) return fail(h, UL_EINVAL, "barrier_unreachable must be 0 or 1");
        h->barrier_unreachable = v != 0.0;
    } else if (!std::strcmp(key, "pdl")) {
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(h, UL_EINVAL, "pdl must be 0, 1 or 2");
        h->use_pdl = static_cast<int>(v);
        drop_graphs(h, 0); // captured sequences carry the launch attribute
    } else if (!std::strcmp(key, "graphs")) {
        if (v != 0.0 && v != 1.0) return fail(h, UL_EINVAL, "graphs must be 0 or 1");
        h->use_graphs = v != 0.0;
    } else if (!std::strcmp(key, "slab_resident")) {
        if (v != 0.0 && v != 1.0) return fail(h, UL_EINVAL, "slab_resident must be 0 or 1");
        h->slab_mode = static_cast<int>(v);
    } else if (!std::strcmp(key, "slab_cluster")) {
        if (!(v >= 0.0) || v > 16.0 || v != static_cast<int>(v))
            return fail(h, UL_EINVAL, "slab_cluster must be an integer in [0, 16]");
        h->slab_cluster = static_cast<int>(v);
    } else if (!std::strcmp(key, "contract_tiled")) {
        if (v != 0.0 && v != 1.0) return fail(h, UL_EINVAL, "contract_tiled must be 0 or 1");
        h->contract_tiled = v != 0.0;
        drop_graphs(h, 0); // captured sequences hold the contraction launch
    } else if (!std::strcmp(key, "copy_stall_test")) {
        if (!(v >= 0.0) || v > static_cast<double>(ul::kCopyWaitLimit) || v != static_cast<double>(static_cast<long long>(v)))
            return fail(h, UL_EINVAL, "copy_stall_test must be an integer in [0, 2e9]");
        h->copy_wait_cycles = v > 0.0 ? -static_cast<long long>(v) : ul::kCopyWaitLimit;
        drop_graphs(h, 0); // captured sequences hold the contraction launch
    } else if (!std::strcmp(key, "insertion_chunk_mb")) {
        if (!(v >= 1.0) || v > 1e6 || v != static_cast<int>(v))
            return fail(h, UL_EINVAL, "insertion_chunk_mb must be an integer in [1, 1e6]");
        h->chunk_mb = static_cast<int>(v);
    } else if (!std::strcmp(key, "beta")) {
        if (!(v >= 0.0)) return fail(h, UL_EINVAL, "beta must be >= 0");
        h->beta = v;
    } else {
        return fail(h, UL_EINVAL, std::string("ul_set_option: unknown key '") + key + "'");
    }
    return UL_OK;
}

int ul_get_links(ul_lattice* h, double* theta_host)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_get_links: NULL handle");
    if (!theta_host) return fail(h, UL_EINVAL, "ul_get_links: NULL buffer");
    cudaError_t e = is_f64(h) ? ul::launch_to_canonical<double>(h->g, static_cast<double*>(h->theta), h->canon, h->stream)
                              : ul::launch_to_canonical<float>(h->g, static_cast<float*>(h->theta), h->canon, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "layout kernel launch");
    h->launches += 1;
    UL_CK(h, cudaMemcpyAsync(theta_host, h->canon, 4ull * h->g.V * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    return check_device_status(h);
}

int ul_set_links(ul_lattice* h, const double* theta_host)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_set_links: NULL handle");
    if (!theta_host) return fail(h, UL_EINVAL, "ul_set_links: NULL buffer");
    UL_CK(h, cudaMemcpyAsync(h->canon, theta_host, 4ull * h->g.V * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    cudaError_t e = is_f64(h)
        ? ul::launch_from_canonical<double>(h->g, h->canon, static_cast<double*>(h->theta), h->cs, h->stream)
        : ul::launch_from_canonical<float>(h->g, h->canon, static_cast<float*>(h->theta), h->cs, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "layout kernel launch");
    h->launches += 1;
    UL_CK(h, cudaStreamSynchronize(h->stream));
    return UL_OK;
}

int ul_get_state(ul_lattice* h, uint64_t* seed, uint64_t* metro_pass)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_get_state: NULL handle");
    if (seed) *seed = h->seed;
    if (metro_pass) *metro_pass = h->metro_pass;
    return UL_OK;
}

int ul_set_state(ul_lattice* h, uint64_t seed, uint64_t metro_pass)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_set_state: NULL handle");
    h->seed = seed;
    h->metro_pass = metro_pass;
    return UL_OK;
}

int ul_get_stats(ul_lattice* h, uint64_t* accepted, uint64_t* proposed)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_get_stats: NULL handle");
    unsigned long long a = 0;
    UL_CK(h, cudaMemcpyAsync(&a, h->d_accepted, sizeof(a), cudaMemcpyDeviceToHost, h->stream));
    UL_CK(h, cudaStreamSynchronize(h->stream));
    if (accepted) *accepted = a;
    if (proposed) *proposed = h->proposed;
    return UL_OK;
}

int ul_get_launch_count(ul_lattice* h, uint64_t* launches)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_get_launch_count: NULL handle");
    if (launches) *launches = h->launches;
    return UL_OK;
}

int ul_synchronize(ul_lattice* h)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_synchronize: NULL handle");
    UL_CK(h, cudaStreamSynchronize(h->stream));
    return check_device_status(h);
}

int ul_set_stream(ul_lattice* h, void* cuda_stream)
{
    if (!h) return fail(nullptr, UL_EINVAL, "ul_set_stream: NULL handle");
    UL_CK(h, cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own_stream;
    return UL_OK;
}

int ul_rng_uniforms(int precision, uint64_t seed, uint64_t pass, uint64_t link0, int n, double* out)
{
    if (precision != UL_FP64 && precision != UL_FP32_ACC64)
        return fail(nullptr, UL_EINVAL, "ul_rng_uniforms: precision must be UL_FP64 or UL_FP32_ACC64");
    if (n < 0 || n > (1 << 24) || (n > 0 && !out))
        return fail(nullptr, UL_EINVAL, "ul_rng_uniforms: n must be in [0, 2^24] and out non-NULL");
    if (n == 0) return UL_OK;
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2ull * n * sizeof(double));
    if (e == cudaSuccess)
        e = precision == UL_FP64 ? ul::launch_rng_uniforms<double>(seed, pass, link0, n, d, nullptr)
                                 : ul::launch_rng_uniforms<float>(seed, pass, link0, n, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, 2ull * n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? UL_ENOMEM : UL_ECUDA,
                    std::string("ul_rng_uniforms: ") + cudaGetErrorString(e));
    }
    return UL_OK;
}

int ul_check_enabled(void)
{
#ifdef UL_CHECK
    return 1;
#else
    return 0;
#endif
}

int ul_check_status(unsigned long long* first_failure, int clear)
{
    if (!first_failure) return UL_EINVAL;
    unsigned long long w64 = 0, w32 = 0;
    if (ul::check_word<double>(&w64, clear != 0) != cudaSuccess) return UL_ECUDA;
    if (ul::check_word<float>(&w32, clear != 0) != cudaSuccess) return UL_ECUDA;
    *first_failure = w64 ? w64 : w32;
    return UL_OK;
}

const char* ul_last_error(const ul_lattice* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

int ul_precision(const ul_lattice* h) { return h ? h->precision : UL_EINVAL; }

} // extern "C"
