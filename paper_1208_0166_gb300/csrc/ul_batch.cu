// ul_batch.cu — the batch engine behind ul_batch_* (include/ul.h): many independent
// lattices of different shapes, couplings and seeds advanced together on one GPU.
//
// Every job runs the same program as a single handle: n_sweeps compound sweeps, then one
// multilevel level of n_sub sub-samples (masked passes + transporter measurement), then
// the cross-slab reduction and the plaquette.  The engine advances all resident jobs in
// lockstep by update passes: each pass is 8 batched class launches that cover every
// resident lattice (each at its own position in its program), followed by one batched
// measurement launch for the jobs that just finished a sub-sample.  Jobs are admitted
// from a FIFO queue as soon as their device memory fits in the batch's HBM budget
// (first-fit arena) and a parameter-table slot is free, and leave when their results
// are on the host: continuous batching.  A job only ever touches its own memory and its
// own random numbers, so its results are bit for bit the same alone or in any mix.
#include <atomic>
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/ul.h"
#include "ul_device.cuh"
#include "ul_internal.h"

namespace {

size_t round256(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }

// First-fit allocator over one device region; offsets are 256-byte aligned.
class Arena {
public:
    void init(size_t size)
    {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    long long alloc(size_t n)
    {
        n = round256(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used_ += n;
            return static_cast<long long>(off);
        }
        return -1;
    }
    void release(size_t off, size_t n)
    {
        n = round256(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

private:
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

enum { kQueued = 0, kRunning = 1, kReducing = 2, kFinished = 3 };

struct Job {
    uint64_t id = 0;
    ul_job spec{};
    ul::Geo g{};
    int S = 0;
    long long off = -1;
    size_t bytes = 0;
    void* theta = nullptr;
    void* cs = nullptr;
    double2* asum = nullptr;
    double* partials = nullptr;
    double* dout = nullptr;
    double* plaq_partials = nullptr;
    unsigned long long* accepted = nullptr;
    long pos = 0, sweep_passes = 0, total_passes = 0;
    uint64_t metro_pass = 0, proposed = 0;
    int state = kQueued;
    double* host = nullptr; // pinned: 2 r_max correlator + plaquette + accepted count
    cudaEvent_t done = nullptr;
};

struct Layout {
    size_t theta, cs, asum, partials, dout, plaq, acc, total;
};

Layout layout_of(const Job& j, size_t rs)
{
    Layout l{};
    const size_t n_link = 4ull * j.g.V;
    size_t o = 0;
    l.theta = o;
    o += round256(n_link * rs);
    l.cs = o;
    o += round256(n_link * 2 * rs);
    l.asum = o;
    o += round256(static_cast<size_t>(j.S) * j.spec.r_max * j.g.L3 * sizeof(double2));
    l.partials = o;
    o += round256(ul::ml_partials_doubles(j.g, j.spec.r_max, 0) * sizeof(double));
    l.dout = o;
    o += round256((2ull * j.spec.r_max + 8) * sizeof(double));
    l.plaq = o;
    o += round256(static_cast<size_t>(ul::plaquette_partials(j.g)) * sizeof(double));
    l.acc = o;
    o += round256(sizeof(unsigned long long));
    l.total = o;
    return l;
}

// Block sizes tried by the batched update kernel's autotuner, and the choice per precision.
const int kTuneCandidates[3] = {64, 96, 128};
std::atomic<int> g_tuned_threads[2]; // 0 until tuned; written by any thread

} // namespace

struct ul_batch {
    int precision = UL_FP64;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    char* base = nullptr;
    Arena arena;
    std::deque<Job*> queue;
    std::vector<Job*> resident; // running or reducing
    std::map<uint64_t, Job*> jobs;
    uint64_t next_id = 1;
    int threads = 128;
    // autotuning: timed passes per candidate, then the fastest block size
    struct Sample {
        int threads;
        cudaEvent_t a, b;
    };
    std::vector<Sample> tune;
    bool tuned = false;
    uint64_t link_updates = 0, launches = 0, passes = 0;
    std::string err;
};

namespace {

int bfail(ul_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    return code;
}

int bcuda(ul_batch* b, cudaError_t e, const char* what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? UL_ENOMEM : UL_ECUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define UB_CK(b, call)                                                                                          \
    do {                                                                                                        \
        cudaError_t e_ = (call);                                                                                \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call);                                                    \
    } while (0)

size_t real_size(const ul_batch* b) { return b->precision == UL_FP64 ? sizeof(double) : sizeof(float); }

uint64_t updatable(const Job& j, int slab_t)
{
    long n = 4L * j.g.V;
    if (slab_t > 0) n -= 3L * j.g.L3 * (j.g.Nt / slab_t);
    return static_cast<uint64_t>(n);
}

// Position pos of the job's program: Metropolis or overrelaxation, masked or not, and
// whether a sub-sample ends with this pass.
void pass_kind(const Job& j, bool* metro, int* slab_t, bool* measure)
{
    if (j.pos < j.sweep_passes) {
        const int per = j.spec.sweep_metro + j.spec.sweep_or;
        *metro = (j.pos % per) < j.spec.sweep_metro;
        *slab_t = 0;
        *measure = false;
        return;
    }
    const int per = j.spec.sub_metro + j.spec.sub_or;
    const long k = (j.pos - j.sweep_passes) % per;
    *metro = k < j.spec.sub_metro;
    *slab_t = j.spec.slab_t;
    *measure = k == per - 1;
}

void destroy_job(Job* j)
{
    if (j->host) cudaFreeHost(j->host);
    if (j->done) cudaEventDestroy(j->done);
    delete j;
}

int admit(ul_batch* b)
{
    while (!b->queue.empty()) {
        int running = 0;
        for (Job* j : b->resident) running += j->state == kRunning;
        if (running >= ul::kMaxBatchJobs) break;
        Job* j = b->queue.front();
        const Layout l = layout_of(*j, real_size(b));
        const long long off = b->arena.alloc(l.total);
        if (off < 0) break; // first in line waits until memory frees up
        b->queue.pop_front();
        j->off = off;
        j->bytes = l.total;
        char* p = b->base + off;
        j->theta = p + l.theta;
        j->cs = p + l.cs;
        j->asum = reinterpret_cast<double2*>(p + l.asum);
        j->partials = reinterpret_cast<double*>(p + l.partials);
        j->dout = reinterpret_cast<double*>(p + l.dout);
        j->plaq_partials = reinterpret_cast<double*>(p + l.plaq);
        j->accepted = reinterpret_cast<unsigned long long*>(p + l.acc);
        UB_CK(b, cudaMemsetAsync(j->asum, 0, static_cast<size_t>(j->S) * j->spec.r_max * j->g.L3 * sizeof(double2),
                                 b->stream));
        UB_CK(b, cudaMemsetAsync(j->accepted, 0, sizeof(unsigned long long), b->stream));
        cudaError_t e = b->precision == UL_FP64
            ? ul::launch_hot_start<double>(j->g, static_cast<double*>(j->theta), j->cs, j->spec.seed, b->stream)
            : ul::launch_hot_start<float>(j->g, static_cast<float*>(j->theta), j->cs, j->spec.seed, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "hot start launch");
        b->launches += 1;
        j->state = kRunning;
        b->resident.push_back(j);
    }
    return UL_OK;
}

int finalize_job(ul_batch* b, Job* j)
{
    const int r_max = j->spec.r_max;
    cudaError_t e = ul::launch_ml_reduce(j->g, j->spec.slab_t, j->spec.n_sub, r_max, 0, j->asum, nullptr, nullptr,
                                         j->partials, j->dout, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "reduction launch");
    e = b->precision == UL_FP64
        ? ul::launch_plaquette<double>(j->g, j->cs, j->plaq_partials, j->dout + 2 * r_max, b->stream)
        : ul::launch_plaquette<float>(j->g, j->cs, j->plaq_partials, j->dout + 2 * r_max, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "plaquette launch");
    b->launches += 4;
    UB_CK(b, cudaMemcpyAsync(j->host, j->dout, (2ull * r_max + 1) * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    UB_CK(b, cudaMemcpyAsync(j->host + 2 * r_max + 1, j->accepted, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             b->stream));
    UB_CK(b, cudaEventRecord(j->done, b->stream));
    j->state = kReducing;
    return UL_OK;
}

void retire_finished(ul_batch* b)
{
    std::vector<Job*> keep;
    for (Job* j : b->resident) {
        if (j->state == kReducing && cudaEventQuery(j->done) == cudaSuccess) {
            b->arena.release(static_cast<size_t>(j->off), j->bytes);
            j->state = kFinished;
        } else {
            keep.push_back(j);
        }
    }
    b->resident.swap(keep);
}

void collect_tuning(ul_batch* b)
{
    if (b->tuned || b->tune.size() < 6) return;
    for (auto& s : b->tune)
        if (cudaEventQuery(s.b) != cudaSuccess) return;
    float best = 1e30f;
    int pick = 128;
    for (int c : kTuneCandidates) {
        float sum = 0.f;
        int n = 0;
        for (auto& s : b->tune)
            if (s.threads == c) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, s.a, s.b);
                sum += ms;
                ++n;
            }
        if (n && sum / n < best) {
            best = sum / n;
            pick = c;
        }
    }
    for (auto& s : b->tune) {
        cudaEventDestroy(s.a);
        cudaEventDestroy(s.b);
    }
    b->tune.clear();
    b->threads = pick;
    b->tuned = true;
    g_tuned_threads[b->precision == UL_FP64 ? 0 : 1] = pick;
}

// One lockstep pass over every resident running job.  Returns UL_OK, or a negative status.
int one_pass(ul_batch* b, bool* did_work)
{
    *did_work = false;
    // Two tables per pass: temporal classes (every link) and spatial classes (for a masked
    // job only the unfrozen slices); they differ only in the block offsets.
    ul::BatchUpdateTable t{};
    ul::BatchUpdateTable ts{};
    ul::BatchMeasureTable m{};
    std::vector<Job*> in_pass;
    for (Job* j : b->resident)
        if (j->state == kRunning && j->pos < j->total_passes) in_pass.push_back(j);
    if (in_pass.empty()) return UL_OK;
    *did_work = true;

    // block size: a timed rotation over the candidates during the first passes
    int threads = b->threads;
    bool timing = false;
    if (!b->tuned && b->tune.size() < 6) {
        threads = kTuneCandidates[b->tune.size() % 3];
        timing = true;
    }
    int blocks = 0, blocks_s = 0;
    std::vector<bool> measure(in_pass.size(), false);
    for (size_t q = 0; q < in_pass.size(); ++q) {
        Job* j = in_pass[q];
        bool metro;
        int slab_t;
        bool meas;
        pass_kind(*j, &metro, &slab_t, &meas);
        ul::BatchUpdateJob& u = t.job[t.njobs++];
        u.theta = j->theta;
        u.cs = j->cs;
        u.accepted = j->accepted;
        u.L = j->g.L;
        u.Nt = j->g.Nt;
        u.V = j->g.V;
        u.Vh = j->g.Vh;
        u.L3 = j->g.L3;
        u.block0 = blocks;
        u.metro = metro ? 1 : 0;
        u.slab_t = slab_t;
        u.frozen_mask = 0;
        if (slab_t > 0 && j->g.Nt <= 64)
            for (int tt = 0; tt < j->g.Nt; tt += slab_t) u.frozen_mask |= 1ull << tt;
        u.pass = j->metro_pass;
        u.seed = j->spec.seed;
        u.beta = j->spec.beta;
        u.width = j->spec.metro_width;
        blocks += (j->g.Vh + threads - 1) / threads;
        ts.job[ts.njobs] = u;
        ts.job[ts.njobs].block0 = blocks_s;
        ts.njobs += 1;
        const long spatial_work = slab_t > 1 ? static_cast<long>(j->g.Nt / slab_t) * (slab_t - 1) * (j->g.L3 / 2)
                                             : (slab_t == 1 ? 0L : static_cast<long>(j->g.Vh));
        blocks_s += static_cast<int>((spatial_work + threads - 1) / threads);
        b->link_updates += updatable(*j, slab_t);
        if (metro) {
            j->metro_pass += 1;
            j->proposed += updatable(*j, slab_t);
        }
        measure[q] = meas;
    }
    b->passes += 1;
    ul_batch::Sample smp{threads, nullptr, nullptr};
    if (timing) {
        UB_CK(b, cudaEventCreate(&smp.a));
        UB_CK(b, cudaEventCreate(&smp.b));
        UB_CK(b, cudaEventRecord(smp.a, b->stream));
    }
    const bool pdl = b->precision == UL_FP32_ACC64;
    for (int mu = 0; mu < 4; ++mu)
        for (int par = 0; par < 2; ++par) {
            const ul::BatchUpdateTable& tab = mu == 0 ? t : ts;
            const int nb = mu == 0 ? blocks : blocks_s;
            if (nb == 0) continue; // every spatial link of every job is frozen (slab_t == 1)
            cudaError_t e = b->precision == UL_FP64
                ? ul::launch_batched_update<double>(tab, nb, threads, mu, par, b->stream, pdl)
                : ul::launch_batched_update<float>(tab, nb, threads, mu, par, b->stream, pdl);
            if (e != cudaSuccess) return bcuda(b, e, "batched update launch");
            b->launches += 1;
        }
    if (timing) {
        UB_CK(b, cudaEventRecord(smp.b, b->stream));
        b->tune.push_back(smp);
    }
    // measurements of the jobs whose sub-sample ended with this pass
    int mblocks = 0;
    for (size_t q = 0; q < in_pass.size(); ++q) {
        Job* j = in_pass[q];
        j->pos += 1;
        if (!measure[q]) continue;
        ul::BatchMeasureJob& mj = m.job[m.njobs++];
        mj.cs = j->cs;
        mj.asum = j->asum;
        mj.L = j->g.L;
        mj.Nt = j->g.Nt;
        mj.V = j->g.V;
        mj.Vh = j->g.Vh;
        mj.L3 = j->g.L3;
        mj.block0 = mblocks;
        mj.slab_t = j->spec.slab_t;
        mj.r_max = j->spec.r_max;
        mblocks += (j->S * j->g.L3 + 255) / 256;
    }
    if (m.njobs) {
        cudaError_t e = b->precision == UL_FP64 ? ul::launch_batched_measure<double>(m, mblocks, b->stream)
                                                : ul::launch_batched_measure<float>(m, mblocks, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "batched measurement launch");
        b->launches += 1;
    }
    for (Job* j : in_pass)
        if (j->pos == j->total_passes) {
            const int rc = finalize_job(b, j);
            if (rc) return rc;
        }
    return UL_OK;
}

} // namespace

extern "C" {

int ul_batch_create(ul_batch** out, int precision, size_t hbm_budget_bytes, void* cuda_stream)
{
    if (!out) return UL_EINVAL;
    *out = nullptr;
    if (precision != UL_FP64 && precision != UL_FP32_ACC64) return UL_EINVAL;
    if (hbm_budget_bytes < (1u << 20)) return UL_EINVAL;
    ul_batch* b = new (std::nothrow) ul_batch();
    if (!b) return UL_ENOMEM;
    b->precision = precision;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
        b->stream = b->own_stream;
    }
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->base), hbm_budget_bytes);
    if (e == cudaSuccess) e = ul::prepare_ml_reduce();
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (b->own_stream) cudaStreamDestroy(b->own_stream);
        delete b;
        return e == cudaErrorMemoryAllocation ? UL_ENOMEM : UL_ECUDA;
    }
    b->arena.init(hbm_budget_bytes);
    const int cached = g_tuned_threads[precision == UL_FP64 ? 0 : 1];
    if (cached) {
        b->threads = cached;
        b->tuned = true;
    }
    *out = b;
    return UL_OK;
}

int ul_batch_submit(ul_batch* b, const ul_job* job, uint64_t* job_id)
{
    if (!b) return UL_EINVAL;
    if (!job || !job_id) return bfail(b, UL_EINVAL, "ul_batch_submit: NULL argument");
    const ul_job& s = *job;
    if (s.L < 2 || s.Nt < 2 || (s.L & 1) || (s.Nt & 1))
        return bfail(b, UL_EINVAL, "ul_batch_submit: L and Nt must be even and >= 2");
    const long long V = static_cast<long long>(s.L) * s.L * s.L * s.Nt;
    if (V > (1LL << 28)) return bfail(b, UL_EINVAL, "ul_batch_submit: L^3 Nt must not exceed 2^28");
    if (!(s.beta >= 0.0) || !(s.metro_width > 0.0)) return bfail(b, UL_EINVAL, "ul_batch_submit: beta or width");
    if (s.n_sweeps < 0 || s.sweep_metro < 0 || s.sweep_or < 0 || (s.n_sweeps > 0 && s.sweep_metro + s.sweep_or < 1))
        return bfail(b, UL_EINVAL, "ul_batch_submit: sweep schedule");
    if (s.slab_t < 1 || s.Nt % s.slab_t || s.Nt / s.slab_t > ul::kMaxSlabs)
        return bfail(b, UL_EINVAL, "ul_batch_submit: slab_t must divide Nt");
    if (s.n_sub < 1 || s.sub_metro < 0 || s.sub_or < 0 || s.sub_metro + s.sub_or < 1)
        return bfail(b, UL_EINVAL, "ul_batch_submit: sub-sample schedule (n_sub >= 1, at least one pass)");
    if (s.r_max < 1 || s.r_max > s.L / 2) return bfail(b, UL_EINVAL, "ul_batch_submit: r_max must be in [1, L/2]");
    Job* j = new (std::nothrow) Job();
    if (!j) return bfail(b, UL_ENOMEM, "ul_batch_submit: host allocation");
    j->spec = s;
    j->g.L = s.L;
    j->g.Nt = s.Nt;
    j->g.Lh = s.L / 2;
    j->g.L3 = s.L * s.L * s.L;
    j->g.V = static_cast<int>(V);
    j->g.Vh = static_cast<int>(V / 2);
    j->S = s.Nt / s.slab_t;
    j->sweep_passes = static_cast<long>(s.n_sweeps) * (s.sweep_metro + s.sweep_or);
    j->total_passes = j->sweep_passes + static_cast<long>(s.n_sub) * (s.sub_metro + s.sub_or);
    const size_t need = layout_of(*j, real_size(b)).total;
    if (need > b->arena.size()) {
        delete j;
        return bfail(b, UL_ENOMEM, "ul_batch_submit: the job needs " + std::to_string(need) +
                                       " bytes, more than the batch's whole budget");
    }
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&j->host), (2ull * s.r_max + 2) * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_job(j);
        return bcuda(b, e, "ul_batch_submit");
    }
    j->id = b->next_id++;
    b->queue.push_back(j);
    b->jobs[j->id] = j;
    *job_id = j->id;
    return UL_OK;
}

int ul_batch_step(ul_batch* b, int max_passes, int* n_active)
{
    if (!b) return UL_EINVAL;
    if (max_passes < 0) return bfail(b, UL_EINVAL, "ul_batch_step: max_passes must be >= 0");
    for (int it = 0; it < max_passes; ++it) {
        int rc = admit(b);
        if (rc) return rc;
        bool work = false;
        rc = one_pass(b, &work);
        if (rc) return rc;
        retire_finished(b);
        collect_tuning(b);
        if (!work) break;
    }
    retire_finished(b);
    collect_tuning(b);
    if (n_active) *n_active = static_cast<int>(b->queue.size() + b->resident.size());
    return UL_OK;
}

int ul_batch_poll(ul_batch* b, uint64_t job_id, double* out, int* state)
{
    if (!b) return UL_EINVAL;
    if (!state) return bfail(b, UL_EINVAL, "ul_batch_poll: NULL state");
    auto it = b->jobs.find(job_id);
    if (it == b->jobs.end()) return bfail(b, UL_EINVAL, "ul_batch_poll: unknown or already collected job");
    Job* j = it->second;
    if (j->state == kReducing) retire_finished(b);
    if (j->state != kFinished) {
        *state = j->state == kQueued ? UL_JOB_QUEUED : UL_JOB_RUNNING;
        return UL_OK;
    }
    if (!out) return bfail(b, UL_EINVAL, "ul_batch_poll: NULL output for a finished job");
    const int r_max = j->spec.r_max;
    std::memcpy(out, j->host, (2ull * r_max + 1) * sizeof(double));
    unsigned long long acc = 0;
    std::memcpy(&acc, j->host + 2 * r_max + 1, sizeof acc);
    out[2 * r_max + 1] = j->proposed ? static_cast<double>(acc) / static_cast<double>(j->proposed) : 0.0;
    b->jobs.erase(it);
    destroy_job(j);
    *state = UL_JOB_DONE;
    return UL_OK;
}

int ul_batch_job_info(ul_batch* b, uint64_t job_id, int* state, uint64_t* passes_done, uint64_t* passes_total)
{
    if (!b) return UL_EINVAL;
    auto it = b->jobs.find(job_id);
    if (it == b->jobs.end()) return bfail(b, UL_EINVAL, "ul_batch_job_info: unknown or already collected job");
    const Job* j = it->second;
    if (state)
        *state = j->state == kQueued ? UL_JOB_QUEUED : (j->state == kFinished ? UL_JOB_DONE : UL_JOB_RUNNING);
    if (passes_done) *passes_done = static_cast<uint64_t>(j->pos);
    if (passes_total) *passes_total = static_cast<uint64_t>(j->total_passes);
    return UL_OK;
}

int ul_batch_stats(ul_batch* b, uint64_t* link_updates, uint64_t* launches, int* block_threads, size_t* bytes_in_use)
{
    if (!b) return UL_EINVAL;
    if (link_updates) *link_updates = b->link_updates;
    if (launches) *launches = b->launches;
    if (block_threads) *block_threads = b->threads;
    if (bytes_in_use) *bytes_in_use = b->arena.used();
    return UL_OK;
}

int ul_batch_free(ul_batch* b)
{
    if (!b) return UL_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& s : b->tune) {
        cudaEventDestroy(s.a);
        cudaEventDestroy(s.b);
    }
    for (auto& kv : b->jobs) destroy_job(kv.second);
    cudaFree(b->base);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return UL_OK;
}

const char* ul_batch_last_error(const ul_batch* b) { return b ? b->err.c_str() : ""; }

} // extern "C"
