// ul_batch.cu — the batch engine behind ul_batch_* (include/ul.h): many independent
// lattices of different shapes, couplings and seeds advanced together on one GPU.
//
// Every job runs the same program as a single handle: n_sweeps compound sweeps, then one
// multilevel level of n_sub sub-samples (masked passes + transporter measurement), then
// the cross-slab reduction and the plaquette.  The engine advances the jobs in lockstep by
// update passes, in groups of one shape whose links fit L2 (option group_mb): a pass of a
// group is 8 class launches that cover every lattice of the group (each at its own position
// in its program; the grid's y index selects the lattice), followed by one measurement
// launch for the lattices that just finished a sub-sample.  A group runs a whole step's
// passes in a row (its links stay in L2); each shape has a stream of its own, the largest
// shapes the highest-priority ones, so shapes overlap.  A job whose slab fits
// the shared memory of a thread-block cluster runs its whole level as a slab-resident
// launch instead (all sub-samples, cluster barriers between classes, measurements inside):
// the jobs of one shape that reach their level in the same step share one such launch
// (slab_jobs_kernel), on a second stream beside the lockstep passes of the others.  The
// cluster size per shape is chosen by an autotuner that times each feasible size on a
// scratch lattice once and keeps the choice in a JSON file (with the lockstep block size).  Jobs are admitted
// from a FIFO queue as soon as their device memory fits in the batch's HBM budget
// (first-fit arena) and a parameter-table slot is free, and leave when their results
// are on the host: continuous batching.  A job only ever touches its own memory and its
// own random numbers, so its results are bit for bit the same alone or in any mix.
#include <atomic>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <sys/stat.h>
#include <vector>

#include "../../include/ul.h"
#include "ul_device.cuh"
#include "ul_internal.h"

// Optional trace of the engine's host steps on stderr (environment variable
// UL_BATCH_TRACE=1), to locate a call that does not return.
static bool ub_trace_on()
{
    static const bool on = [] {
        const char* v = std::getenv("UL_BATCH_TRACE");
        return v && v[0] == '1';
    }();
    return on;
}
#define UB_TRACE(...)                                      \
    do {                                                   \
        if (ub_trace_on()) {                               \
            std::fprintf(stderr, "ul_batch: " __VA_ARGS__); \
            std::fputc('\n', stderr);                      \
            std::fflush(stderr);                           \
        }                                                  \
    } while (0)

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
    int sidx = 0;           // lockstep stream of the job's shape
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


// Autotuned launch shapes, kept in a JSON file: {"<device>/<sms>/<key>": value, ...}.
// Path: $UL_TUNE_CACHE, else $XDG_CACHE_HOME/paper_1208_0166_gb300/tune.json, else
// $HOME/.cache/paper_1208_0166_gb300/tune.json; an empty UL_TUNE_CACHE keeps the choices in
// memory only.  A file that cannot be read or written is ignored (the shapes are then tuned
// again); values only choose launch shapes, never results.
class TuneCache {
public:
    bool get(const std::string& key, int* out)
    {
        std::lock_guard<std::mutex> lock(m_);
        load_locked();
        auto it = v_.find(prefix() + key);
        if (it == v_.end()) return false;
        *out = it->second;
        return true;
    }
    void put(const std::string& key, int value)
    {
        std::lock_guard<std::mutex> lock(m_);
        load_locked();
        v_[prefix() + key] = value;
        save_locked();
    }
    std::string path()
    {
        const char* env = std::getenv("UL_TUNE_CACHE");
        if (env) return env;
        const char* xdg = std::getenv("XDG_CACHE_HOME");
        if (xdg && *xdg) return std::string(xdg) + "/paper_1208_0166_gb300/tune.json";
        const char* home = std::getenv("HOME");
        if (home && *home) return std::string(home) + "/.cache/paper_1208_0166_gb300/tune.json";
        return "";
    }

private:
    std::string prefix()
    {
        int dev = 0;
        cudaDeviceProp prop{};
        if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return "unknown/";
        }
        std::string name = prop.name;
        for (char& c : name)
            if (c == '"' || c == '\\' || c == '/') c = '_';
        return name + "/" + std::to_string(prop.multiProcessorCount) + "/";
    }
    static long long mtime_of(const std::string& p)
    {
        struct stat st {};
        if (p.empty() || stat(p.c_str(), &st) != 0) return -1;
        return static_cast<long long>(st.st_mtim.tv_sec) * 1000000000LL + st.st_mtim.tv_nsec;
    }
    void load_locked()
    {
        const std::string p = path();
        const long long mt = mtime_of(p);
        if (loaded_ && p == loaded_path_ && mt == loaded_mtime_) return; // unchanged since read or written
        loaded_ = true;
        loaded_path_ = p;
        loaded_mtime_ = mt;
        v_.clear();
        if (p.empty()) return;
        FILE* f = std::fopen(p.c_str(), "r");
        if (!f) return;
        std::string text;
        char buf[4096];
        size_t n;
        while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
        std::fclose(f);
        // entries "key": integer; keys hold no quotes
        size_t pos = 0;
        while ((pos = text.find('"', pos)) != std::string::npos) {
            const size_t end = text.find('"', pos + 1);
            if (end == std::string::npos) break;
            const std::string key = text.substr(pos + 1, end - pos - 1);
            size_t c = text.find(':', end);
            if (c == std::string::npos) break;
            char* stop = nullptr;
            const long val = std::strtol(text.c_str() + c + 1, &stop, 10);
            if (stop != text.c_str() + c + 1) v_[key] = static_cast<int>(val);
            pos = stop ? static_cast<size_t>(stop - text.c_str()) : c + 1;
        }
    }
    void save_locked()
    {
        const std::string p = path();
        if (p.empty()) return;
        // create the directory chain
        for (size_t i = 1; i < p.size(); ++i)
            if (p[i] == '/') mkdir(p.substr(0, i).c_str(), 0755);
        const std::string tmp = p + ".tmp" + std::to_string(static_cast<long>(reinterpret_cast<uintptr_t>(this) & 0xffff));
        FILE* f = std::fopen(tmp.c_str(), "w");
        if (!f) return;
        std::fputs("{\n", f);
        size_t k = 0;
        for (const auto& kv : v_)
            std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < v_.size() ? "," : "");
        std::fputs("}\n", f);
        const bool ok = std::fclose(f) == 0;
        if (ok) std::rename(tmp.c_str(), p.c_str());
        else std::remove(tmp.c_str());
        loaded_mtime_ = mtime_of(p);
    }

    std::mutex m_;
    std::map<std::string, int> v_;
    bool loaded_ = false;
    std::string loaded_path_;
    long long loaded_mtime_ = -1;
};

TuneCache& tune_cache()
{
    static TuneCache c;
    return c;
}

std::string shape_key(int precision, const ul::Geo& g, int slab_t)
{
    return std::string(precision == UL_FP64 ? "fp64" : "fp32") + "/slab_cluster/L" + std::to_string(g.L) + "_Nt" +
           std::to_string(g.Nt) + "_tau" + std::to_string(slab_t);
}

} // namespace

struct ul_batch {
    int precision = UL_FP64;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    static constexpr int kLevelStreams = 4;
    cudaStream_t level_streams[kLevelStreams] = {}; // slab-resident levels and their reductions
    cudaStream_t level_stream = nullptr;            // level_streams[0] (tuning runs there)
    static constexpr int kLockStreams = 4;
    cudaStream_t lock_streams[kLockStreams] = {}; // lockstep passes, one stream per shape (round robin)
    cudaEvent_t ev_lock[kLockStreams] = {};       // the passes enqueued so far on each
    cudaEvent_t ev_admit = nullptr;               // hot starts of the jobs admitted so far
    std::map<std::pair<int, int>, int> shape_stream;
    int slab_levels = 2;                 // option "slab_levels": 0 never, 1 where the slab fits, 2 auto
    bool tune_slab = true;               // option "tune": time the cluster sizes (else slab_plan's choice)
    std::map<std::string, std::pair<int, int>> plans; // shape key -> (cluster, threads); (0, 0): lockstep
    char* base = nullptr;
    Arena arena;
    std::deque<Job*> queue;
    std::vector<Job*> resident; // running or reducing
    std::map<uint64_t, Job*> jobs;
    uint64_t next_id = 1;
    int threads = 0; // lockstep block size of the last shape tuned (reported by ul_batch_stats)
    // lockstep block size per shape (precision, L, Nt): tuned by timing candidate sizes on
    // the first passes of that shape, or read from the tune cache
    struct Sample {
        int threads;
        cudaEvent_t a, b;
        double links;
    };
    struct ShapeTune {
        int chosen = 0;
        int next = 0; // passes timed so far
        std::vector<Sample> samples;
    };
    std::map<std::string, ShapeTune> tunes;
    size_t group_bytes = 64ull << 20; // option "group_mb": links of one lockstep group
    uint64_t link_updates = 0, launches = 0, passes = 0, slab_launches = 0;
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
    std::vector<Job*> admitted;
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
        admitted.push_back(j);
    }
    if (!admitted.empty()) {
        // streams of new shapes: in order of decreasing lattice volume, so that the largest
        // shape of an admission (the longest levels) gets the highest-priority streams
        std::vector<Job*> order = admitted;
        std::stable_sort(order.begin(), order.end(), [](const Job* x, const Job* y) { return x->g.V > y->g.V; });
        for (Job* j : order) {
            auto ss = b->shape_stream.find({j->g.L, j->g.Nt});
            if (ss == b->shape_stream.end())
                ss = b->shape_stream.emplace(std::make_pair(j->g.L, j->g.Nt),
                                             static_cast<int>(b->shape_stream.size()) % ul_batch::kLockStreams).first;
            j->sidx = ss->second;
        }
        // every lockstep stream sees the hot starts before its next pass
        UB_CK(b, cudaEventRecord(b->ev_admit, b->stream));
        for (cudaStream_t ls : b->lock_streams) UB_CK(b, cudaStreamWaitEvent(ls, b->ev_admit, 0));
    }
    return UL_OK;
}

int finalize_job(ul_batch* b, Job* j, cudaStream_t st)
{
    const int r_max = j->spec.r_max;
    cudaError_t e = ul::launch_ml_reduce(j->g, j->spec.slab_t, j->spec.n_sub, r_max, 0, j->asum, nullptr, nullptr,
                                         j->partials, j->dout, st);
    if (e != cudaSuccess) return bcuda(b, e, "reduction launch");
    e = b->precision == UL_FP64
        ? ul::launch_plaquette<double>(j->g, j->cs, j->plaq_partials, j->dout + 2 * r_max, st)
        : ul::launch_plaquette<float>(j->g, j->cs, j->plaq_partials, j->dout + 2 * r_max, st);
    if (e != cudaSuccess) return bcuda(b, e, "plaquette launch");
    b->launches += 4;
    UB_CK(b, cudaMemcpyAsync(j->host, j->dout, (2ull * r_max + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    UB_CK(b, cudaMemcpyAsync(j->host + 2 * r_max + 1, j->accepted, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             st));
    UB_CK(b, cudaEventRecord(j->done, st));
    j->state = kReducing;
    return UL_OK;
}

// Slab-resident plan (cluster size, threads) of one shape; (0, 0) when the slab does not fit
// a cluster.  With tuning on, every feasible cluster size is timed once on a scratch lattice
// of that shape (a hot start, then one sub-sample of 1 Metropolis + 3 overrelaxation passes
// and a measurement per size, best of three) and the fastest is kept, in memory and in the
// tune cache.  The cluster size changes no result.
template <typename R>
int slab_level_plan(ul_batch* b, const ul::Geo& g, int slab_t, int* cluster, int* threads)
{
    const std::string key = shape_key(b->precision, g, slab_t);
    auto it = b->plans.find(key);
    if (it != b->plans.end()) {
        *cluster = it->second.first;
        *threads = it->second.second;
        return UL_OK;
    }
    *cluster = 0;
    *threads = 0;
    int cached = 0;
    if (b->tune_slab && tune_cache().get(key, &cached)) {
        int c = 0, t = 0;
        if (cached > 0) UB_CK(b, ul::slab_plan<R>(g, slab_t, cached, &c, &t));
        *cluster = c;
        *threads = t;
        b->plans[key] = {c, t};
        return UL_OK;
    }
    int c0 = 0, t0 = 0;
    UB_CK(b, ul::slab_plan<R>(g, slab_t, 0, &c0, &t0));
    if (!c0 || !b->tune_slab) {
        *cluster = c0;
        *threads = t0;
        b->plans[key] = {c0, t0};
        if (b->tune_slab) tune_cache().put(key, c0);
        return UL_OK;
    }
    // scratch lattice of this shape
    const size_t n_link = 4ull * g.V;
    const int S = g.Nt / slab_t;
    char* mem = nullptr;
    const size_t bytes_theta = round256(n_link * sizeof(R)), bytes_cs = round256(n_link * 2 * sizeof(R));
    const size_t bytes_asum = round256(static_cast<size_t>(S) * g.L3 * sizeof(double2));
    UB_CK(b, cudaMalloc(reinterpret_cast<void**>(&mem), bytes_theta + bytes_cs + bytes_asum + 256));
    R* theta = reinterpret_cast<R*>(mem);
    void* cs = mem + bytes_theta;
    double2* asum = reinterpret_cast<double2*>(mem + bytes_theta + bytes_cs);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(mem + bytes_theta + bytes_cs + bytes_asum);
    cudaStream_t st = b->level_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best_c = c0, best_t = t0;
    float best_ms = 1e30f;
    cudaError_t e = ul::launch_hot_start<R>(g, theta, cs, 12345, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(asum, 0, bytes_asum + 256, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    UB_TRACE("slab tuning L=%d Nt=%d slab_t=%d", g.L, g.Nt, slab_t);
    for (int c = 1; c <= 16 && e == cudaSuccess; ++c) {
        int cc = 0, tt = 0;
        e = ul::slab_plan<R>(g, slab_t, c, &cc, &tt);
        if (e != cudaSuccess || cc != c) continue;
        UB_TRACE("slab tuning trial cluster=%d threads=%d", c, tt);
        ul::SlabArgs a{};
        a.u.slab_t = slab_t;
        if (g.Nt <= 64)
            for (int t = 0; t < g.Nt; t += slab_t) a.u.frozen_mask |= 1ull << t;
        a.u.seed = 12345;
        a.u.beta = 1.0;
        a.u.width = 1.0;
        a.u.beta_f = 1.0f;
        a.u.width_f = 1.0f;
        a.u.accepted = acc;
        a.n_units = 1;
        a.n_metro = 1;
        a.n_or = 3;
        a.cluster = c;
        a.nz = g.L / c;
        a.r_max = 1;
        a.asum = asum;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = ul::launch_slab<R>(g, theta, cs, a, tt, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && ms < ms_best) ms_best = ms; // rep 0 warms up
        }
        if (e == cudaSuccess && ms_best < best_ms) {
            best_ms = ms_best;
            best_c = c;
            best_t = tt;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    UB_TRACE("slab tuning trials done, freeing scratch");
    const cudaError_t ef = cudaFree(mem);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return bcuda(b, e, "slab cluster tuning");
    *cluster = best_c;
    *threads = best_t;
    b->plans[key] = {best_c, best_t};
    tune_cache().put(key, best_c);
    return UL_OK;
}

// Option "slab_levels" = 2 (auto): a slab-resident level only where two of its CTAs fit one
// SM's shared memory.  A level of larger slabs holds whole SMs for its duration, which the
// lockstep passes of other shapes cannot share (measured on a batch of 32 lattices of 12^4 to
// 24^4: 24^4 slab-resident levels made the batch 6 % slower than lockstep levels).
bool shares_sm(ul_batch* b, const ul::Geo& g, int slab_t, int cluster)
{
    int dev = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t smem = b->precision == UL_FP64 ? ul::slab_level_smem<double>(g, slab_t, cluster)
                                                : ul::slab_level_smem<float>(g, slab_t, cluster);
    return 2 * smem <= static_cast<size_t>(per_sm);
}

// Jobs at the start of their level whose slab fits a cluster: grouped by shape, each group's
// whole level as one slab-resident launch on the level stream (after the lockstep passes
// enqueued so far), followed there by each job's reduction and result copy.
int offload_levels(ul_batch* b)
{
    if (b->slab_levels == 0) return UL_OK;
    std::map<std::string, std::vector<Job*>> groups;
    for (Job* j : b->resident)
        if (j->state == kRunning && j->pos == j->sweep_passes && j->pos < j->total_passes)
            groups[shape_key(b->precision, j->g, j->spec.slab_t)].push_back(j);
    if (groups.empty()) return UL_OK;
    for (auto& kv : groups) {
        std::vector<Job*>& js = kv.second;
        const ul::Geo g = js[0]->g;
        const int slab_t = js[0]->spec.slab_t;
        int cluster = 0, threads = 0;
        const int rc = b->precision == UL_FP64 ? slab_level_plan<double>(b, g, slab_t, &cluster, &threads)
                                               : slab_level_plan<float>(b, g, slab_t, &cluster, &threads);
        if (rc) return rc;
        if (!cluster) continue; // the lockstep passes run this level
        if (b->slab_levels == 2 && !shares_sm(b, g, slab_t, cluster)) continue;
        // each shape on its own stream (round robin), after the passes enqueued so far for
        // these jobs (all of one shape, so on one lockstep stream)
        const int si = js[0]->sidx;
        UB_CK(b, cudaEventRecord(b->ev_lock[si], b->lock_streams[si]));
        cudaStream_t lst = b->level_streams[si % ul_batch::kLevelStreams]; // the shape's priority
        UB_CK(b, cudaStreamWaitEvent(lst, b->ev_lock[si], 0));
        for (size_t k0 = 0; k0 < js.size(); k0 += ul::kMaxSlabJobs) {
            const size_t k1 = std::min(js.size(), k0 + static_cast<size_t>(ul::kMaxSlabJobs));
            ul::SlabJobTable t{};
            ul::SlabArgs a{};
            a.u.slab_t = slab_t;
            a.cluster = cluster;
            a.nz = g.L / cluster;
            for (size_t k = k0; k < k1; ++k) {
                Job* j = js[k];
                ul::SlabJob& sj = t.job[t.njobs++];
                sj.theta = j->theta;
                sj.cs = j->cs;
                sj.asum = j->asum;
                sj.u.slab_t = slab_t;
                sj.u.frozen_mask = 0;
                if (g.Nt <= 64)
                    for (int tt = 0; tt < g.Nt; tt += slab_t) sj.u.frozen_mask |= 1ull << tt;
                sj.u.pass = j->metro_pass;
                sj.u.pass_base = nullptr;
                sj.u.seed = j->spec.seed;
                sj.u.beta = j->spec.beta;
                sj.u.width = j->spec.metro_width;
                sj.u.beta_f = static_cast<float>(j->spec.beta);
                sj.u.width_f = static_cast<float>(j->spec.metro_width);
                sj.u.accepted = j->accepted;
                sj.n_units = j->spec.n_sub;
                sj.n_metro = j->spec.sub_metro;
                sj.n_or = j->spec.sub_or;
                sj.r_max = j->spec.r_max;
            }
            UB_TRACE("slab level launch L=%d jobs=%d cluster=%d threads=%d stream=%d", g.L, t.njobs, cluster, threads,
                     si % ul_batch::kLevelStreams);
            cudaError_t e = b->precision == UL_FP64 ? ul::launch_slab_jobs<double>(g, a, t, threads, lst)
                                                    : ul::launch_slab_jobs<float>(g, a, t, threads, lst);
            if (e != cudaSuccess) return bcuda(b, e, "slab-resident level launch");
            b->launches += 1;
            b->slab_launches += 1;
            for (size_t k = k0; k < k1; ++k) {
                Job* j = js[k];
                const uint64_t per = updatable(*j, slab_t);
                const uint64_t nsub = static_cast<uint64_t>(j->spec.n_sub);
                b->link_updates += nsub * static_cast<uint64_t>(j->spec.sub_metro + j->spec.sub_or) * per;
                j->metro_pass += nsub * static_cast<uint64_t>(j->spec.sub_metro);
                j->proposed += nsub * static_cast<uint64_t>(j->spec.sub_metro) * per;
                j->pos = j->total_passes;
                const int rc2 = finalize_job(b, j, lst);
                if (rc2) return rc2;
            }
        }
    }
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

// Candidate lockstep block sizes; each is timed on kTunePasses consecutive passes (whole
// compound sweeps, so every candidate sees the same mix of Metropolis and overrelaxation).
constexpr int kTunePasses = 4;

std::vector<int> lockstep_candidates(int precision)
{
    if (precision == UL_FP64) return {64, 128, 256};
    return {128, 288, 576};
}

std::string lockstep_key(int precision, const ul::Geo& g)
{
    return std::string(precision == UL_FP64 ? "fp64" : "fp32") + "/lockstep_threads/L" + std::to_string(g.L) + "_Nt" +
           std::to_string(g.Nt);
}

// Block size for the next pass of a group of shape g: the tuned or cached choice, else the
// candidate under test (returns 0 with *timing = true while timing).
int lockstep_threads(ul_batch* b, const ul::Geo& g, bool* timing)
{
    *timing = false;
    ul_batch::ShapeTune& st = b->tunes[lockstep_key(b->precision, g)];
    if (st.chosen) return st.chosen;
    int cached = 0;
    const std::vector<int> cands = lockstep_candidates(b->precision);
    if (tune_cache().get(lockstep_key(b->precision, g), &cached) &&
        std::find(cands.begin(), cands.end(), cached) != cands.end()) {
        st.chosen = cached;
        return cached;
    }
    const int total = kTunePasses * static_cast<int>(cands.size());
    if (st.next < total) {
        *timing = true;
        return cands[st.next / kTunePasses];
    }
    return 0; // all timed; collect_tuning picks
}

// When every timed pass of a shape has completed: the candidate with the least time per
// link wins (kept in the tune cache).
void collect_tuning(ul_batch* b)
{
    const std::vector<int> cands = lockstep_candidates(b->precision);
    for (auto& kv : b->tunes) {
        ul_batch::ShapeTune& st = kv.second;
        if (st.chosen || st.next < kTunePasses * static_cast<int>(cands.size())) continue;
        bool ready = true;
        for (auto& smp : st.samples) ready = ready && cudaEventQuery(smp.b) == cudaSuccess;
        if (!ready) continue;
        double best = 1e300;
        int pick = cands[0];
        for (int c : cands) {
            double ms_sum = 0.0, links = 0.0;
            for (auto& smp : st.samples)
                if (smp.threads == c) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, smp.a, smp.b);
                    ms_sum += ms;
                    links += smp.links;
                }
            if (links > 0 && ms_sum / links < best) {
                best = ms_sum / links;
                pick = c;
            }
        }
        for (auto& smp : st.samples) {
            cudaEventDestroy(smp.a);
            cudaEventDestroy(smp.b);
        }
        st.samples.clear();
        st.chosen = pick;
        b->threads = pick;
        tune_cache().put(kv.first, pick);
    }
}

size_t job_link_bytes(const ul_batch* b, const Job& j) { return 4ull * j.g.V * 3 * real_size(b); }

// Lockstep jobs (running, not offloaded) in groups of one shape whose links fit
// b->group_bytes (at least one job, at most kMaxBatchJobs), in job order.
std::vector<std::vector<Job*>> lockstep_groups(ul_batch* b)
{
    std::map<std::pair<int, int>, std::vector<Job*>> by_shape;
    for (Job* j : b->resident)
        if (j->state == kRunning && j->pos < j->total_passes) by_shape[{j->g.L, j->g.Nt}].push_back(j);
    std::vector<std::vector<Job*>> groups;
    for (auto& kv : by_shape) {
        std::vector<Job*> cur;
        size_t bytes = 0;
        for (Job* j : kv.second) {
            const size_t jb = job_link_bytes(b, *j);
            if (!cur.empty() && (bytes + jb > b->group_bytes || static_cast<int>(cur.size()) == ul::kMaxBatchJobs)) {
                groups.push_back(cur);
                cur.clear();
                bytes = 0;
            }
            cur.push_back(j);
            bytes += jb;
        }
        if (!cur.empty()) groups.push_back(cur);
    }
    return groups;
}

// One lockstep pass of one group (jobs of one shape): 8 class launches, then the measurement
// of the jobs whose sub-sample ended with this pass.  *did_work = false when no job of the
// group had a pass left.
int group_pass(ul_batch* b, const std::vector<Job*>& group, bool* did_work)
{
    *did_work = false;
    std::vector<Job*> in_pass;
    for (Job* j : group)
        if (j->state == kRunning && j->pos < j->total_passes) in_pass.push_back(j);
    if (in_pass.empty()) return UL_OK;
    *did_work = true;
    const ul::Geo g = in_pass[0]->g;
    cudaStream_t st = b->lock_streams[in_pass[0]->sidx];
    bool timing = false;
    int threads = lockstep_threads(b, g, &timing);
    if (!threads) threads = ul::class_block_threads(g.Vh, b->precision == UL_FP32_ACC64); // waiting for timings
    b->threads = threads;
    ul::BatchUpdateTable t{};
    ul::BatchMeasureTable m{};
    long work_t = 0, work_s = 0; // links per lattice of the temporal / spatial classes (largest in the group)
    std::vector<bool> measure(in_pass.size(), false);
    double links = 0.0;
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
        u.metro = metro ? 1 : 0;
        u.slab_t = slab_t;
        u.frozen_mask = 0;
        if (slab_t > 0 && j->g.Nt <= 64)
            for (int tt = 0; tt < j->g.Nt; tt += slab_t) u.frozen_mask |= 1ull << tt;
        u.pass = j->metro_pass;
        u.seed = j->spec.seed;
        u.beta = j->spec.beta;
        u.width = j->spec.metro_width;
        work_t = std::max<long>(work_t, j->g.Vh);
        const long spatial = slab_t > 1 ? static_cast<long>(j->g.Nt / slab_t) * (slab_t - 1) * (j->g.L3 / 2)
                                        : (slab_t == 1 ? 0L : static_cast<long>(j->g.Vh));
        work_s = std::max(work_s, spatial);
        const uint64_t n_up = updatable(*j, slab_t);
        b->link_updates += n_up;
        links += static_cast<double>(n_up);
        if (metro) {
            j->metro_pass += 1;
            j->proposed += n_up;
        }
        measure[q] = meas;
    }
    b->passes += 1;
    ul_batch::Sample smp{threads, nullptr, nullptr, links};
    if (timing) {
        UB_CK(b, cudaEventCreate(&smp.a));
        UB_CK(b, cudaEventCreate(&smp.b));
        UB_CK(b, cudaEventRecord(smp.a, st));
    }
    const bool pdl = b->precision == UL_FP32_ACC64;
    for (int mu = 0; mu < 4; ++mu)
        for (int par = 0; par < 2; ++par) {
            const long work = mu == 0 ? work_t : work_s;
            if (work == 0) continue; // every spatial link of every lattice of the group is frozen
            const int bx = static_cast<int>((work + threads - 1) / threads);
            cudaError_t e = b->precision == UL_FP64
                ? ul::launch_group_update<double>(t, g.L, bx, threads, mu, par, st, pdl)
                : ul::launch_group_update<float>(t, g.L, bx, threads, mu, par, st, pdl);
            if (e != cudaSuccess) return bcuda(b, e, "lockstep update launch");
            b->launches += 1;
        }
    if (timing) {
        UB_CK(b, cudaEventRecord(smp.b, st));
        ul_batch::ShapeTune& st = b->tunes[lockstep_key(b->precision, g)];
        st.samples.push_back(smp);
        st.next += 1;
    }
    // measurements of the jobs whose sub-sample ended with this pass
    long mwork = 0;
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
        mj.slab_t = j->spec.slab_t;
        mj.r_max = j->spec.r_max;
        mwork = std::max<long>(mwork, static_cast<long>(j->S) * j->g.L3);
    }
    if (m.njobs) {
        const int bx = static_cast<int>((mwork + 255) / 256);
        cudaError_t e = b->precision == UL_FP64 ? ul::launch_group_measure<double>(m, bx, st)
                                                : ul::launch_group_measure<float>(m, bx, st);
        if (e != cudaSuccess) return bcuda(b, e, "lockstep measurement launch");
        b->launches += 1;
    }
    for (Job* j : in_pass)
        if (j->pos == j->total_passes) {
            const int rc = finalize_job(b, j, st);
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
    // stream k (lockstep and level) gets the k-th highest priority: shapes are assigned to
    // streams in order of decreasing volume (admit)
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    auto prio = [&](int k) { return std::min(least, greatest + k); };
    for (int k = 0; k < ul_batch::kLevelStreams && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithPriority(&b->level_streams[k], cudaStreamNonBlocking, prio(k));
    b->level_stream = b->level_streams[0];
    for (int k = 0; k < ul_batch::kLockStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithPriority(&b->lock_streams[k], cudaStreamNonBlocking, prio(k));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_lock[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_admit, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->base), hbm_budget_bytes);
    if (e == cudaSuccess) e = ul::prepare_ml_reduce();
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (b->base) cudaFree(b->base);
        if (b->ev_admit) cudaEventDestroy(b->ev_admit);
        for (int k = 0; k < ul_batch::kLockStreams; ++k) {
            if (b->ev_lock[k]) cudaEventDestroy(b->ev_lock[k]);
            if (b->lock_streams[k]) cudaStreamDestroy(b->lock_streams[k]);
        }
        for (cudaStream_t ls : b->level_streams)
            if (ls) cudaStreamDestroy(ls);
        if (b->own_stream) cudaStreamDestroy(b->own_stream);
        delete b;
        return e == cudaErrorMemoryAllocation ? UL_ENOMEM : UL_ECUDA;
    }
    b->arena.init(hbm_budget_bytes);
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
    UB_TRACE("step: %zu queued, %zu resident", b->queue.size(), b->resident.size());
    if (max_passes > 0) {
        int rc = admit(b);
        if (rc) return rc;
        UB_TRACE("admitted: %zu resident", b->resident.size());
        rc = offload_levels(b);
        if (rc) return rc;
        // each group runs its passes back to back, so that its links stay in L2
        for (const std::vector<Job*>& group : lockstep_groups(b)) {
            for (int it = 0; it < max_passes; ++it) {
                bool work = false;
                rc = group_pass(b, group, &work);
                if (rc) return rc;
                if (!work) break;
                rc = offload_levels(b);
                if (rc) return rc;
            }
            collect_tuning(b);
        }
        rc = offload_levels(b);
        if (rc) return rc;
    }
    UB_TRACE("step: retire");
    retire_finished(b);
    collect_tuning(b);
    UB_TRACE("step: done");
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

int ul_batch_plan(ul_batch* b, int L, int Nt, int slab_t, int* cluster, uint64_t* slab_launches)
{
    if (!b) return UL_EINVAL;
    if (L < 2 || Nt < 2 || (L & 1) || (Nt & 1) || slab_t < 1 || Nt % slab_t)
        return bfail(b, UL_EINVAL, "ul_batch_plan: L, Nt even >= 2 and slab_t dividing Nt");
    if (slab_launches) *slab_launches = b->slab_launches;
    if (!cluster) return UL_OK;
    ul::Geo g{};
    g.L = L;
    g.Nt = Nt;
    g.Lh = L / 2;
    g.L3 = L * L * L;
    g.V = g.L3 * Nt;
    g.Vh = g.V / 2;
    int c = 0, t = 0;
    const int rc = b->precision == UL_FP64 ? slab_level_plan<double>(b, g, slab_t, &c, &t)
                                           : slab_level_plan<float>(b, g, slab_t, &c, &t);
    if (rc) return rc;
    *cluster = b->slab_levels == 0 || (b->slab_levels == 2 && c && !shares_sm(b, g, slab_t, c)) ? 0 : c;
    return UL_OK;
}

int ul_batch_counters(ul_batch* b, uint64_t* slab_level_launches)
{
    if (!b) return UL_EINVAL;
    if (slab_level_launches) *slab_level_launches = b->slab_launches;
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
    for (cudaStream_t ls : b->level_streams)
        if (ls) cudaStreamSynchronize(ls);
    for (cudaStream_t ls : b->lock_streams)
        if (ls) cudaStreamSynchronize(ls);
    for (auto& kv : b->tunes)
        for (auto& smp : kv.second.samples) {
            cudaEventDestroy(smp.a);
            cudaEventDestroy(smp.b);
        }
    for (auto& kv : b->jobs) destroy_job(kv.second);
    cudaFree(b->base);
    if (b->ev_admit) cudaEventDestroy(b->ev_admit);
    for (int k = 0; k < ul_batch::kLockStreams; ++k) {
        if (b->ev_lock[k]) cudaEventDestroy(b->ev_lock[k]);
        if (b->lock_streams[k]) cudaStreamDestroy(b->lock_streams[k]);
    }
    for (cudaStream_t ls : b->level_streams)
        if (ls) cudaStreamDestroy(ls);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return UL_OK;
}

int ul_batch_set_option(ul_batch* b, const char* key, double v)
{
    if (!b) return UL_EINVAL;
    if (!key) return bfail(b, UL_EINVAL, "ul_batch_set_option: NULL key");
    if (!std::strcmp(key, "group_mb")) {
        if (!(v >= 1.0 && v <= 65536.0)) return bfail(b, UL_EINVAL, "ul_batch_set_option: group_mb must be in [1, 65536]");
        b->group_bytes = static_cast<size_t>(v) << 20;
        return UL_OK;
    }
    if (!std::strcmp(key, "slab_levels")) {
        if (v != 0.0 && v != 1.0 && v != 2.0) return bfail(b, UL_EINVAL, "ul_batch_set_option: slab_levels must be 0, 1 or 2");
        b->slab_levels = static_cast<int>(v);
        return UL_OK;
    }
    if (!std::strcmp(key, "tune")) {
        if (v != 0.0 && v != 1.0) return bfail(b, UL_EINVAL, "ul_batch_set_option: tune must be 0 or 1");
        b->tune_slab = v != 0.0;
        b->plans.clear();
        return UL_OK;
    }
    return bfail(b, UL_EINVAL, std::string("ul_batch_set_option: unknown option ") + key);
}

const char* ul_batch_last_error(const ul_batch* b) { return b ? b->err.c_str() : ""; }

} // extern "C"
