// ul_noalloc.cu — ul_plaquette_noalloc: the mean plaquette of a caller-owned angle array,
// computed without allocating any device memory.
//
// Some callers cannot let a library allocate: a host that runs under a fixed device-memory
// budget handed out by its own allocator (a framework's caching allocator, an embedded
// service with a hard cap) must not see memory appear outside that budget, and a loop that
// cannot afford the device-wide synchronisation cudaMalloc/cudaFree may imply cannot call
// them at all.  This entry point takes the input and output buffers from the caller and
// keeps its only scratch — one partial sum per block of 256 sites — in the file-scope
// device array below, which every GPU that loads the library holds until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it names a
// stand-in, not GPU memory), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
#include <cstdint>
#include <mutex>

#include "../../include/ul.h"
#include "ul_math.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
// One partial sum per block of 256 sites: lattices up to 2^24 sites (e.g. 64^4).
constexpr int kNoAllocMaxBlocks = 1 << 16;
constexpr long long kNoAllocMaxSites = static_cast<long long>(kNoAllocMaxBlocks) * kNoAllocThreads;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_setup_mutex;
double* g_partials_dev[kMaxDevices] = {};

__device__ __forceinline__ double warp_block_sum(double v, double* smem)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = v;
    __syncthreads();
    double total = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNoAllocThreads / 32; ++w) total += smem[w];
    return total;
}

// Per-site sum over the six planes of Re U_mu nu(x) = cos(theta_mu(x) + theta_nu(x+mu)
// - theta_mu(x+nu) - theta_nu(x)); canonical layout theta[mu*V + i].
__global__ void __launch_bounds__(kNoAllocThreads)
    noalloc_plaquette_partials(const double* __restrict__ theta, int L, int Nt, double* __restrict__ partials)
{
    __shared__ double smem[kNoAllocThreads / 32];
    const long long V = static_cast<long long>(L) * L * L * Nt;
    const long long i = static_cast<long long>(blockIdx.x) * kNoAllocThreads + threadIdx.x;
    double v = 0.0;
    if (i < V) {
        int c[4];
        c[1] = static_cast<int>(i % L);
        c[2] = static_cast<int>((i / L) % L);
        c[3] = static_cast<int>((i / (static_cast<long long>(L) * L)) % L);
        c[0] = static_cast<int>(i / (static_cast<long long>(L) * L * L));
        auto shifted = [&](int d) {
            int e[4] = {c[0], c[1], c[2], c[3]};
            const int n = d == 0 ? Nt : L;
            e[d] = e[d] + 1 == n ? 0 : e[d] + 1;
            return e[1] + static_cast<long long>(L) * (e[2] + static_cast<long long>(L) * (e[3] + static_cast<long long>(L) * e[0]));
        };
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                const double a = theta[mu * V + i] + theta[nu * V + shifted(mu)] - theta[mu * V + shifted(nu)] -
                                 theta[nu * V + i];
                v += cos(a);
            }
    }
    const double t = warp_block_sum(v, smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kNoAllocThreads)
    noalloc_plaquette_finish(const double* __restrict__ partials, int n, double scale, double* __restrict__ out)
{
    __shared__ double smem[kNoAllocThreads / 32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += kNoAllocThreads) v += partials[k];
    const double t = warp_block_sum(v, smem);
    if (threadIdx.x == 0) *out = t * scale;
}

// Device address of the partials array for the current device (looked up once per device).
cudaError_t partials_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_dev[dev] = static_cast<double*>(p);
    }
    *out = g_partials_dev[dev];
    return cudaSuccess;
}

} // namespace

extern "C" {

int ul_plaquette_noalloc(const double* theta_dev, int L, int Nt, double* out_dev, void* cuda_stream)
{
    if (!theta_dev || !out_dev) return UL_EINVAL;
    if (L < 2 || Nt < 2) return UL_EINVAL;
    const long long V = static_cast<long long>(L) * L * L * Nt;
    if (V > kNoAllocMaxSites) return UL_EINVAL; // larger than the built-in scratch array covers
    double* partials = nullptr;
    if (partials_for_current_device(&partials) != cudaSuccess) return UL_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nb = static_cast<int>((V + kNoAllocThreads - 1) / kNoAllocThreads);
    // An error left pending on this thread by earlier, unrelated work is cleared here, so
    // that only this call's own launch errors are reported below.
    (void)cudaGetLastError();
    noalloc_plaquette_partials<<<nb, kNoAllocThreads, 0, st>>>(theta_dev, L, Nt, partials);
    noalloc_plaquette_finish<<<1, kNoAllocThreads, 0, st>>>(partials, nb, 1.0 / (6.0 * static_cast<double>(V)),
                                                             out_dev);
    return cudaGetLastError() == cudaSuccess ? UL_OK : UL_ECUDA;
}

} // extern "C"
