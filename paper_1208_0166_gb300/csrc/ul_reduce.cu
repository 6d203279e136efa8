// ul_reduce.cu — cross-slab products, reduction over x0 and normalisation of the
// multilevel estimators (Section 2.2 of arXiv:1208.0166):
//   C(r)        = (1/L^3) sum_x0 prod_s A_s(x0, r),                 A_s = <T>_s
//   N(r, d, ch) = (1/V)   sum_x0 sum_s B_s(x0, r, d, ch) prod_{s' != s} A_s'(x0, r),
//                                                                  B_s = <T O>_s
// The product over the other slabs is prefix(s) * suffix(s+1) (no division).  All sums
// run in a fixed order, so results are bitwise reproducible for a fixed lattice shape.
#include <atomic>
#include "ul_device.cuh"
#include "ul_internal.h"
#include "ul_math.cuh"

namespace ul {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double bsum(double v, double* smem)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double total = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; ++w) total += smem[w];
    return total;
}

// Mean of a sample sum: multiplication by the reciprocal of the sample count (one DMUL
// instead of an FP64 division per component).
__device__ __forceinline__ Cx<double> mean_of(double2 v, double inv_n) { return Cx<double>{v.x * inv_n, v.y * inv_n}; }

// grid (chunks, r_max); partials[((r*Q + q)*chunks + chunk)*2 + part], Q = 1 + nd*8.
__global__ void __launch_bounds__(kT) ml_reduce_kernel(Geo g, int S, int n_sub, int r_max, int nd,
                                                        const double2* __restrict__ asum,
                                                        const double2* __restrict__ bsum_in,
                                                        double* __restrict__ partials)
{
    __shared__ double smem[kT / 32];
    const int chunks = gridDim.x, chunk = blockIdx.x, r = blockIdx.y;
    const int x0 = chunk * kT + threadIdx.x;
    const bool valid = x0 < g.L3;
    const int Q = 1 + nd * 8;
    const double n = 1.0 / static_cast<double>(n_sub);
    Cx<double> pre[kMaxSlabs + 1];
    pre[0] = Cx<double>{1.0, 0.0};
    for (int s = 0; s < S; ++s) {
        const Cx<double> A = valid ? mean_of(asum[static_cast<long>(s * r_max + r) * g.L3 + x0], n) : Cx<double>{0.0, 0.0};
        pre[s + 1] = cmul(pre[s], A);
    }
    const Cx<double> c = valid ? pre[S] : Cx<double>{0.0, 0.0};
    double re = bsum(c.re, smem);
    double im = bsum(c.im, smem);
    if (threadIdx.x == 0) {
        const long o = ((static_cast<long>(r) * Q + 0) * chunks + chunk) * 2;
        partials[o] = re;
        partials[o + 1] = im;
    }
    for (int d = 0; d < nd; ++d) {
        Cx<double> acc[8];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) acc[ch] = Cx<double>{0.0, 0.0};
        if (valid) {
            Cx<double> suf{1.0, 0.0};
            for (int s = S - 1; s >= 0; --s) {
                const Cx<double> W = cmul(pre[s], suf);
                const long base = ((static_cast<long>(s * r_max + r) * nd + d) * 8) * g.L3 + x0;
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) acc[ch] = cadd(acc[ch], cmul(mean_of(bsum_in[base + ch * g.L3], n), W));
                suf = cmul(mean_of(asum[static_cast<long>(s * r_max + r) * g.L3 + x0], n), suf);
            }
        }
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            re = bsum(acc[ch].re, smem);
            im = bsum(acc[ch].im, smem);
            if (threadIdx.x == 0) {
                const long o = ((static_cast<long>(r) * Q + 1 + d * 8 + ch) * chunks + chunk) * 2;
                partials[o] = re;
                partials[o + 1] = im;
            }
        }
    }
}

// The same reduction with the other-slab weights W_s = (1/n_sub) prod_{s' != s} A_s'(x0, r)
// formed once per (x0, r) and kept in shared memory (column tid of wsm[S][kT]: no thread
// reads another's), so the offsets d reuse them; a term of the field sums is then four
// FP64 fused multiply-adds, B_s W_s (the mean of B folded into W).  The correlator is
// summed exactly as in ml_reduce_kernel.
constexpr int kReduceSmemBytes = 200 * 1024;

__global__ void __launch_bounds__(kT) ml_reduce_w_kernel(Geo g, int S, int n_sub, int r_max, int nd,
                                                          const double2* __restrict__ asum,
                                                          const double2* __restrict__ bsum_in,
                                                          double* __restrict__ partials)
{
    extern __shared__ double2 wsm[];
    __shared__ double smem[kT / 32];
    const int chunks = gridDim.x, chunk = blockIdx.x, r = blockIdx.y;
    const int tid = static_cast<int>(threadIdx.x);
    const int x0 = chunk * kT + tid;
    const bool valid = x0 < g.L3;
    const int Q = 1 + nd * 8;
    const double n = 1.0 / static_cast<double>(n_sub);
    Cx<double> p{1.0, 0.0};
    for (int s = 0; s < S; ++s) {
        const Cx<double> A = valid ? mean_of(asum[static_cast<long>(s * r_max + r) * g.L3 + x0], n) : Cx<double>{0.0, 0.0};
        wsm[s * kT + tid] = make_double2(p.re, p.im); // prefix prod_{s' < s} A_s'
        p = cmul(p, A);
    }
    const Cx<double> c = valid ? p : Cx<double>{0.0, 0.0};
    double re = bsum(c.re, smem);
    double im = bsum(c.im, smem);
    if (threadIdx.x == 0) {
        const long o = ((static_cast<long>(r) * Q + 0) * chunks + chunk) * 2;
        partials[o] = re;
        partials[o + 1] = im;
    }
    if (nd == 0) return;
    if (valid) {
        Cx<double> suf{1.0, 0.0};
        for (int s = S - 1; s >= 0; --s) {
            const double2 pre = wsm[s * kT + tid];
            const Cx<double> W = cmul(Cx<double>{pre.x, pre.y}, suf);
            wsm[s * kT + tid] = make_double2(W.re * n, W.im * n);
            suf = cmul(mean_of(asum[static_cast<long>(s * r_max + r) * g.L3 + x0], n), suf);
        }
    }
    for (int d = 0; d < nd; ++d) {
        double ar[8], ai[8];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) ar[ch] = ai[ch] = 0.0;
        if (valid) {
            for (int s = S - 1; s >= 0; --s) {
                const double2 W = wsm[s * kT + tid];
                const long base = ((static_cast<long>(s * r_max + r) * nd + d) * 8) * g.L3 + x0;
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    const double2 B = bsum_in[base + ch * g.L3];
                    ar[ch] = fma(B.x, W.x, fma(-B.y, W.y, ar[ch]));
                    ai[ch] = fma(B.x, W.y, fma(B.y, W.x, ai[ch]));
                }
            }
        }
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            re = bsum(ar[ch], smem);
            im = bsum(ai[ch], smem);
            if (threadIdx.x == 0) {
                const long o = ((static_cast<long>(r) * Q + 1 + d * 8 + ch) * chunks + chunk) * 2;
                partials[o] = re;
                partials[o + 1] = im;
            }
        }
    }
}

// One thread per output double: sum over chunks in order, then normalise.
__global__ void ml_finalize_kernel(int r_max, int nd, int chunks, const double* __restrict__ partials, double L3,
                                   double V, double* __restrict__ out)
{
    const int Q = 1 + nd * 8;
    const int k = blockIdx.x * blockDim.x + threadIdx.x; // (r*Q + q)*2 + part
    if (k >= r_max * Q * 2) return;
    const int part = k & 1;
    const int rq = k >> 1;
    const int r = rq / Q, q = rq - r * Q;
    double v = 0.0;
    for (int c = 0; c < chunks; ++c) v += partials[(static_cast<long>(rq) * chunks + c) * 2 + part];
    if (q == 0) {
        out[2 * r + part] = v / L3;
    } else {
        out[2 * r_max + ((r * nd) * 8 + (q - 1)) * 2 + part] = v / V;
    }
}

// Vacuum channel averages: block ch sums osum[ch][0..SL3) and divides by n_sub V.
__global__ void __launch_bounds__(kT) ml_vacuum_kernel(int SL3, const double* __restrict__ osum, double nV,
                                                        double* __restrict__ out)
{
    __shared__ double smem[kT / 32];
    const int ch = blockIdx.x;
    double v = 0.0;
    for (int k = threadIdx.x; k < SL3; k += kT) v += osum[static_cast<long>(ch) * SL3 + k];
    const double t = bsum(v, smem);
    if (threadIdx.x == 0) out[ch] = t / nV;
}

__global__ void set_u64_kernel(unsigned long long* p, unsigned long long v) { *p = v; }

// Two-level multilevel: one level-1 sample per (level-1 slab s1, r, x0) is the product of
// the level-2 means of the m level-2 slabs inside s1, added to the level-1 accumulator.
//   asum1[(s1*R + r)*L3 + x0] += prod_{j<m} asum2[((s1*m + j)*R + r)*L3 + x0] / n2
__global__ void __launch_bounds__(kT) fold_level2_kernel(int L3, int S1, int m, int r_max, int n2,
                                                         const double2* __restrict__ asum2,
                                                         double2* __restrict__ asum1)
{
    const long k = static_cast<long>(blockIdx.x) * kT + threadIdx.x;
    const long total = static_cast<long>(S1) * r_max * L3;
    if (k >= total) return;
    const int x0 = static_cast<int>(k % L3);
    const long sr = k / L3;
    const int r = static_cast<int>(sr % r_max);
    const int s1 = static_cast<int>(sr / r_max);
    const double n = 1.0 / static_cast<double>(n2);
    Cx<double> prod{1.0, 0.0};
    for (int j = 0; j < m; ++j)
        prod = cmul(prod, mean_of(asum2[(static_cast<long>(s1 * m + j) * r_max + r) * L3 + x0], n));
    double2 a = asum1[k];
    a.x += prod.re;
    a.y += prod.im;
    asum1[k] = a;
}

// Two-level multilevel with insertions: one level-1 sample per (level-1 slab s1, r, x0) from
// the level-2 means of the m level-2 slabs j inside s1,
//   asum1 += prod_j A2(j),   bsum1[d, ch] += sum_j B2(j, d, ch) prod_{j' != j} A2(j'),
// with A2 = asum2 / n2 and B2 = bsum2 / n2 (products in j order, sums in j order).
constexpr int kMaxFoldM = 16;

__global__ void __launch_bounds__(kT) fold_level2_fields_kernel(int L3, int S1, int m, int r_max, int nd, int n2,
                                                                const double2* __restrict__ asum2,
                                                                const double2* __restrict__ bsum2,
                                                                double2* __restrict__ asum1,
                                                                double2* __restrict__ bsum1)
{
    const long k = static_cast<long>(blockIdx.x) * kT + threadIdx.x;
    const long total = static_cast<long>(S1) * r_max * L3;
    if (k >= total) return;
    const int x0 = static_cast<int>(k % L3);
    const long sr = k / L3;
    const int r = static_cast<int>(sr % r_max);
    const int s1 = static_cast<int>(sr / r_max);
    const double n = 1.0 / static_cast<double>(n2);
    Cx<double> A[kMaxFoldM];
    Cx<double> prod{1.0, 0.0};
    for (int j = 0; j < m; ++j) {
        A[j] = mean_of(asum2[(static_cast<long>(s1 * m + j) * r_max + r) * L3 + x0], n);
        prod = cmul(prod, A[j]);
    }
    double2 a = asum1[k];
    a.x += prod.re;
    a.y += prod.im;
    asum1[k] = a;
    for (int d = 0; d < nd; ++d)
        for (int ch = 0; ch < 8; ++ch) {
            Cx<double> b{0.0, 0.0};
            for (int j = 0; j < m; ++j) {
                const long i2 = ((static_cast<long>(s1 * m + j) * r_max + r) * nd + d) * 8 + ch;
                Cx<double> term = mean_of(bsum2[i2 * L3 + x0], n);
                for (int j2 = 0; j2 < m; ++j2)
                    if (j2 != j) term = cmul(term, A[j2]);
                b = cadd(b, term);
            }
            const long i1 = ((static_cast<long>(s1) * r_max + r) * nd + d) * 8 + ch;
            double2 v = bsum1[i1 * L3 + x0];
            v.x += b.re;
            v.y += b.im;
            bsum1[i1 * L3 + x0] = v;
        }
}

// The same fold for a compile-time number M of level-2 slabs per level-1 slab: the weights
// W_j = (1/n2) prod_{j' != j} A2(j') are formed once per (s1, r, x0) in registers, and a
// term of the field sums is four FP64 fused multiply-adds, B_j W_j (the sample mean of B
// folded into W).  The correlator product is formed exactly as in the generic kernel.
template <int M>
__global__ void __launch_bounds__(kT) fold_level2_fields_m_kernel(int L3, int S1, int r_max, int nd, int n2,
                                                                  const double2* __restrict__ asum2,
                                                                  const double2* __restrict__ bsum2,
                                                                  double2* __restrict__ asum1,
                                                                  double2* __restrict__ bsum1)
{
    const long k = static_cast<long>(blockIdx.x) * kT + threadIdx.x;
    const long total = static_cast<long>(S1) * r_max * L3;
    if (k >= total) return;
    const int x0 = static_cast<int>(k % L3);
    const long sr = k / L3;
    const int r = static_cast<int>(sr % r_max);
    const int s1 = static_cast<int>(sr / r_max);
    const double n = 1.0 / static_cast<double>(n2);
    Cx<double> A[M];
    Cx<double> prod{1.0, 0.0};
#pragma unroll
    for (int j = 0; j < M; ++j) {
        A[j] = mean_of(asum2[(static_cast<long>(s1 * M + j) * r_max + r) * L3 + x0], n);
        prod = cmul(prod, A[j]);
    }
    double2 a = asum1[k];
    a.x += prod.re;
    a.y += prod.im;
    asum1[k] = a;
    Cx<double> W[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        Cx<double> w{n, 0.0};
#pragma unroll
        for (int j2 = 0; j2 < M; ++j2)
            if (j2 != j) w = cmul(w, A[j2]);
        W[j] = w;
    }
    for (int d = 0; d < nd; ++d) {
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            double br = 0.0, bi = 0.0;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const long i2 = ((static_cast<long>(s1 * M + j) * r_max + r) * nd + d) * 8 + ch;
                const double2 B = bsum2[i2 * L3 + x0];
                br = fma(B.x, W[j].re, fma(-B.y, W[j].im, br));
                bi = fma(B.x, W[j].im, fma(B.y, W[j].re, bi));
            }
            const long i1 = ((static_cast<long>(s1) * r_max + r) * nd + d) * 8 + ch;
            double2 v = bsum1[i1 * L3 + x0];
            v.x += br;
            v.y += bi;
            bsum1[i1 * L3 + x0] = v;
        }
    }
}

} // namespace

cudaError_t launch_fold_level2_fields(const Geo& g, int tau1, int tau2, int r_max, int nd, int n2,
                                      const double2* asum2, const double2* bsum2, double2* asum1, double2* bsum1,
                                      cudaStream_t st)
{
    const int S1 = g.Nt / tau1, m = tau1 / tau2;
    if (m > kMaxFoldM) return cudaErrorInvalidValue;
    const long total = static_cast<long>(S1) * r_max * g.L3;
    const int nb = static_cast<int>((total + kT - 1) / kT);
    switch (m) {
    case 1: fold_level2_fields_m_kernel<1><<<nb, kT, 0, st>>>(g.L3, S1, r_max, nd, n2, asum2, bsum2, asum1, bsum1); break;
    case 2: fold_level2_fields_m_kernel<2><<<nb, kT, 0, st>>>(g.L3, S1, r_max, nd, n2, asum2, bsum2, asum1, bsum1); break;
    case 4: fold_level2_fields_m_kernel<4><<<nb, kT, 0, st>>>(g.L3, S1, r_max, nd, n2, asum2, bsum2, asum1, bsum1); break;
    default:
        fold_level2_fields_kernel<<<nb, kT, 0, st>>>(g.L3, S1, m, r_max, nd, n2, asum2, bsum2, asum1, bsum1);
        break;
    }
    return cudaGetLastError();
}

// set once the shared-memory limit has been raised: until then a launch that needs more
// than the default 48 KB takes the prefix-array form
std::atomic<bool> g_reduce_prepared{false};

cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st)
{
    set_u64_kernel<<<1, 1, 0, st>>>(p, v);
    return cudaGetLastError();
}

size_t ml_partials_doubles(const Geo& g, int r_max, int nd)
{
    const size_t chunks = (g.L3 + kT - 1) / kT;
    return static_cast<size_t>(r_max) * (1 + nd * 8) * chunks * 2;
}

cudaError_t launch_ml_reduce(const Geo& g, int slab_t, int n_sub, int r_max, int nd, const double2* asum,
                             const double2* bsum_in, const double* osum, double* partials, double* out_dev,
                             cudaStream_t st)
{
    const int S = g.Nt / slab_t;
    if (S > kMaxSlabs) return cudaErrorInvalidValue;
    const int chunks = (g.L3 + kT - 1) / kT;
    const size_t wbytes = static_cast<size_t>(S) * kT * sizeof(double2);
    if (wbytes <= 48 * 1024 || (wbytes <= kReduceSmemBytes && g_reduce_prepared.load()))
        ml_reduce_w_kernel<<<dim3(chunks, r_max), kT, wbytes, st>>>(g, S, n_sub, r_max, nd, asum, bsum_in, partials);
    else
        ml_reduce_kernel<<<dim3(chunks, r_max), kT, 0, st>>>(g, S, n_sub, r_max, nd, asum, bsum_in, partials);
    const int nout = r_max * (1 + nd * 8) * 2;
    ml_finalize_kernel<<<(nout + kT - 1) / kT, kT, 0, st>>>(r_max, nd, chunks, partials, static_cast<double>(g.L3),
                                                             static_cast<double>(g.V), out_dev);
    if (nd > 0 && osum)
        ml_vacuum_kernel<<<8, kT, 0, st>>>(S * g.L3, osum, static_cast<double>(n_sub) * static_cast<double>(g.V),
                                           out_dev + 2 * r_max + 2 * r_max * nd * 8);
    return cudaGetLastError();
}

cudaError_t prepare_ml_reduce()
{
    const cudaError_t e =
        cudaFuncSetAttribute(ml_reduce_w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kReduceSmemBytes);
    if (e == cudaSuccess) g_reduce_prepared.store(true);
    return e;
}

cudaError_t launch_ml_vacuum(int SL3, const double* osum, int nch, double nV, double* out, cudaStream_t st)
{
    ml_vacuum_kernel<<<nch, kT, 0, st>>>(SL3, osum, nV, out);
    return cudaGetLastError();
}

int plaquette_partials(const Geo& g) { return (g.V + kT - 1) / kT; }

cudaError_t launch_fold_level2(const Geo& g, int tau1, int tau2, int r_max, int n2, const double2* asum2,
                               double2* asum1, cudaStream_t st)
{
    const int S1 = g.Nt / tau1, m = tau1 / tau2;
    const long total = static_cast<long>(S1) * r_max * g.L3;
    fold_level2_kernel<<<static_cast<int>((total + kT - 1) / kT), kT, 0, st>>>(g.L3, S1, m, r_max, n2, asum2, asum1);
    return cudaGetLastError();
}

} // namespace ul
