// ul_kernels.cuh — link-update and measurement kernels, templated on the link precision.
// Included by ul_kernels_f64.cu (R = double, compiled with -fmad=false) and
// ul_kernels_f32.cu (R = float).
//
// Paper: arXiv:1208.0166, Section 2 (Wilson action, plaquette), Section 2.1 (Metropolis
// and overrelaxation), Section 2.2 (multilevel: slabs with frozen spatial links,
// transporters T, insertion operator, multilevel field estimator).
#pragma once
#include "ul_device.cuh"
#include "ul_internal.h"
#include "ul_math.cuh"

namespace ul {

constexpr int kThreads = 256;

template <typename R>
using cs_t = typename Prec<R>::cs_t;

template <typename R>
__device__ __forceinline__ Cx<R> link_u(const cs_t<R>* __restrict__ cs, int off)
{
    const cs_t<R> v = cs[off];
    return Cx<R>{v.x, v.y};
}

template <typename R>
__device__ __forceinline__ Cx<double> link_u64(const cs_t<R>* __restrict__ cs, int off)
{
    const cs_t<R> v = cs[off];
    return Cx<double>{static_cast<double>(v.x), static_cast<double>(v.y)};
}

inline int blocks_for(long n) { return static_cast<int>((n + kThreads - 1) / kThreads); }

// ---------------------------------------------------------------------------
// Hot start: theta = -pi + 2 pi u, u from Philox(counter (mu V + i, 0, 0, 0), key (seed, 0)).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) hot_start_kernel(Geo g, R* __restrict__ theta,
                                                             cs_t<R>* __restrict__ cs, uint64_t seed)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x; // [mu][parity][h]
    if (k >= 4 * g.V) return;
    const int mu = k / g.V;
    const int rem = k - mu * g.V;
    const int par = rem / g.Vh;
    const Site s = site_from_half(g, par, rem - par * g.Vh);
    const uint64_t link_id = static_cast<uint64_t>(mu) * g.V + lex_index(g, s);
    const Philox4 w = philox4x64_10(link_id, 0, 0, 0, seed, kStreamHotStart);
    const double u = static_cast<double>(w.w[0] >> 11) * 0x1.0p-53;
    const double th = -dm::PI + 2.0 * dm::PI * u;
    R t = static_cast<R>(th);
    if constexpr (sizeof(R) == 4) t = Prec<R>::wrap(t); // rounding may reach float(pi)
    theta[k] = t;
    R sn, cn;
    Prec<R>::sincos(t, &sn, &cn);
    cs[k] = cs_t<R>{cn, sn};
}

template <typename R>
__global__ void __launch_bounds__(kThreads) refresh_cs_kernel(Geo g, const R* __restrict__ theta,
                                                              cs_t<R>* __restrict__ cs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 4 * g.V) return;
    R sn, cn;
    Prec<R>::sincos(theta[k], &sn, &cn);
    cs[k] = cs_t<R>{cn, sn};
}

// ---------------------------------------------------------------------------
// Staple sum of link (mu, x), Section 2:
//   A = sum_{nu != mu} [ U_nu(x+mu) U*_mu(x+nu) U*_nu(x) + U*_nu(x+mu-nu) U*_mu(x-nu) U_nu(x-nu) ]
// so that the plaquettes containing U_mu(x) contribute Re(U_mu(x) A).  The terms are
// formed and summed in this order (nu ascending, forward before backward).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ Cx<R> staple_sum(const Geo& g, const cs_t<R>* __restrict__ cs, int mu, const Site& x)
{
    Cx<R> A{R(0), R(0)};
    const Site xpm = site_step(g, x, mu, +1);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const Site xpn = site_step(g, x, nu, +1);
        const Site xmn = site_step(g, x, nu, -1);
        const Site xpm_mn = site_step(g, xpm, nu, -1);
        const Cx<R> fwd = cmul(cmul(link_u<R>(cs, link_offset(g, nu, xpm)), cconj(link_u<R>(cs, link_offset(g, mu, xpn)))),
                               cconj(link_u<R>(cs, link_offset(g, nu, x))));
        const Cx<R> bwd = cmul(cmul(cconj(link_u<R>(cs, link_offset(g, nu, xpm_mn))),
                                    cconj(link_u<R>(cs, link_offset(g, mu, xmn)))),
                               link_u<R>(cs, link_offset(g, nu, xmn)));
        A = cadd(A, cadd(fwd, bwd));
    }
    return A;
}

// ---------------------------------------------------------------------------
// One sub-sweep of the links of class (mu, parity); Section 2.1.
//   Metropolis:      theta' = wrap(theta + width (2 u1 - 1)),
//                    dS = -beta Re(e^{i theta'} A) - (-beta Re(e^{i theta} A)),
//                    accept iff u2 < exp(-dS);
//   Overrelaxation:  theta' = wrap(-2 arg(A) - theta).
// With slab_t > 0, spatial links on slices t % slab_t == 0 are frozen (Section 2.2).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads)
    update_class_kernel(Geo g, R* __restrict__ theta, cs_t<R>* __restrict__ cs, int mu, int parity, int metro,
                        uint64_t pass, uint64_t seed, R beta, R width, int slab_t,
                        unsigned long long* __restrict__ accepted)
{
    using P = Prec<R>;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    bool acc = false;
    if (h < g.Vh) {
        const Site x = site_from_half(g, parity, h);
        const bool frozen = slab_t > 0 && mu != 0 && (x.c[0] % slab_t) == 0;
        if (!frozen) {
            const Cx<R> A = staple_sum<R>(g, cs, mu, x);
            const int off = (mu * 2 + parity) * g.Vh + h;
            const R th = theta[off];
            if (metro) {
                const uint64_t link_id = static_cast<uint64_t>(mu) * g.V + lex_index(g, x);
                const Philox4 w = philox4x64_10(link_id, pass, 0, 0, seed, kStreamMetropolis);
                const R u1 = P::uniform(w.w[0]);
                const R u2 = P::uniform(w.w[1]);
                const R prop = P::wrap(th + width * (R(2) * u1 - R(1)));
                const cs_t<R> old = cs[off];
                const R s_old = -beta * (old.x * A.re - old.y * A.im);
                R sn, cn;
                P::sincos(prop, &sn, &cn);
                const R s_new = -beta * (cn * A.re - sn * A.im);
                const R dS = s_new - s_old;
                if (u2 < P::exp(-dS)) {
                    theta[off] = prop;
                    cs[off] = cs_t<R>{cn, sn};
                    acc = true;
                }
            } else {
                const R alpha = P::atan2(A.im, A.re);
                const R nth = P::wrap(R(-2) * alpha - th);
                R sn, cn;
                P::sincos(nth, &sn, &cn);
                theta[off] = nth;
                cs[off] = cs_t<R>{cn, sn};
            }
        }
    }
    if (metro) {
        const unsigned mask = __ballot_sync(0xffffffffu, acc);
        if ((threadIdx.x & 31) == 0 && mask) atomicAdd(accepted, static_cast<unsigned long long>(__popc(mask)));
    }
}

// ---------------------------------------------------------------------------
// Layout conversion between the canonical host order theta[mu*V + i] and the device
// order [mu][parity][h].
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) to_canonical_kernel(Geo g, const R* __restrict__ theta,
                                                                double* __restrict__ canon)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x; // canonical index
    if (k >= 4 * g.V) return;
    const int mu = k / g.V;
    const Site s = site_from_lex(g, k - mu * g.V);
    canon[k] = static_cast<double>(theta[link_offset(g, mu, s)]);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) from_canonical_kernel(Geo g, const double* __restrict__ canon,
                                                                  R* __restrict__ theta, cs_t<R>* __restrict__ cs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 4 * g.V) return;
    const int mu = k / g.V;
    const Site s = site_from_lex(g, k - mu * g.V);
    const int off = link_offset(g, mu, s);
    const R t = static_cast<R>(canon[k]);
    theta[off] = t;
    R sn, cn;
    Prec<R>::sincos(t, &sn, &cn);
    cs[off] = cs_t<R>{cn, sn};
}

// ---------------------------------------------------------------------------
// Block sum of a double in a fixed order (bitwise reproducible for a fixed launch).
// ---------------------------------------------------------------------------
static __device__ __forceinline__ double block_sum(double v, double* smem /* kThreads/32 */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double total = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) total += smem[w];
    return total; // valid in thread 0
}

// Plaquette U_mu nu(x) = U_mu(x) U_nu(x+mu) U*_mu(x+nu) U*_nu(x), in FP64.
template <typename R>
__device__ __forceinline__ Cx<double> plaquette64(const Geo& g, const cs_t<R>* __restrict__ cs, int mu, int nu,
                                                  const Site& x)
{
    const Site xpm = site_step(g, x, mu, +1);
    const Site xpn = site_step(g, x, nu, +1);
    return cmul(cmul(cmul(link_u64<R>(cs, link_offset(g, mu, x)), link_u64<R>(cs, link_offset(g, nu, xpm))),
                     cconj(link_u64<R>(cs, link_offset(g, mu, xpn)))),
                cconj(link_u64<R>(cs, link_offset(g, nu, x))));
}

template <typename R>
__global__ void __launch_bounds__(kThreads) plaquette_kernel(Geo g, const cs_t<R>* __restrict__ cs,
                                                             double* __restrict__ partials)
{
    __shared__ double smem[kThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < g.V) {
        const Site x = site_from_lex(g, i);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) v += plaquette64<R>(g, cs, mu, nu, x).re;
    }
    const double t = block_sum(v, smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

static __global__ void __launch_bounds__(kThreads) sum_partials_kernel(const double* __restrict__ partials, int n,
                                                                double scale, double* __restrict__ out)
{
    __shared__ double smem[kThreads / 32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partials[k];
    const double t = block_sum(v, smem);
    if (threadIdx.x == 0) *out = t * scale;
}

// ---------------------------------------------------------------------------
// Multilevel measurement (Section 2.2).
// Field channels: ch = 2c + part, planes c = (0,1) E_x, (0,2) E_y, (0,3) E_z, (2,3) B_x,
// part 0 = Im P, part 1 = Re P.
// ---------------------------------------------------------------------------
__device__ __constant__ static const int kPlaneMu[4] = {0, 0, 0, 2};
__device__ __constant__ static const int kPlaneNu[4] = {1, 2, 3, 3};

// O[ch][s*L3 + y] = sum_{t in slab s} channel_ch(y, t); osum accumulates O over samples.
template <typename R>
__global__ void __launch_bounds__(kThreads) slab_channels_kernel(Geo g, const cs_t<R>* __restrict__ cs,
                                                                 int slab_t, double* __restrict__ O,
                                                                 double* __restrict__ osum)
{
    const int S = g.Nt / slab_t;
    const int k = blockIdx.x * blockDim.x + threadIdx.x; // s*L3 + y
    if (k >= S * g.L3) return;
    const int s = k / g.L3;
    const int y = k - s * g.L3;
    const int SL3 = S * g.L3;
    double acc[8];
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) acc[ch] = 0.0;
    for (int t = s * slab_t; t < (s + 1) * slab_t; ++t) {
        const Site x = site_from_lex(g, y + g.L3 * t);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const Cx<double> P = plaquette64<R>(g, cs, kPlaneMu[c], kPlaneNu[c], x);
            acc[2 * c] += P.im;
            acc[2 * c + 1] += P.re;
        }
    }
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        O[ch * SL3 + k] = acc[ch];
        osum[ch * SL3 + k] += acc[ch];
    }
}

// T(s, x0, r) = prod_{t in slab} U*_0(x0,t) U_0(x0 + r xhat, t);
// asum += T;  bsum += T * O(s, x0 + floor(r/2) xhat + d yhat).
template <typename R>
__global__ void __launch_bounds__(kThreads)
    measure_kernel(Geo g, const cs_t<R>* __restrict__ cs, int slab_t, int r_max, int nd, const double* __restrict__ O,
                   double2* __restrict__ asum, double2* __restrict__ bsum)
{
    const int S = g.Nt / slab_t;
    const int k = blockIdx.x * blockDim.x + threadIdx.x; // s*L3 + x0
    if (k >= S * g.L3) return;
    const int s = k / g.L3;
    const int x0 = k - s * g.L3;
    const int SL3 = S * g.L3;
    const int px = x0 % g.L, py = (x0 / g.L) % g.L, pz = x0 / (g.L * g.L);
    for (int r = 1; r <= r_max; ++r) {
        const int x1 = (px + r) % g.L + g.L * (py + g.L * pz);
        Cx<double> T{1.0, 0.0};
        for (int t = s * slab_t; t < (s + 1) * slab_t; ++t) {
            const Cx<double> a = link_u64<R>(cs, link_offset(g, 0, site_from_lex(g, x0 + g.L3 * t)));
            const Cx<double> b = link_u64<R>(cs, link_offset(g, 0, site_from_lex(g, x1 + g.L3 * t)));
            T = cmul(T, cmul(cconj(a), b));
        }
        const long ai = static_cast<long>(s * r_max + (r - 1)) * g.L3 + x0;
        double2 av = asum[ai];
        av.x += T.re;
        av.y += T.im;
        asum[ai] = av;
        for (int d = 0; d < nd; ++d) {
            const int yy = (px + r / 2) % g.L + g.L * ((py + d) % g.L + g.L * pz);
            for (int ch = 0; ch < 8; ++ch) {
                const double o = O[ch * SL3 + s * g.L3 + yy];
                const long bi = ((static_cast<long>(s * r_max + (r - 1)) * nd + d) * 8 + ch) * g.L3 + x0;
                double2 bv = bsum[bi];
                bv.x += T.re * o;
                bv.y += T.im * o;
                bsum[bi] = bv;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename R>
cudaError_t launch_hot_start(const Geo& g, R* theta, void* cs, uint64_t seed, cudaStream_t st)
{
    hot_start_kernel<R><<<blocks_for(4L * g.V), kThreads, 0, st>>>(g, theta, static_cast<cs_t<R>*>(cs), seed);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_refresh_cs(const Geo& g, const R* theta, void* cs, cudaStream_t st)
{
    refresh_cs_kernel<R><<<blocks_for(4L * g.V), kThreads, 0, st>>>(g, theta, static_cast<cs_t<R>*>(cs));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_update_class(const Geo& g, R* theta, void* cs, int mu, int parity, bool metro, uint64_t pass,
                                uint64_t seed, double beta, double width, int slab_t,
                                unsigned long long* accepted, cudaStream_t st)
{
    update_class_kernel<R><<<blocks_for(g.Vh), kThreads, 0, st>>>(g, theta, static_cast<cs_t<R>*>(cs), mu, parity,
                                                                   metro ? 1 : 0, pass, seed, static_cast<R>(beta),
                                                                   static_cast<R>(width), slab_t, accepted);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_to_canonical(const Geo& g, const R* theta, double* canon, cudaStream_t st)
{
    to_canonical_kernel<R><<<blocks_for(4L * g.V), kThreads, 0, st>>>(g, theta, canon);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_from_canonical(const Geo& g, const double* canon, R* theta, void* cs, cudaStream_t st)
{
    from_canonical_kernel<R><<<blocks_for(4L * g.V), kThreads, 0, st>>>(g, canon, theta, static_cast<cs_t<R>*>(cs));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_plaquette(const Geo& g, const void* cs, double* partials, double* out_dev, cudaStream_t st)
{
    const int nb = blocks_for(g.V);
    plaquette_kernel<R><<<nb, kThreads, 0, st>>>(g, static_cast<const cs_t<R>*>(cs), partials);
    sum_partials_kernel<<<1, kThreads, 0, st>>>(partials, nb, 1.0 / (6.0 * static_cast<double>(g.V)), out_dev);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_slab_channels(const Geo& g, const void* cs, int slab_t, double* O, double* osum, cudaStream_t st)
{
    const int S = g.Nt / slab_t;
    slab_channels_kernel<R><<<blocks_for(static_cast<long>(S) * g.L3), kThreads, 0, st>>>(
        g, static_cast<const cs_t<R>*>(cs), slab_t, O, osum);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_measure(const Geo& g, const void* cs, int slab_t, int r_max, int nd, const double* O,
                           double2* asum, double2* bsum, cudaStream_t st)
{
    const int S = g.Nt / slab_t;
    measure_kernel<R><<<blocks_for(static_cast<long>(S) * g.L3), kThreads, 0, st>>>(
        g, static_cast<const cs_t<R>*>(cs), slab_t, r_max, nd, O, asum, bsum);
    return cudaGetLastError();
}

#define UL_INSTANTIATE_KERNELS(R)                                                                                  \
    template cudaError_t launch_hot_start<R>(const Geo&, R*, void*, uint64_t, cudaStream_t);                        \
    template cudaError_t launch_refresh_cs<R>(const Geo&, const R*, void*, cudaStream_t);                           \
    template cudaError_t launch_update_class<R>(const Geo&, R*, void*, int, int, bool, uint64_t, uint64_t, double, \
                                                double, int, unsigned long long*, cudaStream_t);                   \
    template cudaError_t launch_to_canonical<R>(const Geo&, const R*, double*, cudaStream_t);                       \
    template cudaError_t launch_from_canonical<R>(const Geo&, const double*, R*, void*, cudaStream_t);              \
    template cudaError_t launch_plaquette<R>(const Geo&, const void*, double*, double*, cudaStream_t);               \
    template cudaError_t launch_slab_channels<R>(const Geo&, const void*, int, double*, double*, cudaStream_t);      \
    template cudaError_t launch_measure<R>(const Geo&, const void*, int, int, int, const double*, double2*,         \
                                           double2*, cudaStream_t);

} // namespace ul
