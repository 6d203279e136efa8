// ul_kernels.cuh — link-update and measurement kernels, templated on the link precision.
// Included by ul_kernels_f64.cu (R = double, compiled with -fmad=false) and
// ul_kernels_f32.cu (R = float).
//
// Paper: arXiv:1208.0166, Section 2 (Wilson action, plaquette), Section 2.1 (Metropolis
// and overrelaxation), Section 2.2 (multilevel: slabs with frozen spatial links,
// transporters T, insertion operator, multilevel field estimator).
#pragma once
#include <algorithm>
#include <atomic>
#include <cooperative_groups.h>
#include "ul_device.cuh"
#include "ul_batch_types.h"
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
// Link update of one (mu, parity) class, Sections 2 and 2.1.
//
// Staple sum of link (mu, x):
//   A = sum_{nu != mu} [ U_nu(x+mu) U*_mu(x+nu) U*_nu(x) + U*_nu(x+mu-nu) U*_mu(x-nu) U_nu(x-nu) ]
// so that the plaquettes containing U_mu(x) contribute Re(U_mu(x) A); the terms are formed
// and summed in this order (nu ascending, forward before backward).
//   Metropolis:      theta' = wrap(theta + width (2 u1 - 1)),
//                    dS = -beta Re(e^{i theta'} A) - (-beta Re(e^{i theta} A)),
//                    accept iff u2 < exp(-dS);
//   Overrelaxation:  theta' = wrap(-2 arg(A) - theta).
// With a nonzero frozen mask, spatial links on slices t with bit t set stay frozen
// (Section 2.2: the spatial links on the slab boundaries are held fixed).
//
// Index arithmetic: the spatial extent is a compile-time constant LC for the common
// lattice sizes (LC = 0: runtime L), the direction MU is a template parameter, and
// neighbour sites are reached by adding direction strides to the lexicographic index
// with a wrap correction, so no coordinate array is indexed at run time.
// ---------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ R beta_of(const UpdateArgs& a) { return sizeof(R) == 8 ? static_cast<R>(a.beta) : static_cast<R>(a.beta_f); }
template <typename R>
__device__ __forceinline__ R width_of(const UpdateArgs& a) { return sizeof(R) == 8 ? static_cast<R>(a.width) : static_cast<R>(a.width_f); }

template <int LC>
struct Extent {
    int L, Nt;
    __device__ __forceinline__ Extent(const Geo& g) : L(LC ? LC : g.L), Nt(g.Nt) {}
};

// Lexicographic offset of a +1 / -1 step along direction D from coordinate c.
template <int D>
__device__ __forceinline__ int step_up(int c, int L, int Nt)
{
    const int n = D == 0 ? Nt : L;
    const int st = D == 0 ? L * L * L : (D == 1 ? 1 : (D == 2 ? L : L * L));
    return c == n - 1 ? -(n - 1) * st : st;
}
template <int D>
__device__ __forceinline__ int step_down(int c, int L, int Nt)
{
    const int n = D == 0 ? Nt : L;
    const int st = D == 0 ? L * L * L : (D == 1 ? 1 : (D == 2 ? L : L * L));
    return c == 0 ? (n - 1) * st : -st;
}

// Loads of link data.  CG = true reads through L2 only (ld.global.cg): inside a
// persistent kernel other SMs rewrite links between classes and L1 is not coherent.
template <typename T, bool CG>
__device__ __forceinline__ T ld_link(const T* p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

template <typename R, bool CG = false>
__device__ __forceinline__ Cx<R> load_link(const cs_t<R>* __restrict__ cs, int Vh, int dir, int par, int j)
{
#ifdef UL_CHECK
    j = static_cast<int>(UL_IDX(j, 2LL * Vh, kChkNeighbour));
    const cs_t<R> v = ld_link<cs_t<R>, CG>(cs + UL_IDX((dir * 2 + par) * Vh + (j >> 1), 8LL * Vh, kChkStaple));
#else
    const cs_t<R> v = ld_link<cs_t<R>, CG>(cs + (dir * 2 + par) * Vh + (j >> 1));
#endif
    return Cx<R>{v.x, v.y};
}

// One plane's contribution to the staple sum, from its six links:
//   A += U_nu(x+mu) U*_mu(x+nu) U*_nu(x)   (forward, staple_acc_fwd)
//   A += U*_nu(x+mu-nu) U*_mu(x-nu) U_nu(x-nu)   (backward, staple_acc_bwd)
// each term's last product accumulated into A by fused multiply-adds (cmul_acc), the
// forward term before the backward one.  Every update kernel (one class per launch,
// persistent, batched, slab-resident) uses these functions, so a link's new value does not
// depend on the kernel.
template <typename R>
__device__ __forceinline__ void staple_acc_fwd(Cx<R>& A, Cx<R> nu_up_mu, Cx<R> mu_up_nu, Cx<R> nu_here)
{
    cmul_acc(A, cmul(nu_up_mu, cconj(mu_up_nu)), cconj(nu_here));
}
template <typename R>
__device__ __forceinline__ void staple_acc_bwd(Cx<R>& A, Cx<R> nu_diag, Cx<R> mu_dn_nu, Cx<R> nu_dn_nu)
{
    cmul_acc(A, cmul(cconj(nu_diag), cconj(mu_dn_nu)), nu_dn_nu);
}

template <typename R, int MU, int NU, bool CG>
__device__ __forceinline__ void staple_term(Cx<R>& A, const cs_t<R>* __restrict__ cs, int Vh, int p, int i,
                                            const int c[4], int L, int Nt, int up_mu)
{
    const int q = p ^ 1;
    const int up_nu = step_up<NU>(c[NU], L, Nt);
    const int dn_nu = step_down<NU>(c[NU], L, Nt);
    staple_acc_fwd(A, load_link<R, CG>(cs, Vh, NU, q, i + up_mu), load_link<R, CG>(cs, Vh, MU, q, i + up_nu),
                   load_link<R, CG>(cs, Vh, NU, p, i));
    staple_acc_bwd(A, load_link<R, CG>(cs, Vh, NU, p, i + up_mu + dn_nu), load_link<R, CG>(cs, Vh, MU, q, i + dn_nu),
                   load_link<R, CG>(cs, Vh, NU, q, i + dn_nu));
}

// Metropolis proposal and decision for a link with angle th, phase old = (cos th, sin th)
// and staple sum A; the two uniforms come from Philox(counter (link_id, pass, 0, 0), key
// (seed, 1)).  Proposal th' = wrap(fma(width, 2 u1 - 1, th)) with its phase (cn, sn);
// action change dS = beta [(cos th - cos th') Re A - (sin th - sin th') Im A]
// = beta fma(dc, Re A, -(ds Im A)); accept iff u2 < exp(-dS).  metro_propose needs no
// neighbour link, so a kernel may form the proposal before the links it reads are final.
template <typename R>
__device__ __forceinline__ void metro_propose(R th, uint64_t link_id, uint64_t pass, uint64_t seed, R width, R& prop,
                                              R& sn, R& cn, R& u2)
{
    using P = Prec<R>;
    R u1;
    P::metro_uniforms(link_id, pass, seed, &u1, &u2);
    prop = P::wrap(fma_r(width, P::two_u_minus_one(u1), th));
    P::sincos(prop, &sn, &cn);
}

template <typename R>
__device__ __forceinline__ bool metro_accept(cs_t<R> old, Cx<R> A, R beta, R prop, R sn, R cn, R u2, R& nth,
                                             cs_t<R>& ncs)
{
    const R dS = beta * fma_r(old.x - cn, A.re, -((old.y - sn) * A.im));
    if (Prec<R>::less_nonneg(u2, Prec<R>::exp(-dS))) {
        nth = prop;
        ncs = cs_t<R>{cn, sn};
        return true;
    }
    return false;
}

// One Metropolis hit (the phase old() is read after the proposal is formed, which keeps it
// out of registers during the generator).  On acceptance returns true with the new angle
// and phase in nth, ncs.
template <typename R, class OldPhase>
__device__ __forceinline__ bool metropolis_new(R th, OldPhase old_phase, Cx<R> A, uint64_t link_id, uint64_t pass,
                                               uint64_t seed, R width, R beta, R& nth, cs_t<R>& ncs)
{
    R prop, sn, cn, u2;
    metro_propose<R>(th, link_id, pass, seed, width, prop, sn, cn, u2);
    return metro_accept<R>(old_phase(), A, beta, prop, sn, cn, u2, nth, ncs);
}

// Overrelaxation: the reflection th' = wrap(-2 arg(A) - th) with its phase.
template <typename R>
__device__ __forceinline__ void overrelax_new(R th, Cx<R> A, R& nth, cs_t<R>& ncs)
{
    using P = Prec<R>;
    const R alpha = P::atan2(A.im, A.re);
    nth = P::wrap(P::minus_twice(alpha) - th);
    R sn, cn;
    P::sincos(nth, &sn, &cn);
    ncs = cs_t<R>{cn, sn};
}

template <typename R, int LC, int MU, bool CG = false>
__device__ __forceinline__ bool update_link(const Geo& g, R* __restrict__ theta, cs_t<R>* __restrict__ cs, int h,
                                            const UpdateArgs& a)
{
    const Extent<LC> e(g);
    const int L = e.L, Nt = e.Nt, Lh = L / 2, Vh = g.Vh;
    const int p = a.parity;
    const int row = h / Lh;
    const int xh = h - row * Lh;
    const int y = row % L;
    const int zt = row / L;
    const int z = zt % L;
    const int t = zt / L;
    if (MU != 0 && a.slab_t > 0) {
        const bool frozen = a.frozen_mask ? ((a.frozen_mask >> t) & 1ull) != 0 : (t % a.slab_t) == 0;
        if (frozen) return false;
    }
    const int b = (p + y + z + t) & 1; // x = 2 xh + b
    const int x = 2 * xh + b;
    const int i = 2 * h + b;           // lexicographic site index
    const int c[4] = {t, x, y, z};
    const int up_mu = step_up<MU>(c[MU], L, Nt);
    Cx<R> A{R(0), R(0)};
    if (MU != 0) staple_term<R, MU, (MU == 0 ? 1 : 0), CG>(A, cs, Vh, p, i, c, L, Nt, up_mu);
    if (MU != 1) staple_term<R, MU, (MU == 1 ? 2 : 1), CG>(A, cs, Vh, p, i, c, L, Nt, up_mu);
    if (MU != 2) staple_term<R, MU, (MU == 2 ? 3 : 2), CG>(A, cs, Vh, p, i, c, L, Nt, up_mu);
    if (MU != 3) staple_term<R, MU, (MU == 3 ? 0 : 3), CG>(A, cs, Vh, p, i, c, L, Nt, up_mu);
    const int off = static_cast<int>(UL_IDX((MU * 2 + p) * Vh + h, 8LL * Vh, kChkOwnLink));
    const R th = ld_link<R, CG>(theta + off);
    R nth;
    cs_t<R> ncs;
    if (a.metro) {
        uint64_t pass = a.pass;
        if (a.pass_base) pass += *a.pass_base;
        const uint64_t link_id = static_cast<uint64_t>(MU) * g.V + static_cast<uint64_t>(i);
        if (!metropolis_new<R>(th, [&] { return ld_link<cs_t<R>, CG>(cs + off); }, A, link_id, pass, a.seed,
                               width_of<R>(a), beta_of<R>(a), nth, ncs))
            return false;
        theta[off] = nth;
        cs[off] = ncs;
        return true;
    }
    overrelax_new<R>(th, A, nth, ncs);
    theta[off] = nth;
    cs[off] = ncs;
    return false;
}

// The Metropolis uniforms (u1, u2) of links link0 .. link0 + n - 1 in pass `pass`, as the update
// kernels draw them (for tests of the generator against its reference).
template <typename R>
__global__ void __launch_bounds__(kThreads) rng_uniforms_kernel(uint64_t seed, uint64_t pass, uint64_t link0, int n,
                                                                 double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R u1, u2;
    Prec<R>::metro_uniforms(link0 + static_cast<uint64_t>(i), pass, seed, &u1, &u2);
    out[2 * i] = static_cast<double>(u1);
    out[2 * i + 1] = static_cast<double>(u2);
}

template <typename R>
cudaError_t launch_rng_uniforms(uint64_t seed, uint64_t pass, uint64_t link0, int n, double* out, cudaStream_t st)
{
    rng_uniforms_kernel<R><<<blocks_for(n), kThreads, 0, st>>>(seed, pass, link0, n, out);
    return cudaGetLastError();
}

// Threads per block of the one-class-per-launch update kernel: at most kUpdateThreads (eight
// warps) for the FP64 kernel, at most kWideThreads (eighteen warps) for the FP32 one;
// update_block_threads / wide_block_threads pick the size per launch.
constexpr int kUpdateThreads = 256;
constexpr int kWideThreads = 576;

inline int sm_count_cached()
{
    static std::atomic<int> sms_of[16]; // SM count per device, queried once (any thread)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) dev = 0;
    int sms = sms_of[dev].load(std::memory_order_relaxed);
    if (!sms) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
        sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

// Warps on the busiest SM when `warps` warps in blocks of k warps spread evenly in one wave.
inline long busiest_sm_warps(long warps, int k, int sms)
{
    const long blocks = (warps + k - 1) / k;
    return (blocks + sms - 1) / sms * k;
}

// Block size (in threads, 2 to 8 warps) for a class launch of `work` links: the size whose
// blocks, spread evenly over the SMs in one wave, put the fewest warps on the busiest SM
// (each SM's share is bound by its FP64 pipe or its issue rate), the larger block on a
// tie.  24^4: a full class (5,184 warps) 5 warps per block (35 warps on the busiest SM,
// against 36 with 4), a masked spatial class (2,592 warps) 6 warps (18 against 20).
inline int update_block_threads(long work)
{
    const int sms = sm_count_cached();
    const long warps = (work + 31) / 32;
    int best_k = 4;
    long best = -1;
    for (int k = 2; k <= kUpdateThreads / 32; ++k) {
        const long busiest = busiest_sm_warps(warps, k, sms);
        if (best < 0 || busiest < best || (busiest == best && k > best_k)) {
            best = busiest;
            best_k = k;
        }
    }
    return best_k * 32;
}

// Block size (2 to 18 warps) of the FP32 class launch: among the sizes whose busiest SM holds
// at most 3 % more warps than the best balance, the one with the fewest blocks.  A launch
// pays for every block it dispatches (a chain of empty kernels of ~1,000 blocks measured
// 1.4 us per kernel, of 152 blocks 0.6 us), which matters for the FP32 class kernel of a
// few microseconds.  24^4: a full class 18 warps (288 blocks, 36 warps on the busiest SM,
// against 1,037 blocks and 35 warps with 5), a masked spatial class 18 warps (144 blocks).
inline int wide_block_threads(long work)
{
    const int sms = sm_count_cached();
    const long warps = (work + 31) / 32;
    long best = -1;
    for (int k = 2; k <= kWideThreads / 32; ++k) {
        const long b = busiest_sm_warps(warps, k, sms);
        if (best < 0 || b < best) best = b;
    }
    int pick = 2;
    for (int k = 2; k <= kWideThreads / 32; ++k)
        if (busiest_sm_warps(warps, k, sms) * 100 <= best * 103) pick = k; // largest k = fewest blocks
    return pick * 32;
}

// With compact_tau > 1 and mu != 0 the grid covers only the unfrozen time slices (those
// with t % compact_tau != 0): thread q maps to the q-th link of those slices.
template <typename R, int LC>
__device__ __forceinline__ void update_class_body(const Geo& g, R* __restrict__ theta, cs_t<R>* __restrict__ cs,
                                                  int mu, const UpdateArgs& a, int compact_tau)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = h < g.Vh;
    if (compact_tau > 1 && mu != 0) {
        const int L = LC ? LC : g.L;
        const int hs = (L * L * L) / 2; // links of one parity on one time slice
        const int per = compact_tau - 1; // unfrozen slices per slab
        const int q = h;
        valid = q < (g.Nt / compact_tau) * per * hs;
        const int slice = q / hs;
        const int t = (slice / per) * compact_tau + 1 + slice % per;
        h = t * hs + (q - slice * hs);
    }
    // Programmatic dependent launch: once every block of this grid has started, the next
    // class kernel of the stream may be scheduled; no link is read before the previous
    // kernel of the stream has completed and its writes are visible.  (Both instructions
    // are no-ops for a kernel launched without the programmatic-serialization attribute.)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    bool acc = false;
    if (valid) {
        switch (mu) {
        case 0: acc = update_link<R, LC, 0>(g, theta, cs, h, a); break;
        case 1: acc = update_link<R, LC, 1>(g, theta, cs, h, a); break;
        case 2: acc = update_link<R, LC, 2>(g, theta, cs, h, a); break;
        default: acc = update_link<R, LC, 3>(g, theta, cs, h, a); break;
        }
    }
    if (a.metro) {
        const unsigned mask = __ballot_sync(0xffffffffu, acc);
        if ((threadIdx.x & 31) == 0 && mask) atomicAdd(a.accepted, static_cast<unsigned long long>(__popc(mask)));
    }
}

template <typename R, int LC>
__global__ void __launch_bounds__(kUpdateThreads, 5)
    update_class_kernel(Geo g, R* __restrict__ theta, cs_t<R>* __restrict__ cs, int mu, UpdateArgs a, int compact_tau)
{
    update_class_body<R, LC>(g, theta, cs, mu, a, compact_tau);
}

// The same update in blocks of up to 18 warps, two blocks per SM (FP32 class launches).
template <typename R, int LC>
__global__ void __launch_bounds__(kWideThreads, 2)
    update_class_wide_kernel(Geo g, R* __restrict__ theta, cs_t<R>* __restrict__ cs, int mu, UpdateArgs a,
                             int compact_tau)
{
    update_class_body<R, LC>(g, theta, cs, mu, a, compact_tau);
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

// ---------------------------------------------------------------------------
// Per-sample storage of the deferred insertion contraction (Section 2.2: the insertion
// term of a slab is the sample mean of T O).  FP32 links: T as a complex float, the 8
// channel sums of a site as 8 floats.  FP64 links: every value as a double-single pair
// (hi, lo) of floats in the value's own 8 bytes, so that the contraction runs in
// double-single arithmetic on the FP32 pipes instead of on the FP64 pipe:
//   T: one float4 {re hi, im hi, re lo, im lo} in the 16 bytes of the complex double;
//   O: the 64 bytes per site of an x-row of L sites hold four parts {hi ch 0-3, hi ch 4-7,
//      lo ch 0-3, lo ch 4-7}, part-major: part q of site x at float4 (row start) + q L + x,
//      so that one part of consecutive sites is contiguous.
// ---------------------------------------------------------------------------

// x = hi + lo: hi the leading 24 significant bits of x (truncated), lo the remaining 29
// bits rounded to a float, so |lo| < 2^-23 |hi| and |x - hi - lo| <= max(2^-48 |x|, 2^-126):
// integer operations only; a part below the normal float range (2^-126) is stored as 0,
// |x| >= 2^128 as infinity (the stored samples are bounded by the slab thickness).
__device__ __forceinline__ float2 ds_split(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int hw = static_cast<unsigned int>(b >> 32), lw = static_cast<unsigned int>(b);
    const unsigned int sign = hw & 0x80000000u;
    const int e = static_cast<int>((hw >> 20) & 0x7ffu); // biased FP64 exponent
    const int ef = e - 1023 + 127;                       // biased FP32 exponent of hi
    if (ef <= 0) return make_float2(0.f, 0.f);
    if (ef >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
    const float hi = __uint_as_float(sign | (static_cast<unsigned int>(ef) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const unsigned int rem = lw & 0x1fffffffu; // the remaining bits, in units of 2^(e - 1075)
    float lo = 0.f;
    if (rem != 0) {
        const unsigned int fr = __float_as_uint(__uint2float_rn(rem));
        const int ex = static_cast<int>(fr >> 23) + (e - 1075); // biased exponent of rem 2^(e - 1075)
        if (ex > 0) lo = __uint_as_float(sign | (static_cast<unsigned int>(ex) << 23) | (fr & 0x7fffffu));
    }
    return make_float2(hi, lo);
}

template <typename R>
struct SampleStore;

template <>
struct SampleStore<float> {
    static __device__ __forceinline__ void put_T(Cx<float>* tk, long i, Cx<float> T) { tk[i] = T; }
    // site: index of the site in the buffer (slot S L3 + s L3 + x0); x: its x coordinate
    static __device__ __forceinline__ void put_O(float* ok, long site, int /*x*/, int /*L*/, const float v[8])
    {
        float4* o = reinterpret_cast<float4*>(ok + site * 8);
        o[0] = make_float4(v[0], v[1], v[2], v[3]);
        o[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    static __device__ __forceinline__ Cx<float> get_T(const Cx<float>* tk, long i) { return tk[i]; }
    static __device__ __forceinline__ void get_O(const float* ok, long site, int /*x*/, int /*L*/, float v[8])
    {
        const float4 a = reinterpret_cast<const float4*>(ok + site * 8)[0];
        const float4 b = reinterpret_cast<const float4*>(ok + site * 8)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};

template <>
struct SampleStore<double> {
    static __device__ __forceinline__ void put_T(Cx<double>* tk, long i, Cx<double> T)
    {
        const float2 re = ds_split(T.re), im = ds_split(T.im);
        reinterpret_cast<float4*>(tk)[i] = make_float4(re.x, im.x, re.y, im.y);
    }
    static __device__ __forceinline__ void put_O(double* ok, long site, int x, int L, const double v[8])
    {
        float2 d[8];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) d[ch] = ds_split(v[ch]);
        float4* o = reinterpret_cast<float4*>(ok) + (site - x) * 4 + x;
        o[0] = make_float4(d[0].x, d[1].x, d[2].x, d[3].x);
        o[L] = make_float4(d[4].x, d[5].x, d[6].x, d[7].x);
        o[2 * L] = make_float4(d[0].y, d[1].y, d[2].y, d[3].y);
        o[3 * L] = make_float4(d[4].y, d[5].y, d[6].y, d[7].y);
    }
    // the stored pairs as doubles (hi + lo is exact in FP64)
    static __device__ __forceinline__ Cx<double> get_T(const Cx<double>* tk, long i)
    {
        const float4 v = reinterpret_cast<const float4*>(tk)[i];
        return Cx<double>{static_cast<double>(v.x) + static_cast<double>(v.z),
                          static_cast<double>(v.y) + static_cast<double>(v.w)};
    }
    static __device__ __forceinline__ void get_O(const double* ok, long site, int x, int L, double v[8])
    {
        const float4* o = reinterpret_cast<const float4*>(ok) + (site - x) * 4 + x;
        const float4 h0 = o[0], h1 = o[L], l0 = o[2 * L], l1 = o[3 * L];
        v[0] = static_cast<double>(h0.x) + static_cast<double>(l0.x);
        v[1] = static_cast<double>(h0.y) + static_cast<double>(l0.y);
        v[2] = static_cast<double>(h0.z) + static_cast<double>(l0.z);
        v[3] = static_cast<double>(h0.w) + static_cast<double>(l0.w);
        v[4] = static_cast<double>(h1.x) + static_cast<double>(l1.x);
        v[5] = static_cast<double>(h1.y) + static_cast<double>(l1.y);
        v[6] = static_cast<double>(h1.z) + static_cast<double>(l1.z);
        v[7] = static_cast<double>(h1.w) + static_cast<double>(l1.w);
    }
};

// One measurement after sub-sample k, thread per (s, x0).  With the slab line
// W(s, x) = prod_{t in slab s} U_0(x, t) (partial Polyakov line),
//   T(s, x0, r) = prod_{t in slab} U*_0(x0,t) U_0(x0 + r xhat, t) = W*(s, x0) W(s, x0 + r xhat),
//   asum[(s*R + r-1)*L3 + x0] += T            (FP64 slab accumulator, r = 1..r_max)
// and, with fields, the slab sums of the 8 plaquette channels at x0,
//   O(s, x0, ch) = sum_{t in slab s} channel_ch(x0, t),   osum[ch*SL3 + s*L3 + x0] += O,
// with T and O stored for the deferred insertion contraction:
//   tk[((slot*S + s)*R + r-1)*L3 + x0] = T,   ok at site (slot*S + s)*L3 + x0 = O
// (SampleStore: plain values for FP32 links, double-single pairs for FP64 links).
// The per-sample products are formed in the link precision R (FP64 or FP32); every
// accumulator is FP64.
template <typename R, bool CG = false>
__device__ __forceinline__ Cx<R> link_at(const cs_t<R>* __restrict__ cs, int off)
{
    const cs_t<R> v = ld_link<cs_t<R>, CG>(cs + off);
    return Cx<R>{v.x, v.y};
}

template <typename R, bool CG = false>
__device__ __forceinline__ Cx<R> slab_line(const Geo& g, const cs_t<R>* __restrict__ cs, int x, int t0, int slab_t)
{
    Cx<R> w = link_at<R, CG>(cs, link_offset(g, 0, site_from_lex(g, x + g.L3 * t0)));
    for (int t = t0 + 1; t < t0 + slab_t; ++t)
        w = cmul_rn(w, link_at<R, CG>(cs, link_offset(g, 0, site_from_lex(g, x + g.L3 * t))));
    return w;
}

// Product over the slab's slices of the multihit temporal links ubar[x + L3 t].
template <typename R, bool CG = false>
__device__ __forceinline__ Cx<R> slab_line_mh(const Geo& g, const Cx<R>* __restrict__ ubar, int x, int t0, int slab_t)
{
    const cs_t<R>* u = reinterpret_cast<const cs_t<R>*>(ubar);
    cs_t<R> v = ld_link<cs_t<R>, CG>(u + x + g.L3 * t0);
    Cx<R> w{v.x, v.y};
    for (int t = t0 + 1; t < t0 + slab_t; ++t) {
        v = ld_link<cs_t<R>, CG>(u + x + g.L3 * t);
        w = cmul_rn(w, Cx<R>{v.x, v.y});
    }
    return w;
}

// ubar (may be null): multihit temporal links by lexicographic site; when set, the
// correlator at r >= 2 uses them (the insertion samples keep the links themselves).
// wrow (may be null): the slab lines W(s, x) of the x-row of site k, indexed by x (formed
// once per row by the caller); when null each line is formed here.  Same products either way.
template <typename R, bool CG = false>
__device__ __forceinline__ void measure_store_site(const Geo& g, const cs_t<R>* __restrict__ cs, int slab_t,
                                                   int r_max, int fields, int slot, double2* __restrict__ asum,
                                                   Cx<R>* __restrict__ tk, R* __restrict__ ok,
                                                   double* __restrict__ osum, int k,
                                                   const Cx<R>* __restrict__ ubar = nullptr,
                                                   const Cx<R>* wrow = nullptr)
{
    const int S = g.Nt / slab_t;
    const int s = k / g.L3;
    const int x0 = k - s * g.L3;
    const int px = x0 % g.L, pyz = x0 - px;
    const int t0 = s * slab_t;
    const Cx<R> w0 = cconj(wrow ? wrow[px] : slab_line<R, CG>(g, cs, x0, t0, slab_t));
    const Cx<R> w0m = ubar ? cconj(slab_line_mh<R, CG>(g, ubar, x0, t0, slab_t)) : w0;
    for (int r = 1; r <= r_max; ++r) {
        const int x1 = (px + r) % g.L + pyz;
        const Cx<R> T = cmul_rn(w0, wrow ? wrow[(px + r) % g.L] : slab_line<R, CG>(g, cs, x1, t0, slab_t));
        const Cx<R> Tc = (ubar && r >= 2) ? cmul_rn(w0m, slab_line_mh<R, CG>(g, ubar, x1, t0, slab_t)) : T;
        const long ai = UL_IDX(static_cast<long>(s * r_max + (r - 1)) * g.L3 + x0,
                               static_cast<long long>(S) * r_max * g.L3, kChkAsum);
        double2 av = ld_link<double2, CG>(asum + ai);
        av.x += static_cast<double>(Tc.re);
        av.y += static_cast<double>(Tc.im);
        asum[ai] = av;
#ifdef UL_CHECK
        if (fields && (slot < 0 || x1 < 0 || x1 >= g.L3)) (void)UL_IDX(-1, 0, kChkSample);
#endif
        if (fields) SampleStore<R>::put_T(tk, (static_cast<long>(slot * S + s) * r_max + (r - 1)) * g.L3 + x0, T);
    }
    if (!fields) return;
    R acc[8];
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) acc[ch] = R(0);
    for (int t = t0; t < t0 + slab_t; ++t) {
        const Site x = site_from_lex(g, x0 + g.L3 * t);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int mu = kPlaneMu[c], nu = kPlaneNu[c];
            const Site xpm = site_step(g, x, mu, +1);
            const Site xpn = site_step(g, x, nu, +1);
            const Cx<R> P = cmul_rn(cmul_rn(cmul_rn(link_at<R, CG>(cs, link_offset(g, mu, x)),
                                                    link_at<R, CG>(cs, link_offset(g, nu, xpm))),
                                            cconj(link_at<R, CG>(cs, link_offset(g, mu, xpn)))),
                                    cconj(link_at<R, CG>(cs, link_offset(g, nu, x))));
            acc[2 * c] += P.im;
            acc[2 * c + 1] += P.re;
        }
    }
    const int SL3 = S * g.L3;
    SampleStore<R>::put_O(ok, static_cast<long>(slot) * SL3 + k, px, g.L, acc);
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
#ifdef UL_CHECK
        const long oi = UL_IDX(static_cast<long>(ch) * SL3 + k, 8LL * SL3, kChkOsum);
        osum[oi] = ld_link<double, CG>(osum + oi) + static_cast<double>(acc[ch]);
#else
        osum[ch * SL3 + k] = ld_link<double, CG>(osum + ch * SL3 + k) + static_cast<double>(acc[ch]);
#endif
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    measure_store_kernel(Geo g, const cs_t<R>* __restrict__ cs, int slab_t, int r_max, int fields, int slot,
                         double2* __restrict__ asum, Cx<R>* __restrict__ tk, R* __restrict__ ok,
                         double* __restrict__ osum, const Cx<R>* __restrict__ ubar)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x; // s*L3 + x0
    if (k >= (g.Nt / slab_t) * g.L3) return;
    measure_store_site<R>(g, cs, slab_t, r_max, fields, slot, asum, tk, ok, osum, k, ubar);
}

// The same with blocks of whole x-rows (blockDim a multiple of L): each thread forms the
// slab line of its own site into shared memory, and the transporters T(x0, r) take the
// lines of the row from there (each line formed once instead of r_max + 1 times).
template <typename R>
__global__ void __launch_bounds__(kThreads)
    measure_store_rows_kernel(Geo g, const cs_t<R>* __restrict__ cs, int slab_t, int r_max, int fields, int slot,
                              double2* __restrict__ asum, Cx<R>* __restrict__ tk, R* __restrict__ ok,
                              double* __restrict__ osum)
{
    __shared__ Cx<R> w[kThreads];
    const int tid = static_cast<int>(threadIdx.x);
    const int k = blockIdx.x * blockDim.x + tid; // s*L3 + x0
    const bool valid = k < (g.Nt / slab_t) * g.L3;
    if (valid) {
        const int s = k / g.L3;
        w[tid] = slab_line<R>(g, cs, k - s * g.L3, s * slab_t, slab_t);
    }
    __syncthreads();
    if (!valid) return;
    measure_store_site<R>(g, cs, slab_t, r_max, fields, slot, asum, tk, ok, osum, k, nullptr, w + (tid - k % g.L));
}

// ---------------------------------------------------------------------------
// Analytic multihit (Section 2.2): the temporal link at lexicographic site i replaced by
// its mean over its own Boltzmann weight exp(beta Re(U A)) with the staple A fixed,
//   ubar = (I1(beta |A|) / I0(beta |A|)) A* / |A|   (0 when A = 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double bessel_ratio_i1_i0(double x)
{
    if (x <= 0.0) return 0.0;
    if (x > 600.0) return 1.0 - 1.0 / (2.0 * x) - 1.0 / (8.0 * x * x) - 1.0 / (8.0 * x * x * x);
    return cyl_bessel_i1(x) / cyl_bessel_i0(x);
}

template <typename R, int LC, bool CG = false>
__device__ __forceinline__ void multihit_site(const Geo& g, const cs_t<R>* __restrict__ cs, double beta,
                                              Cx<R>* __restrict__ ubar, int i)
{
    const Extent<LC> e(g);
    const int L = e.L, Nt = e.Nt;
    const int x = i % L;
    const int rest = i / L;
    const int y = rest % L;
    const int z = (rest / L) % L;
    const int t = rest / (L * L);
    const int c[4] = {t, x, y, z};
    const int p = (x + y + z + t) & 1;
    const int up_mu = step_up<0>(t, L, Nt);
    Cx<R> A{R(0), R(0)};
    staple_term<R, 0, 1, CG>(A, cs, g.Vh, p, i, c, L, Nt, up_mu);
    staple_term<R, 0, 2, CG>(A, cs, g.Vh, p, i, c, L, Nt, up_mu);
    staple_term<R, 0, 3, CG>(A, cs, g.Vh, p, i, c, L, Nt, up_mu);
    const double are = static_cast<double>(A.re), aim = static_cast<double>(A.im);
    const double a = sqrt(are * are + aim * aim);
    const double f = a > 0.0 ? bessel_ratio_i1_i0(beta * a) / a : 0.0;
    ubar[i] = Cx<R>{static_cast<R>(f * are), static_cast<R>(-f * aim)};
}

template <typename R, int LC>
__global__ void __launch_bounds__(kThreads) multihit_kernel(Geo g, const cs_t<R>* __restrict__ cs, double beta,
                                                            Cx<R>* __restrict__ ubar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.V) multihit_site<R, LC>(g, cs, beta, ubar, i);
}

// Accumulator of a complex x real product sum over the samples of one chunk.
// FP64: fused multiply-add.  FP32: Kahan-compensated sums (error independent of the
// number of terms), folded into the FP64 slab accumulator once per chunk.
template <typename R>
struct InsertionAcc;

template <>
struct InsertionAcc<double> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(Cx<double> T, double o)
    {
        re = fma(T.re, o, re);
        im = fma(T.im, o, im);
    }
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ double total_re() const { return re; }
    __device__ __forceinline__ double total_im() const { return im; }
};

// FP32: the products of a block of samples are summed by fused multiply-adds into a block
// partial; fold() adds the partial to a compensated (Kahan) sum, so the rounding error grows
// with the block length (kInsertionBlock) and not with the number of samples.
constexpr int kInsertionBlock = 8;

// The real and imaginary parts are the two lanes of paired FP32 instructions (FFMA2 / FADD2:
// each lane rounded as the scalar operation).
template <>
struct InsertionAcc<float> {
    float2 sum = make_float2(0.f, 0.f), comp = make_float2(0.f, 0.f); // Kahan sums of block partials
    float2 blk = make_float2(0.f, 0.f);                               // partial sums of the current block
    __device__ __forceinline__ void add(Cx<float> T, float o)
    {
        blk = __ffma2_rn(make_float2(T.re, T.im), make_float2(o, o), blk);
    }
    __device__ __forceinline__ void fold()
    {
        const float2 y = __fadd2_rn(blk, make_float2(-comp.x, -comp.y));
        const float2 t = __fadd2_rn(sum, y);
        const float2 d = __fadd2_rn(t, make_float2(-sum.x, -sum.y));
        comp = __fadd2_rn(d, make_float2(-y.x, -y.y));
        sum = t;
        blk = make_float2(0.f, 0.f);
    }
    // the compensated sum rounded once to FP32, then widened (one FP64-pipe conversion)
    __device__ __forceinline__ double total_re() const { return static_cast<double>(__fsub_rn(sum.x, comp.x)); }
    __device__ __forceinline__ double total_im() const { return static_cast<double>(__fsub_rn(sum.y, comp.y)); }
};

template <typename R>
struct Vec8;
template <>
struct Vec8<float> {
    static __device__ __forceinline__ void load(const float* p, float v[8])
    {
        const float4 a = reinterpret_cast<const float4*>(p)[0];
        const float4 b = reinterpret_cast<const float4*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};
template <>
struct Vec8<double> {
    static __device__ __forceinline__ void load(const double* p, double v[8])
    {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 a = reinterpret_cast<const double2*>(p)[q];
            v[2 * q] = a.x;
            v[2 * q + 1] = a.y;
        }
    }
};

// Deferred insertion contraction over the `count` samples stored in tk/ok:
//   bsum[(((s*R + r-1)*nd + d)*8 + ch)*L3 + x0] += sum_k T_k(s,x0,r) O_k(s, x0 + floor(r/2) xhat + d yhat, ch)
// (with `first`, the level's first chunk, bsum is not read: the sums start from 0)
// thread per output (s, r, d, x0), one block per kThreads consecutive x0 of one (s, r, d);
// the blocks of a tile of x0 are neighbours in the grid for all (r, d) (d fastest, then r),
// so the transporters and channel rows they share are read from DRAM about once.  Each
// output is summed over k in order by one thread.  The register bound keeps three
// 256-thread blocks per SM (the FP32 form holds 48 accumulator registers).
constexpr int kContractMinBlocks = 3;

template <typename R>
__global__ void __launch_bounds__(kThreads, kContractMinBlocks)
    insertion_contract_kernel(Geo g, int S, int r_max, int nd, int count, const Cx<R>* __restrict__ tk,
                              const R* __restrict__ ok, double2* __restrict__ bsum, bool first)
{
    const int tiles = (g.L3 + kThreads - 1) / kThreads;
    int b = static_cast<int>(blockIdx.x);
    const int d = b % nd;
    b /= nd;
    const int r = b % r_max + 1;
    b /= r_max;
    const int tile = b % tiles;
    const int s = b / tiles;
    const int x0 = tile * kThreads + static_cast<int>(threadIdx.x);
    if (x0 >= g.L3) return;
    const int px = x0 % g.L, py = (x0 / g.L) % g.L, pz = x0 / (g.L * g.L);
    const int yx = (px + r / 2) % g.L;
    const int y = yx + g.L * ((py + d) % g.L + g.L * pz);
    const long SL3 = static_cast<long>(S) * g.L3;
    InsertionAcc<R> acc[8];
    for (int k = 0; k < count; ++k) {
        const Cx<R> T = SampleStore<R>::get_T(tk, (static_cast<long>(k * S + s) * r_max + (r - 1)) * g.L3 + x0);
        R o[8];
        SampleStore<R>::get_O(ok, k * SL3 + static_cast<long>(s) * g.L3 + y, yx, g.L, o);
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) acc[ch].add(T, o[ch]);
        if (k % kInsertionBlock == kInsertionBlock - 1)
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) acc[ch].fold();
    }
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) acc[ch].fold();
    const long base = (((static_cast<long>(s) * r_max + (r - 1)) * nd + d) * 8) * g.L3 + x0;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        double2 b = first ? make_double2(0.0, 0.0) : bsum[base + ch * g.L3];
        b.x += acc[ch].total_re();
        b.y += acc[ch].total_im();
        bsum[base + ch * g.L3] = b;
    }
}

// ---------------------------------------------------------------------------
// Persistent sweep kernel: one cooperative launch runs n_units units, each n_metro
// Metropolis + n_or overrelaxation passes (8 classes each) and, with `measure`, one
// measurement; classes are separated by a grid-wide barrier.  Every link is updated by
// the same device function as in the one-class-per-launch kernel (loads through L2),
// so the trajectory is the same bit for bit.
//
// The barrier is one arrival counter in device memory, zeroed before the launch.  Every
// wait is bounded: after spin_limit polls a waiting block writes a nonzero status word
// and the kernel returns; the host reports UL_ETIMEOUT at its next synchronising call.
// ---------------------------------------------------------------------------

// Barrier number `epoch` (1, 2, ...) of a launch completes when the arrival counter, which
// is zero at launch and only grows, reaches epoch * expected.
__device__ __forceinline__ bool grid_barrier(const PersistArgs& a, unsigned int& epoch)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        epoch += 1;
        const unsigned int target = epoch * a.expected;
        __threadfence();
        atomicAdd(a.bar, 1u);
        volatile unsigned int* vcount = a.bar;
        unsigned long long polls = 0;
        while (*vcount < target) {
            if (++polls > a.spin_limit) {
                atomicExch(a.status, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        if (ok && *reinterpret_cast<volatile int*>(a.status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename R, int LC>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 5 : 4) persistent_kernel(Geo g, R* __restrict__ theta, cs_t<R>* __restrict__ cs,
                                                         PersistArgs a)
{
    if (*reinterpret_cast<volatile int*>(a.status) != 0) return;
    const int stride = static_cast<int>(gridDim.x * blockDim.x);
    const int tid = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    unsigned int epoch = 0;
    UpdateArgs u = a.u;
    for (int unit = 0; unit < a.n_units; ++unit) {
        for (int k = 0; k < a.n_metro + a.n_or; ++k) {
            u.metro = k < a.n_metro ? 1 : 0;
            for (int mu = 0; mu < 4; ++mu)
                for (int par = 0; par < 2; ++par) {
                    u.parity = par;
                    int accepted = 0;
                    for (int h = tid; h < g.Vh; h += stride) {
                        bool acc;
                        switch (mu) {
                        case 0: acc = update_link<R, LC, 0, true>(g, theta, cs, h, u); break;
                        case 1: acc = update_link<R, LC, 1, true>(g, theta, cs, h, u); break;
                        case 2: acc = update_link<R, LC, 2, true>(g, theta, cs, h, u); break;
                        default: acc = update_link<R, LC, 3, true>(g, theta, cs, h, u); break;
                        }
                        accepted += acc ? 1 : 0;
                    }
                    if (u.metro) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) accepted += __shfl_xor_sync(0xffffffffu, accepted, o);
                        if ((threadIdx.x & 31) == 0 && accepted)
                            atomicAdd(u.accepted, static_cast<unsigned long long>(accepted));
                    }
                    if (!grid_barrier(a, epoch)) return;
                }
            if (u.metro) u.pass += 1;
        }
        if (a.measure) {
            Cx<R>* ubar = static_cast<Cx<R>*>(a.ubar);
            if (ubar) {
                for (int q = tid; q < g.V; q += stride) multihit_site<R, LC, true>(g, cs, u.beta, ubar, q);
                if (!grid_barrier(a, epoch)) return;
            }
            const int SL3 = (g.Nt / u.slab_t) * g.L3;
            for (int q = tid; q < SL3; q += stride)
                measure_store_site<R, true>(g, cs, u.slab_t, a.r_max, a.fields, a.slot0 + unit, a.asum,
                                            static_cast<Cx<R>*>(a.tk), static_cast<R*>(a.ok), a.osum, q, ubar);
            if (!grid_barrier(a, epoch)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// Batch kernels: one launch updates class (mu, parity) of every lattice of a group of one
// shape (couplings, seeds and schedule positions may differ).  The per-lattice parameters
// travel in the kernel's parameter block; the grid's y index selects the lattice.  Each
// link is updated by the same device function as in the single-lattice kernel, so a
// lattice's trajectory does not depend on its batch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Geo geo_of(int L, int Nt, int V, int Vh, int L3)
{
    Geo g;
    g.L = L;
    g.Nt = Nt;
    g.Lh = L / 2;
    g.L3 = L3;
    g.V = V;
    g.Vh = Vh;
    return g;
}

// Lockstep class update of a group of lattices of one shape: the grid's y index selects the
// lattice, its x extent covers the lattice's links of the class (threads beyond a lattice's
// work do nothing).  Each link is updated by update_class_body with the lattice's own
// arguments, so its new value is the single-lattice kernel's.
template <typename R, int LC>
__device__ __forceinline__ void group_update(const BatchUpdateTable& t, int mu, int parity)
{
    const BatchUpdateJob& J = t.job[blockIdx.y];
    const Geo g = geo_of(J.L, J.Nt, J.V, J.Vh, J.L3);
    UpdateArgs a;
    a.parity = parity;
    a.metro = J.metro;
    a.slab_t = J.slab_t;
    a.frozen_mask = J.frozen_mask;
    a.pass = J.pass;
    a.pass_base = nullptr;
    a.seed = J.seed;
    a.beta = J.beta;
    a.width = J.width;
    a.beta_f = static_cast<float>(J.beta);
    a.width_f = static_cast<float>(J.width);
    a.accepted = J.accepted;
    const int compact = (J.slab_t > 1 && mu != 0) ? J.slab_t : 0;
    update_class_body<R, LC>(g, static_cast<R*>(J.theta), static_cast<cs_t<R>*>(J.cs), mu, a, compact);
}

template <typename R, int LC>
__global__ void __launch_bounds__(kUpdateThreads, 5)
    group_update_kernel(const __grid_constant__ BatchUpdateTable t, int mu, int parity)
{
    group_update<R, LC>(t, mu, parity);
}

template <typename R, int LC>
__global__ void __launch_bounds__(kWideThreads, 2)
    group_update_wide_kernel(const __grid_constant__ BatchUpdateTable t, int mu, int parity)
{
    group_update<R, LC>(t, mu, parity);
}

// Measurement of a group of lattices (y index: lattice), as measure_store_kernel.
template <typename R>
__global__ void __launch_bounds__(kThreads) group_measure_kernel(const __grid_constant__ BatchMeasureTable t)
{
    const BatchMeasureJob& J = t.job[blockIdx.y];
    const int k = static_cast<int>(blockIdx.x) * kThreads + static_cast<int>(threadIdx.x);
    const Geo g = geo_of(J.L, J.Nt, J.V, J.Vh, J.L3);
    if (k >= (J.Nt / J.slab_t) * J.L3) return;
    measure_store_site<R>(g, static_cast<const cs_t<R>*>(J.cs), J.slab_t, J.r_max, 0, 0, J.asum, nullptr, nullptr,
                          nullptr, k);
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
                                const unsigned long long* pass_base, uint64_t seed, double beta, double width,
                                int slab_t, unsigned long long* accepted, cudaStream_t st, int* launched, bool pdl)
{
    UpdateArgs a;
    a.parity = parity;
    a.metro = metro ? 1 : 0;
    a.slab_t = slab_t;
    a.frozen_mask = 0;
    if (slab_t > 0 && g.Nt <= 64)
        for (int t = 0; t < g.Nt; t += slab_t) a.frozen_mask |= 1ull << t;
    a.pass = pass;
    a.pass_base = pass_base;
    a.seed = seed;
    a.beta = beta;
    a.width = width;
    a.beta_f = static_cast<float>(beta);
    a.width_f = static_cast<float>(width);
    a.accepted = accepted;
    cs_t<R>* c = static_cast<cs_t<R>*>(cs);
    const int compact = (slab_t > 1 && mu != 0) ? slab_t : 0;
    const long work = compact ? static_cast<long>(g.Nt / slab_t) * (slab_t - 1) * (g.L3 / 2) : g.Vh;
    *launched = 0;
    if (work == 0) return cudaSuccess; // slab_t == 1: every spatial link is frozen
    *launched = 1;
    cudaLaunchConfig_t cfg{};
    const bool wide = sizeof(R) == 4;
    const int threads = wide ? wide_block_threads(work) : update_block_threads(work);
    cfg.gridDim = dim3(static_cast<unsigned>((work + threads - 1) / threads));
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (wide) {
        switch (g.L) {
        case 8: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 8>, g, theta, c, mu, a, compact);
        case 12: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 12>, g, theta, c, mu, a, compact);
        case 16: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 16>, g, theta, c, mu, a, compact);
        case 20: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 20>, g, theta, c, mu, a, compact);
        case 24: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 24>, g, theta, c, mu, a, compact);
        case 32: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 32>, g, theta, c, mu, a, compact);
        default: return cudaLaunchKernelEx(&cfg, update_class_wide_kernel<R, 0>, g, theta, c, mu, a, compact);
        }
    }
    switch (g.L) {
    case 8: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 8>, g, theta, c, mu, a, compact);
    case 12: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 12>, g, theta, c, mu, a, compact);
    case 16: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 16>, g, theta, c, mu, a, compact);
    case 20: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 20>, g, theta, c, mu, a, compact);
    case 24: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 24>, g, theta, c, mu, a, compact);
    case 32: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 32>, g, theta, c, mu, a, compact);
    default: return cudaLaunchKernelEx(&cfg, update_class_kernel<R, 0>, g, theta, c, mu, a, compact);
    }
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
cudaError_t launch_measure_store(const Geo& g, const void* cs, int slab_t, int r_max, bool fields, int slot,
                                 double2* asum, void* tk, void* ok, double* osum, const void* ubar, cudaStream_t st)
{
    const int S = g.Nt / slab_t;
    const long n = static_cast<long>(S) * g.L3;
    if (!ubar && g.L <= kThreads) {
        // blocks of whole x-rows, about 192 threads
        const int threads = g.L * std::max(1, std::min(kThreads / g.L, 192 / g.L));
        measure_store_rows_kernel<R><<<static_cast<unsigned int>((n + threads - 1) / threads), threads, 0, st>>>(
            g, static_cast<const cs_t<R>*>(cs), slab_t, r_max, fields ? 1 : 0, slot, asum, static_cast<Cx<R>*>(tk),
            static_cast<R*>(ok), osum);
        return cudaGetLastError();
    }
    const int threads = update_block_threads(n); // balanced over the SMs, as the class updates
    measure_store_kernel<R><<<static_cast<unsigned int>((n + threads - 1) / threads), threads, 0, st>>>(
        g, static_cast<const cs_t<R>*>(cs), slab_t, r_max, fields ? 1 : 0, slot, asum, static_cast<Cx<R>*>(tk),
        static_cast<R*>(ok), osum, static_cast<const Cx<R>*>(ubar));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_multihit(const Geo& g, const void* cs, double beta, void* ubar, cudaStream_t st)
{
    const cs_t<R>* c = static_cast<const cs_t<R>*>(cs);
    Cx<R>* u = static_cast<Cx<R>*>(ubar);
    const int nb = blocks_for(g.V);
    switch (g.L) {
    case 8: multihit_kernel<R, 8><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    case 12: multihit_kernel<R, 12><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    case 16: multihit_kernel<R, 16><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    case 20: multihit_kernel<R, 20><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    case 24: multihit_kernel<R, 24><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    case 32: multihit_kernel<R, 32><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    default: multihit_kernel<R, 0><<<nb, kThreads, 0, st>>>(g, c, beta, u); break;
    }
    return cudaGetLastError();
}

template <typename R>
bool launch_contract_tiled(const Geo& g, int S, int r_max, int nd, int count, const void* tk, const void* ok,
                           double2* bsum, bool first, int* status, cudaStream_t st, cudaError_t* err, bool sym,
                           long long wait_cycles);

template <typename R>
cudaError_t launch_insertion_contract(const Geo& g, int slab_t, int r_max, int nd, int count, const void* tk,
                                      const void* ok, double2* bsum, bool first, cudaStream_t st, bool tiled,
                                      int* status, long long wait_cycles)
{
    const int S = g.Nt / slab_t;
    cudaError_t err = cudaSuccess;
    if (tiled && launch_contract_tiled<R>(g, S, r_max, nd, count, tk, ok, bsum, first, status, st, &err, false,
                                          wait_cycles))
        return err;
    const long total = static_cast<long>(S) * r_max * nd * ((g.L3 + kThreads - 1) / kThreads) * kThreads;
    insertion_contract_kernel<R><<<blocks_for(total), kThreads, 0, st>>>(
        g, S, r_max, nd, count, static_cast<const Cx<R>*>(tk), static_cast<const R*>(ok), bsum, first);
    return cudaGetLastError();
}

// Class (mu, parity) of every lattice of a group of one extent L: grid (blocks_x, t.njobs).
// FP32 uses the wide kernel (blocks of up to kWideThreads), FP64 blocks of up to
// kUpdateThreads.
template <typename R>
cudaError_t launch_group_update(const BatchUpdateTable& t, int L, int blocks_x, int threads, int mu, int parity,
                                cudaStream_t st, bool pdl)
{
    if (t.njobs < 1 || blocks_x < 1) return cudaErrorInvalidValue;
    const bool wide = sizeof(R) == 4;
    if (threads > (wide ? kWideThreads : kUpdateThreads)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks_x), static_cast<unsigned>(t.njobs));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define UL_GROUP_LAUNCH(K)                                                                                     \
    switch (L) {                                                                                               \
    case 8: return cudaLaunchKernelEx(&cfg, K<R, 8>, t, mu, parity);                                           \
    case 12: return cudaLaunchKernelEx(&cfg, K<R, 12>, t, mu, parity);                                         \
    case 16: return cudaLaunchKernelEx(&cfg, K<R, 16>, t, mu, parity);                                         \
    case 20: return cudaLaunchKernelEx(&cfg, K<R, 20>, t, mu, parity);                                         \
    case 24: return cudaLaunchKernelEx(&cfg, K<R, 24>, t, mu, parity);                                         \
    case 32: return cudaLaunchKernelEx(&cfg, K<R, 32>, t, mu, parity);                                         \
    default: return cudaLaunchKernelEx(&cfg, K<R, 0>, t, mu, parity);                                          \
    }
    if (wide) {
        UL_GROUP_LAUNCH(group_update_wide_kernel)
    }
    UL_GROUP_LAUNCH(group_update_kernel)
#undef UL_GROUP_LAUNCH
}

template <typename R>
cudaError_t launch_group_measure(const BatchMeasureTable& t, int blocks_x, cudaStream_t st)
{
    if (t.njobs < 1 || blocks_x < 1) return cudaErrorInvalidValue;
    group_measure_kernel<R><<<dim3(static_cast<unsigned>(blocks_x), static_cast<unsigned>(t.njobs)), kThreads, 0, st>>>(t);
    return cudaGetLastError();
}

template <typename R, int LC>
cudaError_t launch_persistent_lc(const Geo& g, R* theta, void* cs, const PersistArgs& in, int threads, cudaStream_t st)
{
    // occupancy of this instantiation and SM count, queried once (any thread; one GPU model)
    static std::atomic<int> cached_blocks_per_sm{0}, cached_n_sm{0};
    auto fn = persistent_kernel<R, LC>;
    threads = 256;
    int blocks_per_sm = cached_blocks_per_sm.load(std::memory_order_relaxed);
    int n_sm = cached_n_sm.load(std::memory_order_relaxed);
    if (!blocks_per_sm || !n_sm) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, threads, 0);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
        cached_n_sm.store(n_sm, std::memory_order_relaxed);
        cached_blocks_per_sm.store(blocks_per_sm, std::memory_order_relaxed);
    }
    const int work = in.measure ? std::max(g.Vh, (g.Nt / in.u.slab_t) * g.L3) : g.Vh;
    int grid = blocks_per_sm * n_sm;
    grid = std::min(grid, (work + threads - 1) / threads);
    grid = std::max(grid, 1);
    PersistArgs a = in;
    a.expected = in.expected == 0 ? static_cast<unsigned int>(grid)
                 : (in.expected == 0xffffffffu ? static_cast<unsigned int>(grid) + 1u : in.expected);
    Geo gg = g;
    cs_t<R>* c = static_cast<cs_t<R>*>(cs);
    void* args[] = {static_cast<void*>(&gg), static_cast<void*>(&theta), static_cast<void*>(&c), static_cast<void*>(&a)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fn), dim3(grid), dim3(threads), args, 0, st);
}

// in.expected == 0: the barrier waits for the whole grid; 0xffffffff: for one block more
// than the grid, so every wait runs into its limit (exercises the timeout path).
template <typename R>
cudaError_t launch_persistent(const Geo& g, R* theta, void* cs, const PersistArgs& in, int threads, cudaStream_t st)
{
    switch (g.L) {
    case 8: return launch_persistent_lc<R, 8>(g, theta, cs, in, threads, st);
    case 12: return launch_persistent_lc<R, 12>(g, theta, cs, in, threads, st);
    case 16: return launch_persistent_lc<R, 16>(g, theta, cs, in, threads, st);
    case 20: return launch_persistent_lc<R, 20>(g, theta, cs, in, threads, st);
    case 24: return launch_persistent_lc<R, 24>(g, theta, cs, in, threads, st);
    case 32: return launch_persistent_lc<R, 32>(g, theta, cs, in, threads, st);
    default: return launch_persistent_lc<R, 0>(g, theta, cs, in, threads, st);
    }
}

// Check word of this translation unit (bounds-checked build; 0 and nothing to clear in the
// default build).  The template parameter only selects the FP64 or FP32 unit.
template <typename R>
cudaError_t check_word(unsigned long long* out, bool clear)
{
#ifdef UL_CHECK
    cudaError_t e = cudaMemcpyFromSymbol(out, g_ul_check_word, sizeof(unsigned long long));
    if (e == cudaSuccess && clear) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(g_ul_check_word, &zero, sizeof zero);
    }
    return e;
#else
    (void)clear;
    *out = 0;
    return cudaSuccess;
#endif
}

#define UL_INSTANTIATE_KERNELS(R)                                                                                  \
    template cudaError_t check_word<R>(unsigned long long*, bool);                                                 \
    template cudaError_t launch_measure_sym<R>(const Geo&, const void*, int, int, int, int, double2*, void*,       \
                                               void*, void*, double*, cudaStream_t);                              \
    template cudaError_t launch_insertion_contract_sym<R>(const Geo&, int, int, int, int, const void*,             \
                                                          const void*, double2*, bool, cudaStream_t, bool, int*,  \
                                                          long long);                                             \
    template cudaError_t launch_rng_uniforms<R>(uint64_t, uint64_t, uint64_t, int, double*, cudaStream_t);        \
    template cudaError_t slab_plan<R>(const Geo&, int, int, int*, int*);                                           \
    template size_t slab_level_smem<R>(const Geo&, int, int);                                                      \
    template cudaError_t launch_slab<R>(const Geo&, R*, void*, const SlabArgs&, int, cudaStream_t);               \
    template cudaError_t launch_slab_jobs<R>(const Geo&, const SlabArgs&, const SlabJobTable&, int, cudaStream_t); \
    template cudaError_t launch_persistent<R>(const Geo&, R*, void*, const PersistArgs&, int, cudaStream_t);       \
    template cudaError_t launch_group_update<R>(const BatchUpdateTable&, int, int, int, int, int, cudaStream_t,    \
                                                bool);                                                             \
    template cudaError_t launch_group_measure<R>(const BatchMeasureTable&, int, cudaStream_t);                     \
    template cudaError_t launch_hot_start<R>(const Geo&, R*, void*, uint64_t, cudaStream_t);                        \
    template cudaError_t launch_refresh_cs<R>(const Geo&, const R*, void*, cudaStream_t);                           \
    template cudaError_t launch_update_class<R>(const Geo&, R*, void*, int, int, bool, uint64_t,                    \
                                                const unsigned long long*, uint64_t, double, double, int,          \
                                                unsigned long long*, cudaStream_t, int*, bool);                    \
    template cudaError_t launch_to_canonical<R>(const Geo&, const R*, double*, cudaStream_t);                       \
    template cudaError_t launch_from_canonical<R>(const Geo&, const double*, R*, void*, cudaStream_t);              \
    template cudaError_t launch_plaquette<R>(const Geo&, const void*, double*, double*, cudaStream_t);               \
    template cudaError_t launch_measure_store<R>(const Geo&, const void*, int, int, bool, int, double2*, void*,     \
                                                 void*, double*, const void*, cudaStream_t);                        \
    template cudaError_t launch_multihit<R>(const Geo&, const void*, double, void*, cudaStream_t);                 \
    template cudaError_t launch_insertion_contract<R>(const Geo&, int, int, int, int, const void*, const void*,     \
                                                      double2*, bool, cudaStream_t, bool, int*, long long);        \
    template cudaError_t prepare_insertion_contract<R>();

} // namespace ul

#include "ul_slab.cuh"
#include "ul_sym.cuh"
#include "ul_contract.cuh"
