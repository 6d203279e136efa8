// ul_slab.cuh — slab-resident sub-sample kernel (Section 2.2), included by ul_kernels.cuh.
//
// While the sub-samples of a multilevel level run, the spatial links on the slab boundaries
// are frozen, so the updates inside slab s read only the links of that slab and of its two
// boundary slices: temporal links on slices t0 .. t0+tau-1 (t0 = s tau), spatial links on
// t0+1 .. t0+tau-1 (updated) and on t0 and t0+tau (frozen).  One thread-block cluster owns
// one slab: its CTAs copy the slab's links into shared memory, run n_units sub-samples
// (n_metro Metropolis then n_or overrelaxation passes of the 8 (mu, parity) classes, then
// the measurement) with a cluster barrier between classes, and write the updated links
// back.  CTA r of the cluster holds the z planes [r nz, (r+1) nz); the staple of a link on
// the first or last of those planes reads links of the neighbouring CTA through
// distributed shared memory.
//
// Links are updated by the same staple and decision functions as in the other update
// kernels with the same Philox counters, and the measurement forms the same products in
// the same order as measure_store_site, so the trajectory, the accumulators and the stored
// samples equal those of the one-class-per-launch path.
//
// Shared memory of one CTA (P = L L nz sites per time slice, Ph = P / 2 per parity):
//   phases [NS][2][Ph] (cos, sin): slot tl for the temporal links of slice t0+tl
//          (0 <= tl < tau), slot tau + (k-1)(tau+1) + tl for spatial direction k on slice
//          t0+tl (0 <= tl <= tau);
//   angles [NT][2][Ph]: slot tl (temporal, 0 <= tl < tau), slot tau + (k-1)(tau-1) + tl-1
//          (spatial, 1 <= tl <= tau-1);
// with NS = tau + 3 (tau+1), NT = tau + 3 (tau-1); inside a slot, parity p and half index
// (x + L (y + L zl)) >> 1, p being the parity of the site's global coordinates.
#pragma once
#include <cooperative_groups.h>

#include "ul_batch_types.h"
#include "ul_device.cuh"
#include "ul_math.cuh"

namespace ul {

__host__ __device__ __forceinline__ int slab_phase_slots(int tau) { return tau + 3 * (tau + 1); }
__host__ __device__ __forceinline__ int slab_angle_slots(int tau) { return tau + 3 * (tau - 1); }

// Phase arrays of a CTA and of the CTAs holding the z planes below and above it.  A site
// is addressed by its local lexicographic index li = x + L (y + L zl); after a step in z,
// li < 0 or li >= P addresses the neighbouring CTA (its local index li + P or li - P).
// TC, NZC: the slab thickness and the z planes per CTA when known at compile time (0: taken
// from the launch), so that every shared-memory offset of a staple folds to a constant.
template <typename R, int LC, int TC = 0, int NZC = 0>
struct SlabLinks {
    cs_t<R>* own; // this CTA's phases (shared memory)
    cs_t<R>* dn;  // the CTA below (distributed shared memory)
    cs_t<R>* up;  // the CTA above
    int P_rt, Ph_rt, tau_rt;

    __device__ __forceinline__ int P() const { return (LC && NZC) ? LC * LC * NZC : P_rt; }
    __device__ __forceinline__ int Ph() const { return (LC && NZC) ? LC * LC * NZC / 2 : Ph_rt; }
    __device__ __forceinline__ int tau() const { return TC ? TC : tau_rt; }
    __device__ __forceinline__ int slot(int dir, int tl) const
    {
        return dir == 0 ? tl : tau() + (dir - 1) * (tau() + 1) + tl;
    }
    // ZS: the z step (-1, 0, +1) taken to reach the site.
    template <int ZS>
    __device__ __forceinline__ Cx<R> ld(int dir, int tl, int li, int par) const
    {
        const int base = (slot(dir, tl) * 2 + par) * Ph();
        cs_t<R> v;
        if constexpr (ZS > 0) {
            if (li >= P()) v = up[base + ((li - P()) >> 1)];
            else v = own[base + (li >> 1)];
        } else if constexpr (ZS < 0) {
            if (li < 0) v = dn[base + ((li + P()) >> 1)];
            else v = own[base + (li >> 1)];
        } else {
            v = own[base + (li >> 1)];
        }
        return Cx<R>{v.x, v.y};
    }
    // The same by half index hh = li >> 1 of the site in this CTA's numbering; edge: the
    // site before the z step lies on the CTA's last (ZS > 0) or first (ZS < 0) plane, so
    // the step leaves the CTA (the neighbour's half index is hh -+ Ph).
    template <int ZS>
    __device__ __forceinline__ Cx<R> ldh(int dir, int tl, int hh, int par, bool edge) const
    {
        const int base = (slot(dir, tl) * 2 + par) * Ph();
        cs_t<R> v;
        if constexpr (ZS > 0) {
            v = edge ? up[base + hh - Ph()] : own[base + hh];
        } else if constexpr (ZS < 0) {
            v = edge ? dn[base + hh + Ph()] : own[base + hh];
        } else {
            v = own[base + hh];
        }
        return Cx<R>{v.x, v.y};
    }
};

// Local-index offsets of the +1 / -1 steps from site (x, y) (periodic in x and y; a z step
// is +-L^2 and never wraps inside a CTA; a t step changes the slice instead).
struct SlabSteps {
    int xu, xd, yu, yd, zs;
    __device__ __forceinline__ SlabSteps(int x, int y, int L)
    {
        xu = x == L - 1 ? -(L - 1) : 1;
        xd = x == 0 ? L - 1 : -1;
        yu = y == L - 1 ? -(L - 1) * L : L;
        yd = y == 0 ? (L - 1) * L : -L;
        zs = L * L;
    }
    template <int D>
    __device__ __forceinline__ int up() const
    {
        return D == 0 ? 0 : (D == 1 ? xu : (D == 2 ? yu : zs));
    }
    template <int D>
    __device__ __forceinline__ int dn() const
    {
        return D == 0 ? 0 : (D == 1 ? xd : (D == 2 ? yd : -zs));
    }
};

// Half-index offsets of the +1 / -1 steps from site (x, y): a step s of the local index li
// moves the half index h = li >> 1 to (li + s) >> 1 = h + ((b + s) >> 1), b = x & 1, so an
// even step (in y or z) moves it by s / 2 and two steps add their offsets (at most one of
// them in x).  A z step moves it by L^2 / 2 (leaving the CTA on its edge planes).
struct SlabHalfSteps {
    int xu, xd, yu, yd, zs;
    __device__ __forceinline__ SlabHalfSteps(int x, int y, int L)
    {
        const int b = x & 1;
        xu = x == L - 1 ? (b - (L - 1)) >> 1 : (b + 1) >> 1;
        xd = x == 0 ? (b + L - 1) >> 1 : (b - 1) >> 1;
        yu = y == L - 1 ? -(L - 1) * L / 2 : L / 2;
        yd = y == 0 ? (L - 1) * L / 2 : -L / 2;
        zs = L * L / 2;
    }
    template <int D>
    __device__ __forceinline__ int up() const
    {
        return D == 0 ? 0 : (D == 1 ? xu : (D == 2 ? yu : zs));
    }
    template <int D>
    __device__ __forceinline__ int dn() const
    {
        return D == 0 ? 0 : (D == 1 ? xd : (D == 2 ? yd : -zs));
    }
};

// One plane's staple contribution by half indices (the loads of slab_staple_term):
// zup / zdn: the site lies on the CTA's last / first z plane.
template <typename R, int LC, int TC, int NZC, int MU, int NU>
__device__ __forceinline__ void slab_staple_term_h(Cx<R>& A, const SlabLinks<R, LC, TC, NZC>& S,
                                                   const SlabHalfSteps& hs, int tl, int h, int p, bool zup, bool zdn)
{
    constexpr int ZM = MU == 3 ? 1 : 0;
    constexpr int ZN = NU == 3 ? 1 : 0;
    constexpr int TM = MU == 0 ? 1 : 0;
    constexpr int TN = NU == 0 ? 1 : 0;
    constexpr int ZD = ZM - ZN; // z step of the diagonal site x + mu - nu
    const int q = p ^ 1;
    const int h_mu = h + hs.up<MU>();
    const int h_nu = h + hs.up<NU>();
    const int h_nd = h + hs.dn<NU>();
    const int h_dg = h_mu + hs.dn<NU>();
    staple_acc_fwd(A, S.template ldh<ZM>(NU, tl + TM, h_mu, q, zup), S.template ldh<ZN>(MU, tl + TN, h_nu, q, zup),
                   S.template ldh<0>(NU, tl, h, p, false));
    staple_acc_bwd(A, S.template ldh<ZD>(NU, tl + TM - TN, h_dg, p, ZD > 0 ? zup : zdn),
                   S.template ldh<-ZN>(MU, tl - TN, h_nd, q, zdn), S.template ldh<-ZN>(NU, tl - TN, h_nd, q, zdn));
}

// Global offset in [dir][parity][h] of link dir at site (x, y, zg, tg).
__device__ __forceinline__ int slab_global_offset(const Geo& g, int dir, int x, int y, int zg, int tg)
{
    const int i = x + g.L * (y + g.L * (zg + g.L * tg));
    return static_cast<int>(UL_IDX((dir * 2 + ((x + y + zg + tg) & 1)) * g.Vh + (i >> 1), 8LL * g.Vh,
                                   kChkSlabGlobal));
}

// Class (MU, p) of this CTA: thread tid updates the links at half index hl = tid (+ nthr ...)
// on every updatable slice.  Returns the number of Metropolis acceptances.
template <typename R, int LC, int TC, int NZC, int MU>
__device__ __forceinline__ int slab_class(const SlabLinks<R, LC, TC, NZC>& S, R* th_own, const Geo& g, int L, int z0,
                                          int t0, int p, bool metro, uint64_t pass, const UpdateArgs& a)
{
    const int Lh = L / 2, tau = S.tau(), Ph = S.Ph();
    const int nz = S.P() / (L * L);
    const int nsl = MU == 0 ? tau : tau - 1;
    int accepted = 0;
    for (int hl = static_cast<int>(threadIdx.x); hl < Ph; hl += static_cast<int>(blockDim.x)) {
        const int row = hl / Lh;
        const int xh = hl - row * Lh;
        const int y = row % L;
        const int zl = row / L;
        for (int sl = 0; sl < nsl; ++sl) {
            const int tl = MU == 0 ? sl : sl + 1;
            const int x = 2 * xh + ((p + y + z0 + zl + t0 + tl) & 1);
            const SlabHalfSteps hs(x, y, L);
            const bool zup = zl == nz - 1, zdn = zl == 0;
            Cx<R> A{R(0), R(0)};
            if (MU != 0) slab_staple_term_h<R, LC, TC, NZC, MU, 0>(A, S, hs, tl, hl, p, zup, zdn);
            if (MU != 1) slab_staple_term_h<R, LC, TC, NZC, MU, 1>(A, S, hs, tl, hl, p, zup, zdn);
            if (MU != 2) slab_staple_term_h<R, LC, TC, NZC, MU, 2>(A, S, hs, tl, hl, p, zup, zdn);
            if (MU != 3) slab_staple_term_h<R, LC, TC, NZC, MU, 3>(A, S, hs, tl, hl, p, zup, zdn);
            const int ph_idx = (S.slot(MU, tl) * 2 + p) * Ph + hl;
            const int th_slot = MU == 0 ? tl : tau + (MU - 1) * (tau - 1) + tl - 1;
            const int th_idx = (th_slot * 2 + p) * Ph + hl;
            const R th = th_own[th_idx];
            R nth;
            cs_t<R> ncs;
            if (metro) {
                const uint64_t link_id = static_cast<uint64_t>(MU) * g.V +
                                         static_cast<uint64_t>(x + L * (y + L * (z0 + zl + L * (t0 + tl))));
                if (metropolis_new<R>(th, [&] { return S.own[ph_idx]; }, A, link_id, pass, a.seed, width_of<R>(a),
                                      beta_of<R>(a), nth, ncs)) {
                    th_own[th_idx] = nth;
                    S.own[ph_idx] = ncs;
                    ++accepted;
                }
            } else {
                overrelax_new<R>(th, A, nth, ncs);
                th_own[th_idx] = nth;
                S.own[ph_idx] = ncs;
            }
        }
    }
    return accepted;
}

// Measurement of one sub-sample for this CTA's sites (same products, order and stores as
// measure_store_site).
template <typename R, int LC, int TC, int NZC>
__device__ __forceinline__ void slab_measure(const SlabLinks<R, LC, TC, NZC>& S, const Geo& g, int L, int z0, int t0, int s,
                                             int slot, const SlabArgs& a)
{
    const int tau = S.tau(), P = S.P();
    const int nS = g.Nt / tau, SL3 = nS * g.L3;
    for (int q = static_cast<int>(threadIdx.x); q < P; q += static_cast<int>(blockDim.x)) {
        const int x = q % L;
        const int yz = q / L;
        const int y = yz % L;
        const int zl = yz / L;
        const int x0 = x + L * (y + L * (z0 + zl));
        const int kk = s * g.L3 + x0;
        const int pbase = y + z0 + zl + t0;
        auto line = [&](int xx) {
            const int lx = q - x + xx;
            Cx<R> w = S.template ld<0>(0, 0, lx, (xx + pbase) & 1);
            for (int tl = 1; tl < tau; ++tl) w = cmul_rn(w, S.template ld<0>(0, tl, lx, (xx + pbase + tl) & 1));
            return w;
        };
        const Cx<R> w0 = cconj(line(x));
        for (int r = 1; r <= a.r_max; ++r) {
            const int x1 = x + r < L ? x + r : x + r - L;
            const Cx<R> T = cmul_rn(w0, line(x1));
            const long ai = static_cast<long>(s * a.r_max + (r - 1)) * g.L3 + x0;
            double2 av = a.asum[ai];
            av.x += static_cast<double>(T.re);
            av.y += static_cast<double>(T.im);
            a.asum[ai] = av;
            if (a.fields)
                SampleStore<R>::put_T(static_cast<Cx<R>*>(a.tk),
                                      (static_cast<long>(slot * nS + s) * a.r_max + (r - 1)) * g.L3 + x0, T);
        }
        if (!a.fields) continue;
        const SlabSteps st(x, y, L);
        R acc[8];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) acc[ch] = R(0);
        for (int tl = 0; tl < tau; ++tl) {
            const int pc = (x + pbase + tl) & 1;
            const Cx<R> u0 = S.template ld<0>(0, tl, q, pc);
            // planes (0, k): U_0(x) U_k(x + t) U*_0(x + k) U*_k(x)
            const Cx<R> e1 = cmul_rn(cmul_rn(cmul_rn(u0, S.template ld<0>(1, tl + 1, q, pc ^ 1)),
                                             cconj(S.template ld<0>(0, tl, q + st.xu, pc ^ 1))),
                                     cconj(S.template ld<0>(1, tl, q, pc)));
            const Cx<R> e2 = cmul_rn(cmul_rn(cmul_rn(u0, S.template ld<0>(2, tl + 1, q, pc ^ 1)),
                                             cconj(S.template ld<0>(0, tl, q + st.yu, pc ^ 1))),
                                     cconj(S.template ld<0>(2, tl, q, pc)));
            const Cx<R> e3 = cmul_rn(cmul_rn(cmul_rn(u0, S.template ld<0>(3, tl + 1, q, pc ^ 1)),
                                             cconj(S.template ld<1>(0, tl, q + st.zs, pc ^ 1))),
                                     cconj(S.template ld<0>(3, tl, q, pc)));
            // plane (2, 3): U_2(x) U_3(x + y) U*_2(x + z) U*_3(x)
            const Cx<R> b1 = cmul_rn(cmul_rn(cmul_rn(S.template ld<0>(2, tl, q, pc), S.template ld<0>(3, tl, q + st.yu, pc ^ 1)),
                                             cconj(S.template ld<1>(2, tl, q + st.zs, pc ^ 1))),
                                     cconj(S.template ld<0>(3, tl, q, pc)));
            acc[0] += e1.im;
            acc[1] += e1.re;
            acc[2] += e2.im;
            acc[3] += e2.re;
            acc[4] += e3.im;
            acc[5] += e3.re;
            acc[6] += b1.im;
            acc[7] += b1.re;
        }
        SampleStore<R>::put_O(static_cast<R*>(a.ok), static_cast<long>(slot) * SL3 + kk, x, L, acc);
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) a.osum[ch * SL3 + kk] += static_cast<double>(acc[ch]);
    }
}

template <typename R, int LC, int TC = 0, int NZC = 0>
__device__ __forceinline__ void slab_body(const Geo& g, R* __restrict__ theta, cs_t<R>* __restrict__ cs,
                                          const SlabArgs& a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = static_cast<int>(cl.block_rank());
    const int ncl = a.cluster;
    const int s = static_cast<int>(blockIdx.x) / ncl;
    const int tau = TC ? TC : a.u.slab_t;
    const int L = LC ? LC : g.L, Lh = L / 2, nz = NZC ? NZC : a.nz;
    const int P = L * L * nz, Ph = P / 2;
    const int z0 = rank * nz, t0 = s * tau;
    const int NS = slab_phase_slots(tau), NT = slab_angle_slots(tau);
    const int tid = static_cast<int>(threadIdx.x), nthr = static_cast<int>(blockDim.x);

    extern __shared__ __align__(16) unsigned char slab_smem[];
    cs_t<R>* ph = reinterpret_cast<cs_t<R>*>(slab_smem);
    R* th = reinterpret_cast<R*>(ph + NS * P);

    SlabLinks<R, LC, TC, NZC> S;
    S.own = ph;
    S.dn = cl.map_shared_rank(ph, (rank + ncl - 1) % ncl);
    S.up = cl.map_shared_rank(ph, (rank + 1) % ncl);
    S.P_rt = P;
    S.Ph_rt = Ph;
    S.tau_rt = tau;

    // entry e of the phase (angle) array -> direction, slice and site
    auto decode = [&](int e, bool angle, int& dir, int& tl, int& par, int& x, int& y, int& zl) {
        const int slot = e / P;
        const int rem = e - slot * P;
        par = rem >= Ph ? 1 : 0;
        const int hl = rem - par * Ph;
        if (slot < tau) {
            dir = 0;
            tl = slot;
        } else {
            const int per = angle ? tau - 1 : tau + 1;
            const int k = (slot - tau) / per;
            dir = k + 1;
            tl = (slot - tau) - k * per + (angle ? 1 : 0);
        }
        const int row = hl / Lh;
        const int xh = hl - row * Lh;
        y = row % L;
        zl = row / L;
        x = 2 * xh + ((par + y + z0 + zl + t0 + tl) & 1);
    };

    for (int e = tid; e < NS * P; e += nthr) {
        int dir, tl, par, x, y, zl;
        decode(e, false, dir, tl, par, x, y, zl);
        ph[e] = cs[slab_global_offset(g, dir, x, y, z0 + zl, (t0 + tl) % g.Nt)];
    }
    for (int e = tid; e < NT * P; e += nthr) {
        int dir, tl, par, x, y, zl;
        decode(e, true, dir, tl, par, x, y, zl);
        th[e] = theta[slab_global_offset(g, dir, x, y, z0 + zl, t0 + tl)];
    }
    cl.sync();

    // first Metropolis pass: an offset plus a device-side base where the launch is replayed
    // from a CUDA graph (as for the one-class-per-launch kernel)
    uint64_t pass = a.u.pass + (a.u.pass_base ? *a.u.pass_base : 0ull);
    for (int unit = 0; unit < a.n_units; ++unit) {
        for (int k = 0; k < a.n_metro + a.n_or; ++k) {
            const bool metro = k < a.n_metro;
            for (int mu = 0; mu < 4; ++mu) {
                if (mu != 0 && tau == 1) continue; // no updatable spatial link (uniform over the cluster)
                for (int p = 0; p < 2; ++p) {
                    int accepted;
                    switch (mu) {
                    case 0: accepted = slab_class<R, LC, TC, NZC, 0>(S, th, g, L, z0, t0, p, metro, pass, a.u); break;
                    case 1: accepted = slab_class<R, LC, TC, NZC, 1>(S, th, g, L, z0, t0, p, metro, pass, a.u); break;
                    case 2: accepted = slab_class<R, LC, TC, NZC, 2>(S, th, g, L, z0, t0, p, metro, pass, a.u); break;
                    default: accepted = slab_class<R, LC, TC, NZC, 3>(S, th, g, L, z0, t0, p, metro, pass, a.u); break;
                    }
                    if (metro) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) accepted += __shfl_xor_sync(0xffffffffu, accepted, o);
                        if ((tid & 31) == 0 && accepted)
                            atomicAdd(a.u.accepted, static_cast<unsigned long long>(accepted));
                    }
                    cl.sync();
                }
            }
            if (metro) pass += 1;
        }
        if (!a.skip_measure) {
            slab_measure<R, LC, TC, NZC>(S, g, L, z0, t0, s, a.slot0 + unit, a);
            cl.sync(); // the next updates may change links that other CTAs just measured
        }
    }

    for (int e = tid; e < NT * P; e += nthr) {
        int dir, tl, par, x, y, zl;
        decode(e, true, dir, tl, par, x, y, zl);
        const int off = slab_global_offset(g, dir, x, y, z0 + zl, t0 + tl);
        theta[off] = th[e];
        cs[off] = ph[(S.slot(dir, tl) * 2 + par) * Ph + (e - (e / Ph) * Ph)];
    }
}

// The block has one thread per half-site of a CTA's planes (rounded up to warps): the
// compile-time shape bounds it exactly.
template <typename R, int LC, int TC = 0, int NZC = 0>
__global__ void __launch_bounds__((LC && NZC) ? (LC * LC * NZC / 2 + 31) / 32 * 32 : 1024, 1)
    slab_kernel(Geo g, R* __restrict__ theta, cs_t<R>* __restrict__ cs, SlabArgs a)
{
    slab_body<R, LC, TC, NZC>(g, theta, cs, a);
}

// The same slab-resident level for several lattices of one shape in one launch: the grid's
// y index selects the lattice (clusters never span two lattices), whose links, Metropolis
// arguments, accumulator and schedule come from the table; every lattice's results are
// those of its own slab_kernel launch.
template <typename R, int LC>
__global__ void __launch_bounds__(1024, 1) slab_jobs_kernel(Geo g, SlabArgs a, const __grid_constant__ SlabJobTable t)
{
    const SlabJob& j = t.job[blockIdx.y];
    SlabArgs b = a;
    b.u = j.u;
    b.asum = j.asum;
    b.n_units = j.n_units;
    b.n_metro = j.n_metro;
    b.n_or = j.n_or;
    b.r_max = j.r_max;
    slab_body<R, LC>(g, static_cast<R*>(j.theta), static_cast<cs_t<R>*>(j.cs), b);
}

// Kernel instances for extent L (compile-time extents for the common sizes; for FP32 links
// at L = 24 with slabs of 2 slices and 3 z planes per CTA, the benchmark's shape, also the
// slab thickness and the planes per CTA).
template <typename R>
auto slab_kernel_for(int L, int tau = 0, int nz = 0)
{
    if constexpr (sizeof(R) == 4)
        if (L == 24 && tau == 2 && nz == 3) return slab_kernel<R, 24, 2, 3>;
    switch (L) {
    case 16: return slab_kernel<R, 16>;
    case 24: return slab_kernel<R, 24>;
    case 32: return slab_kernel<R, 32>;
    default: return slab_kernel<R, 0>;
    }
}

template <typename R>
auto slab_jobs_kernel_for(int L)
{
    switch (L) {
    case 16: return slab_jobs_kernel<R, 16>;
    case 24: return slab_jobs_kernel<R, 24>;
    case 32: return slab_jobs_kernel<R, 32>;
    default: return slab_jobs_kernel<R, 0>;
    }
}

template <typename R>
size_t slab_smem_bytes(int L, int nz, int tau)
{
    const size_t P = static_cast<size_t>(L) * L * nz;
    return P * (static_cast<size_t>(slab_phase_slots(tau)) * 2 * sizeof(R) +
                static_cast<size_t>(slab_angle_slots(tau)) * sizeof(R));
}

// Shared memory of one CTA of a slab-resident launch of shape g with `cluster` CTAs per slab.
template <typename R>
size_t slab_level_smem(const Geo& g, int tau, int cluster)
{
    return slab_smem_bytes<R>(g.L, g.L / cluster, tau);
}

template <typename R>
cudaError_t slab_plan(const Geo& g, int tau, int force_cluster, int* cluster, int* threads)
{
    *cluster = 0;
    *threads = 0;
    int dev = 0, optin = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int S = g.Nt / tau;
    auto fits = [&](int c) {
        return c >= 1 && c <= 16 && g.L % c == 0 && slab_smem_bytes<R>(g.L, g.L / c, tau) <= static_cast<size_t>(optin);
    };
    int best = 0;
    if (force_cluster > 0) {
        if (fits(force_cluster)) best = force_cluster;
    } else {
        // the most CTAs per slab (up to the portable 8) with every slab's cluster resident at once
        for (int c = 1; c <= 8; ++c)
            if (fits(c) && S * c <= sms) best = c;
        if (!best)
            for (int c = 1; c <= 16 && !best; ++c)
                if (fits(c)) best = c;
    }
    if (!best) return cudaSuccess;
    const int nz = g.L / best;
    const int Ph = g.L * g.L * nz / 2;
    int nt = ((Ph + 31) / 32) * 32; // one half index per thread in each class
    nt = nt > 1024 ? 1024 : nt;
    const size_t smem = slab_smem_bytes<R>(g.L, nz, tau);
    auto fn = slab_kernel_for<R>(g.L, tau, nz);
    auto fnj = slab_jobs_kernel_for<R>(g.L);
    // the attribute is an upper bound shared by every shape that uses this kernel instance:
    // the device's opt-in maximum, so that no later plan lowers it below another's need
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fnj, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess && best > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess && best > 8) e = cudaFuncSetAttribute(fnj, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(S * best));
    cfg.blockDim = dim3(static_cast<unsigned>(nt));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(best);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, fn, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess; // not launchable in this shape: no slab plan
    }
    if (active < 1) return cudaSuccess;
    *cluster = best;
    *threads = nt;
    return cudaSuccess;
}

// The level of t.njobs lattices of shape g (slab thickness a.u.slab_t, a.cluster CTAs of
// `threads` threads per slab, a plan of slab_plan) in one launch; a supplies the uniform
// part (cluster, nz, skip_measure = 0, fields = 0), the table the rest.
template <typename R>
cudaError_t launch_slab_jobs(const Geo& g, const SlabArgs& a, const SlabJobTable& t, int threads, cudaStream_t st)
{
    if (t.njobs < 1 || t.njobs > kMaxSlabJobs) return cudaErrorInvalidValue;
    const int S = g.Nt / a.u.slab_t;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(S * a.cluster), static_cast<unsigned>(t.njobs));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = slab_smem_bytes<R>(g.L, a.nz, a.u.slab_t);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(a.cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, slab_jobs_kernel_for<R>(g.L), g, a, t);
}

template <typename R>
cudaError_t launch_slab(const Geo& g, R* theta, void* cs, const SlabArgs& a, int threads, cudaStream_t st)
{
    const int S = g.Nt / a.u.slab_t;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(S * a.cluster));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = slab_smem_bytes<R>(g.L, a.nz, a.u.slab_t);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(a.cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, slab_kernel_for<R>(g.L, a.u.slab_t, a.nz), g, theta, static_cast<cs_t<R>*>(cs), a);
}

} // namespace ul
