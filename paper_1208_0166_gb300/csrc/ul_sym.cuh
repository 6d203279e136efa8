// ul_sym.cuh — symmetrised insertion measurement and contraction (Section 2.2), included
// by ul_kernels.cuh.
//
// The one-level estimator is averaged over the 24 frames of the source pair: separation
// axis +e_a (a = 1, 2, 3), insertion offset direction sb e_b and third direction sc e_c
// ((a, b, c) a permutation of the spatial axes, sb, sc = +-1), i.e. over the lattice
// symmetries that keep the time axis and the orientation of the pair.  The channels of a
// frame are the planes (0, +a), (0, sb b), (0, sc c), (sb b, sc c) at y = x0 + floor(r/2) e_a
// + d sb e_b.  A plaquette in negative directions is the conjugate of a stored plaquette at
// a shifted corner:
//   P_{mu,-nu}(x) = P*_{mu nu}(x - nu),  P_{-mu,nu}(x) = P*_{mu nu}(x - mu),
//   P_{-mu,-nu}(x) = P_{mu nu}(x - mu - nu),  P_{nu mu}(x) = P*_{mu nu}(x),
// so the measurement stores the six planes (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) once per site,
// a second kernel sums every axis's 8 frames per insertion midpoint, and the contraction
// multiplies those sums by the axis's transporters.
//
// Everything indexed by a site for one axis a (the accumulators asum3 / bsum3, the stored
// transporters tk3 and the frame sums csym) uses the axis-major site order of a: position
// along e_a fastest, then the other two axes in increasing order.  The midpoint shift
// x0 + floor(r/2) e_a then stays inside a row of L consecutive entries, as the shift along
// x does for the single-frame estimator; the reduction over x0 takes the entries in this
// order.  The frame sums of a midpoint are stored as 8 consecutive channels.
#pragma once

namespace ul {

__device__ __constant__ static const int kSymPlaneMu[6] = {0, 0, 0, 1, 1, 2};
__device__ __constant__ static const int kSymPlaneNu[6] = {1, 2, 3, 2, 3, 3};

// Spatial coordinates of a site, moved along one axis without integer division.
struct SymSite {
    int c1, c2, c3; // coordinates along the spatial axes 1, 2, 3 (x, y, z)
    __device__ __forceinline__ SymSite moved(int L, int axis, int n) const // |n| < L
    {
        SymSite q = *this;
        int& v = axis == 1 ? q.c1 : (axis == 2 ? q.c2 : q.c3);
        v += n;
        v = v >= L ? v - L : (v < 0 ? v + L : v);
        return q;
    }
    __device__ __forceinline__ int lex(int L) const { return c1 + L * (c2 + L * c3); }
    // index in the axis-major order of axis a
    __device__ __forceinline__ int axis_major(int L, int a) const
    {
        return a == 1 ? c1 + L * (c2 + L * c3) : (a == 2 ? c2 + L * (c1 + L * c3) : c3 + L * (c1 + L * c2));
    }
    // the site at index i of the axis-major order of axis a
    static __device__ __forceinline__ SymSite from_axis_major(int L, int a, int i)
    {
        const int u = i % L, v = (i / L) % L, w = i / (L * L);
        return a == 1 ? SymSite{u, v, w} : (a == 2 ? SymSite{v, u, w} : SymSite{v, w, u});
    }
};

// Index reached from axis-major index i of axis a by n (0 <= n < L) steps along e_a.
__device__ __forceinline__ int axis_major_step(int L, int i, int n)
{
    const int u = i % L;
    const int v = u + n;
    return i - u + (v >= L ? v - L : v);
}

// slab_line of the spatial site with lexicographic index x0 and coordinate sum csum (x+y+z):
// the same loads and products, the temporal link offsets formed without decoding the site.
template <typename R>
__device__ __forceinline__ Cx<R> slab_line_at(const Geo& g, const cs_t<R>* __restrict__ cs, int x0, int csum, int t0,
                                              int slab_t)
{
    Cx<R> w = link_at<R>(cs, ((csum + t0) & 1) * g.Vh + ((x0 + g.L3 * t0) >> 1));
    for (int t = t0 + 1; t < t0 + slab_t; ++t)
        w = cmul_rn(w, link_at<R>(cs, ((csum + t) & 1) * g.Vh + ((x0 + g.L3 * t) >> 1)));
    return w;
}

// Measurement after one sub-sample, one launch of 4 S L3 threads:
// threads [0, 3 S L3), one per (a, s, i) with i the axis-major index of site x0:
//   T_a(s, x0, r) = W*(s, x0) W(s, x0 + r e_a)  (W the slab line),
//   asum3[(a-1) nA + (s R + r-1) L3 + i] += T,  tk3[(((slot*3 + a-1) S + s) R + r-1) L3 + i] = T;
// threads [3 S L3, 4 S L3), one per (s, x0) in lexicographic order:
//   O(s, x0, 2p + part) = sum_{t in slab} {Im, Re} P_p(x0, t)  (the six planes p),
//   o12[ch SL3 + s L3 + x0] = O (this sample only),  osum12[ch SL3 + s L3 + x0] += O.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    measure_sym_kernel(Geo g, const cs_t<R>* __restrict__ cs, int slab_t, int r_max, int slot,
                       double2* __restrict__ asum3, Cx<R>* __restrict__ tk3, R* __restrict__ o12,
                       double* __restrict__ osum12)
{
    const int S = g.Nt / slab_t;
    const long SL3 = static_cast<long>(S) * g.L3;
    long idx = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= 4 * SL3) return;
    if (idx < 3 * SL3) {
        const int a = static_cast<int>(idx / SL3) + 1;
        const long rem = idx - (a - 1) * SL3;
        const int s = static_cast<int>(rem / g.L3);
        const int i = static_cast<int>(rem - static_cast<long>(s) * g.L3);
        const int t0 = s * slab_t;
        const SymSite p0 = SymSite::from_axis_major(g.L, a, i);
        const Cx<R> w0 = cconj(slab_line_at<R>(g, cs, p0.lex(g.L), p0.c1 + p0.c2 + p0.c3, t0, slab_t));
        const long nA = SL3 * r_max;
        for (int r = 1; r <= r_max; ++r) {
            const SymSite p = p0.moved(g.L, a, r);
            const Cx<R> T = cmul_rn(w0, slab_line_at<R>(g, cs, p.lex(g.L), p.c1 + p.c2 + p.c3, t0, slab_t));
            const long ai = (a - 1) * nA + static_cast<long>(s * r_max + (r - 1)) * g.L3 + i;
            double2 av = asum3[ai];
            av.x += static_cast<double>(T.re);
            av.y += static_cast<double>(T.im);
            asum3[ai] = av;
            tk3[((static_cast<long>(slot * 3 + a - 1) * S + s) * r_max + (r - 1)) * g.L3 + i] = T;
        }
        return;
    }
    const int k = static_cast<int>(idx - 3 * SL3); // s*L3 + x0
    const int s = k / g.L3;
    const int x0 = k - s * g.L3;
    const int t0 = s * slab_t;
    R acc[12];
#pragma unroll
    for (int ch = 0; ch < 12; ++ch) acc[ch] = R(0);
    for (int t = t0; t < t0 + slab_t; ++t) {
        const Site x = site_from_lex(g, x0 + g.L3 * t);
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const int mu = kSymPlaneMu[p], nu = kSymPlaneNu[p];
            const Cx<R> P = cmul_rn(cmul_rn(cmul_rn(link_at<R>(cs, link_offset(g, mu, x)),
                                                    link_at<R>(cs, link_offset(g, nu, site_step(g, x, mu, +1)))),
                                            cconj(link_at<R>(cs, link_offset(g, mu, site_step(g, x, nu, +1))))),
                                    cconj(link_at<R>(cs, link_offset(g, nu, x))));
            acc[2 * p] += P.im;
            acc[2 * p + 1] += P.re;
        }
    }
#pragma unroll
    for (int ch = 0; ch < 12; ++ch) {
        o12[ch * SL3 + k] = acc[ch];
        osum12[ch * SL3 + k] += static_cast<double>(acc[ch]);
    }
}

// Index of the stored plane (mu, nu), mu < nu.
__device__ __forceinline__ int sym_plane(int mu, int nu)
{
    return mu == 0 ? nu - 1 : (mu == 1 ? (nu == 2 ? 3 : 4) : 5);
}

// Frame sums of one sub-sample, thread per (a, s, d, m), m fastest in lexicographic order (the
// channel loads of neighbouring threads are neighbours); the 8 frames (b, c, sb, sc) of axis a
// put their channels at y = m + d sb e_b; their sum does not depend on how the midpoint
// m = x0 + floor(r/2) e_a was reached, so it is formed once per (a, s, d, m) and stored at
// the axis-major index i(m) of a as 8 consecutive channels (one 32-byte sector in FP32):
//   csym[(((((slot*3 + a-1) S + s) nd + d) L3 + i(m)) 8 + ch] = sum over the frames of channel ch,
// the frames taken in the order (b, c) = (o1, o2), (o2, o1) (o1 < o2 the axes other than a),
// sb = +, -, sc = +, -, summed in precision R.
// The 8 channel sums over the frames of axis a at midpoint pm and offset d (channel ch of site
// y of the slab: O[ch SL3 + y]), in the order stated above.
template <typename R>
__device__ __forceinline__ void frame_sums(int L, long SL3, const R* __restrict__ O, int a, int d, SymSite pm, R C[8])
{
    const int o1 = a == 1 ? 2 : 1, o2 = a == 3 ? 2 : 3;
    const int pa = a - 1;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) C[ch] = R(0);
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const int b = pair == 0 ? o1 : o2, c = pair == 0 ? o2 : o1;
        const int pb = b - 1, pc = c - 1;
        const int pbc = sym_plane(b < c ? b : c, b < c ? c : b);
        const R ori = b < c ? R(1) : R(-1); // Im of P_{bc} = ori Im of the stored plane
#pragma unroll
        for (int sbi = 0; sbi < 2; ++sbi) {
            const SymSite py = pm.moved(L, b, sbi == 0 ? d : -d);
            const SymSite pyb = py.moved(L, b, -1);
            const int y = py.lex(L), yb = pyb.lex(L), yc = py.moved(L, c, -1).lex(L), ybc = pyb.moved(L, c, -1).lex(L);
#pragma unroll
            for (int sci = 0; sci < 2; ++sci) {
                // (0, +a)
                C[0] += O[(2 * pa) * SL3 + y];
                C[1] += O[(2 * pa + 1) * SL3 + y];
                // (0, sb b)
                if (sbi == 0) {
                    C[2] += O[(2 * pb) * SL3 + y];
                    C[3] += O[(2 * pb + 1) * SL3 + y];
                } else {
                    C[2] -= O[(2 * pb) * SL3 + yb];
                    C[3] += O[(2 * pb + 1) * SL3 + yb];
                }
                // (0, sc c)
                if (sci == 0) {
                    C[4] += O[(2 * pc) * SL3 + y];
                    C[5] += O[(2 * pc + 1) * SL3 + y];
                } else {
                    C[4] -= O[(2 * pc) * SL3 + yc];
                    C[5] += O[(2 * pc + 1) * SL3 + yc];
                }
                // (sb b, sc c)
                const int q = sbi == 0 ? (sci == 0 ? y : yc) : (sci == 0 ? yb : ybc);
                const R sgn = (sbi == sci) ? ori : -ori;
                C[6] += sgn * O[(2 * pbc) * SL3 + q];
                C[7] += O[(2 * pbc + 1) * SL3 + q];
            }
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    combine_sym_kernel(Geo g, int S, int nd, int slot, const R* __restrict__ o12, R* __restrict__ csym)
{
    const long idx = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long per_axis = static_cast<long>(S) * nd * g.L3;
    if (idx >= 3 * per_axis) return;
    const int a = static_cast<int>(idx / per_axis) + 1;
    long rest = idx - (a - 1) * per_axis;
    const int m = static_cast<int>(rest % g.L3);
    rest /= g.L3;
    const int d = static_cast<int>(rest % nd);
    const int s = static_cast<int>(rest / nd);
    const int L = g.L;
    const SymSite pm{m % L, (m / L) % L, m / (L * L)};
    R C[8];
    frame_sums<R>(L, static_cast<long>(S) * g.L3, o12 + static_cast<long>(s) * g.L3, a, d, pm, C);
    R* out = csym + (((static_cast<long>(slot * 3 + a - 1) * S + s) * nd + d) * g.L3 + pm.axis_major(L, a)) * 8;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) out[ch] = C[ch];
}

// The same frame sums, one block of L^2 threads per (a, s, d, plane): the plane holds the
// axis-major indices [L^2 w, L^2 (w + 1)) of axis a (z = w for a = 1, 2; y = w for a = 3).
// Thread t takes the site with x = t mod L (the channel loads of neighbouring threads are
// neighbours) and v = t / L as its other in-plane coordinate (y for a = 1, the coordinate
// along e_a for a = 2, 3); the block stages the plane's sums in shared memory in axis-major
// order and writes them as one contiguous run of 8 L^2 values.
template <typename R>
__global__ void __launch_bounds__(1024)
    combine_sym_plane_kernel(Geo g, int S, int nd, int slot, const R* __restrict__ o12, R* __restrict__ csym)
{
    extern __shared__ __align__(16) unsigned char tile_raw[];
    R* tile = reinterpret_cast<R*>(tile_raw);
    const int L = g.L, L2 = g.L * g.L;
    int b = static_cast<int>(blockIdx.x); // ((a - 1) S + s) nd + d) L + w
    const int w = b % L;
    b /= L;
    const int d = b % nd;
    b /= nd;
    const int s = b % S;
    const int a = b / S + 1;
    const int t = static_cast<int>(threadIdx.x);
    const int x = t % L, v = t / L;
    const SymSite pm = a == 3 ? SymSite{x, w, v} : SymSite{x, v, w};
    const int il = a == 1 ? x + L * v : v + L * x; // axis-major index within the plane
    R C[8];
    frame_sums<R>(L, static_cast<long>(S) * g.L3, o12 + static_cast<long>(s) * g.L3, a, d, pm, C);
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) tile[il * 8 + ch] = C[ch];
    __syncthreads();
    R* out = csym + (((static_cast<long>(slot * 3 + a - 1) * S + s) * nd + d) * g.L3 + static_cast<long>(L2) * w) * 8;
    for (int e = t; e < 8 * L2; e += blockDim.x) out[e] = tile[e];
}

// Symmetrised contraction over the `count` stored samples, m = x0 + floor(r/2) e_a, sites in
// the axis-major order of a:
//   bsum3[(a-1) nB + (((s R + r-1) nd + d) 8 + ch) L3 + x0] += sum_k T_a,k(s, x0, r) csym_k(a, s, d, m, ch),
// thread per output (a, s, r, d, x0) summing over k in order, blocks ordered as in
// insertion_contract_kernel (a tile of x0 for all (r, d) together); with `first` (the
// level's first chunk) bsum3 is written, not read.
template <typename R>
__global__ void __launch_bounds__(kThreads, kContractMinBlocks)
    insertion_contract_sym_kernel(Geo g, int S, int r_max, int nd, int count, const Cx<R>* __restrict__ tk3,
                                  const R* __restrict__ csym, double2* __restrict__ bsum3, bool first)
{
    const long per_axis = static_cast<long>(S) * r_max * nd * g.L3;
    const int tiles = (g.L3 + kThreads - 1) / kThreads;
    int b = static_cast<int>(blockIdx.x);
    const int d = b % nd;
    b /= nd;
    const int r = b % r_max + 1;
    b /= r_max;
    const int tile = b % tiles;
    b /= tiles;
    const int s = b % S;
    const int a = b / S + 1;
    const int x0 = tile * kThreads + static_cast<int>(threadIdx.x);
    if (x0 >= g.L3) return;
    const int m = axis_major_step(g.L, x0, r / 2);
    InsertionAcc<R> acc[8];
    for (int k = 0; k < count; ++k) {
        const Cx<R> T = tk3[((static_cast<long>(k * 3 + a - 1) * S + s) * r_max + (r - 1)) * g.L3 + x0];
        R C[8];
        Vec8<R>::load(csym + (((static_cast<long>(k * 3 + a - 1) * S + s) * nd + d) * g.L3 + m) * 8, C);
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) acc[ch].add(T, C[ch]);
        if (k % kInsertionBlock == kInsertionBlock - 1)
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) acc[ch].fold();
    }
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) acc[ch].fold();
    const long base = (a - 1) * (per_axis * 8) + (((static_cast<long>(s) * r_max + (r - 1)) * nd + d) * 8) * g.L3 + x0;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        double2 bv = first ? make_double2(0.0, 0.0) : bsum3[base + ch * g.L3];
        bv.x += acc[ch].total_re();
        bv.y += acc[ch].total_im();
        bsum3[base + ch * g.L3] = bv;
    }
}

template <typename R>
cudaError_t launch_measure_sym(const Geo& g, const void* cs, int slab_t, int r_max, int nd, int slot, double2* asum3,
                               void* tk3, void* o12, void* csym, double* osum12, cudaStream_t st)
{
    const int S = g.Nt / slab_t;
    measure_sym_kernel<R><<<blocks_for(4L * S * g.L3), kThreads, 0, st>>>(
        g, static_cast<const cs_t<R>*>(cs), slab_t, r_max, slot, asum3, static_cast<Cx<R>*>(tk3),
        static_cast<R*>(o12), osum12);
    const size_t tile_bytes = static_cast<size_t>(g.L) * g.L * 8 * sizeof(R);
    if (g.L * g.L <= 1024 && tile_bytes <= 48 * 1024)
        combine_sym_plane_kernel<R><<<static_cast<unsigned int>(3L * S * nd * g.L), g.L * g.L, tile_bytes, st>>>(
            g, S, nd, slot, static_cast<const R*>(o12), static_cast<R*>(csym));
    else
        combine_sym_kernel<R><<<blocks_for(3L * S * nd * g.L3), kThreads, 0, st>>>(
            g, S, nd, slot, static_cast<const R*>(o12), static_cast<R*>(csym));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_insertion_contract_sym(const Geo& g, int slab_t, int r_max, int nd, int count, const void* tk3,
                                          const void* csym, double2* bsum3, bool first, cudaStream_t st, bool tiled,
                                          int* status, long long wait_cycles)
{
    const int S = g.Nt / slab_t;
    cudaError_t err = cudaSuccess;
    if (tiled && launch_contract_tiled<R>(g, S, r_max, nd, count, tk3, csym, bsum3, first, status, st, &err, true,
                                          wait_cycles))
        return err;
    const long total = 3L * S * r_max * nd * ((g.L3 + kThreads - 1) / kThreads) * kThreads;
    insertion_contract_sym_kernel<R><<<blocks_for(total), kThreads, 0, st>>>(
        g, S, r_max, nd, count, static_cast<const Cx<R>*>(tk3), static_cast<const R*>(csym), bsum3, first);
    return cudaGetLastError();
}

} // namespace ul
