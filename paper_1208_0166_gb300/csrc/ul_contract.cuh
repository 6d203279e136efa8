// ul_contract.cuh — tiled forms of the deferred insertion contraction: FP32 arithmetic for
// FP32 links, double-single arithmetic for FP64 links.  Included at the end of ul_kernels.cuh.
//
// Paper: arXiv:1208.0166, Section 2.2 (the insertion term of a slab is the slab average of
// T(s,x0,r) times the insertion O at the plaquette x0 + floor(r/2) xhat + d yhat).
//
// The per-sample buffers hold, for every stored sub-sample k, the transporters
// T_k(s, x0, r) and the channel sums O_k(s, site, ch) of every slab.  The contraction is
//   bsum(s, r, d, ch, x0) += sum_k T_k(s, x0, r) O_k(s, x0 + floor(r/2) xhat + d yhat, ch).
// Both shifts stay inside the z-plane of x0 (periodic in x and y), so one block owns
//   one slab s, one z-plane, a tile of `ny` y-rows of that plane (all L x values),
//   one group of two separations (ra, rb) and a subset of `ndb` offsets d,
// and runs over the samples in batches of kInsertionBlock: each batch of transporters (the
// tile's x0, both separations) and channel rows (rows py0 + d0 ... py0 + ny - 1 + d0 +
// ndb - 1 of the plane) is copied into shared memory with cp.async, double-buffered, while
// the previous batch is contracted.  A thread owns the 8 channels of one output (x0, r, d);
// the two separations of a pair sit in neighbouring lanes, so that for the pairs (2,3),
// (4,5), ... (equal shift floor(r/2)) the two lanes read the same channel row (one
// shared-memory access serves both).  The remaining separation 1 pairs with r_max for
// even r_max and is alone for odd r_max.
//
// Per output the arithmetic is that of insertion_contract_kernel<float> (the products of
// the samples in order, blocks of kInsertionBlock folded into a compensated sum, the FP64
// update of bsum), so both forms give the same bits.
#pragma once
#include <atomic>

namespace ul {

// Block shape: at most kContractItems threads (a multiple of 32) and kContractSmem bytes of
// shared memory, so that two blocks share an SM and one block's barriers and FP64 epilogue
// overlap the other's contraction (measured faster than one block of 672 threads per SM).
constexpr int kContractItems = 352, kContractSmem = 110 * 1024, kContractBlocksPerSM = 2;

struct ContractTile {
    int ny = 0, ndb = 0, rows = 0, bs = 0, tpad = 0;
    int threads = 0, smem = 0;
    int ytiles = 0, dsubs = 0, groups = 0;
    bool ok = false;
};

// Tile plan of one launch with at most `max_items` threads and `max_smem` bytes of shared
// memory per block; ok = false where a batch of kInsertionBlock samples does not fit (large
// L with many offsets): the untiled kernel runs instead.
// The second transporter plane of a sample starts tpad floats after the first, so that
// the two lanes of a pair hit different banks (its byte offset is 64 modulo 128).
inline ContractTile contract_tile(const Geo& g, int r_max, int nd, int max_items, int max_smem, bool sym = false)
{
    ContractTile t;
    const int L = g.L;
    const int per_row = 2 * L; // threads per (y-row, offset): two separations x L
    t.ndb = std::min(nd, std::max(1, max_items / per_row));
    t.ny = std::max(1, std::min(L, max_items / (per_row * t.ndb)));
    t.bs = kInsertionBlock;
    auto tpad = [&](int ny) { return ((64 - 8 * L * ny) % 128 + 128) % 128 / 4; };
    // staged channel rows: the rows the offsets reach (single frame), or the tile's rows once
    // per offset (24-frame sums, which are stored per offset)
    auto rows_for = [&](int ny) { return sym ? ny * t.ndb : std::min(L, ny + t.ndb - 1); };
    auto smem_for = [&](int ny) {
        const long rows = rows_for(ny);
        const long per_sample = (4L * L * ny + tpad(ny)) * sizeof(float) // T: (ra, rb) planes of L ny complex
                                + rows * L * 8 * sizeof(float);          // O rows
        return 2 * t.bs * per_sample;
    };
    while (t.ny > 1 && smem_for(t.ny) > max_smem) --t.ny; // fewer y-rows per tile to fit
    t.tpad = tpad(t.ny);
    t.rows = rows_for(t.ny);
    const int items = per_row * t.ny * t.ndb;
    t.threads = (items + 31) / 32 * 32;
    t.smem = static_cast<int>(smem_for(t.ny));
    t.ytiles = (L + t.ny - 1) / t.ny;
    t.dsubs = (nd + t.ndb - 1) / t.ndb;
    t.groups = (r_max + 1) / 2;
    t.ok = items <= max_items && t.smem <= max_smem;
    return t;
}

__device__ __forceinline__ void contract_group(int gi, int r_max, int& ra, int& rb)
{
    const int npairs = (r_max - 1) / 2;
    if (gi < npairs) {
        ra = 2 * gi + 2;
        rb = 2 * gi + 3;
    } else {
        ra = 1;
        rb = (r_max % 2 == 0) ? r_max : 0;
    }
}

__device__ __forceinline__ unsigned int smem_u32(const void* p)
{
    return static_cast<unsigned int>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// one arrival that also announces `bytes` of bulk copies completing on the barrier's phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity)
{
    unsigned int done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

// Waits for the phase `parity` of the barrier, at most about kCopyWaitCycles SM cycles
// (about a second); false when the limit was reached.
constexpr long long kCopyWaitCycles = kCopyWaitLimit;

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned int parity,
                                                  long long limit = kCopyWaitCycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Bulk copy global -> shared memory of this CTA (16-byte aligned addresses, size a multiple
// of 16), completing `bytes` on the barrier.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned int bytes,
                                              unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// One sample of one output: the transporter (re, im) at t, the 8 channels of the shifted
// site at o.
__device__ __forceinline__ void contract_sample(const float* t, const float* o, InsertionAcc<float>* acc)
{
    const float2 tv = *reinterpret_cast<const float2*>(t);
    const float4 lo = *reinterpret_cast<const float4*>(o);
    const float4 hi = *reinterpret_cast<const float4*>(o + 4);
    const Cx<float> T{tv.x, tv.y};
    acc[0].add(T, lo.x);
    acc[1].add(T, lo.y);
    acc[2].add(T, lo.z);
    acc[3].add(T, lo.w);
    acc[4].add(T, hi.x);
    acc[5].add(T, hi.y);
    acc[6].add(T, hi.z);
    acc[7].add(T, hi.w);
}

// The copies of one batch into buffer `buf`, issued by the 32 lanes of one warp (lane j:
// sample k0 + j): per sample the transporter rows of the tile for each separation and the
// staged channel rows (two copies where the rows wrap past L - 1); lane 0 first announces
// the batch's bytes on the buffer's barrier.
// For the 24-frame sums (SYM) the channel part is one copy per offset d of the tile (ndv
// offsets, o_ds floats apart in global memory, blk floats apart in shared memory).
template <bool SYM>
__device__ __forceinline__ void issue_batch(float* smem, unsigned long long* bars, int k0, int buf, int nb, int bufsz,
                                            int tsz, int osz, int o_at, int tplane, int nr,
                                            const Cx<float>* tsrc0, long t_db, long t_ks, unsigned int t_bytes,
                                            const float* osrc0, long o_ks, int row0, int n1, int rows, int L,
                                            unsigned int o_bytes, int ndv, long o_ds, int blk,
                                            unsigned int extra_tx = 0)
{
    float* base = smem + buf * bufsz;
    const int lane = static_cast<int>(threadIdx.x) & 31;
    if (lane == 0) mbar_arrive_expect_tx(&bars[buf], (nr * t_bytes + o_bytes) * nb + extra_tx);
    __syncwarp();
    for (int j = lane; j < nb; j += 32) {
        const long k = k0 + j;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const Cx<float>* ts = tsrc0 + k * t_ks;
        bulk_copy_g2s(base + j * tsz, ts, t_bytes, &bars[buf]);
        if (nr == 2) bulk_copy_g2s(base + j * tsz + tplane, ts + t_db, t_bytes, &bars[buf]);
        const float* os = osrc0 + k * o_ks;
        float* od = base + o_at + j * osz;
        if constexpr (SYM) {
            for (int q = 0; q < ndv; ++q) bulk_copy_g2s(od + q * blk, os + q * o_ds, o_bytes / ndv, &bars[buf]);
        } else {
            const unsigned int seg1 = static_cast<unsigned int>(n1 * L * 8 * sizeof(float));
            bulk_copy_g2s(od, os + static_cast<long>(row0) * L * 8, seg1, &bars[buf]);
            if (n1 < rows) bulk_copy_g2s(od + n1 * L * 8, os, o_bytes - seg1, &bars[buf]);
        }
    }
}

// Shared memory of one batch buffer (floats):
//   T[j][ri][x0l] complex, j < kInsertionBlock, ri < 2, x0l < L ny   (4 L ny + tpad floats per
//                          sample; plane ri = 1 starts 2 L ny + tpad floats after plane 0)
//   O[j][rl][x][ch],       rl < rows, x < L, ch < 8                  (8 rows L floats per sample)
// The two lanes of a pair read the same O site (one access); eight lanes read four sites 32
// bytes apart, one 128-byte line, so the 128-bit loads need no swizzle.
// SYM: the 24-frame estimator.  Sites of one separation axis a are in that axis's
// axis-major order (the midpoint shift runs along the rows, "x" below), the channel part is
// the frame sums of each offset d of the tile (O[j][dl][y-row][x][ch], ny rows per offset),
// tk and ok hold the three axes per sample, and the grid has the axis slowest.
template <typename R, bool SYM>
__global__ void __launch_bounds__(kContractItems, kContractBlocksPerSM)
    insertion_contract_tiled_kernel(Geo g, int S, int r_max, int nd, int count, ContractTile t,
                                    const Cx<float>* __restrict__ tk, const float* __restrict__ ok,
                                    double2* __restrict__ bsum, bool first, int* __restrict__ status,
                                    long long wait_cycles)
{
    // wait_cycles < 0: the timeout test.  The first batch's barrier then expects 16 bytes
    // more than its copies deliver, so its phase cannot complete: the first wait gives up
    // after -wait_cycles cycles, the block reports status 2, waits (the full limit) while the
    // copies it issued land, and leaves.
    const bool stall_test = wait_cycles < 0;
    const long long first_wait = stall_test ? -wait_cycles : wait_cycles;
    extern __shared__ __align__(16) float smem[];
    __shared__ unsigned long long bars[2];
    constexpr int BS = kInsertionBlock;
    const int L = g.L, L2 = g.L * g.L;
    // block -> (axis, s, pz, ytile, group, dsub), dsub fastest: the blocks of one plane run together
    int b = static_cast<int>(blockIdx.x);
    const int blocks_per_axis = S * L * t.ytiles * t.groups * t.dsubs;
    const int ax = SYM ? b / blocks_per_axis : 0; // separation axis - 1
    b -= ax * blocks_per_axis;
    const int dsub = b % t.dsubs;
    b /= t.dsubs;
    const int gi = b % t.groups;
    b /= t.groups;
    const int ytile = b % t.ytiles;
    b /= t.ytiles;
    const int pz = b % L;
    const int s = b / L;
    int ra, rb;
    contract_group(gi, r_max, ra, rb);
    const int nr = rb ? 2 : 1;
    const int py0 = ytile * t.ny, d0 = dsub * t.ndb;
    const int nyv = min(t.ny, L - py0);          // y-rows of this tile
    const int XT = L * t.ny;                     // x0 slots per staged sample
    const int row0 = (py0 + d0) % L;             // first staged channel row
    const int tsz = XT * 4 + t.tpad, osz = t.rows * L * 8; // floats per staged sample
    const int bufsz = BS * (tsz + osz);          // floats per batch buffer: T then O
    const long plane = static_cast<long>(L2) * pz;

    // this thread's output (x0, r, d): separation fastest, then x, y-row, offset
    const int tid = static_cast<int>(threadIdx.x);
    const int ri = tid & 1, item = tid >> 1;
    const int px = item % L, pyl = (item / L) % t.ny, dl = item / (L * t.ny);
    const int r = ri ? rb : ra;
    const bool active = item < L * t.ny * t.ndb && r != 0 && pyl < nyv && d0 + dl < nd;
    const int toff = ri * (2 * XT + t.tpad) + 2 * (px + L * pyl);         // transporter in a staged sample
    const int ooff = SYM ? ((dl * t.ny + pyl) * L + (px + r / 2) % L) * 8    // frame sums of offset dl
                         : (((pyl + dl) % L) * L + (px + r / 2) % L) * 8; // shifted channel site

    // batch copies, issued by the lanes of warp 0 (lane j: sample j of the batch)
    const int n1 = min(t.rows, L - row0); // staged rows before the wrap to row 0
    const unsigned int t_bytes = static_cast<unsigned int>(nyv * L * sizeof(Cx<float>));
    const int ndv = min(t.ndb, nd - d0); // offsets of this block (SYM)
    const unsigned int o_bytes = static_cast<unsigned int>((SYM ? ndv * nyv : t.rows) * L * 8 * sizeof(float));
    const int na = SYM ? 3 : 1;             // separation axes per stored sample
    const long sa = static_cast<long>(ax) * S + s;
    const Cx<float>* tsrc0 = tk + (sa * r_max + (ra - 1)) * g.L3 + plane + static_cast<long>(L) * py0;
    const long t_db = static_cast<long>(rb - ra) * g.L3;         // second separation's plane
    const long t_ks = static_cast<long>(na) * S * r_max * g.L3;  // per sample (complex)
    const float* osrc0 = SYM ? ok + ((sa * nd + d0) * g.L3 + plane + static_cast<long>(L) * py0) * 8
                             : ok + (static_cast<long>(s) * g.L3 + plane) * 8;
    const long o_ks = static_cast<long>(na) * S * (SYM ? nd : 1) * g.L3 * 8; // per sample (floats)
    const long o_ds = static_cast<long>(g.L3) * 8;                          // per offset (SYM)
    const int tplane = 2 * XT + t.tpad;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // this thread's outputs bsum[out + ch L3]
    const long out = (((sa * r_max + (r - 1)) * nd + d0 + dl) * 8) * g.L3 + px + L * (py0 + pyl) + plane;
    InsertionAcc<float> acc[8];
    const int nbatch = (count + BS - 1) / BS;
    if (tid < 32)
        issue_batch<SYM>(smem, bars, 0, 0, min(BS, count), bufsz, tsz, osz, BS * tsz, tplane, nr, tsrc0, t_db, t_ks,
                         t_bytes, osrc0, o_ks, row0, n1, t.rows, L, o_bytes, ndv, o_ds, t.ny * L * 8,
                         stall_test ? 16u : 0u);
    for (int bi = 0; bi < nbatch; ++bi) {
        const int buf = bi & 1;
        const int k0 = bi * BS;
        const int nb = min(BS, count - k0);
        // the other buffer was last read in batch bi - 1, which every thread has finished
        if (bi + 1 < nbatch && tid < 32)
            issue_batch<SYM>(smem, bars, k0 + BS, buf ^ 1, min(BS, count - k0 - BS), bufsz, tsz, osz, BS * tsz, tplane,
                             nr, tsrc0, t_db, t_ks, t_bytes, osrc0, o_ks, row0, n1, t.rows, L, o_bytes, ndv, o_ds,
                             t.ny * L * 8);
        // the last batch: bring this thread's FP64 sums into L2 for the epilogue
        if (bi + 1 == nbatch && active && !first) {
#pragma unroll
            for (int ch = 0; ch < 8; ++ch)
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(bsum + out + ch * g.L3));
        }
        const bool arrived = mbar_wait_bounded(&bars[buf], (bi >> 1) & 1, first_wait);
        if (__syncthreads_or(!arrived)) {
            // a copy did not complete in time: report it, give the copies in flight a bounded
            // wait (the full limit, whatever wait_cycles is) so that none lands after the
            // block has left, and stop
            if (tid == 0) {
                atomicExch(status, 2);
                mbar_wait_bounded(&bars[buf], (bi >> 1) & 1);
                if (bi + 1 < nbatch) mbar_wait_bounded(&bars[buf ^ 1], ((bi + 1) >> 1) & 1);
            }
            return;
        }
        if (active) {
            const float* sT = smem + buf * bufsz + toff;
            const float* sO = smem + buf * bufsz + BS * tsz + ooff;
            if (nb == BS) {
                // a whole block of kInsertionBlock samples (k0 is a multiple of it): fold after it
#pragma unroll
                for (int j = 0; j < BS; ++j) contract_sample(sT + j * tsz, sO + j * osz, acc);
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) acc[ch].fold();
            } else {
                for (int j = 0; j < nb; ++j) contract_sample(sT + j * tsz, sO + j * osz, acc);
            }
        }
        __syncthreads(); // the next batch overwrites this buffer
    }
    if (!active) return;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) acc[ch].fold();
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        double2 v = first ? make_double2(0.0, 0.0) : bsum[out + ch * g.L3];
        v.x += acc[ch].total_re();
        v.y += acc[ch].total_im();
        bsum[out + ch * g.L3] = v;
    }
}

// ---------------------------------------------------------------------------
// FP64 links: the same contraction over the double-single samples (SampleStore<double>),
// in double-single arithmetic on the FP32 pipes.  A product a b of a = ah + al and
// b = bh + bl is p = fl(ah bh) plus e = (ah bh - p) + ah bl + al bh (the first term exact by
// a fused multiply-add; al bl, below 2^-46 |ah bh|, is left out), so with the 2^-48
// representation error of each factor a term is within 2^-44 |a b|.  The running sum is a
// pair (s, c): s takes p by an error-free two-sum whose error, with e, goes to c; after
// each staged batch the pair is renormalised by a two-sum, so |c| stays near 2^-24 |s| and
// a chunk of n samples is summed within (n 2^-48 + 2^-43) sum |T O|.  Once per output the
// pair is widened to FP64 (exactly, by integer operations) and added into bsum.  Same tiles,
// copies and bounded waits as the FP32 form; a value takes two floats, so a staged batch
// holds kDsBatch samples.  The real and imaginary parts run as the two lanes of paired FP32
// instructions.
// ---------------------------------------------------------------------------
constexpr int kDsBatch = 4;
// Threads per block of the double-single kernel (2 L ny ndb, at most kDsItems): 96-thread
// blocks measured faster alone than 352-thread ones (2.75 against 2.88 ms for 32 samples at
// 24^4: more blocks resident, fewer warps per batch barrier), and fit beside the FP64 class
// updates of the next chunk (a full 24^4 class holds about 50 K of an SM's 64 K registers).
constexpr int kDsItems = 96;

// Paired FP32 arithmetic on (re, im) lanes (FFMA2 / FADD2 / FMUL2: two IEEE single
// operations per instruction, each lane rounded as the scalar operation would be).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

// Running double-single sums of the real and imaginary parts of one output channel.
struct DsSum2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    // (s + c) += (ah + al)(bh + bl) in each lane
    __device__ __forceinline__ void add_prod(float2 ah, float2 al, float2 bh, float2 bl)
    {
        const float2 p = __fmul2_rn(ah, bh);
        float2 e = __ffma2_rn(ah, bh, neg2(p));
        e = __ffma2_rn(ah, bl, e);
        e = __ffma2_rn(al, bh, e);
        const float2 t = __fadd2_rn(s, p);
        const float2 z = sub2(t, s);
        const float2 err = __fadd2_rn(sub2(s, sub2(t, z)), sub2(p, z));
        s = t;
        c = __fadd2_rn(c, __fadd2_rn(err, e));
    }
    __device__ __forceinline__ void renormalise()
    {
        const float2 t = __fadd2_rn(s, c);
        const float2 z = sub2(t, s);
        c = __fadd2_rn(sub2(s, sub2(t, z)), sub2(c, z));
        s = t;
    }
    // bsum + s + c in FP64 per lane; the widening of s and c to FP64 is exact and done by
    // integer operations (a part below 2^-126 counts as 0), leaving two FP64 additions
    __device__ __forceinline__ double2 added_to(double2 b) const
    {
        return make_double2((b.x + widen(s.x)) + widen(c.x), (b.y + widen(s.y)) + widen(c.y));
    }
    static __device__ __forceinline__ double widen(float x)
    {
        const unsigned int u = __float_as_uint(x);
        const unsigned int e = (u >> 23) & 0xffu;
        if (e == 0) return 0.0;
        const unsigned int hi = (u & 0x80000000u) | ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
    }
};

// Tile plan of the double-single form (see contract_tile): 16 bytes per staged transporter,
// 64 per staged channel site.
inline ContractTile contract_tile_ds(const Geo& g, int r_max, int nd, int max_items, int max_smem)
{
    ContractTile t;
    const int L = g.L;
    const int per_row = 2 * L;
    t.ndb = std::min(nd, std::max(1, max_items / per_row));
    t.ny = std::max(1, std::min(L, max_items / (per_row * t.ndb)));
    t.bs = kDsBatch;
    auto tpad = [&](int ny) { return ((64 - 16 * L * ny) % 128 + 128) % 128 / 4; };
    auto rows_for = [&](int ny) { return std::min(L, ny + t.ndb - 1); };
    auto smem_for = [&](int ny) {
        const long per_sample = (8L * L * ny + tpad(ny) + 16L * rows_for(ny) * L) * sizeof(float);
        return 2 * t.bs * per_sample;
    };
    while (t.ny > 1 && smem_for(t.ny) > max_smem) --t.ny;
    t.tpad = tpad(t.ny);
    t.rows = rows_for(t.ny);
    const int items = per_row * t.ny * t.ndb;
    t.threads = (items + 31) / 32 * 32;
    t.smem = static_cast<int>(smem_for(t.ny));
    t.ytiles = (L + t.ny - 1) / t.ny;
    t.dsubs = (nd + t.ndb - 1) / t.ndb;
    t.groups = (r_max + 1) / 2;
    t.ok = items <= max_items && t.smem <= max_smem;
    return t;
}

// Shared memory of one batch buffer (floats):
//   T[j][ri][x0l] float4 {re hi, im hi, re lo, im lo}   (plane ri = 1 starts 4 L ny + tpad
//                                                        floats after plane 0)
//   O[j][rl][q][x] float4, part q of the channel pairs   (16 L floats per row)
// Eight lanes of a 128-bit load read four consecutive sites of one part (64 contiguous
// bytes) or the two transporter planes (64 bytes apart modulo 128): no bank conflicts.
template <typename R> // double: the kernel of the FP64 links
__global__ void __launch_bounds__(kContractItems, kContractBlocksPerSM)
    insertion_contract_ds_kernel(Geo g, int S, int r_max, int nd, int count, ContractTile t,
                                 const float4* __restrict__ tk, const float4* __restrict__ ok,
                                 double2* __restrict__ bsum, bool first, int* __restrict__ status,
                                 long long wait_cycles)
{
    const bool stall_test = wait_cycles < 0;
    const long long first_wait = stall_test ? -wait_cycles : wait_cycles;
    extern __shared__ __align__(16) float smem[];
    __shared__ unsigned long long bars[2];
    constexpr int BS = kDsBatch;
    const int L = g.L, L2 = g.L * g.L;
    int b = static_cast<int>(blockIdx.x);
    const int dsub = b % t.dsubs;
    b /= t.dsubs;
    const int gi = b % t.groups;
    b /= t.groups;
    const int ytile = b % t.ytiles;
    b /= t.ytiles;
    const int pz = b % L;
    const int s = b / L;
    int ra, rb;
    contract_group(gi, r_max, ra, rb);
    const int nr = rb ? 2 : 1;
    const int py0 = ytile * t.ny, d0 = dsub * t.ndb;
    const int nyv = min(t.ny, L - py0);
    const int XT = L * t.ny;
    const int row0 = (py0 + d0) % L;
    const int tplane = 4 * XT + t.tpad;
    const int tsz = 8 * XT + t.tpad, osz = t.rows * L * 16;
    const int bufsz = BS * (tsz + osz);
    const long plane = static_cast<long>(L2) * pz;

    const int tid = static_cast<int>(threadIdx.x);
    const int ri = tid & 1, item = tid >> 1;
    const int px = item % L, pyl = (item / L) % t.ny, dl = item / (L * t.ny);
    const int r = ri ? rb : ra;
    const bool active = item < L * t.ny * t.ndb && r != 0 && pyl < nyv && d0 + dl < nd;
    const int toff = ri * tplane + 4 * (px + L * pyl);
    const int ooff = ((pyl + dl) % L) * L * 16 + ((px + r / 2) % L) * 4;

    const int n1 = min(t.rows, L - row0);
    const unsigned int t_bytes = static_cast<unsigned int>(nyv * L * sizeof(float4));
    const unsigned int o_bytes = static_cast<unsigned int>(t.rows * L * 4 * sizeof(float4));
    const float4* tsrc0 = tk + (static_cast<long>(s) * r_max + (ra - 1)) * g.L3 + plane + static_cast<long>(L) * py0;
    const long t_db = static_cast<long>(rb - ra) * g.L3;
    const long t_ks = static_cast<long>(S) * r_max * g.L3;       // float4 per sample
    const float4* osrc0 = ok + (static_cast<long>(s) * g.L3 + plane) * 4;
    const long o_ks = static_cast<long>(S) * g.L3 * 4;          // float4 per sample
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // copies of one batch into buffer buf by the lanes of warp 0 (lane j: sample k0 + j)
    auto issue = [&](int k0, int buf, int nb, unsigned int extra_tx) {
        float* base = smem + buf * bufsz;
        const int lane = tid & 31;
        if (lane == 0) mbar_arrive_expect_tx(&bars[buf], (nr * t_bytes + o_bytes) * nb + extra_tx);
        __syncwarp();
        for (int j = lane; j < nb; j += 32) {
            const long k = k0 + j;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            const float4* ts = tsrc0 + k * t_ks;
            bulk_copy_g2s(base + j * tsz, ts, t_bytes, &bars[buf]);
            if (nr == 2) bulk_copy_g2s(base + j * tsz + tplane, ts + t_db, t_bytes, &bars[buf]);
            const float4* os = osrc0 + k * o_ks;
            float* od = base + BS * tsz + j * osz;
            const unsigned int seg1 = static_cast<unsigned int>(n1 * L * 4 * sizeof(float4));
            bulk_copy_g2s(od, os + static_cast<long>(row0) * L * 4, seg1, &bars[buf]);
            if (n1 < t.rows) bulk_copy_g2s(od + n1 * L * 16, os, o_bytes - seg1, &bars[buf]);
        }
    };

    const long out = (((static_cast<long>(s) * r_max + (r - 1)) * nd + d0 + dl) * 8) * g.L3 + px + L * (py0 + pyl) + plane;
    DsSum2 acc[8];
    const int nbatch = (count + BS - 1) / BS;
    if (tid < 32) issue(0, 0, min(BS, count), stall_test ? 16u : 0u);
    for (int bi = 0; bi < nbatch; ++bi) {
        const int buf = bi & 1;
        const int k0 = bi * BS;
        const int nb = min(BS, count - k0);
        if (bi + 1 < nbatch && tid < 32) issue(k0 + BS, buf ^ 1, min(BS, count - k0 - BS), 0u);
        if (bi + 1 == nbatch && active && !first) {
#pragma unroll
            for (int ch = 0; ch < 8; ++ch)
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(bsum + out + ch * g.L3));
        }
        const bool arrived = mbar_wait_bounded(&bars[buf], (bi >> 1) & 1, first_wait);
        if (__syncthreads_or(!arrived)) {
            if (tid == 0) {
                atomicExch(status, 2);
                mbar_wait_bounded(&bars[buf], (bi >> 1) & 1);
                if (bi + 1 < nbatch) mbar_wait_bounded(&bars[buf ^ 1], ((bi + 1) >> 1) & 1);
            }
            return;
        }
        if (active) {
            const float* sT = smem + buf * bufsz + toff;
            const float* sO = smem + buf * bufsz + BS * tsz + ooff;
            auto sample = [&](int j) {
                const float4 tv = *reinterpret_cast<const float4*>(sT + j * tsz);
                const float* o = sO + j * osz;
                const float4 h0 = *reinterpret_cast<const float4*>(o);
                const float4 h1 = *reinterpret_cast<const float4*>(o + 4 * L);
                const float4 l0 = *reinterpret_cast<const float4*>(o + 8 * L);
                const float4 l1 = *reinterpret_cast<const float4*>(o + 12 * L);
                const float oh[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
                const float ol[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
                const float2 th = make_float2(tv.x, tv.y), tl = make_float2(tv.z, tv.w);
#pragma unroll
                for (int ch = 0; ch < 8; ++ch)
                    acc[ch].add_prod(th, tl, make_float2(oh[ch], oh[ch]), make_float2(ol[ch], ol[ch]));
            };
            if (nb == BS) {
#pragma unroll
                for (int j = 0; j < BS; ++j) sample(j);
            } else {
                for (int j = 0; j < nb; ++j) sample(j);
            }
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) acc[ch].renormalise();
        }
        __syncthreads(); // the next batch overwrites this buffer
    }
    if (!active) return;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        const double2 v = first ? make_double2(0.0, 0.0) : bsum[out + ch * g.L3];
        bsum[out + ch * g.L3] = acc[ch].added_to(v);
    }
}

// set (per link precision) once the shared-memory limit has been raised: until then a tile
// that needs more than the default 48 KB runs as the untiled kernel
template <typename R>
inline std::atomic<bool> g_contract_prepared{false};

template <typename R>
cudaError_t prepare_insertion_contract()
{
    if constexpr (sizeof(R) == 8) {
        const cudaError_t e = cudaFuncSetAttribute(insertion_contract_ds_kernel<double>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        if (e == cudaSuccess) g_contract_prepared<R>.store(true);
        return e;
    } else {
        cudaError_t e = cudaFuncSetAttribute(insertion_contract_tiled_kernel<float, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(insertion_contract_tiled_kernel<float, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        if (e == cudaSuccess) g_contract_prepared<R>.store(true);
        return e;
    }
    return cudaSuccess;
}

// Launches the tiled form: for FP32 links the FP32 kernel (sym: the 24-frame sums of three
// axes), for FP64 links the double-single kernel (single-frame sums only); returns false
// (nothing launched) where it does not apply, and the caller runs the untiled kernel.
template <typename R>
bool launch_contract_tiled(const Geo& g, int S, int r_max, int nd, int count, const void* tk, const void* ok,
                           double2* bsum, bool first, int* status, cudaStream_t st, cudaError_t* err, bool sym,
                           long long wait_cycles)
{
    if constexpr (sizeof(R) == 8) {
        const ContractTile t = contract_tile_ds(g, r_max, nd, kDsItems, kContractSmem);
        if (sym || !t.ok || count < 1 || (t.smem > 48 * 1024 && !g_contract_prepared<R>.load())) return false;
        const long blocks = static_cast<long>(S) * g.L * t.ytiles * t.groups * t.dsubs;
        insertion_contract_ds_kernel<double><<<static_cast<unsigned int>(blocks), t.threads, t.smem, st>>>(
            g, S, r_max, nd, count, t, static_cast<const float4*>(tk), static_cast<const float4*>(ok), bsum, first,
            status, wait_cycles);
        *err = cudaGetLastError();
        return true;
    } else {
        const ContractTile t = contract_tile(g, r_max, nd, kContractItems, kContractSmem, sym);
        if (!t.ok || count < 1 || (t.smem > 48 * 1024 && !g_contract_prepared<R>.load())) return false;
        const long blocks = static_cast<long>(sym ? 3 : 1) * S * g.L * t.ytiles * t.groups * t.dsubs;
        const auto* tkf = static_cast<const Cx<float>*>(tk);
        const auto* okf = static_cast<const float*>(ok);
        if (sym)
            insertion_contract_tiled_kernel<float, true><<<static_cast<unsigned int>(blocks), t.threads, t.smem, st>>>(
                g, S, r_max, nd, count, t, tkf, okf, bsum, first, status, wait_cycles);
        else
            insertion_contract_tiled_kernel<float, false><<<static_cast<unsigned int>(blocks), t.threads, t.smem, st>>>(
                g, S, r_max, nd, count, t, tkf, okf, bsum, first, status, wait_cycles);
        *err = cudaGetLastError();
        return true;
    }
}

} // namespace ul
