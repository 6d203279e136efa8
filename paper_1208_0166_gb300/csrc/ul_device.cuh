// ul_device.cuh — lattice geometry in the device layout and the Philox4x64-10 generator.
//
// Device layout of link data: [mu][parity][h] with h = i >> 1 the half index of the
// lexicographic site i = x + L*(y + L*(z + L*t)).  With L even, the two sites 2h and
// 2h+1 of a row have opposite parity, so (parity, h) enumerates each parity class
// densely and the threads of one class read and write contiguous memory.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ul {

// ---------------------------------------------------------------------------
// Bounds-checked build (compiled with -DUL_CHECK, library libul_check.so).  Every index
// passed through UL_IDX is compared with the extent of the array it addresses; an index
// out of range is recorded in this translation unit's check word (the first one only:
// bit 63 set, bits 48..55 the site's tag, bits 0..47 the index) and replaced by 0, so
// the access stays inside the array and the kernel runs on: no trap, no fault.  The host
// reads the words with ul_check_status.  In the default build UL_IDX is the index itself.
// ---------------------------------------------------------------------------
enum : unsigned {
    kChkLinkOffset = 1,  // link_offset: (mu, site) of a link array
    kChkNeighbour = 2,   // a staple's neighbour site index
    kChkStaple = 3,      // a staple's neighbour link offset
    kChkOwnLink = 4,     // the updated link's own offset
    kChkSlabGlobal = 5,  // slab kernel: global link offset
    kChkAsum = 6,        // measurement: transporter accumulator
    kChkSample = 7,      // measurement: stored sample (slab, separation, site)
    kChkOsum = 8,        // measurement: channel sums
};

#ifdef UL_CHECK
static __device__ unsigned long long g_ul_check_word; // one per translation unit
__device__ __forceinline__ long long ul_checked_index(long long idx, long long n, unsigned tag)
{
    if (idx >= 0 && idx < n) return idx;
    atomicCAS(&g_ul_check_word, 0ull,
              (1ull << 63) | (static_cast<unsigned long long>(tag & 0xffu) << 48) |
                  (static_cast<unsigned long long>(idx) & 0xffffffffffffull));
    return 0;
}
#define UL_IDX(idx, n, tag) ::ul::ul_checked_index((idx), (n), (tag))
#else
#define UL_IDX(idx, n, tag) (idx)
#endif

struct Geo {
    int L, Nt;  // extent of x, y, z and of t
    int Lh;     // L / 2
    int L3;     // L^3 spatial sites
    int V;      // L^3 Nt sites
    int Vh;     // V / 2 sites per parity
};

// Coordinates indexed by direction: c[0] = t, c[1] = x, c[2] = y, c[3] = z.
struct Site {
    int c[4];
};

__device__ __forceinline__ Site site_from_half(const Geo& g, int parity, int h)
{
    const int row = h / g.Lh;
    const int xh = h - row * g.Lh;
    const int y = row % g.L;
    const int rest = row / g.L;
    const int z = rest % g.L;
    const int t = rest / g.L;
    Site s;
    s.c[0] = t;
    s.c[2] = y;
    s.c[3] = z;
    s.c[1] = 2 * xh + ((parity + y + z + t) & 1);
    return s;
}

__device__ __forceinline__ int lex_index(const Geo& g, const Site& s)
{
    return s.c[1] + g.L * (s.c[2] + g.L * (s.c[3] + g.L * s.c[0]));
}

__device__ __forceinline__ int site_parity(const Site& s) { return (s.c[0] + s.c[1] + s.c[2] + s.c[3]) & 1; }

__device__ __forceinline__ Site site_step(const Geo& g, Site s, int d, int delta)
{
    const int n = d == 0 ? g.Nt : g.L;
    int v = s.c[d] + delta;
    v = v < 0 ? v + n : (v >= n ? v - n : v);
    s.c[d] = v;
    return s;
}

// Offset of link (mu, s) in a [mu][parity][h] array.
__device__ __forceinline__ int link_offset(const Geo& g, int mu, const Site& s)
{
    return static_cast<int>(UL_IDX((mu * 2 + site_parity(s)) * g.Vh + (lex_index(g, s) >> 1), 8LL * g.Vh,
                                   kChkLinkOffset));
}

// Site from a lexicographic index.
__device__ __forceinline__ Site site_from_lex(const Geo& g, int i)
{
    Site s;
    s.c[1] = i % g.L;
    int r = i / g.L;
    s.c[2] = r % g.L;
    r /= g.L;
    s.c[3] = r % g.L;
    s.c[0] = r / g.L;
    return s;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications
// with a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
struct Philox4 {
    uint64_t w[4];
};

__device__ __forceinline__ Philox4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                  uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ULL;
    constexpr uint64_t kMulB = 0xCA5A826395121157ULL;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ULL;
    constexpr uint64_t kWeylB = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t hiA = __umul64hi(kMulA, c0), loA = kMulA * c0;
        const uint64_t hiB = __umul64hi(kMulB, c2), loB = kMulB * c2;
        const uint64_t n0 = hiB ^ c1 ^ k0;
        const uint64_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    Philox4 r;
    r.w[0] = c0;
    r.w[1] = c1;
    r.w[2] = c2;
    r.w[3] = c3;
    return r;
}

// Philox4x32-10 (same paper): ten rounds of two 32x32->64 multiplications, 32-bit Weyl key
// schedule; used for the Metropolis uniforms of the FP32 path, which need 48 random bits.
struct Philox4x32 {
    uint32_t w[4];
};

__device__ __forceinline__ Philox4x32 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                     uint32_t k1)
{
    constexpr uint32_t kMulA = 0xD2511F53u;
    constexpr uint32_t kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u;
    constexpr uint32_t kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    Philox4x32 r;
    r.w[0] = c0;
    r.w[1] = c1;
    r.w[2] = c2;
    r.w[3] = c3;
    return r;
}

// Philox stream ids (second key word of Philox4x64, fourth counter word of Philox4x32)
enum : uint64_t { kStreamHotStart = 0, kStreamMetropolis = 1 };

} // namespace ul
