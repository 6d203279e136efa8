/*
 * Plain, slow CPU oracle (FP64) for the multilevel U(1) hot path of arXiv:1208.0166.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark.  It is written straight from the paper's
 * definitions with no blocking, fusion or reordering, and shares no code with
 * the CUDA path.  Every link variable is formed as U = cos(theta) + i sin(theta)
 * and every product is the complex product the paper writes down.
 *
 * Paper passages followed:
 *   Section 2 (Wilson action):     beta S = beta sum_x sum_{mu<nu} [1 - Re U_mu nu(x)],
 *                                  U_mu nu(x) = U_mu(x) U_nu(x+mu) U*_mu(x+nu) U*_nu(x)
 *   Section 2.1 (Configurations):  Metropolis + overrelaxation updates
 *   Section 2.2 (Multilevel):      time layers whose spatial boundary links are held fixed, updates of the rest;
 *                                  V(r) = -(1/Nt) ln <P*(0) P(r)>;
 *                                  insertion operator O(x0,x,t,r) = U*_0(x0,t) U_0(x0+r,t) O(x,t);
 *                                  TO^(2) = T(t) O(t+1) + O(t) T(t+1);
 *                                  <P* P O(x)> = (1/V) sum_x0 sum_t < products over slabs >.
 */
#include "ul_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Elementary functions with a fixed operation sequence.                     */
/*                                                                           */
/* The update dynamics is chaotic: a one-ulp difference in any cos/sin grows */
/* to O(1e-4) rad within one compound sweep.  An independent device         */
/* implementation can only be compared link by link if both evaluate the    */
/* same IEEE operations, so sin/cos/exp/atan2 are written here from          */
/* published methods instead of taken from libm:                             */
/*   - sin/cos: additive range reduction by pi/2 with a three-part constant  */
/*     (W. J. Cody, W. Waite, "Software Manual for the Elementary Functions",*/
/*     1980), Taylor series on [-pi/4, pi/4] evaluated by Horner's rule;     */
/*   - exp: reduction by ln 2 (same method), Taylor series on                */
/*     [-ln2/2, ln2/2], scaling by 2^k;                                      */
/*   - atan2: octant reduction to t in [0,1], t = j/8 + u with the addition */
/*     formula atan(t) = atan(j/8) + atan((t-j/8)/(1+t j/8)), Taylor series  */
/*     of atan on |u| <= 1/16.                                               */
/* Every fused multiply-add is written as fma(); the file is compiled with   */
/* floating-point contraction off.  The constants are pi/2, ln 2 and         */
/* atan(j/8) split into a double and its rounding remainder.                 */
/* ------------------------------------------------------------------------ */

static const double PIO2_1 = 0x1.921fb54442d18p+0;   /* double(pi/2) */
static const double PIO2_2 = 0x1.1a62633145c07p-54;  /* double(pi/2 - PIO2_1) */
static const double PIO2_3 = -0x1.f1976b7ed8fbcp-110; /* double(pi/2 - PIO2_1 - PIO2_2) */
static const double INV_PIO2 = 0x1.45f306dc9c883p-1; /* double(2/pi) */
static const double PI_D = 0x1.921fb54442d18p+1;     /* double(pi) */
static const double LN2_HI = 0x1.62e42fefa39efp-1;   /* double(ln 2) */
static const double LN2_LO = 0x1.abc9e3b39803fp-56;  /* double(ln 2 - LN2_HI) */
static const double INV_LN2 = 0x1.71547652b82fep+0;  /* double(1/ln 2) */
/* atan(j/8), j = 0..8, as double + remainder */
static const double ATAN_J8_HI[9] = {
    0.0,
    0x1.fd5ba9aac2f6ep-4, 0x1.f5b75f92c80ddp-3, 0x1.6f61941e4def1p-2, 0x1.dac670561bb4fp-2,
    0x1.1e00babdefeb4p-1, 0x1.4978fa3269ee1p-1, 0x1.700a7c5784634p-1, 0x1.921fb54442d18p-1};
static const double ATAN_J8_LO[9] = {
    0.0,
    -0x1.cd37686760c17p-59, 0x1.8ab6e3cf7afbdp-57, -0x1.c63aae6f6e918p-56, 0x1.a2b7f222f65e2p-56,
    -0x1.928df287a668fp-58, 0x1.2419a87f2a458p-56, -0x1.8c34d25aadef6p-56, 0x1.1a62633145c07p-55};

void ulo_sincos(double x, double* s_out, double* c_out)
{
    double k = rint(x * INV_PIO2);
    double r = fma(-k, PIO2_1, x);
    r = fma(-k, PIO2_2, r);
    r = fma(-k, PIO2_3, r);
    double z = r * r;
    /* sin r = r + r z (-1/3! + z (1/5! - ... + z 1/17!)) */
    double ps = 1.0 / 355687428096000.0;     /* 1/17! */
    ps = fma(ps, z, -1.0 / 1307674368000.0); /* 1/15! */
    ps = fma(ps, z, 1.0 / 6227020800.0);     /* 1/13! */
    ps = fma(ps, z, -1.0 / 39916800.0);      /* 1/11! */
    ps = fma(ps, z, 1.0 / 362880.0);         /* 1/9! */
    ps = fma(ps, z, -1.0 / 5040.0);          /* 1/7! */
    ps = fma(ps, z, 1.0 / 120.0);            /* 1/5! */
    ps = fma(ps, z, -1.0 / 6.0);             /* 1/3! */
    double sn = fma(r * z, ps, r);
    /* cos r = 1 + z (-1/2! + z (1/4! - ... + z 1/16!)) */
    double pc = 1.0 / 20922789888000.0;      /* 1/16! */
    pc = fma(pc, z, -1.0 / 87178291200.0);   /* 1/14! */
    pc = fma(pc, z, 1.0 / 479001600.0);      /* 1/12! */
    pc = fma(pc, z, -1.0 / 3628800.0);       /* 1/10! */
    pc = fma(pc, z, 1.0 / 40320.0);          /* 1/8! */
    pc = fma(pc, z, -1.0 / 720.0);           /* 1/6! */
    pc = fma(pc, z, 1.0 / 24.0);             /* 1/4! */
    pc = fma(pc, z, -0.5);                   /* 1/2! */
    double cs = fma(z, pc, 1.0);
    long q = ((long)k) & 3;
    if (q == 0) { *s_out = sn; *c_out = cs; }
    else if (q == 1) { *s_out = cs; *c_out = -sn; }
    else if (q == 2) { *s_out = -sn; *c_out = -cs; }
    else { *s_out = -cs; *c_out = sn; }
}

double ulo_exp(double x)
{
    if (x > 700.0) return INFINITY;
    if (x < -700.0) return 0.0;
    double k = rint(x * INV_LN2);
    double r = fma(-k, LN2_HI, x);
    r = fma(-k, LN2_LO, r);
    /* e^r = sum_{n=0}^{13} r^n / n! */
    double p = 1.0 / 6227020800.0;     /* 1/13! */
    p = fma(p, r, 1.0 / 479001600.0);  /* 1/12! */
    p = fma(p, r, 1.0 / 39916800.0);   /* 1/11! */
    p = fma(p, r, 1.0 / 3628800.0);    /* 1/10! */
    p = fma(p, r, 1.0 / 362880.0);     /* 1/9! */
    p = fma(p, r, 1.0 / 40320.0);      /* 1/8! */
    p = fma(p, r, 1.0 / 5040.0);       /* 1/7! */
    p = fma(p, r, 1.0 / 720.0);        /* 1/6! */
    p = fma(p, r, 1.0 / 120.0);        /* 1/5! */
    p = fma(p, r, 1.0 / 24.0);         /* 1/4! */
    p = fma(p, r, 1.0 / 6.0);          /* 1/3! */
    p = fma(p, r, 0.5);                /* 1/2! */
    p = fma(p, r, 1.0);                /* 1/1! */
    p = fma(p, r, 1.0);                /* 1/0! */
    return ldexp(p, (int)k);
}

/* atan(u) for |u| <= 1/16: u - u^3/3 + u^5/5 - ... - u^15/15 */
static double atan_series(double u)
{
    double z = u * u;
    double p = -1.0 / 15.0;
    p = fma(p, z, 1.0 / 13.0);
    p = fma(p, z, -1.0 / 11.0);
    p = fma(p, z, 1.0 / 9.0);
    p = fma(p, z, -1.0 / 7.0);
    p = fma(p, z, 1.0 / 5.0);
    p = fma(p, z, -1.0 / 3.0);
    return fma(u * z, p, u);
}

double ulo_atan2(double y, double x)
{
    double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0) return 0.0;
    int swap = ay > ax;
    double t = swap ? ax / ay : ay / ax;
    int j = (int)rint(t * 8.0);
    double a;
    if (j == 0) {
        a = atan_series(t);
    } else {
        double c = (double)j * 0.125;
        double u = (t - c) / (1.0 + t * c);
        a = ATAN_J8_HI[j] + (ATAN_J8_LO[j] + atan_series(u));
    }
    if (swap) a = (PIO2_1 - a) + PIO2_2;
    if (x < 0.0) a = (2.0 * PIO2_1 - a) + 2.0 * PIO2_2;
    if (y < 0.0) a = -a;
    return a;
}

/* ------------------------------------------------------------------------ */
/* Complex numbers as (re, im) pairs.  A product (a + ib)(c + id) is formed  */
/* as re = fma(a, c, -(b d)), im = fma(a, d, b c): each component is one     */
/* fused multiply-add of one exact product and one rounded product.          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double re, im;
} cplx;

static cplx cmk(double re, double im)
{
    cplx z;
    z.re = re;
    z.im = im;
    return z;
}
static cplx cmul(cplx a, cplx b) { return cmk(fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)); }
static cplx cconj(cplx a) { return cmk(a.re, -a.im); }
static cplx cadd(cplx a, cplx b) { return cmk(a.re + b.re, a.im + b.im); }
static cplx cscale(cplx a, double s) { return cmk(a.re * s, a.im * s); }
static cplx cdivr(cplx a, double s) { return cmk(a.re / s, a.im / s); }

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from the definition in Salmon et al., SC'11, Section 4.     */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void ulo_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        uint64_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double ulo_u53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

/* Philox4x32-10 (same paper): per round (hi, lo) = M * c for M0 = 0xD2511F53 on c0 and
 * M1 = 0xCD9E8D57 on c2, c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), then the key is bumped
 * by (0x9E3779B9, 0xBB67AE85).  The FP32 path draws its Metropolis uniforms from it. */
void ulo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t pa = (uint64_t)0xD2511F53u * c0, pb = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hiA = (uint32_t)(pa >> 32), loA = (uint32_t)pa;
        uint32_t hiB = (uint32_t)(pb >> 32), loB = (uint32_t)pb;
        uint32_t n0 = hiB ^ c1 ^ k0, n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L, Nt;
    long V;
} lat_t;

static lat_t mk(int L, int Nt)
{
    lat_t g;
    g.L = L;
    g.Nt = Nt;
    g.V = (long)L * L * L * Nt;
    return g;
}

/* c[0] = t, c[1] = x, c[2] = y, c[3] = z (indexed by direction). */
static void coords(const lat_t* g, long i, int c[4])
{
    c[1] = (int)(i % g->L);
    c[2] = (int)((i / g->L) % g->L);
    c[3] = (int)((i / ((long)g->L * g->L)) % g->L);
    c[0] = (int)(i / ((long)g->L * g->L * g->L));
}

static int extent(const lat_t* g, int mu) { return mu == 0 ? g->Nt : g->L; }

static long index_of(const lat_t* g, const int c[4])
{
    int w[4];
    for (int mu = 0; mu < 4; mu++) {
        int n = extent(g, mu);
        w[mu] = ((c[mu] % n) + n) % n;
    }
    return w[1] + (long)g->L * (w[2] + (long)g->L * (w[3] + (long)g->L * w[0]));
}

/* Index of the site c + a*e_mu + b*e_nu. */
static long shifted(const lat_t* g, const int c[4], int mu, int a, int nu, int b)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] += a;
    d[nu] += b;
    return index_of(g, d);
}

/* U_mu(x) = cos(theta_mu(x)) + i sin(theta_mu(x)) */
static cplx link(const lat_t* g, const double* theta, int mu, long i)
{
    double s, c;
    ulo_sincos(theta[(long)mu * g->V + i], &s, &c);
    return cmk(c, s);
}

/* ------------------------------------------------------------------------ */
/* Action pieces (Section 2)                                                 */
/* ------------------------------------------------------------------------ */

double ulo_wrap(double theta)
{
    const double two_pi = 2.0 * PI_D;
    return theta - two_pi * floor((theta + PI_D) / two_pi);
}

/* A += p * q with both components accumulated by fused multiply-adds:
 * Re: fma(p.re, q.re, fma(-p.im, q.im, A.re)),  Im: fma(p.re, q.im, fma(p.im, q.re, A.im)). */
static cplx cmul_acc(cplx A, cplx p, cplx q)
{
    return cmk(fma(p.re, q.re, fma(-p.im, q.im, A.re)), fma(p.re, q.im, fma(p.im, q.re, A.im)));
}

/* A(x,mu) = sum_{nu != mu} [ U_nu(x+mu) U*_mu(x+nu) U*_nu(x)
 *                           + U*_nu(x+mu-nu) U*_mu(x-nu) U_nu(x-nu) ]
 * The first term completes the plaquette U_mu nu(x); the second is the conjugate of
 * the plaquette U_mu nu(x-nu) with U*_mu(x) removed, so that both enter as Re(U_mu(x) A).
 * Terms in the order nu ascending, forward before backward; each term's last product is
 * accumulated into A (cmul_acc). */
static cplx staple(const lat_t* g, const double* theta, int mu, long i)
{
    int c[4];
    coords(g, i, c);
    cplx A = cmk(0.0, 0.0);
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        cplx f = cmul(link(g, theta, nu, shifted(g, c, mu, 1, nu, 0)),
                      cconj(link(g, theta, mu, shifted(g, c, nu, 1, mu, 0))));
        A = cmul_acc(A, f, cconj(link(g, theta, nu, i)));
        cplx b = cmul(cconj(link(g, theta, nu, shifted(g, c, mu, 1, nu, -1))),
                      cconj(link(g, theta, mu, shifted(g, c, nu, -1, mu, 0))));
        A = cmul_acc(A, b, link(g, theta, nu, shifted(g, c, nu, -1, mu, 0)));
    }
    return A;
}

void ulo_staple(int L, int Nt, const double* theta, int mu, long i, double* re, double* im)
{
    lat_t g = mk(L, Nt);
    cplx A = staple(&g, theta, mu, i);
    *re = A.re;
    *im = A.im;
}

/* Re(exp(i th) A) = cos(th) Re A - sin(th) Im A */
static double re_link_times(double th, double a_re, double a_im)
{
    double s, c;
    ulo_sincos(th, &s, &c);
    return c * a_re - s * a_im;
}

double ulo_local_action(int L, int Nt, double beta, const double* theta, int mu, long i)
{
    lat_t g = mk(L, Nt);
    cplx A = staple(&g, theta, mu, i);
    return -beta * re_link_times(theta[(long)mu * g.V + i], A.re, A.im);
}

/* Metropolis: propose theta' = wrap(theta + width (2 u1 - 1)) (2 u1 - 1 is exact; the step
 * is added by one fused multiply-add); with S_loc = -beta Re(e^{i theta} A),
 * dS = S_loc(theta') - S_loc(theta) = beta [(cos theta - cos theta') Re A - (sin theta - sin theta') Im A],
 * formed as beta * fma(dc, Re A, -(ds Im A)); accept iff u2 < exp(-dS). */
double ulo_metropolis_link(double theta, double a_re, double a_im, double beta,
                           double width, double u1, double u2, int* accepted)
{
    double proposal = ulo_wrap(fma(width, 2.0 * u1 - 1.0, theta));
    double s0, c0, s1, c1;
    ulo_sincos(theta, &s0, &c0);
    ulo_sincos(proposal, &s1, &c1);
    double dS = beta * fma(c0 - c1, a_re, -((s0 - s1) * a_im));
    if (u2 < ulo_exp(-dS)) {
        *accepted = 1;
        return proposal;
    }
    *accepted = 0;
    return theta;
}

/* Overrelaxation: S_loc = -beta |A| cos(theta + alpha), alpha = arg A; the reflection
 * theta + alpha -> -(theta + alpha) keeps S_loc, i.e. theta' = -2 alpha - theta. */
double ulo_overrelax_link(double theta, double a_re, double a_im)
{
    double alpha = ulo_atan2(a_im, a_re);
    return ulo_wrap(-2.0 * alpha - theta);
}

/* ------------------------------------------------------------------------ */
/* Sweeps (Section 2.1, Section 2.2 layers with fixed spatial links)         */
/* ------------------------------------------------------------------------ */

static int is_frozen(const lat_t* g, int mu, long i, int slab_t)
{
    if (slab_t <= 0 || mu == 0) return 0;
    int c[4];
    coords(g, i, c);
    return (c[0] % slab_t) == 0;
}

static int parity_of(const lat_t* g, long i)
{
    int c[4];
    coords(g, i, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

long ulo_sweep(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
               uint64_t* metro_pass, int n_metro, int n_or, int slab_t)
{
    lat_t g = mk(L, Nt);
    long accepted_total = 0;
    for (int pass = 0; pass < n_metro + n_or; pass++) {
        int metropolis = pass < n_metro;
        for (int mu = 0; mu < 4; mu++) {
            for (int p = 0; p < 2; p++) {
                /* The links of one (mu, parity) class share no staple (checkerboard), so the
                 * timing build (-fopenmp) may update them on several threads; the default
                 * build ignores the pragma.  Either way each link gets the same value. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : accepted_total)
#endif
                for (long i = 0; i < g.V; i++) {
                    if (parity_of(&g, i) != p) continue;
                    if (is_frozen(&g, mu, i, slab_t)) continue;
                    cplx A = staple(&g, theta, mu, i);
                    long li = (long)mu * g.V + i;
                    if (metropolis) {
                        uint64_t ctr[4] = {(uint64_t)li, *metro_pass, 0, 0};
                        uint64_t key[2] = {seed, 1};
                        uint64_t w[4];
                        ulo_philox4x64_10(ctr, key, w);
                        int acc = 0;
                        theta[li] = ulo_metropolis_link(theta[li], A.re, A.im, beta, width,
                                                        ulo_u53(w[0]), ulo_u53(w[1]), &acc);
                        accepted_total += acc;
                    } else {
                        theta[li] = ulo_overrelax_link(theta[li], A.re, A.im);
                    }
                }
            }
        }
        if (metropolis) (*metro_pass)++;
    }
    return accepted_total;
}

int ulo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ulo_hot_start(int L, int Nt, uint64_t seed, double* theta)
{
    lat_t g = mk(L, Nt);
    for (int mu = 0; mu < 4; mu++) {
        for (long i = 0; i < g.V; i++) {
            long li = (long)mu * g.V + i;
            uint64_t ctr[4] = {(uint64_t)li, 0, 0, 0};
            uint64_t key[2] = {seed, 0};
            uint64_t w[4];
            ulo_philox4x64_10(ctr, key, w);
            theta[li] = -PI_D + 2.0 * PI_D * ulo_u53(w[0]);
        }
    }
}

void ulo_gauge_transform(int L, int Nt, uint64_t seed, double* theta)
{
    lat_t g = mk(L, Nt);
    double* lambda = (double*)malloc(sizeof(double) * g.V);
    for (long i = 0; i < g.V; i++) {
        uint64_t ctr[4] = {(uint64_t)i, 0, 0, 0};
        uint64_t key[2] = {seed, 2};
        uint64_t w[4];
        ulo_philox4x64_10(ctr, key, w);
        lambda[i] = -PI_D + 2.0 * PI_D * ulo_u53(w[0]);
    }
    for (int mu = 0; mu < 4; mu++) {
        for (long i = 0; i < g.V; i++) {
            int c[4];
            coords(&g, i, c);
            long j = shifted(&g, c, mu, 1, mu, 0);
            long li = (long)mu * g.V + i;
            theta[li] = ulo_wrap(theta[li] + lambda[i] - lambda[j]);
        }
    }
    free(lambda);
}

/* ------------------------------------------------------------------------ */
/* Observables                                                               */
/* ------------------------------------------------------------------------ */

/* U_mu nu(x) = U_mu(x) U_nu(x+mu) U*_mu(x+nu) U*_nu(x) (Section 2) */
static cplx plaquette_at(const lat_t* g, const double* theta, int mu, int nu, long i)
{
    int c[4];
    coords(g, i, c);
    return cmul(cmul(cmul(link(g, theta, mu, i), link(g, theta, nu, shifted(g, c, mu, 1, nu, 0))),
                     cconj(link(g, theta, mu, shifted(g, c, nu, 1, mu, 0)))),
                cconj(link(g, theta, nu, i)));
}

void ulo_plaquette_at(int L, int Nt, const double* theta, int mu, int nu, long i,
                      double* re, double* im)
{
    lat_t g = mk(L, Nt);
    cplx P = plaquette_at(&g, theta, mu, nu, i);
    *re = P.re;
    *im = P.im;
}

double ulo_plaquette(int L, int Nt, const double* theta)
{
    lat_t g = mk(L, Nt);
    double sum = 0.0;
    for (long i = 0; i < g.V; i++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) sum += plaquette_at(&g, theta, mu, nu, i).re;
    return sum / (6.0 * (double)g.V);
}

static long spatial_to_site(const lat_t* g, long x0, int t)
{
    long L3 = (long)g->L * g->L * g->L;
    return x0 + L3 * t;
}

/* Spatial site x0 shifted by a along x and b along y. */
static long spatial_shift(const lat_t* g, long x0, int a, int b)
{
    int c[4];
    coords(g, x0, c); /* t = 0 */
    int d[4] = {0, c[1] + a, c[2] + b, c[3]};
    return index_of(g, d);
}

/* P(x0) = prod_t U_0(x0, t) */
static cplx polyakov_at(const lat_t* g, const double* theta, long x0)
{
    cplx P = cmk(1.0, 0.0);
    for (int t = 0; t < g->Nt; t++) P = cmul(P, link(g, theta, 0, spatial_to_site(g, x0, t)));
    return P;
}

void ulo_polyakov(int L, int Nt, const double* theta, double* out)
{
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    for (long x0 = 0; x0 < L3; x0++) {
        cplx P = polyakov_at(&g, theta, x0);
        out[2 * x0] = P.re;
        out[2 * x0 + 1] = P.im;
    }
}

void ulo_polyakov_correlator(int L, int Nt, const double* theta, int r_max, double* out)
{
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    for (int r = 1; r <= r_max; r++) {
        cplx sum = cmk(0.0, 0.0);
        for (long x0 = 0; x0 < L3; x0++)
            sum = cadd(sum, cmul(cconj(polyakov_at(&g, theta, x0)),
                                 polyakov_at(&g, theta, spatial_shift(&g, x0, r, 0))));
        sum = cdivr(sum, (double)L3);
        out[2 * (r - 1)] = sum.re;
        out[2 * (r - 1) + 1] = sum.im;
    }
}

/* Field channel ch of the plaquette with lower corner at site i:
 * ch = 2c + part, planes c = (0,1) E_x, (0,2) E_y, (0,3) E_z, (2,3) B_x; part 0 Im, 1 Re. */
static double channel_value(const lat_t* g, const double* theta, int ch, long i)
{
    static const int planes[4][2] = {{0, 1}, {0, 2}, {0, 3}, {2, 3}};
    int c = ch / 2, part = ch % 2;
    cplx P = plaquette_at(g, theta, planes[c][0], planes[c][1], i);
    return part == 0 ? P.im : P.re;
}

void ulo_field_correlator(int L, int Nt, const double* theta, int r_max, int d_max, double* out)
{
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    int nd = d_max + 1;
    for (int r = 1; r <= r_max; r++)
        for (int d = 0; d < nd; d++)
            for (int ch = 0; ch < 8; ch++) {
                cplx sum = cmk(0.0, 0.0);
                for (long x0 = 0; x0 < L3; x0++) {
                    cplx pp = cmul(cconj(polyakov_at(&g, theta, x0)),
                                   polyakov_at(&g, theta, spatial_shift(&g, x0, r, 0)));
                    long y = spatial_shift(&g, x0, r / 2, d);
                    for (int t = 0; t < Nt; t++)
                        sum = cadd(sum, cscale(pp, channel_value(&g, theta, ch, spatial_to_site(&g, y, t))));
                }
                sum = cdivr(sum, (double)g.V);
                long o = (((long)(r - 1) * nd + d) * 8 + ch) * 2;
                out[o] = sum.re;
                out[o + 1] = sum.im;
            }
}

/* One element of the direct field correlator (same definition, one (r, d, ch)). */
void ulo_field_correlator_one(int L, int Nt, const double* theta, int r, int d, int ch, double* re, double* im)
{
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    cplx sum = cmk(0.0, 0.0);
    for (long x0 = 0; x0 < L3; x0++) {
        cplx pp = cmul(cconj(polyakov_at(&g, theta, x0)), polyakov_at(&g, theta, spatial_shift(&g, x0, r, 0)));
        long y = spatial_shift(&g, x0, r / 2, d);
        for (int t = 0; t < Nt; t++)
            sum = cadd(sum, cscale(pp, channel_value(&g, theta, ch, spatial_to_site(&g, y, t))));
    }
    sum = cdivr(sum, (double)g.V);
    *re = sum.re;
    *im = sum.im;
}

/* ------------------------------------------------------------------------ */
/* Analytic multihit (Section 2.2: temporal links replaced by their average  */
/* over the link's own Boltzmann weight with all other links fixed)          */
/* ------------------------------------------------------------------------ */

/* I1(x)/I0(x) for x >= 0 from the power series
 *   I0(x) = sum_k (x^2/4)^k / (k!)^2,   I1(x) = (x/2) sum_k (x^2/4)^k / (k! (k+1)!),
 * summed until the terms stop changing the sums; for x > 600 (beyond any coupling used
 * here) the asymptotic series 1 - 1/(2x) - 1/(8x^2) - 1/(8x^3). */
double ulo_bessel_ratio(double x)
{
    if (x <= 0.0) return 0.0;
    if (x > 600.0) return 1.0 - 1.0 / (2.0 * x) - 1.0 / (8.0 * x * x) - 1.0 / (8.0 * x * x * x);
    const double q = 0.25 * x * x;
    double t0 = 1.0, s0 = 1.0;       /* I0 terms and sum */
    double t1 = 0.5 * x, s1 = t1;    /* I1 terms and sum */
    for (int k = 1; k < 2000; k++) {
        t0 *= q / ((double)k * (double)k);
        t1 *= q / ((double)k * (double)(k + 1));
        double n0 = s0 + t0, n1 = s1 + t1;
        if (n0 == s0 && n1 == s1) break;
        s0 = n0;
        s1 = n1;
    }
    return s1 / s0;
}

/* Multihit link: the mean of e^{i theta} under exp(beta Re(e^{i theta} A)) with A the
 * staple of the temporal link at site i: (I1(beta |A|) / I0(beta |A|)) A* / |A|. */
static cplx multihit_link(const lat_t* g, const double* theta, double beta, long i)
{
    cplx A = staple(g, theta, 0, i);
    double a = sqrt(A.re * A.re + A.im * A.im);
    if (a == 0.0) return cmk(0.0, 0.0);
    double f = ulo_bessel_ratio(beta * a) / a;
    return cmk(f * A.re, -f * A.im);
}

void ulo_multihit_link(int L, int Nt, double beta, const double* theta, long i, double* re, double* im)
{
    lat_t g = mk(L, Nt);
    cplx u = multihit_link(&g, theta, beta, i);
    *re = u.re;
    *im = u.im;
}

/* ------------------------------------------------------------------------ */
/* One-level multilevel estimator (Section 2.2)                              */
/* ------------------------------------------------------------------------ */

/* T^(tau)(s, x0, r) = prod over the slab's slices t of U*_0(x0,t) U_0(x0 + r xhat, t):
 * the product of the two-link transporters T(x0,t,r) of the slab. */
static cplx slab_transporter(const lat_t* g, const double* theta, int slab_t, int s, long x0, int r,
                             int multihit, double beta)
{
    cplx T = cmk(1.0, 0.0);
    long x1 = spatial_shift(g, x0, r, 0);
    /* Multihit only where the two temporal links share no plaquette (r >= 2). */
    int mh = multihit && r >= 2;
    for (int t = s * slab_t; t < (s + 1) * slab_t; t++) {
        long i0 = spatial_to_site(g, x0, t), i1 = spatial_to_site(g, x1, t);
        cplx a = mh ? multihit_link(g, theta, beta, i0) : link(g, theta, 0, i0);
        cplx b = mh ? multihit_link(g, theta, beta, i1) : link(g, theta, 0, i1);
        T = cmul(T, cmul(cconj(a), b));
    }
    return T;
}

int ulo_multilevel(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                   uint64_t* metro_pass, int slab_t, int n_sub, int sub_metro, int sub_or,
                   int r_max, int d_max, double* corr, double* fields, double* vac,
                   double* samples_T, int multihit)
{
    if (slab_t < 1 || Nt % slab_t != 0 || n_sub < 1 || r_max < 1 || r_max > L / 2 ||
        (fields && (d_max < 0 || d_max >= L)))
        return -1;
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    int S = Nt / slab_t;
    int nd = fields ? d_max + 1 : 0;
    long nA = (long)S * L3 * r_max;
    cplx* Asum = (cplx*)calloc((size_t)nA, sizeof(cplx));
    cplx* Bsum = NULL;
    if (fields) Bsum = (cplx*)calloc((size_t)(nA * nd * 8), sizeof(cplx));
    double Osum[8] = {0};

    for (int k = 0; k < n_sub; k++) {
        ulo_sweep(L, Nt, beta, seed, width, theta, metro_pass, sub_metro, sub_or, slab_t);
        for (int s = 0; s < S; s++)
            for (long x0 = 0; x0 < L3; x0++)
                for (int r = 1; r <= r_max; r++) {
                    cplx T = slab_transporter(&g, theta, slab_t, s, x0, r, multihit, beta);
                    cplx Tplain = multihit ? slab_transporter(&g, theta, slab_t, s, x0, r, 0, beta) : T;
                    long a = ((long)s * L3 + x0) * r_max + (r - 1);
                    Asum[a] = cadd(Asum[a], T);
                    if (samples_T) {
                        long o = ((long)k * nA + a) * 2;
                        samples_T[o] = T.re;
                        samples_T[o + 1] = T.im;
                    }
                    if (!fields) continue;
                    /* TO^(tau) = T^(tau) * sum over the slab's slices of O(x, t) */
                    for (int d = 0; d < nd; d++) {
                        long y = spatial_shift(&g, x0, r / 2, d);
                        for (int ch = 0; ch < 8; ch++) {
                            double O = 0.0;
                            for (int t = s * slab_t; t < (s + 1) * slab_t; t++)
                                O += channel_value(&g, theta, ch, spatial_to_site(&g, y, t));
                            long b = (a * nd + d) * 8 + ch;
                            Bsum[b] = cadd(Bsum[b], cscale(Tplain, O));
                        }
                    }
                }
        if (vac)
            for (int ch = 0; ch < 8; ch++)
                for (long i = 0; i < g.V; i++) Osum[ch] += channel_value(&g, theta, ch, i);
    }

    /* Per-slab averages, their product over slabs, then the average over x0. */
    for (int r = 1; r <= r_max; r++) {
        cplx sum = cmk(0.0, 0.0);
        for (long x0 = 0; x0 < L3; x0++) {
            cplx prod = cmk(1.0, 0.0);
            for (int s = 0; s < S; s++)
                prod = cmul(prod, cdivr(Asum[((long)s * L3 + x0) * r_max + (r - 1)], (double)n_sub));
            sum = cadd(sum, prod);
        }
        sum = cdivr(sum, (double)L3);
        corr[2 * (r - 1)] = sum.re;
        corr[2 * (r - 1) + 1] = sum.im;
    }
    /* Insertion: one slab carries <T O>, every other slab its <T>; summed over the slab
     * that carries the operator and over x0, divided by V = L^3 Nt. */
    if (fields) {
        for (int r = 1; r <= r_max; r++)
            for (int d = 0; d < nd; d++)
                for (int ch = 0; ch < 8; ch++) {
                    cplx sum = cmk(0.0, 0.0);
                    for (long x0 = 0; x0 < L3; x0++)
                        for (int s = 0; s < S; s++) {
                            long a = ((long)s * L3 + x0) * r_max + (r - 1);
                            cplx term = cdivr(Bsum[(a * nd + d) * 8 + ch], (double)n_sub);
                            for (int s2 = 0; s2 < S; s2++) {
                                if (s2 == s) continue;
                                term = cmul(term, cdivr(Asum[((long)s2 * L3 + x0) * r_max + (r - 1)],
                                                        (double)n_sub));
                            }
                            sum = cadd(sum, term);
                        }
                    sum = cdivr(sum, (double)g.V);
                    long o = (((long)(r - 1) * nd + d) * 8 + ch) * 2;
                    fields[o] = sum.re;
                    fields[o + 1] = sum.im;
                }
    }
    if (vac)
        for (int ch = 0; ch < 8; ch++) vac[ch] = Osum[ch] / ((double)n_sub * (double)g.V);
    free(Asum);
    free(Bsum);
    return 0;
}

/* Two-level estimator with field insertions (Section 2.2: the bracketed factors of the field
 * estimator are level-1 averages over the level-2 slabs inside a level-1 slab).  Level-2
 * means over the n2 samples of one level-1 iteration, per level-2 slab s2:
 *   A2(s2) = <T>,  B2(s2, d, ch) = <T O(x0 + floor(r/2) xhat + d yhat, ch)>;
 * one level-1 sample per level-1 slab s1 (level-2 slabs j = 0..m-1 inside it):
 *   a1 = prod_j A2(j),  b1 = sum_j B2(j) prod_{j' != j} A2(j');
 * with A1, B1 their means over the n1 level-1 samples,
 *   corr = (1/L^3) sum_x0 prod_s1 A1(s1),  fields = (1/V) sum_x0 sum_s1 B1(s1) prod_{s1' != s1} A1(s1'),
 *   vac = <O> over all sites, slices and the n1 n2 level-2 samples. */
int ulo_multilevel2_fields(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                           uint64_t* metro_pass, int tau1, int n1, int tau2, int n2, int sub_metro, int sub_or,
                           int r_max, int d_max, double* corr, double* fields, double* vac)
{
    if (tau1 < 1 || tau2 < 1 || Nt % tau1 != 0 || tau1 % tau2 != 0 || n1 < 1 || n2 < 1 || r_max < 1 ||
        r_max > L / 2 || d_max < 0 || d_max >= L)
        return -1;
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    int S1 = Nt / tau1, S2 = Nt / tau2, m = tau1 / tau2, nd = d_max + 1;
    long nA1 = (long)S1 * L3 * r_max, nA2 = (long)S2 * L3 * r_max;
    cplx* A1 = (cplx*)calloc((size_t)nA1, sizeof(cplx));
    cplx* B1 = (cplx*)calloc((size_t)(nA1 * nd * 8), sizeof(cplx));
    cplx* A2 = (cplx*)calloc((size_t)nA2, sizeof(cplx));
    cplx* B2 = (cplx*)calloc((size_t)(nA2 * nd * 8), sizeof(cplx));
    double Osum[8] = {0};
    if (!A1 || !B1 || !A2 || !B2) {
        free(A1);
        free(B1);
        free(A2);
        free(B2);
        return -2;
    }
    for (int k1 = 0; k1 < n1; k1++) {
        ulo_sweep(L, Nt, beta, seed, width, theta, metro_pass, sub_metro, sub_or, tau1);
        memset(A2, 0, sizeof(cplx) * (size_t)nA2);
        memset(B2, 0, sizeof(cplx) * (size_t)(nA2 * nd * 8));
        for (int k2 = 0; k2 < n2; k2++) {
            ulo_sweep(L, Nt, beta, seed, width, theta, metro_pass, sub_metro, sub_or, tau2);
            for (int s = 0; s < S2; s++)
                for (long x0 = 0; x0 < L3; x0++)
                    for (int r = 1; r <= r_max; r++) {
                        cplx T = slab_transporter(&g, theta, tau2, s, x0, r, 0, beta);
                        long a = ((long)s * L3 + x0) * r_max + (r - 1);
                        A2[a] = cadd(A2[a], T);
                        for (int d = 0; d < nd; d++) {
                            long y = spatial_shift(&g, x0, r / 2, d);
                            for (int ch = 0; ch < 8; ch++) {
                                double O = 0.0;
                                for (int t = s * tau2; t < (s + 1) * tau2; t++)
                                    O += channel_value(&g, theta, ch, spatial_to_site(&g, y, t));
                                long b = (a * nd + d) * 8 + ch;
                                B2[b] = cadd(B2[b], cscale(T, O));
                            }
                        }
                    }
            if (vac)
                for (int ch = 0; ch < 8; ch++)
                    for (long i = 0; i < g.V; i++) Osum[ch] += channel_value(&g, theta, ch, i);
        }
        for (int s1 = 0; s1 < S1; s1++)
            for (long x0 = 0; x0 < L3; x0++)
                for (int r = 1; r <= r_max; r++) {
                    long a1 = ((long)s1 * L3 + x0) * r_max + (r - 1);
                    cplx prod = cmk(1.0, 0.0);
                    for (int j = 0; j < m; j++)
                        prod = cmul(prod, cdivr(A2[((long)(s1 * m + j) * L3 + x0) * r_max + (r - 1)], (double)n2));
                    A1[a1] = cadd(A1[a1], prod);
                    for (int d = 0; d < nd; d++)
                        for (int ch = 0; ch < 8; ch++) {
                            cplx b = cmk(0.0, 0.0);
                            for (int j = 0; j < m; j++) {
                                long a2 = ((long)(s1 * m + j) * L3 + x0) * r_max + (r - 1);
                                cplx term = cdivr(B2[(a2 * nd + d) * 8 + ch], (double)n2);
                                for (int j2 = 0; j2 < m; j2++) {
                                    if (j2 == j) continue;
                                    term = cmul(term, cdivr(A2[((long)(s1 * m + j2) * L3 + x0) * r_max + (r - 1)],
                                                            (double)n2));
                                }
                                b = cadd(b, term);
                            }
                            long ib = (a1 * nd + d) * 8 + ch;
                            B1[ib] = cadd(B1[ib], b);
                        }
                }
    }
    for (int r = 1; r <= r_max; r++) {
        cplx sum = cmk(0.0, 0.0);
        for (long x0 = 0; x0 < L3; x0++) {
            cplx prod = cmk(1.0, 0.0);
            for (int s1 = 0; s1 < S1; s1++)
                prod = cmul(prod, cdivr(A1[((long)s1 * L3 + x0) * r_max + (r - 1)], (double)n1));
            sum = cadd(sum, prod);
        }
        sum = cdivr(sum, (double)L3);
        corr[2 * (r - 1)] = sum.re;
        corr[2 * (r - 1) + 1] = sum.im;
    }
    for (int r = 1; r <= r_max; r++)
        for (int d = 0; d < nd; d++)
            for (int ch = 0; ch < 8; ch++) {
                cplx sum = cmk(0.0, 0.0);
                for (long x0 = 0; x0 < L3; x0++)
                    for (int s1 = 0; s1 < S1; s1++) {
                        long a1 = ((long)s1 * L3 + x0) * r_max + (r - 1);
                        cplx term = cdivr(B1[(a1 * nd + d) * 8 + ch], (double)n1);
                        for (int s2 = 0; s2 < S1; s2++) {
                            if (s2 == s1) continue;
                            term = cmul(term, cdivr(A1[((long)s2 * L3 + x0) * r_max + (r - 1)], (double)n1));
                        }
                        sum = cadd(sum, term);
                    }
                sum = cdivr(sum, (double)g.V);
                long o = (((long)(r - 1) * nd + d) * 8 + ch) * 2;
                fields[o] = sum.re;
                fields[o + 1] = sum.im;
            }
    if (vac)
        for (int ch = 0; ch < 8; ch++) vac[ch] = Osum[ch] / ((double)n1 * (double)n2 * (double)g.V);
    free(A1);
    free(B1);
    free(A2);
    free(B2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Symmetrised insertions: the one-level estimator averaged over the 24      */
/* lattice symmetries that keep the time axis and send the separation        */
/* direction to a positive spatial axis                                      */
/* ------------------------------------------------------------------------ */

/* Link in a signed direction: U_{+mu}(x) = U_mu(x); U_{-mu}(x) = U*_mu(x - mu), the link
 * from x to x - mu traversed backwards. */
static cplx signed_link(const lat_t* g, const double* theta, int mu, int sgn, long i)
{
    if (sgn > 0) return link(g, theta, mu, i);
    int c[4];
    coords(g, i, c);
    return cconj(link(g, theta, mu, shifted(g, c, mu, -1, mu, 0)));
}

/* Oriented plaquette at site i spanned by the signed directions (s1 e_mu, s2 e_nu):
 * U_{s1 mu}(x) U_{s2 nu}(x + s1 mu) U*_{s1 mu}(x + s2 nu) U*_{s2 nu}(x). */
static cplx signed_plaquette(const lat_t* g, const double* theta, int mu, int s1, int nu, int s2, long i)
{
    int c[4];
    coords(g, i, c);
    long x_mu = shifted(g, c, mu, s1, mu, 0);
    long x_nu = shifted(g, c, nu, s2, nu, 0);
    return cmul(cmul(cmul(signed_link(g, theta, mu, s1, i), signed_link(g, theta, nu, s2, x_mu)),
                     cconj(signed_link(g, theta, mu, s1, x_nu))),
                cconj(signed_link(g, theta, nu, s2, i)));
}

/* Spatial site x0 moved by n steps along spatial axis a (1 = x, 2 = y, 3 = z). */
static long spatial_step(const lat_t* g, long x0, int a, int n)
{
    int c[4];
    coords(g, x0, c);
    return shifted(g, c, a, n, a, 0);
}

/* A frame: separation axis +e_a, insertion offset direction sb e_b, third direction sc e_c
 * ((a, b, c) a permutation of (1, 2, 3)).  Its four channel planes, in the order of the
 * unsymmetrised channels (0,x) (0,y) (0,z) (y,z), are (0, +a), (0, sb b), (0, sc c),
 * (sb b, sc c). */
typedef struct {
    int a, b, c, sb, sc;
} frame_t;

static int frames24(frame_t* f)
{
    int n = 0;
    for (int a = 1; a <= 3; a++) {
        int o1 = a == 1 ? 2 : 1, o2 = a == 3 ? 2 : 3;
        int pairs[2][2] = {{o1, o2}, {o2, o1}};
        for (int p = 0; p < 2; p++)
            for (int sb = 1; sb >= -1; sb -= 2)
                for (int sc = 1; sc >= -1; sc -= 2) {
                    f[n].a = a;
                    f[n].b = pairs[p][0];
                    f[n].c = pairs[p][1];
                    f[n].sb = sb;
                    f[n].sc = sc;
                    n++;
                }
    }
    return n;
}

/* Channel ch = 2 plane + part (part 0 Im, 1 Re) of frame f at site i. */
static double frame_channel(const lat_t* g, const double* theta, const frame_t* f, int ch, long i)
{
    int plane = ch / 2, part = ch % 2;
    cplx P;
    switch (plane) {
    case 0: P = signed_plaquette(g, theta, 0, 1, f->a, 1, i); break;
    case 1: P = signed_plaquette(g, theta, 0, 1, f->b, f->sb, i); break;
    case 2: P = signed_plaquette(g, theta, 0, 1, f->c, f->sc, i); break;
    default: P = signed_plaquette(g, theta, f->b, f->sb, f->c, f->sc, i); break;
    }
    return part == 0 ? P.im : P.re;
}

int ulo_multilevel_sym(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                       uint64_t* metro_pass, int slab_t, int n_sub, int sub_metro, int sub_or,
                       int r_max, int d_max, double* corr, double* fields, double* vac)
{
    if (slab_t < 1 || Nt % slab_t != 0 || n_sub < 1 || r_max < 1 || r_max > L / 2 || d_max < 0 || d_max >= L)
        return -1;
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    int S = Nt / slab_t, nd = d_max + 1;
    frame_t fr[24];
    int nf = frames24(fr);
    long nA = (long)S * L3 * r_max;
    /* Asum per separation axis, Bsum per frame, Osum per frame and channel */
    cplx* Asum = (cplx*)calloc((size_t)(3 * nA), sizeof(cplx));
    cplx* Bsum = (cplx*)calloc((size_t)(nf * nA * nd * 8), sizeof(cplx));
    double* Osum = (double*)calloc((size_t)(nf * 8), sizeof(double));
    if (!Asum || !Bsum || !Osum) {
        free(Asum);
        free(Bsum);
        free(Osum);
        return -2;
    }

    for (int k = 0; k < n_sub; k++) {
        ulo_sweep(L, Nt, beta, seed, width, theta, metro_pass, sub_metro, sub_or, slab_t);
        for (int s = 0; s < S; s++)
            for (long x0 = 0; x0 < L3; x0++)
                for (int r = 1; r <= r_max; r++)
                    for (int a = 1; a <= 3; a++) {
                        /* T^(tau) along +e_a: product over the slab of U*_0(x0,t) U_0(x0 + r e_a, t) */
                        long x1 = spatial_step(&g, x0, a, r);
                        cplx T = cmk(1.0, 0.0);
                        for (int t = s * slab_t; t < (s + 1) * slab_t; t++)
                            T = cmul(T, cmul(cconj(link(&g, theta, 0, spatial_to_site(&g, x0, t))),
                                             link(&g, theta, 0, spatial_to_site(&g, x1, t))));
                        long ia = (long)(a - 1) * nA + ((long)s * L3 + x0) * r_max + (r - 1);
                        Asum[ia] = cadd(Asum[ia], T);
                        for (int f = 0; f < nf; f++) {
                            if (fr[f].a != a) continue;
                            for (int d = 0; d < nd; d++) {
                                long y = spatial_step(&g, spatial_step(&g, x0, a, r / 2), fr[f].b, fr[f].sb * d);
                                for (int ch = 0; ch < 8; ch++) {
                                    double O = 0.0;
                                    for (int t = s * slab_t; t < (s + 1) * slab_t; t++)
                                        O += frame_channel(&g, theta, &fr[f], ch, spatial_to_site(&g, y, t));
                                    long ib = (((long)f * nA + ((long)s * L3 + x0) * r_max + (r - 1)) * nd + d) * 8 + ch;
                                    Bsum[ib] = cadd(Bsum[ib], cscale(T, O));
                                }
                            }
                        }
                    }
        for (int f = 0; f < nf; f++)
            for (int ch = 0; ch < 8; ch++)
                for (long i = 0; i < g.V; i++) Osum[f * 8 + ch] += frame_channel(&g, theta, &fr[f], ch, i);
    }

    /* Per frame: the one-level products and reductions of ulo_multilevel; then the mean over
     * the frames. */
    for (int r = 1; r <= r_max; r++) {
        cplx sum = cmk(0.0, 0.0);
        for (int f = 0; f < nf; f++) {
            long base = (long)(fr[f].a - 1) * nA;
            cplx sf = cmk(0.0, 0.0);
            for (long x0 = 0; x0 < L3; x0++) {
                cplx prod = cmk(1.0, 0.0);
                for (int s = 0; s < S; s++)
                    prod = cmul(prod, cdivr(Asum[base + ((long)s * L3 + x0) * r_max + (r - 1)], (double)n_sub));
                sf = cadd(sf, prod);
            }
            sum = cadd(sum, cdivr(sf, (double)L3));
        }
        sum = cdivr(sum, (double)nf);
        corr[2 * (r - 1)] = sum.re;
        corr[2 * (r - 1) + 1] = sum.im;
    }
    for (int r = 1; r <= r_max; r++)
        for (int d = 0; d < nd; d++)
            for (int ch = 0; ch < 8; ch++) {
                cplx sum = cmk(0.0, 0.0);
                for (int f = 0; f < nf; f++) {
                    long base = (long)(fr[f].a - 1) * nA;
                    cplx sf = cmk(0.0, 0.0);
                    for (long x0 = 0; x0 < L3; x0++)
                        for (int s = 0; s < S; s++) {
                            long ia = ((long)s * L3 + x0) * r_max + (r - 1);
                            cplx term = cdivr(Bsum[(((long)f * nA + ia) * nd + d) * 8 + ch], (double)n_sub);
                            for (int s2 = 0; s2 < S; s2++) {
                                if (s2 == s) continue;
                                term = cmul(term, cdivr(Asum[base + ((long)s2 * L3 + x0) * r_max + (r - 1)],
                                                        (double)n_sub));
                            }
                            sf = cadd(sf, term);
                        }
                    sum = cadd(sum, cdivr(sf, (double)g.V));
                }
                sum = cdivr(sum, (double)nf);
                long o = (((long)(r - 1) * nd + d) * 8 + ch) * 2;
                fields[o] = sum.re;
                fields[o + 1] = sum.im;
            }
    if (vac)
        for (int ch = 0; ch < 8; ch++) {
            double v = 0.0;
            for (int f = 0; f < nf; f++) v += Osum[f * 8 + ch] / ((double)n_sub * (double)g.V);
            vac[ch] = v / (double)nf;
        }
    free(Asum);
    free(Bsum);
    free(Osum);
    return 0;
}

/* Image of a configuration under the lattice symmetry g that keeps t and maps the spatial
 * unit vector e_i to sign_of[i] e_{axis_of[i]} (i = 1, 2, 3; a signed permutation), sites
 * x -> g x with coordinates taken mod L.  The image U' satisfies U'_{g v}(g x) = U_v(x) for
 * every signed direction v, so a positive link of U' is a link of U or the conjugate of the
 * link one step back. */
void ulo_symmetry_transform(int L, int Nt, const double* theta, const int axis_of[4], const int sign_of[4],
                            double* out)
{
    lat_t g = mk(L, Nt);
    for (long ip = 0; ip < g.V; ip++) {
        int cp[4];
        coords(&g, ip, cp);
        /* x = g^-1 x': x_i = sign_i x'_{axis_i} */
        int c[4];
        c[0] = cp[0];
        for (int i = 1; i <= 3; i++) c[i] = sign_of[i] * cp[axis_of[i]];
        long i0 = index_of(&g, c);
        out[ip] = theta[i0]; /* time links */
        for (int mp = 1; mp <= 3; mp++) {
            int i = 1;
            while (axis_of[i] != mp) i++;
            /* g^-1 e_{mp} = sign_i e_i */
            double th;
            if (sign_of[i] > 0) th = theta[(long)i * g.V + i0];
            else th = ulo_wrap(-theta[(long)i * g.V + shifted(&g, c, i, -1, i, 0)]);
            out[(long)mp * g.V + ip] = th;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Two-level multilevel estimator of the correlator (Section 2.2: two       */
/* nested levels of layers with frozen spatial links)                        */
/* ------------------------------------------------------------------------ */

int ulo_multilevel2(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                    uint64_t* metro_pass, int tau1, int n1, int tau2, int n2, int sub_metro, int sub_or,
                    int r_max, double* corr, int multihit)
{
    if (tau1 < 1 || tau2 < 1 || Nt % tau1 != 0 || tau1 % tau2 != 0 || n1 < 1 || n2 < 1 || r_max < 1 ||
        r_max > L / 2)
        return -1;
    lat_t g = mk(L, Nt);
    long L3 = (long)L * L * L;
    int S1 = Nt / tau1, S2 = Nt / tau2, m = tau1 / tau2;
    cplx* A1 = (cplx*)calloc((size_t)S1 * L3 * r_max, sizeof(cplx));
    cplx* A2 = (cplx*)calloc((size_t)S2 * L3 * r_max, sizeof(cplx));
    for (int k1 = 0; k1 < n1; k1++) {
        /* level 1: update with the spatial links on t = 0 mod tau1 frozen */
        ulo_sweep(L, Nt, beta, seed, width, theta, metro_pass, sub_metro, sub_or, tau1);
        memset(A2, 0, sizeof(cplx) * (size_t)S2 * L3 * r_max);
        for (int k2 = 0; k2 < n2; k2++) {
            /* level 2: also the spatial links on t = 0 mod tau2 frozen */
            ulo_sweep(L, Nt, beta, seed, width, theta, metro_pass, sub_metro, sub_or, tau2);
            for (int s = 0; s < S2; s++)
                for (long x0 = 0; x0 < L3; x0++)
                    for (int r = 1; r <= r_max; r++) {
                        long a = ((long)s * L3 + x0) * r_max + (r - 1);
                        A2[a] = cadd(A2[a], slab_transporter(&g, theta, tau2, s, x0, r, multihit, beta));
                    }
        }
        /* one level-1 sample per level-1 slab: product of its level-2 slab means */
        for (int s1 = 0; s1 < S1; s1++)
            for (long x0 = 0; x0 < L3; x0++)
                for (int r = 1; r <= r_max; r++) {
                    cplx prod = cmk(1.0, 0.0);
                    for (int j = 0; j < m; j++)
                        prod = cmul(prod, cdivr(A2[((long)(s1 * m + j) * L3 + x0) * r_max + (r - 1)], (double)n2));
                    long a = ((long)s1 * L3 + x0) * r_max + (r - 1);
                    A1[a] = cadd(A1[a], prod);
                }
    }
    for (int r = 1; r <= r_max; r++) {
        cplx sum = cmk(0.0, 0.0);
        for (long x0 = 0; x0 < L3; x0++) {
            cplx prod = cmk(1.0, 0.0);
            for (int s1 = 0; s1 < S1; s1++)
                prod = cmul(prod, cdivr(A1[((long)s1 * L3 + x0) * r_max + (r - 1)], (double)n1));
            sum = cadd(sum, prod);
        }
        sum = cdivr(sum, (double)L3);
        corr[2 * (r - 1)] = sum.re;
        corr[2 * (r - 1) + 1] = sum.im;
    }
    free(A1);
    free(A2);
    return 0;
}
