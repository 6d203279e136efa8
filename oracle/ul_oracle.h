/*
 * Plain, slow CPU oracle (FP64) for the multilevel U(1) hot path of
 * Amado, Cardoso, Cardoso, Bicudo, "Study of compact U(1) flux tubes in 3+1
 * dimensions in lattice gauge theory using GPU's" (arXiv:1208.0166).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source with the CUDA path.
 *
 * Conventions (the paper leaves them open; these are the readings taken):
 *   - direction mu = 0 is time, mu = 1,2,3 are x,y,z;
 *   - site index i = x + L*(y + L*(z + L*t)), V = L^3 * Nt;
 *   - link angles are stored canonically as theta[mu*V + i], in [-pi, pi);
 *   - parity of a site is (x+y+z+t) & 1.
 */
#ifndef UL_ORACLE_H
#define UL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = philox(ctr, key). */
void ulo_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Uniform in [0,1) from a 64-bit word: (w >> 11) * 2^-53. */
double ulo_u53(uint64_t w);

/* Philox4x32-10 (Salmon et al., SC'11): out = Philox4x32-10(ctr, key), 32-bit words. */
void ulo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Elementary functions with a fixed IEEE operation sequence (see ul_oracle.c). */
void ulo_sincos(double x, double* s, double* c);
double ulo_exp(double x);
double ulo_atan2(double y, double x);

/* Hot start: theta_mu(x) = -pi + 2 pi u, u from Philox(key=(seed,0), ctr=(mu V + i,0,0,0)) word 0. */
void ulo_hot_start(int L, int Nt, uint64_t seed, double* theta);

/* Staple sum A(x,mu) of the Wilson action (Section 2, Wilson action): the part of
 * sum_{plaquettes} Re U_p that contains U_mu(x) equals Re(U_mu(x) * A). */
void ulo_staple(int L, int Nt, const double* theta, int mu, long i, double* re, double* im);

/* -beta * Re(exp(i theta_mu(x)) A): the local action of one link. */
double ulo_local_action(int L, int Nt, double beta, const double* theta, int mu, long i);

/* One Metropolis hit on a link with a fixed staple: returns the new angle. */
double ulo_metropolis_link(double theta, double a_re, double a_im, double beta,
                           double width, double u1, double u2, int* accepted);

/* Overrelaxation reflection of one link with a fixed staple: theta' = -2 arg(A) - theta. */
double ulo_overrelax_link(double theta, double a_re, double a_im);

/* Wrap into [-pi, pi): theta - 2 pi floor((theta + pi) / (2 pi)). */
double ulo_wrap(double theta);

/*
 * Compound sweep: n_metro Metropolis passes, then n_or overrelaxation passes.
 * A pass visits mu = 0..3, and for each mu the even then the odd sites.
 * If slab_t > 0, spatial links (mu >= 1) on time slices t % slab_t == 0 are
 * frozen (multilevel sublattice update, Section 2.2).
 * *metro_pass counts Metropolis passes; it is the second Philox counter word
 * and is incremented once per Metropolis pass.  Returns accepted hits.
 */
long ulo_sweep(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
               uint64_t* metro_pass, int n_metro, int n_or, int slab_t);

/* Mean plaquette <Re U_p> = (1/6V) sum_x sum_{mu<nu} Re U_mu nu(x). */
double ulo_plaquette(int L, int Nt, const double* theta);

/* Plaquette U_mu nu(x) as a complex number (re, im). */
void ulo_plaquette_at(int L, int Nt, const double* theta, int mu, int nu, long i,
                      double* re, double* im);

/* Polyakov loops P(x0) = prod_t U_0(x0,t), x0 over the L^3 spatial sites. out: 2*L^3. */
void ulo_polyakov(int L, int Nt, const double* theta, double* out);

/* Direct correlator (1/L^3) sum_x0 P*(x0) P(x0 + r xhat), r = 1..r_max. out: 2*r_max. */
void ulo_polyakov_correlator(int L, int Nt, const double* theta, int r_max, double* out);

/* Direct field correlator (1/V) sum_x0 sum_t P*(x0) P(x0 + r xhat) O_ch(x0 + (r/2) xhat + d yhat, t).
 * out: 2 * r_max * (d_max+1) * 8, layout [r-1][d][ch][re,im]. */
void ulo_field_correlator(int L, int Nt, const double* theta, int r_max, int d_max, double* out);

/* One element (r, d, ch) of the direct field correlator. */
void ulo_field_correlator_one(int L, int Nt, const double* theta, int r, int d, int ch, double* re, double* im);

/*
 * One-level Luscher-Weisz multilevel estimator (Section 2.2, Eqs. for V(r),
 * the insertion operator and the multilevel field average).
 *   corr  : 2*r_max doubles, (re,im) of (1/L^3) sum_x0 prod_s <T^(tau)>_s(x0,r)
 *   fields: NULL, or 2*r_max*(d_max+1)*8 doubles, layout [r-1][d][ch][re,im]:
 *           (1/V) sum_x0 sum_s <T^(tau) O_ch>_s(x0,r,d) prod_{s' != s} <T^(tau)>_s'(x0,r)
 *   vac   : NULL, or 8 doubles, <O_ch> over all sites, slices and sub-samples.
 * Channels ch = 2c + part, c: 0 = P_01 (E_x), 1 = P_02 (E_y), 2 = P_03 (E_z),
 * 3 = P_23 (B_x); part 0 = Im, part 1 = Re.
 * Each sub-sample k = 1..n_sub is sub_metro Metropolis + sub_or overrelaxation
 * passes with slab-boundary spatial links frozen, followed by a measurement.
 * samples_T: NULL, or n_sub*S*L^3*r_max*2 doubles recording every T^(tau) sample,
 * layout [k][s][x0][r-1][re,im] (lets tests enumerate the product by brute force).
 * multihit: nonzero to use, for the correlator at r >= 2, the multihit links of the
 * temporal direction (ulo_multihit_link); insertions always use the links themselves.
 */
int ulo_multilevel(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                   uint64_t* metro_pass, int slab_t, int n_sub, int sub_metro, int sub_or,
                   int r_max, int d_max, double* corr, double* fields, double* vac,
                   double* samples_T, int multihit);

/*
 * Two-level multilevel estimator of the correlator (Section 2.2, the bracketed products
 * of the field estimator read as level-1 averages of products of level-2 averages):
 *   n1 times: sub_metro + sub_or passes with spatial links on t = 0 mod tau1 frozen, then
 *             n2 times: the same passes with t = 0 mod tau2 also frozen and a measurement
 *             of T^(tau2) per level-2 slab; one level-1 sample per level-1 slab is the
 *             product of the level-2 means of the tau1/tau2 slabs inside it;
 *   corr[r] = (1/L^3) sum_x0 prod_{level-1 slabs} (mean of the level-1 samples).
 * tau2 divides tau1, tau1 divides Nt.  multihit as in ulo_multilevel.
 */
int ulo_multilevel2(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                    uint64_t* metro_pass, int tau1, int n1, int tau2, int n2, int sub_metro, int sub_or,
                    int r_max, double* corr, int multihit);

/*
 * Symmetrised one-level estimator: ulo_multilevel's correlator, field insertions and
 * vacuum terms (channels (0,x) (0,y) (0,z) (y,z), Im and Re) averaged over the 24 frames
 * (separation axis +e_a, insertion offset direction sb e_b, third axis sc e_c): the lattice
 * symmetries that keep the time axis and the orientation of the source pair.  Plaquettes
 * in negative directions are oriented products of signed links U_{-mu}(x) = U*_mu(x - mu).
 * Same arguments as ulo_multilevel (fields and vac required, d_max >= 0).  0 on success.
 */
int ulo_multilevel_sym(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                       uint64_t* metro_pass, int slab_t, int n_sub, int sub_metro, int sub_or,
                       int r_max, int d_max, double* corr, double* fields, double* vac);

/* Image of the configuration under the spatial signed permutation e_i -> sign_of[i] e_{axis_of[i]}
 * (entries 1..3 used): out_{g v}(g x) = theta_v(x), angles of negative links negated. */
void ulo_symmetry_transform(int L, int Nt, const double* theta, const int axis_of[4], const int sign_of[4],
                            double* out);

/*
 * Two-level estimator with field insertions (the paper's bracketed field estimator, Section
 * 2.2): level-2 means A2 = <T>, B2 = <T O> per level-2 slab over the n2 samples of a level-1
 * iteration; per level-1 slab one sample a1 = prod_j A2(j), b1 = sum_j B2(j) prod_{j' != j} A2(j');
 * corr, fields as ulo_multilevel with the level-1 means of a1, b1 as the slab factors; vac
 * the mean of O over all level-2 samples.  Insertion geometry, channels and output layouts as
 * ulo_multilevel (fields required, vac may be NULL); no multihit.  0 on success.
 */
int ulo_multilevel2_fields(int L, int Nt, double beta, uint64_t seed, double width, double* theta,
                           uint64_t* metro_pass, int tau1, int n1, int tau2, int n2, int sub_metro, int sub_or,
                           int r_max, int d_max, double* corr, double* fields, double* vac);

/* Threads the class loop of ulo_sweep runs on: 1 in the default build; the timing build
 * (compiled with -fopenmp) updates the links of one (mu, parity) class on OpenMP threads,
 * with the same result for every link. */
int ulo_threads(void);

/* I1(x)/I0(x), x >= 0 (power series; asymptotic series beyond x = 600). */
double ulo_bessel_ratio(double x);

/* Analytic multihit value of the temporal link at site i: its average over its own
 * Boltzmann weight exp(beta Re(U A)) with the staple A fixed,
 * (I1(beta|A|) / I0(beta|A|)) A* / |A| (Section 2.2, multihit for the potential). */
void ulo_multihit_link(int L, int Nt, double beta, const double* theta, long i, double* re, double* im);

/* Random gauge transformation theta_mu(x) += lambda(x) - lambda(x + mu),
 * lambda(x) = -pi + 2 pi u53(Philox(key=(seed,2), ctr=(i,0,0,0)) word 0); result wrapped. */
void ulo_gauge_transform(int L, int Nt, uint64_t seed, double* theta);

#ifdef __cplusplus
}
#endif
#endif
