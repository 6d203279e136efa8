/*
 * ul.h — C ABI of libul: the Luscher–Weisz multilevel hot path for 4D compact U(1)
 * lattice gauge theory with the Wilson action, on one GB300 GPU (sm_103a).
 *
 * Method: A. Amado, N. Cardoso, M. Cardoso, P. Bicudo, "Study of compact U(1) flux
 * tubes in 3+1 dimensions in lattice gauge theory using GPU's", arXiv:1208.0166.
 *
 * Conventions used by every entry point
 *   - Direction mu = 0 is time (the paper writes U_0 for temporal links), mu = 1,2,3
 *     are x, y, z.  The lattice is L^3 x Nt, periodic in all directions.
 *   - Canonical host layout of link angles: theta[mu*V + i], V = L^3 Nt,
 *     i = x + L*(y + L*(z + L*t)); U_mu(x) = exp(i theta_mu(x)), theta in [-pi, pi).
 *   - Every call returns UL_OK (0) or a negative status.  On error nothing is written
 *     to the caller's output buffers; ul_last_error() gives a text.  A handle stays
 *     valid after an error (except UL_ENOMEM from ul_init, which sets *h = NULL).
 *   - The library owns all device memory and the handle; the caller owns every host
 *     buffer it passes (outputs are written before the call returns).
 *   - Calls on one handle are serialised on the handle's CUDA stream (the insertion
 *     contractions and a begun level's reduction run on a second, library-owned stream,
 *     ordered by events).  Calls that return results (ul_multilevel*, except
 *     ul_multilevel_fields_begin, ul_plaquette, ul_get_*) block until the results are on
 *     the host.  ul_sweep, ul_set_state and ul_multilevel_fields_begin only enqueue work
 *     and return; an execution error of enqueued work is reported by the next blocking
 *     call.  Different handles may be used from different host threads.
 */
#ifndef UL_H
#define UL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ul_lattice ul_lattice; /* opaque, library-owned */

enum {
    UL_OK = 0,
    UL_EINVAL = -1,   /* an argument is out of range (message says which) */
    UL_ENOMEM = -2,   /* device memory could not be allocated */
    UL_ECUDA = -3,    /* a CUDA runtime call failed (message has the CUDA error) */
    UL_ETIMEOUT = -4, /* a device-side bounded wait gave up */
    UL_ESTATE = -5    /* the handle is not in a state that allows the call */
};

enum {
    UL_FP64 = 0,      /* link angles, updates and accumulation in FP64 */
    UL_FP32_ACC64 = 1 /* link angles, updates and per-sample measurement products in
                         FP32; slab accumulators, cross-slab products and reductions in FP64 */
};

/*
 * ul_init — create a lattice L^3 x Nt at coupling beta with a hot start.
 * Section 2 (Wilson action beta S = beta sum_x sum_{mu<nu}[1 - Re U_mu nu(x)],
 * beta = 1/g^2) and Section 2.1 (configurations of an isotropic lattice).
 * Hot start: theta_mu(x) = -pi + 2 pi u, u = (w0 >> 11) 2^-53 with w0 the first word of
 * Philox4x64-10(counter = (mu V + i, 0, 0, 0), key = (seed, 0)).
 * L, Nt: even, >= 2 (checkerboard), L^3 Nt <= 2^28.  beta >= 0.
 * ul_init is ul_init_ex(..., UL_FP64).
 */
int ul_init(ul_lattice** h, int L, int Nt, double beta, uint64_t seed);
int ul_init_ex(ul_lattice** h, int L, int Nt, double beta, uint64_t seed, int precision);

/*
 * ul_sweep — n_metro Metropolis passes then n_or overrelaxation passes over the whole
 * lattice (Section 2.1: configurations are generated with Metropolis and overrelaxation).
 * A pass updates the 8 classes (mu = 0..3) x (even, odd sites) in that order; links of
 * one class share no plaquette and are updated in parallel.
 *   Metropolis: theta' = wrap(theta + w (2 u1 - 1)), w = option "metro_width" (1.0);
 *     accept iff u2 < exp(-dS), dS = -beta Re[(e^{i theta'} - e^{i theta}) A], with A the
 *     staple sum of the link; u1, u2 from words 0, 1 of Philox4x64-10(counter =
 *     (mu V + i, pass, 0, 0), key = (seed, 1)) (UL_FP32_ACC64: Philox4x32-10, see
 *     ul_rng_uniforms), pass = number of earlier Metropolis passes.
 *   Overrelaxation: theta' = wrap(-2 arg(A) - theta) (leaves Re(e^{i theta} A) unchanged).
 * n_metro, n_or >= 0.  Returns once the passes are enqueued on the handle's stream.
 */
int ul_sweep(ul_lattice* h, int n_metro, int n_or);

/*
 * ul_multilevel — one level of the Luscher–Weisz multilevel algorithm (Section 2.2: the
 * lattice is cut into time layers whose spatial boundary links are held fixed while
 * the remaining links are updated many times) for the Polyakov-loop
 * correlator <P*(0) P(r)> of Section 2.2 (the estimator of V(r) = -(1/Nt) ln <P*P>).
 * The lattice is cut into S = Nt/slab_t time slabs; spatial links on slices
 * t = 0 mod slab_t stay frozen.  n_sub times: options "sub_metro" Metropolis plus
 * "sub_or" overrelaxation passes (defaults 1 and 3) of the unfrozen links, then a
 * measurement of the slab transporters
 *     T(s, x0, r) = prod_{t in slab s} U*_0(x0, t) U_0(x0 + r xhat, t).
 * out (caller-owned host, 2*r_max doubles) receives (re, im) of
 *     C(r) = (1/L^3) sum_x0 prod_s <T(s, x0, r)>,  r = 1..r_max,
 * <.> the mean over the n_sub measurements.  The links keep the last sub-sample state.
 * slab_t >= 1 divides Nt; n_sub >= 1; 1 <= r_max <= L/2.
 */
int ul_multilevel(ul_lattice* h, int slab_t, int n_sub, int r_max, double* out);

/*
 * ul_multilevel_fields — ul_multilevel plus the field insertions of Section 2.2
 * (operator O(x0,x,t,r) = U*_0(x0,t) U_0(x0+r,t) O(x,t); per slab the insertion term is
 * T(s,x0,r) * sum_{t in slab} O(x,t), the general-thickness form of TO^(2); the
 * estimator <P*(0) P(r) O(x)> = (1/V) sum_x0 sum_s <T O>_s prod_{s' != s} <T>_s').
 * The operator sits on the plaquette with lower corner x = x0 + floor(r/2) xhat + d yhat,
 * d = 0..d_max, in channel ch = 2c + part: c = 0 (t,x) plane E_x, 1 (t,y) E_y, 2 (t,z)
 * E_z, 3 (y,z) B_x; part 0 = Im P (a^2 F = sqrt(beta) Im P), 1 = Re P (for
 * a^4 F^2 = beta (1 - Re P)).
 *   out_corr  : 2*r_max doubles, as ul_multilevel;
 *   out_fields: 2*r_max*(d_max+1)*8 doubles, layout [r-1][d][ch][re, im];
 *   out_vac   : 8 doubles (may be NULL), <O_ch> over all sites, slices and sub-samples,
 *               the subtraction term <O> of the connected average.
 * 0 <= d_max < L.
 */
int ul_multilevel_fields(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max,
                         double* out_corr, double* out_fields, double* out_vac);

/*
 * ul_multilevel_fields_begin / ul_multilevel_fields_end — ul_multilevel_fields in two
 * halves, so that the host can queue the next configuration's sweeps while the level's
 * final reduction and result copy are still running.  _begin validates the arguments (as
 * ul_multilevel_fields; d_max < 0 means no insertions, the correlator of ul_multilevel),
 * enqueues the level's sub-samples on the handle's stream, then the reduction and the copy
 * of its results into library-owned pinned host memory on the handle's second stream, and
 * returns without waiting.  _end waits for that copy and writes out_corr (2*r_max doubles),
 * and, when the level was begun with d_max >= 0, out_fields (may be NULL) and out_vac (may
 * be NULL) in the layouts of ul_multilevel_fields.  Between the two calls the handle takes
 * any call except a second _begin, ul_multilevel or ul_multilevel_fields (UL_ESTATE);
 * calls that use the level scratch (the other estimators) wait on the device for the
 * pending reduction.
 * Results are those of ul_multilevel_fields bit for bit.  _end without a _begin:
 * UL_ESTATE.  A grid-barrier timeout of a persistent sweep inside the level is reported by
 * _end (UL_ETIMEOUT).  ul_free with a level pending waits for it and drops its results.
 */
int ul_multilevel_fields_begin(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max);
int ul_multilevel_fields_end(ul_lattice* h, double* out_corr, double* out_fields, double* out_vac);

/*
 * ul_multilevel2_fields — the two-level estimator with field insertions: the paper's
 * field estimator (Section 2.2) with its bracketed factors read as level-1 averages.
 * n1 times: "sub_metro" + "sub_or" passes with the spatial links on t = 0 mod tau1 frozen,
 * then n2 sub-samples with t = 0 mod tau2 also frozen, each measured as in
 * ul_multilevel_fields (thickness tau2); per level-1 iteration the level-2 means
 * A2 = <T>, B2 = <T O> of each level-2 slab, and per level-1 slab (level-2 slabs j inside it)
 * one level-1 sample  a1 = prod_j A2(j),  b1 = sum_j B2(j) prod_{j' != j} A2(j').
 *   out_corr  : (1/L^3) sum_x0 prod_{level-1 slabs} <a1>                     (2*r_max doubles)
 *   out_fields: (1/V) sum_x0 sum_s1 <b1>(s1) prod_{s1' != s1} <a1>(s1')  (layout of ul_multilevel_fields)
 *   out_vac   : <O> over all sites, slices and the n1*n2 level-2 samples (8 doubles, may be NULL).
 * tau2 divides tau1, tau1 divides Nt, tau1/tau2 <= 16, n1, n2 >= 1, 1 <= r_max <= L/2,
 * 0 <= d_max < L; "multihit" must be 0 (UL_EINVAL otherwise).  The level-2 sub-samples run
 * slab-resident under the same conditions as in ul_multilevel_fields.
 */
int ul_multilevel2_fields(ul_lattice* h, int tau1, int n1, int tau2, int n2, int r_max, int d_max,
                          double* out_corr, double* out_fields, double* out_vac);

/*
 * ul_multilevel_fields_sym — ul_multilevel_fields averaged over the 24 frames of the source
 * pair: the estimator of Section 2.2, which the paper evaluates in one frame, evaluated in
 * every frame to which a lattice symmetry keeping the time axis and the orientation of the
 * pair maps that one: separation axis +e_a,
 * a = x, y, z; insertion plaquette at x0 + floor(r/2) e_a + d sb e_b; channel planes
 * (0, +a) "E parallel", (0, sb b) "E along the offset", (0, sc c) "E across", (sb b, sc c)
 * "B parallel", Im and Re, where (a, b, c) is a permutation of the spatial axes and sb, sc
 * = +-1.  A plaquette in negative directions is the oriented product of links traversed
 * backwards, U_{-mu}(x) = U*_mu(x - mu).  The correlator is the mean of the three axes.
 * Outputs and their layouts as in ul_multilevel_fields (out_fields required, out_vac may be
 * NULL).  Runs one launch per class; options "slab_resident" and "persistent" do not apply;
 * "multihit" must be 0 (UL_EINVAL otherwise).  Extra device memory: three transporter and
 * insertion accumulators, 12 (instead of 8) channel sums per site, and per stored sample the
 * transporters of three axes and the frame sums of every insertion midpoint (3 (d_max+1) 8
 * values per site and slab), bounded by the option "insertion_chunk_mb".
 */
int ul_multilevel_fields_sym(ul_lattice* h, int slab_t, int n_sub, int r_max, int d_max,
                             double* out_corr, double* out_fields, double* out_vac);

/*
 * ul_multilevel2 — two-level multilevel correlator (Section 2.2: the paper's two-level
 * scheme, its field estimator grouping pairs of thickness-2 slabs into level-1 factors).
 * n1 times: "sub_metro" + "sub_or" passes with the spatial links on t = 0 mod tau1 frozen,
 * then n2 sub-samples of the same passes with t = 0 mod tau2 also frozen, each followed by
 * a measurement of T (thickness tau2) per level-2 slab; one level-1 sample per level-1 slab
 * is the product of the n2-sample means of the tau1/tau2 level-2 slabs inside it.
 * out (2*r_max doubles): (re, im) of (1/L^3) sum_x0 prod_{level-1 slabs} <level-1 sample>.
 * tau2 divides tau1, tau1 divides Nt, n1, n2 >= 1, 1 <= r_max <= L/2 (and <= 128).
 * Option "multihit" applies as for ul_multilevel.
 */
int ul_multilevel2(ul_lattice* h, int tau1, int n1, int tau2, int n2, int r_max, double* out);

/* ul_plaquette — *out = <Re U_p> = (1/6V) sum_x sum_{mu<nu} Re U_mu nu(x) (Section 2),
 * accumulated in FP64 in a fixed order (bitwise reproducible). */
int ul_plaquette(ul_lattice* h, double* out);

/*
 * ul_check_enabled — 1 if this library is the bounds-checked build (libul_check.so,
 * compiled with -DUL_CHECK), else 0.  The paper has no counterpart: the checked build
 * stands in for a memory sanitizer.  In it, every link offset, neighbour site index and
 * accumulator index the update, measurement, plaquette and slab-resident kernels form is
 * compared with the extent of its array before the access; an index out of range is
 * recorded (first one only) and replaced by 0, so the kernel never faults or traps.
 */
int ul_check_enabled(void);

/*
 * ul_check_status — *first_failure = 0 if no checked index has been out of range since the
 * last clear, else the first failure: bit 63 set, bits 48..55 a tag naming the access
 * (1 link offset, 2 neighbour site, 3 neighbour link, 4 updated link, 5 slab-kernel global
 * offset, 6 transporter accumulator, 7 stored sample, 8 channel sums), bits 0..47 the index.
 * clear != 0 resets the record.  Always 0 in the default build.  Synchronises with the
 * device (reads device memory); call it between kernels, not during stream capture.
 * UL_EINVAL for a NULL pointer, UL_ECUDA if the read fails.
 */
int ul_check_status(unsigned long long* first_failure, int clear);

/*
 * ul_plaquette_noalloc — the mean plaquette <Re U_p> of link angles that already live in
 * device memory, computed without allocating any device memory.  The paper has no
 * counterpart: this exists for callers that cannot let a library allocate, such as a host
 * whose device memory is handed out only by its own allocator under a fixed budget, or a
 * loop that cannot accept the device synchronisation an allocation may cause.
 *   theta_dev : caller-owned device array of 4 L^3 Nt doubles, canonical layout
 *               theta[mu*V + i] (read only).
 *   out_dev   : caller-owned device pointer to one double; receives the mean plaquette.
 *   cuda_stream: cudaStream_t to run on (NULL: the legacy default stream).  The call only
 *               enqueues two kernels and returns; read *out_dev after synchronising the stream.
 * Scratch: one partial sum per block of 256 sites, kept in a fixed array inside the library
 * (512 KiB per GPU that loads it, held until the process exits).  Lattices larger than
 * 2^24 sites (e.g. beyond 64^4) are rejected with UL_EINVAL, as are NULL pointers and
 * L or Nt < 2; UL_ECUDA means a CUDA call of this entry point failed (an error left pending
 * on the calling thread by earlier work is cleared on entry, not reported here).  The first
 * call on each device looks up
 * the array's device address (with that device current); make that first call before any
 * stream capture.  All calls share the one array and each call overwrites every slot it
 * reads, so nothing carries over between calls, but two calls that overlap on the GPU
 * (different streams, same device) race on it: serialise them.  Values agree with
 * ul_plaquette to rounding (the sum order differs).
 */
int ul_plaquette_noalloc(const double* theta_dev, int L, int Nt, double* out_dev, void* cuda_stream);

/*
 * ul_rng_uniforms — the Metropolis uniforms (u1, u2) that the update kernels of `precision`
 * draw for links link0 .. link0+n-1 in Metropolis pass `pass` with `seed` (random numbers
 * are not specified by the paper; the choice is Philox, Salmon et al., SC'11):
 *   UL_FP64:       words 0, 1 of Philox4x64-10(counter (link, pass, 0, 0), key (seed, 1)),
 *                  u = (w >> 11) 2^-53;
 *   UL_FP32_ACC64: words 0, 1 of Philox4x32-10(counter (link, pass low 32 bits, pass high
 *                  32 bits, 1), key (seed low, seed high)), u = (w >> 8) 2^-24.
 * link = mu V + i for link (mu, lexicographic site i).  out: 2n doubles (u1, u2 per link),
 * caller-owned host memory.  0 <= n <= 2^24.  Synchronous (default stream); allocates.
 * For tests and reproduction of the update kernels' random numbers.
 */
int ul_rng_uniforms(int precision, uint64_t seed, uint64_t pass, uint64_t link0, int n, double* out);

/* ul_free — release the handle and its device memory.  NULL is accepted. */
int ul_free(ul_lattice* h);

/*
 * ul_set_option — set a run option (double value):
 *   "metro_width"  half-width of the Metropolis proposal in rad (> 0, default 1.0)
 *   "sub_metro"    Metropolis passes per multilevel sub-sample (>= 0, default 1)
 *   "sub_or"       overrelaxation passes per multilevel sub-sample (>= 0, default 3)
 *   "beta"         coupling (>= 0)
 *   "multihit"     1: ul_multilevel* form the correlator at r >= 2 from the analytic
 *                  multihit values of the temporal links, (I1(beta|A|)/I0(beta|A|)) conj(A)/|A|
 *                  with A the staple (Section 2.2: multihit for the potential); r = 1, whose
 *                  two lines share plaquettes, and the field insertions keep the links
 *                  themselves.  0 (default): links themselves everywhere.
 *   "persistent"   1: each compound sweep, and each chunk of sub-samples with their
 *                  measurements, runs as one cooperative launch whose classes are separated
 *                  by a grid barrier; 0 (default): one launch per class, replayed from
 *                  CUDA graphs.  Results are identical either way.
 *   "barrier_spin_limit"  polls a block spends waiting at a grid barrier before it gives
 *                  up (default 2^24, about a second); a wait that gives up stops the
 *                  launch and the next blocking call returns UL_ETIMEOUT (the handle
 *                  stays usable; the links are then in an incomplete state).
 *   "barrier_unreachable"  1: every barrier waits for one block more than exist, so
 *                  every wait runs into its limit (for testing the timeout path); 0 (default).
 *   "pdl"          1: consecutive class kernels use programmatic dependent launch (the
 *                  next one is scheduled while the previous one runs and waits for its
 *                  completion before reading links); 2: in compound sweeps only, not in
 *                  the passes of sub-samples; 0: plain stream order.  Default 1 for
 *                  UL_FP32_ACC64, 2 for UL_FP64.  Results are identical in every mode.
 *   "graphs"       1 (default): recurring launch sequences (a compound sweep, a chunk of
 *                  sub-samples) are captured once into CUDA graphs and replayed; 0: every
 *                  kernel is launched directly.  Results are identical either way.
 *   "slab_resident"  1: ul_multilevel, ul_multilevel_fields and the level-2 sub-samples of
 *                  ul_multilevel2_fields run each chunk of sub-samples
 *                  as one launch in which a thread-block cluster owns one time slab: its
 *                  links are held in the shared memory of the cluster's CTAs (Section 2.2:
 *                  with the slab boundaries frozen a slab's updates read only its own links)
 *                  and classes are separated by cluster barriers.  Used where the slab fits
 *                  and neither "multihit" nor "persistent" is set; elsewhere, and with 0,
 *                  one launch per class.  Default 1 for UL_FP32_ACC64, 0 for UL_FP64.
 *                  Results are identical either way.
 *   "slab_cluster" CTAs per slab in the slab-resident form (a divisor of L, at most 16;
 *                  0, the default: the most CTAs up to 8 that keep every slab resident).
 *                  A size whose slab share does not fit falls back to one launch per class.
 *   "insertion_chunk_mb"  bound (MiB, default 16384) on the buffers that hold the
 *                  per-sample transporters and channel sums between insertion contractions
 *                  (UL_FP32_ACC64: a level is contracted in chunks of a quarter of its
 *                  sub-samples but at least 48; UL_FP64: in one chunk; smaller where the
 *                  bound requires; in the slab-resident form one chunk's
 *                  contraction overlaps the next chunk's updates); fewer MiB means more,
 *                  smaller contractions (results change only by rounding)
 *   "contract_tiled"  1 (default): the insertion contraction runs in a tiled form (per
 *                  block one slab, one z-plane, a tile of y-rows, two separations and a set
 *                  of offsets d; batches of samples staged in shared memory by bulk copies,
 *                  two blocks per SM); 0: one thread per output reading its operands from
 *                  global memory.  UL_FP32_ACC64: identical results either way.  UL_FP64:
 *                  the per-sample values are stored as double-single pairs of floats (48
 *                  significant bits) and the tiled form contracts them in double-single
 *                  arithmetic on the FP32 pipes (a slab mean of T O within
 *                  (2^-42 + n 2^-48) times the slab thickness for n samples per chunk), the
 *                  untiled form in FP64; the field sums differ by that much, everything else
 *                  is identical.  The 24-frame sums of UL_FP64 keep the untiled FP64 form.
 *                  A staging-copy wait that reaches its time limit (about a second) is
 *                  reported as UL_ETIMEOUT by the level's result call.
 *   "copy_stall_test"  0 (default), or n > 0 (integer <= 2e9): a test of the timeout path
 *                  of the tiled contraction (the FP32 kernel of UL_FP32_ACC64 and the
 *                  double-single kernel of UL_FP64).  Each block's first staged batch then waits for
 *                  16 bytes more than its copies deliver, so that wait gives up after n SM
 *                  cycles; the block reports the timeout, waits (up to the full limit, about
 *                  a second) while the copies it issued land, and leaves.  The level fails
 *                  with UL_ETIMEOUT and writes no results; set 0 to contract normally again.
 */
int ul_set_option(ul_lattice* h, const char* key, double value);

/* ul_get_links / ul_set_links — copy all 4V angles to / from a caller-owned host buffer
 * in the canonical layout, as FP64 (FP32 lattices are widened / rounded to nearest).
 * ul_set_links wraps nothing: inputs must lie in [-pi, pi). */
int ul_get_links(ul_lattice* h, double* theta_host);
int ul_set_links(ul_lattice* h, const double* theta_host);

/* ul_get_state / ul_set_state — the random-number state: seed and the count of
 * Metropolis passes done (the second Philox counter word).  With the links this is
 * the whole state: a restored state continues bit-identically. */
int ul_get_state(ul_lattice* h, uint64_t* seed, uint64_t* metro_pass);
int ul_set_state(ul_lattice* h, uint64_t seed, uint64_t metro_pass);

/* ul_get_stats — accepted Metropolis hits and proposed hits since ul_init. */
int ul_get_stats(ul_lattice* h, uint64_t* accepted, uint64_t* proposed);

/* ul_get_launch_count — number of CUDA kernels launched for this handle since ul_init. */
int ul_get_launch_count(ul_lattice* h, uint64_t* launches);

/* ul_synchronize — wait for all work enqueued on the handle's stream; reports
 * execution errors of earlier ul_sweep calls. */
int ul_synchronize(ul_lattice* h);

/* ul_set_stream — run this handle's work on the caller's CUDA stream (a cudaStream_t,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL returns to the handle's own stream. */
int ul_set_stream(ul_lattice* h, void* cuda_stream);

/* ul_last_error — text of the last error on h (or of the last failed ul_init if h is NULL). */
const char* ul_last_error(const ul_lattice* h);

/* ul_precision — UL_FP64 or UL_FP32_ACC64 for this handle (negative status on NULL). */
int ul_precision(const ul_lattice* h);

/* ---------------------------------------------------------------------------------
 * Batches: many independent lattices (different L, Nt, beta, seeds and schedules) on one
 * GPU.  Each job runs the program of a single handle — n_sweeps compound sweeps of
 * sweep_metro Metropolis + sweep_or overrelaxation passes (Section 2.1), then one
 * multilevel level of n_sub sub-samples of sub_metro + sub_or passes with frozen slab
 * boundaries and a transporter measurement (Section 2.2), the product across slabs and
 * the plaquette — and its results equal, bit for bit in FP64, those of a handle driven
 * by ul_init / ul_sweep / ul_multilevel / ul_plaquette with the same arguments.
 * All resident jobs advance together: one pass is one launch per (mu, parity) class
 * covering every lattice.  Jobs wait in a FIFO queue until their device memory fits in
 * the batch's budget (and one of 48 lattice slots is free) and release it when their
 * results are on the host, so work submitted while others run overlaps with them.
 * --------------------------------------------------------------------------------- */
typedef struct ul_batch ul_batch; /* opaque, library-owned */

typedef struct ul_job {
    int L, Nt;          /* even, >= 2, L^3 Nt <= 2^28 */
    double beta;        /* >= 0 */
    uint64_t seed;      /* Philox key of the hot start and of the Metropolis stream */
    int n_sweeps;       /* compound sweeps before the level (>= 0) */
    int sweep_metro;    /* Metropolis passes per compound sweep */
    int sweep_or;       /* overrelaxation passes per compound sweep */
    int slab_t;         /* slab thickness, divides Nt */
    int n_sub;          /* sub-samples of the level (>= 1) */
    int r_max;          /* correlator separations 1..r_max along x, r_max <= L/2 */
    int sub_metro;      /* Metropolis passes per sub-sample */
    int sub_or;         /* overrelaxation passes per sub-sample (sub_metro + sub_or >= 1) */
    double metro_width; /* Metropolis half-width in rad (> 0) */
} ul_job;

enum { UL_JOB_QUEUED = 0, UL_JOB_RUNNING = 1, UL_JOB_DONE = 2 };

/* ul_batch_create — a batch whose jobs all use `precision`, with a device-memory budget
 * of hbm_budget_bytes (allocated once here, >= 1 MiB) and work on cuda_stream (NULL: a
 * stream of the batch's own). */
int ul_batch_create(ul_batch** b, int precision, size_t hbm_budget_bytes, void* cuda_stream);

/* ul_batch_submit — queue a job; *job_id identifies it.  UL_EINVAL for an invalid job,
 * UL_ENOMEM if the job alone needs more memory than the whole budget. */
int ul_batch_submit(ul_batch* b, const ul_job* job, uint64_t* job_id);

/* ul_batch_step — admit queued jobs that fit, then run up to max_passes lockstep passes
 * (with the measurements and final reductions they reach).  Work is enqueued on the
 * batch's stream; the call blocks only when the launch queue is full (or, the first time a
 * shape reaches a slab-resident level with option "tune" on, while that shape's cluster
 * sizes are timed).  *n_active (may be NULL) receives the number of queued plus resident
 * jobs.  With the environment variable UL_BATCH_TRACE=1 every step prints its host stages
 * (admission, cluster-size tuning, slab-resident level launches, retirement) on stderr. */
int ul_batch_step(ul_batch* b, int max_passes, int* n_active);

/* ul_batch_poll — *state = UL_JOB_QUEUED, UL_JOB_RUNNING or UL_JOB_DONE.  When done, out
 * (2*r_max + 2 doubles) receives the correlator (re, im) for r = 1..r_max, the plaquette
 * and the Metropolis acceptance rate, and the job is released (a second poll of the same
 * id is UL_EINVAL). */
int ul_batch_poll(ul_batch* b, uint64_t job_id, double* out, int* state);

/* ul_batch_job_info — progress of a job that has not been collected yet: *state as in
 * ul_batch_poll (a finished job whose results are not yet collected reads UL_JOB_DONE),
 * *passes_done = update passes the engine has enqueued for it so far (each lockstep step
 * advances every resident job by one pass), *passes_total = its whole program (n_sweeps
 * compound sweeps and n_sub sub-samples).  Serving loops use it to show that jobs admitted
 * at different times advance in the same steps.  Any output may be NULL.  UL_EINVAL for
 * an unknown or already collected job. */
int ul_batch_job_info(ul_batch* b, uint64_t job_id, int* state, uint64_t* passes_done, uint64_t* passes_total);

/* ul_batch_stats — link updates and kernel launches issued so far, the block size the
 * last lockstep pass used (per shape of lattice the autotuner times 64/128/256 threads
 * (FP64) or 128/288/576 (FP32) on the first passes, or reads the choice from the tune cache;
 * results do not depend on it) and the device bytes held by jobs.  Link updates include
 * those of slab-resident levels. */
int ul_batch_stats(ul_batch* b, uint64_t* link_updates, uint64_t* launches, int* block_threads,
                   size_t* bytes_in_use);

/* ul_batch_set_option — batch options (none changes a result):
 *   "group_mb" (default 64, 1 .. 65536): the lockstep passes advance the jobs of one shape in
 *       groups whose links (angles and phases) fit this many MiB, each group for a whole
 *       step's passes in a row, so that its links stay in L2; each shape's passes run on a
 *       stream of their own, the largest shapes on the highest-priority streams.
 *   "slab_levels" (default 2): 1 runs a job's level as one slab-resident cluster launch where
 *       its slab fits (Section 2.2: with the slab boundaries frozen, the sub-samples of a slab
 *       read only its own links), shared by the jobs of one shape that reach their level in
 *       the same step, on a stream beside the lockstep passes; 2 does so only where two of
 *       that launch's CTAs fit one SM's shared memory (a level of larger slabs would hold
 *       whole SMs that the other shapes' passes cannot share); 0 runs every level in the
 *       lockstep passes.
 *   "tune" (default 1): choose each shape's cluster size by timing every feasible size once
 *       on a scratch lattice (a cudaMalloc/cudaFree, the first time a shape is seen) and keep
 *       the choice in the tune cache, a JSON file ($UL_TUNE_CACHE, else $XDG_CACHE_HOME or
 *       $HOME/.cache + /paper_1208_0166_gb300/tune.json; UL_TUNE_CACHE="" keeps it in
 *       memory), which also records the lockstep block size per shape; 0 uses the largest
 *       cluster whose slabs are all resident.
 * UL_EINVAL for a value out of range or an unknown key. */
int ul_batch_set_option(ul_batch* b, const char* key, double value);

/* ul_batch_plan — *cluster = CTAs per slab of the slab-resident level the batch would use
 * for jobs of shape (L, Nt, slab_t) (tuning it now if needed), 0 where the level runs in
 * the lockstep passes; *slab_launches = slab-resident level launches so far.  Either output
 * may be NULL. */
int ul_batch_plan(ul_batch* b, int L, int Nt, int slab_t, int* cluster, uint64_t* slab_launches);

/* ul_batch_counters — slab-resident level launches so far (the output may be NULL). */
int ul_batch_counters(ul_batch* b, uint64_t* slab_level_launches);

/* ul_batch_free — wait for the batch's streams and release everything (NULL accepted). */
int ul_batch_free(ul_batch* b);

/* ul_batch_last_error — text of the last error on b. */
const char* ul_batch_last_error(const ul_batch* b);

#ifdef __cplusplus
}
#endif
#endif
