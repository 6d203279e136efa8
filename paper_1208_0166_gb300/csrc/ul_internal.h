// ul_internal.h — launchers shared between the C-ABI layer and the kernel translation
// units.  Each launcher is instantiated for double (FP64 path, ul_kernels_f64.cu) and
// float (FP32 path, ul_kernels_f32.cu).  Device buffers are passed as plain pointers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ul_batch_types.h"

namespace ul {

struct Geo;

// SM cycles (about a second) a tiled insertion contraction waits for a batch of bulk copies
// before it reports a timeout (status 2).  wait_cycles of the launchers: the limit of that
// first wait of each batch; a negative value -n runs the timeout test (the first batch's
// barrier expects 16 bytes more than its copies deliver, so its wait gives up after n
// cycles).  The wait that lets copies in flight land before a block leaves always has the
// full limit.
constexpr long long kCopyWaitLimit = 2000000000LL;

// Largest number of time slabs one multilevel level may have.
constexpr int kMaxSlabs = 256;

// Check word of the FP64 (R = double) or FP32 (R = float) kernel unit in the
// bounds-checked build (see UL_IDX in ul_device.cuh); 0 in the default build.
template <typename R>
cudaError_t check_word(unsigned long long* out, bool clear);

template <typename R>
cudaError_t launch_hot_start(const Geo& g, R* theta, void* cs, uint64_t seed, cudaStream_t st);

template <typename R>
cudaError_t launch_refresh_cs(const Geo& g, const R* theta, void* cs, cudaStream_t st);

// One sub-sweep of class (mu, parity).  slab_t > 0 freezes spatial links on slices
// t % slab_t == 0.  metro selects Metropolis (else overrelaxation).  The Metropolis pass
// number is pass + *pass_base (pass_base may be null).  *launched is 0 when the class has
// no updatable link (a spatial class with slab_t == 1) and nothing was launched.  pdl:
// launch with programmatic stream serialization (the kernel may be scheduled while the
// previous kernel of the stream runs; it reads no link before that kernel completed).
template <typename R>
cudaError_t launch_update_class(const Geo& g, R* theta, void* cs, int mu, int parity, bool metro,
                                uint64_t pass, const unsigned long long* pass_base, uint64_t seed, double beta,
                                double width, int slab_t, unsigned long long* accepted, cudaStream_t st,
                                int* launched, bool pdl);

// Metropolis uniforms of links link0 .. link0+n-1 (out: 2n doubles, device memory).
template <typename R>
cudaError_t launch_rng_uniforms(uint64_t seed, uint64_t pass, uint64_t link0, int n, double* out, cudaStream_t st);

// *p = v (one thread); sets the pass base read by graph-replayed update kernels.
cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st);

template <typename R>
cudaError_t launch_to_canonical(const Geo& g, const R* theta, double* canon, cudaStream_t st);

template <typename R>
cudaError_t launch_from_canonical(const Geo& g, const double* canon, R* theta, void* cs, cudaStream_t st);

// Mean plaquette into *out_dev; partials must hold plaquette_partials(g) doubles.
int plaquette_partials(const Geo& g);
template <typename R>
cudaError_t launch_plaquette(const Geo& g, const void* cs, double* partials, double* out_dev, cudaStream_t st);

// Measurement after one sub-sample: T into asum (FP64); with fields, T and the slab
// channel sums O stored in sample slot `slot` of tk / ok (precision R) and O added to osum.
template <typename R>
cudaError_t launch_measure_store(const Geo& g, const void* cs, int slab_t, int r_max, bool fields, int slot,
                                 double2* asum, void* tk, void* ok, double* osum, const void* ubar, cudaStream_t st);

// Symmetrised measurement after one sub-sample (transporters along the three axes into
// asum3 / tk3 slot `slot`, the six plaquette planes per site into the one-sample scratch o12
// and osum12, the frame sums per insertion midpoint into csym slot `slot`) and the
// symmetrised contraction of the first `count` stored samples into bsum3 (layouts in
// ul_sym.cuh).
template <typename R>
cudaError_t launch_measure_sym(const Geo& g, const void* cs, int slab_t, int r_max, int nd, int slot, double2* asum3,
                               void* tk3, void* o12, void* csym, double* osum12, cudaStream_t st);
template <typename R>
cudaError_t launch_insertion_contract_sym(const Geo& g, int slab_t, int r_max, int nd, int count, const void* tk3,
                                          const void* csym, double2* bsum3, bool first, cudaStream_t st, bool tiled,
                                          int* status, long long wait_cycles = kCopyWaitLimit);

// Multihit temporal links ubar[i] (lexicographic site i, complex in precision R).
template <typename R>
cudaError_t launch_multihit(const Geo& g, const void* cs, double beta, void* ubar, cudaStream_t st);

// bsum[(((s*R + r-1)*nd + d)*8 + ch)*L3 + x0] += sum over the first `count` stored samples of
// T(s,x0,r) O(s, x0 + floor(r/2) xhat + d yhat, ch); with `first` bsum is written, not read
// (the level's first chunk: no zeroing of the field sums needed).  tiled: FP32 links use the
// shared-memory tiled form where it applies (same bits as the untiled kernel); its bounded
// waits for the staging copies write 2 to *status when they give up.
template <typename R>
cudaError_t launch_insertion_contract(const Geo& g, int slab_t, int r_max, int nd, int count, const void* tk,
                                      const void* ok, double2* bsum, bool first, cudaStream_t st, bool tiled,
                                      int* status, long long wait_cycles = kCopyWaitLimit);

// Raises the dynamic shared-memory limit of the tiled FP32 contraction (once per process,
// before any launch or graph capture that may use it).
template <typename R>
cudaError_t prepare_insertion_contract();

// Raises the dynamic shared-memory limit of the reduction that keeps the other-slab
// weights in shared memory (up to 50 slabs; more slabs use a per-thread prefix array).
cudaError_t prepare_ml_reduce();

// Cross-slab products, x0 reduction and normalisation.  out_dev receives
// 2*r_max doubles (correlator) followed by 2*r_max*nd*8 doubles (fields) and 8 (vacuum).
size_t ml_partials_doubles(const Geo& g, int r_max, int nd);
// out[ch] = sum of osum[ch*SL3 .. ch*SL3 + SL3) / nV for ch < nch.
cudaError_t launch_ml_vacuum(int SL3, const double* osum, int nch, double nV, double* out, cudaStream_t st);
cudaError_t launch_ml_reduce(const Geo& g, int slab_t, int n_sub, int r_max, int nd, const double2* asum,
                             const double2* bsum, const double* osum, double* partials, double* out_dev,
                             cudaStream_t st);

// Two-level multilevel: add the level-1 samples (products of the level-2 means inside each
// level-1 slab) of the level-2 accumulator asum2 to asum1.
cudaError_t launch_fold_level2(const Geo& g, int tau1, int tau2, int r_max, int n2, const double2* asum2,
                               double2* asum1, cudaStream_t st);

// Two-level multilevel with insertions: add the level-1 samples of the level-2 accumulators
// (asum2, bsum2 over n2 samples) to asum1, bsum1 (tau1 / tau2 <= 16).
cudaError_t launch_fold_level2_fields(const Geo& g, int tau1, int tau2, int r_max, int nd, int n2,
                                      const double2* asum2, const double2* bsum2, double2* asum1, double2* bsum1,
                                      cudaStream_t st);

// Persistent cooperative sweep kernel (256 threads per block; `threads` is ignored).
template <typename R>
cudaError_t launch_persistent(const Geo& g, R* theta, void* cs, const PersistArgs& in, int threads, cudaStream_t st);

// Slab-resident sub-samples (one thread-block cluster per slab, links in shared memory).
// slab_plan sets *cluster to the CTAs per slab (0: the slab does not fit, or the cluster
// shape cannot launch) and *threads to the block size; force_cluster > 0 asks for that
// cluster size only.
template <typename R>
cudaError_t slab_plan(const Geo& g, int tau, int force_cluster, int* cluster, int* threads);
// Shared memory of one CTA of a slab-resident launch (cluster CTAs per slab).
template <typename R>
size_t slab_level_smem(const Geo& g, int tau, int cluster);
template <typename R>
cudaError_t launch_slab(const Geo& g, R* theta, void* cs, const SlabArgs& a, int threads, cudaStream_t st);

// One slab-resident level for every lattice of a table (same shape g and plan); see
// slab_jobs_kernel in ul_slab.cuh.
template <typename R>
cudaError_t launch_slab_jobs(const Geo& g, const SlabArgs& a, const SlabJobTable& t, int threads, cudaStream_t st);

// Lockstep class update of a group of lattices of one extent L (grid: blocks_x blocks of
// `threads` per lattice, t.njobs lattices), and its measurement (blocks_x blocks of 256).
template <typename R>
cudaError_t launch_group_update(const BatchUpdateTable& t, int L, int blocks_x, int threads, int mu, int parity,
                                cudaStream_t st, bool pdl);
template <typename R>
cudaError_t launch_group_measure(const BatchMeasureTable& t, int blocks_x, cudaStream_t st);

// Block size of a one-class launch of `work` links (the single-lattice choice): FP32 wide
// blocks, FP64 balanced blocks.
int class_block_threads(long work, bool fp32);

} // namespace ul
