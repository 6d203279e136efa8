// ul_batch_types.h — argument blocks of the update, persistent and batched kernels
// (shared by the kernel translation units and the host layer).  A table travels by value in the kernel's
// parameter block, so it is limited to kMaxBatchJobs lattices per launch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ul {

// Arguments of one class update (uniform over a launch).
struct UpdateArgs {
    int parity, metro, slab_t;
    unsigned long long frozen_mask; // bit t: spatial links on slice t frozen (Nt <= 64)
    uint64_t pass;
    const unsigned long long* pass_base;
    uint64_t seed;
    double beta, width;     // FP64 kernels
    float beta_f, width_f;  // FP32 kernels
    unsigned long long* accepted;
};

// Arguments of a persistent sweep launch (see persistent_kernel).
struct PersistArgs {
    UpdateArgs u;             // u.pass: first Metropolis pass number of this launch
    int n_units;              // compound sweeps, or sub-samples when measure = 1
    int n_metro, n_or;        // passes per unit
    int measure;              // 1: measurement after each unit
    int r_max, fields, slot0; // measurement: correlator separations, insertions, first sample slot
    double2* asum;
    void* tk;
    void* ok;
    double* osum;
    void* ubar;               // multihit temporal links (null: correlator from the links themselves)
    unsigned int* bar;        // arrival counter, zero at launch
    int* status;              // 0 = ok; set when a wait gives up
    unsigned int expected;    // blocks that arrive at each barrier
    unsigned long long spin_limit;
};

// Arguments of a slab-resident sub-sample launch (see slab_kernel).
struct SlabArgs {
    UpdateArgs u;             // u.pass: first Metropolis pass; u.slab_t: slab thickness
    int n_units;              // sub-samples (each: passes, then one measurement)
    int n_metro, n_or;        // passes per sub-sample
    int cluster, nz;          // CTAs per slab (one cluster), z planes per CTA
    int r_max, fields, slot0; // measurement as in PersistArgs
    int skip_measure;         // 1: passes only (the caller measures after the launch)
    double2* asum;
    void* tk;
    void* ok;
    double* osum;
};

constexpr int kMaxBatchJobs = 48;

// One lattice of a slab-resident launch over several lattices of one shape (L, Nt, slab
// thickness): its links, its Metropolis arguments (first pass, seed, coupling, width,
// acceptance counter), its transporter accumulator and its own level schedule.
struct SlabJob {
    void* theta;
    void* cs;
    double2* asum;
    UpdateArgs u;
    int n_units, n_metro, n_or, r_max;
};

constexpr int kMaxSlabJobs = 16;

struct SlabJobTable {
    int njobs;
    SlabJob job[kMaxSlabJobs];
};

struct BatchUpdateJob {
    void* theta;
    void* cs;
    unsigned long long* accepted;
    int L, Nt, V, Vh, L3;
    int metro, slab_t;
    unsigned long long frozen_mask;
    uint64_t pass, seed;
    double beta, width;
};

struct BatchUpdateTable {
    int njobs;
    BatchUpdateJob job[kMaxBatchJobs];
};

struct BatchMeasureJob {
    const void* cs;
    double2* asum;
    int L, Nt, V, Vh, L3;
    int slab_t, r_max;
};

struct BatchMeasureTable {
    int njobs;
    BatchMeasureJob job[kMaxBatchJobs];
};

} // namespace ul
