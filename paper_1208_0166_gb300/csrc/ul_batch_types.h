// ul_batch_types.h — parameter tables of the batched kernels (shared by the kernel
// translation units and the batch engine).  A table travels by value in the kernel's
// parameter block, so it is limited to kMaxBatchJobs lattices per launch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ul {

constexpr int kMaxBatchJobs = 48;

struct BatchUpdateJob {
    void* theta;
    void* cs;
    unsigned long long* accepted;
    int L, Nt, V, Vh, L3;
    int block0;
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
    int block0;
    int slab_t, r_max;
};

struct BatchMeasureTable {
    int njobs;
    BatchMeasureJob job[kMaxBatchJobs];
};

} // namespace ul
