// vegas_batch.cuh -- device-side description of a batch of independent
// integrals that share one launch of every step (the batched form of
// Algorithm 1 of cuVegas; the paper runs one integral per launch).
//
// Every integral keeps its own FillArgs (map, counts, strata, parameters) in
// device memory.  Work lists are prefix sums over the integrals still
// running: tiles for the fill and its fix-up, blocks of kBlockCubes cubes for
// the allocation passes.  A launch over such a list finds the integral of an
// item by a binary search in the prefix array.
#pragma once
#include <cstdint>

#include "vegas_internal.h"

namespace vg {

constexpr int kBatchMaxProblems = 4096;
constexpr int kBatchMaxDim = 16;

// batched fill variants: minimum resident CTAs per SM of the launch bound
constexpr int kBatchVariants = 2;
constexpr int kBatchMinBlocks[kBatchVariants] = {4, 2};
// The fill runs one persistent kernel per group of integrals with the same family and width (3 families x
// widths 4, 8, 16): each kernel holds one instance of the fill's tile code, so its registers are those of that
// instance alone (one kernel over every group spilled to local memory at 64 registers).
constexpr int kBatchGroups = 9;
__host__ __device__ inline int batch_group(int iid, int dmax) {
  const int fam = iid == VEGAS_GAUSS_SUM ? 0 : iid == VEGAS_PRODUCT_PEAK ? 1 : 2;
  return fam * 3 + (dmax == 4 ? 0 : dmax == 8 ? 1 : 2);
}

// per-integral data that only the batched driver uses
struct BatchProblem {
  FillArgs a;       // the fill's arguments; a.iter advances on the device
  double* bins;     // [d*G] map weights, accumulated with FP64 atomics
  uint64_t* bsum;   // [nblocks + 1] allocation block sums
  int64_t nblocks;  // allocation blocks of kBlockCubes cubes
  double* it_est;   // [cap] I_t of every recorded iteration
  double* it_sig;   // [cap] sigma_t
  int dmax;         // 4, 8 or 16: the fill instantiation
  int group;        // batch_group(family, dmax): the fill kernel that runs it
};

// batch-wide state, in device memory
struct BatchCtl {
  int32_t active;     // 1 while the integral takes part in the iterations
  int32_t uniform;    // 1: the next allocation is uniform
  int32_t nrec;       // iterations recorded
  int32_t converged;  // reached the relative-error target
};

// everything the batched kernels read, passed by value
struct BatchLaunch {
  int P, G;
  double alpha, rtol;
  int skip, chunk_tiles;
  BatchProblem* prob;    // [P]
  BatchCtl* ctl;         // [P]
  int32_t* act_tile;     // [P+1] prefix of the tiles of running integrals
  int32_t* grp_tile;     // [kBatchGroups][P+1] the same prefix restricted to each fill group
  int64_t* act_blk;      // [P+1] prefix of their allocation blocks
  uint32_t* counter;     // [2 + kBatchGroups] running integrals after the iteration at [1]; fill work
                         // counter of group g at [2 + g]
  double* acc;           // [P][2] sum of cube means, sum of cube variances
  int* key;              // [P] order-preserving key of the largest ell
  int* flags;            // [P] 1: non-finite value, 2: a split cube was not reassembled
  double* out;           // [P][4] estimate, sigma, chi2/dof, iterations used
  uint32_t rk0[10], rk1[10];  // Philox round keys (one seed for the batch)
};

// integral of item i of a prefix array pre[0..P] (pre[p] <= i < pre[p+1]);
// integrals with no items are skipped because their range is empty
template <typename I>
__device__ __forceinline__ int batch_find(const I* __restrict__ pre, int P, I i) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the fill of group g (batch_group) in register-budget variant v; one definition per family file
int launch_batch_fill(int variant, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s);
int batch_fill_occupancy(int variant, int group, int smem);
int launch_batch_fill_gauss(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s);
int launch_batch_fill_peak(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s);
int launch_batch_fill_osc(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s);
int batch_fill_occupancy_gauss(int variant, int dmax, int smem);
int batch_fill_occupancy_peak(int variant, int dmax, int smem);
int batch_fill_occupancy_osc(int variant, int dmax, int smem);

}  // namespace vg
