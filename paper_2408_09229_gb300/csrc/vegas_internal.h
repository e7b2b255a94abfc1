// vegas_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vegas.h"

namespace vg {

constexpr int kMaxDim = 32;
constexpr int kMaxBins = 4096;
constexpr int kFillThreads = 256;
// Tiles of the fill: 2^tile_log2 consecutive evaluations, 2^(tile_log2 - 8) a thread.  A launch takes 2048
// unless that costs a resident CTA (the shared-memory staging grows with the tile), then 1024.
constexpr int kTileLog2Min = 10, kTileLog2Max = 11;
constexpr int kTileMax = 1 << kTileLog2Max;
static_assert(kFillThreads == 256, "tiles of 2^tile_log2 evaluations: 2^(tile_log2 - 8) a thread");
// how the fill accumulates the map weights
constexpr int kHistShared = 0;    // shared-memory histogram of the evaluation type, atomic adds
constexpr int kHistGlobal = 1;    // per-CTA global histogram, FP64 atomic adds (large d * N_g)
constexpr int kHistTwoPhase = 2;  // FP32: fixed-point tile histogram with shared integer atomics
constexpr int kLongSegment = 32;  // longer cube segments go to a warp
// the cubes a tile of n evaluations can meet (n_h >= 2), and its segments longer than kLongSegment
__host__ __device__ constexpr int tile_max_cubes(int n) { return n / 2 + 3; }
__host__ __device__ constexpr int tile_max_long(int n) { return n / (kLongSegment + 1); }
constexpr int kMaxDerivedParams = 8192;
constexpr int kAllocThreads = 256;
constexpr int kAllocItems = 16;  // cubes per thread in the allocation scan
constexpr int64_t kMaxEval = (int64_t(1) << 31) - 1;
// The FP32 form's evaluation-rounding floor, relative to |I|: the estimate carries a rounding bias of a few FP32
// ulps of each value (map fused multiply-add, ex2 within 2 ulp, the integrand's sums), measured up to 1.1e-6 on
// single-iteration 2-d results and 1.3e-7 at full size.  A stated sigma below 2^-20 |I| (16 ulps) is not a
// statistical error the result can be trusted to: the rtol test uses max(sigma, floor |I|) and the result is flagged.
constexpr double kFp32SigmaFloor = 0x1p-20;
// internal integrand identifiers of the fill (not in the public enumeration):
// tabulated values f_j = values[j] by evaluation index, and a points-only
// pass that writes the evaluation points and nothing else
constexpr int kIntegrandTabulated = 100;
constexpr int kIntegrandPoints = 101;

// Per-tile record of a cube that crosses a tile edge: the tile's part of its
// evaluations as (count, mean, centred second moment).
struct Carry {
  int32_t h;    // cube, -1 when the slot is empty
  int32_t cnt;  // evaluations of the cube inside the tile
  double mean;
  double m2;
};

// Everything the fill kernel needs; passed by value.
struct FillArgs {
  int d, G, NH, ntiles;
  int64_t neval;
  uint32_t key0, key1, iter, pid;
  float half_beta;
  int table_smem;  // 1: map table in shared memory
  int hist_mode;   // kHistShared, kHistGlobal or kHistTwoPhase
  int bin_shift;   // two-phase: log2 of the bits of a packed interval index (3: 8 bits, N_g <= 256; 4: 16 bits)
  int acc32;       // two-phase: 1 when the CTA histogram accumulates in FP32 (large d * N_g), 0 for float-float
  int hist_rep_log2;  // shared FP64 histogram: log2 of its copies; lane l adds into copy l mod 2^hist_rep_log2
  int tile_log2;      // evaluations per tile: 2^tile_log2 (kTileLog2Min .. kTileLog2Max)
  int wv_recompute;   // streamed path: phase B recomputes each evaluation's weight (the layout has no weight slots)
  int np_derived;
  int iid;  // integrand family (the batched fill dispatches on it per tile)
  const double* edges;     // [d][G+1] FP64
  const int64_t* offsets;  // [NH+1]
  const int32_t* tile_first;
  const double* params_raw;  // caller params (device)
  int np_raw;
  float* ell;
  double* cube_mean;
  double* cube_m2;
  int* flags;
  int* ellmax_key;
  Carry* carries;       // [2*ntiles]
  double* cta_part;     // [grid][2]
  double* hist_part;    // [grid][d*G]
  void* gtable;         // global map table when it does not fit in shared memory
  const int* vexp;      // FP32 value scale exponent (see value_exponent), or NULL for 0
  const float* values;  // kIntegrandTabulated: f of evaluation j
  float* points_out;    // kIntegrandPoints: [neval][d] evaluation points
  float* train_w;       // kIntegrandTabulated: (|J f| / n_h)^train_power of evaluations j = i * train_stride
  int train_stride;
  float train_power;
  uint32_t nstrat[kMaxDim], magic[kMaxDim], shift[kMaxDim];
  double gz64[kMaxDim];     // N_g / s_k, rounded in FP64
  float gzb32[kMaxDim];     // RN32(N_g / s_k) 2^-b_k
  float gzn32[kMaxDim];     // -2^23 RN32(N_g / s_k) 2^-b_k
  uint32_t fbits[kMaxDim];  // b_k = 23 - ceil(log2 s_k): fraction bits of an FP32 coordinate
  uint32_t rk0[10], rk1[10];  // Philox round keys
  // shared-memory byte offsets of the regions
  int sm_table, sm_hist, sm_hacc, sm_bins, sm_wv, sm_params, sm_off, sm_raw, sm_invn, sm_vals, sm_long, sm_start, sm_misc,
      sm_total;
};

// launchers (one per precision, defined in vegas_fill_f64.cu / vegas_fill_f32.cu)
int launch_fill_f64(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s);
int launch_fill_f32(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s);
int fill_occupancy_f64(int integrand, int dmax, int tile_log2, int smem);
int fill_occupancy_f32(int integrand, int dmax, int tile_log2, int smem);
// d == dmax (4 or 8) and the map table in shared memory
int launch_fill_f64_exact(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s);
int launch_fill_f32_exact(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s);
int fill_occupancy_f64_exact(int integrand, int dmax, int tile_log2, int smem);
int fill_occupancy_f32_exact(int integrand, int dmax, int tile_log2, int smem);
// DMAX 16 or 32 with the streamed point path (FP32, two-phase histogram, s_k <= 256)
int launch_fill_f32_stream(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s);
int fill_occupancy_f32_stream(int integrand, int dmax, int tile_log2, int smem);

// buffers of the internal integrands (kIntegrandTabulated, kIntegrandPoints)
struct FillExtra {
  const float* values;
  float* points;
  float* train_w;
  int train_stride;
  float train_power;
};

int fill_impl(const vegas_geometry* g, int precision, int integrand, const double* d_params, int64_t nparams,
              int64_t neval, uint64_t seed, int32_t iteration, uint32_t problem_id, double beta,
              const double* d_edges, const int64_t* d_offsets, float* d_ell, double* d_bins, double* d_result,
              double* d_cube_mean, double* d_cube_m2, int* d_flags, void* d_scratch, size_t scratch_bytes,
              void* stream, cudaEvent_t ev_before, cudaEvent_t ev_after, const FillExtra* extra = nullptr);
int allocate_impl(const float* d_ell, int64_t ncubes, int64_t neval, int uniform, int64_t* d_offsets,
                  void* d_scratch, size_t scratch_bytes, cudaStream_t s, const int* d_key);
// device address of the fill's max-ell key inside its scratch area
const int* fill_ellmax_key(const vegas_geometry* g, int64_t neval, const void* d_scratch);
int launch_record_combine(const double* d_result, int t, double* d_est, double* d_sig, int skip, double* d_out,
                          bool lagged, cudaStream_t s);

int dmax_for(int d);
// learned proposal (vegas_flow.cu)
int flow_apply(int d, int direction, const float* d_params, const float* d_xin, float* d_xout, float* d_logdet,
               int64_t n, cudaStream_t s);
// VEGAS_ETIMEOUT when a bounded wait of the tensor-core transform ran out since the last reset
int flow_tc_status(bool reset);
int flow_tc_wait_selftest(int polls, int arrive, cudaStream_t s);
// the same report for the tensor-core training gradient (vegas_flow_grad_tc.cu)
int flow_grad_tc_status(bool reset);
int flow_eval(int integrand, int d, const double* d_params, int64_t nparams, const float* X, const float* logdet,
              float* values, int64_t n, cudaStream_t s);
// training set of an iteration: every kFloorPeriod-th row a uniform point when lambda > 0
constexpr int kFloorPeriod = 4;
int64_t flow_train_rows(int64_t m, float lambda);
int flow_gather(const float* X, int d, int64_t stride, int64_t m, const float* w, float lambda, uint64_t seed,
                uint32_t iter, double* wsum, float* xs, float* ws, cudaStream_t s);
// exploration (vegas_explore.cu): m samples of S maps [S][d][G+1], sample r from map r mod S, as FP32 points X [m][d]
// and the mixture density q [m]; the weights |f| / q (0 where not finite)
constexpr int kMaxExploreMaps = 64;
int explore_points(int d, int G, int S, const double* maps, int64_t m, uint64_t seed, float* X, double* q,
                   cudaStream_t s);
int explore_weights(const float* f, const double* q, int64_t m, float* w, cudaStream_t s);
// A single-integral fill launch: its arguments (tile, layout), the kernel it takes and its resident CTAs per SM.
struct FillPlan {
  FillArgs a;
  bool exact, streamed;
  int per_sm;
};
// The launch plan of the single-integral fill for base (d, G, neval and the rest set): with tile_log2 = 0 the
// tile size that keeps the exact-d path and the most resident CTAs, the larger on a tie; else that tile.
int fill_plan(const FillArgs& base, const int32_t* nstrat, int precision, int integrand, int64_t nparams, int nprm,
              FillPlan& out, int tile_log2 = 0);
// prefetch: reserve the buffer of the next tile's offsets (the single-integral fill; the batched fill does not
// prefetch)
int fill_args_axes(FillArgs& a, const int32_t* nstrat, int precision, int nprm, bool prefetch = true,
                   bool streamed = false);
int derived_param_count(int integrand, int d, const double* host_params_or_null, int64_t np);

// status helpers
inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? VEGAS_OK : VEGAS_ECUDA; }
// At the start of a call that launches kernels: an error that an earlier, unrelated runtime call left in the
// last-error slot (a failed stream capture, the caller's own failed call) is not this call's.  A sticky error
// (a device fault) stays: the call's own runtime calls report it.
inline void clear_stale_error() { cudaGetLastError(); }

}  // namespace vg

// A failed runtime call also leaves its error in the runtime's last-error slot;
// clear it, so that the launch check of a later call (cudaGetLastError) does
// not report this error a second time.
#define VG_CHECK(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) {                            \
      cudaGetLastError();                               \
      return VEGAS_ECUDA;                               \
    }                                                   \
  } while (0)
