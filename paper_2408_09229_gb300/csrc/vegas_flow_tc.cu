// vegas_flow_tc.cu -- the coupling flow's batched transform (vegas_flow_apply)
// on the fifth-generation tensor cores: tcgen05.mma with the accumulators in
// tensor memory.  The flow is defined in vegas_flow.cuh.
//
// A persistent CTA on each SM holds the six layers' weights in shared memory
// and runs several warpgroups, each transforming its own tile of 128 points,
// so that while one waits for its MMAs the others run their element-wise
// work: 8 warpgroups up to 16 axes (flow_apply_u64_kernel), 4 above
// (flow_apply_tc_kernel).  Thread t of a warpgroup owns point t of the tile:
// it keeps the point's z in registers and reads row t of every accumulator
// (tensor-memory lane t).  Per coupling layer:
//   H  = [bf16(z[A]) | 1 1 1 | 0]     128 x K1   (the first K1 columns of U)
//   D  = H W1'^T                      128 x 64   (tensor memory)
//   U  = bf16(relu D)                 128 x 64   (shared memory)
//   D  = [U | ONES] W2'^T;  U = bf16(relu D)
//   D  = [U | ONES] W3'^T             128 x N3
// then s, t from D and the affine update of z[B].  ONES is a 128 x 16 block
// whose first three columns are one: above 16 axes it is the last 16 columns
// of each tile's U (128 x 80), up to 16 axes one shared tile that the bias
// k-step's descriptor points at.  The primed weights carry the bias in three
// extra columns as a bf16 triple (hi, mid, lo) with hi + mid + lo = b to
// 2^-24 relative, multiplied by those ones: the bias enters the FP32
// accumulation at full FP32 precision.  One thread of the warpgroup issues
// the MMAs; every thread waits (bounded) on the warpgroup's mbarrier, which
// the MMAs' completion arrives on.
#include <algorithm>
#include <type_traits>

#include "vegas_flow.cuh"
#include "vegas_internal.h"
#include "vegas_flow_tc.cuh"
#include "vegas_tc.cuh"

namespace vg {

namespace {

// a module-wide status word: bit 2 is set when a bounded wait ran out
__device__ int g_flow_tc_status;

// H or U written: thread 0 issues the GEMM, every thread waits (bounded) for
// its completion; false on every thread of the warpgroup once any wait ran out
__device__ __forceinline__ bool tc_run(TcGroup& G, const unsigned char* A, const unsigned char* B, int KA, int K,
                                       uint32_t idesc) {
  tc_fence_proxy();
  tc_fence_before();
  if (wg_bar_any(1 + G.id, G.failed)) return false;
  if (G.t == 0) {
    tc_fence_after();
    tc_gemm(G.tacc & 0xFFFFu, A, B, KA, K, idesc);  // thread 0 is in lane quarter 0
    tc_commit(G.mbar);
  }
  if (!mbar_wait(G.mbar, G.phase, kTcWaitPolls)) {
    G.failed = true;
    atomicOr(&g_flow_tc_status, 4);
  }
  G.phase ^= 1u;
  tc_fence_after();
  return true;
}

// one coupling layer on the warpgroup's tile; PAR = l mod 2
template <int D, int PAR>
__device__ __forceinline__ bool tc_layer(const unsigned char* wl, unsigned char* U, TcGroup& G, int dir,
                                         float (&z)[D], float& ld) {
  using S = TcShape<D>;
  constexpr int a = PAR == 0 ? (D + 1) / 2 : D / 2, b = D - a;  // conditioning and moved axes
  const int t = G.t;
  // H row t: the conditioning axes 2c + PAR, then the three ones of the bias
#pragma unroll
  for (int q = 0; q < S::K1 / 8; ++q) {
    float hv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = 8 * q + e;
      hv[e] = c < a ? z[2 * c + PAR] : (c < a + 3 ? 1.0f : 0.0f);
    }
    st_shared_v4(U + tc_off(t, 8 * q, kTcK2), bf16x2(hv[0], hv[1]), bf16x2(hv[2], hv[3]), bf16x2(hv[4], hv[5]),
                 bf16x2(hv[6], hv[7]));
  }
  const unsigned char* w1 = wl;
  const unsigned char* w2 = wl + S::W1;
  const unsigned char* w3 = w2 + S::W2;
  if (!tc_run(G, U, w1, kTcK2, S::K1, tc_idesc_bf16(128, 64))) return false;
  tc_hidden_epilogue(G.tacc, U, t);
  tc_fence_before();
  if (!tc_run(G, U, w2, kTcK2, kTcK2, tc_idesc_bf16(128, 64))) return false;
  tc_hidden_epilogue(G.tacc, U, t);
  tc_fence_before();
  if (!tc_run(G, U, w3, kTcK2, kTcK2, tc_idesc_bf16(128, S::N3))) return false;
  float o[S::N3];
  if constexpr (S::N3 == 16) {
    tc_ld16(G.tacc, o);
  } else {
    tc_ld32(G.tacc, o);
  }
  tc_fence_before();
  // pair m = (s_m, t_m) moves axis 2m + 1 - PAR
#pragma unroll
  for (int m = 0; m < b; ++m) {
    const int k = 2 * m + 1 - PAR;
    {
      const float s = flow_soft_clamp(o[2 * m]), tt = o[2 * m + 1];
      if (dir > 0) {
        z[k] = fmaf(z[k], __expf(s), tt);
        ld += s;
      } else {
        z[k] = (z[k] - tt) * __expf(-s);
        ld -= s;
      }
    }
  }
  return true;
}

template <int D>
__global__ void __launch_bounds__(TcShape<D>::threads, 1)
    flow_apply_tc_kernel(const __grid_constant__ FlowArgs fa, int dir, const float* __restrict__ xin,
                         float* __restrict__ xout, float* __restrict__ logdet, int64_t n) {
  using S = TcShape<D>;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int warp = threadIdx.x >> 5;
  uint64_t* mbars = reinterpret_cast<uint64_t*>(sm + S::misc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::misc + 8 * S::G);
  tc_stage_weights<D>(fa, sm);
  if (warp == 0) tc_alloc(tslot, S::tmem_cols);
  if (threadIdx.x == 0) {
    for (int g = 0; g < S::G; ++g) mbar_init(mbars + g, 1);
    mbar_fence_init();
  }
  tc_fence_proxy();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  TcGroup G;
  G.id = threadIdx.x >> 7;
  G.t = threadIdx.x & 127;
  G.tacc = tbase + (uint32_t)(G.id * kTcColsPerGroup) + ((uint32_t)((warp & 3) * 32) << 16);
  G.mbar = mbars + G.id;
  G.phase = 0;
  G.failed = false;
  unsigned char* U = sm + S::weights + G.id * S::U;
  float* stg = reinterpret_cast<float*>(U);
  constexpr int zld = S::ZLD;
  const int t = G.t;
  const int64_t ntiles = (n + 127) / 128;

  for (int64_t tile = (int64_t)blockIdx.x * S::G + G.id; tile < ntiles; tile += (int64_t)gridDim.x * S::G) {
    const int64_t r0 = tile * 128;
    const int rows = (int)min((int64_t)128, n - r0);
    // the tile's x, coalesced, into rows of stride zld (odd: conflict-free row reads); all loads first
    {
      float xl[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int i = t + 128 * j;
        xl[j] = i < rows * D ? xin[r0 * D + i] : 0.5f;
      }
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int i = t + 128 * j;
        stg[(i / D) * zld + i % D] = xl[j];
      }
    }
    wg_bar(1 + G.id);
    float z[D];
    float ld = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      z[k] = flow_logit(stg[t * zld + k]);
      ld -= flow_log_sig_prime(z[k]);
    }
    wg_bar(1 + G.id);
    // the bias block of U: ones in columns 64-66, zeros in 67-79
    st_shared_v4(U + tc_off(t, kFlowHidden, kTcK2), 0x3F803F80u, 0x00003F80u, 0u, 0u);
    st_shared_v4(U + tc_off(t, kFlowHidden + 8, kTcK2), 0u, 0u, 0u, 0u);
    bool ok = true;
    for (int i = 0; i < kFlowLayers && ok; ++i) {
      const int l = dir > 0 ? i : kFlowLayers - 1 - i;
      const unsigned char* wl = sm + l * S::layer;
      ok = (l & 1) ? tc_layer<D, 1>(wl, U, G, dir, z, ld) : tc_layer<D, 0>(wl, U, G, dir, z, ld);
    }
    // the last wait's outcome, agreed by the whole warpgroup
    if (!ok || wg_bar_any(1 + G.id, G.failed)) break;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ld += flow_log_sig_prime(z[k]);
      stg[t * zld + k] = flow_sigmoid(z[k]);
    }
    if (t < rows) logdet[r0 + t] = ld;
    wg_bar(1 + G.id);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int i = t + 128 * j;
      if (i < rows * D) xout[r0 * D + i] = stg[(i / D) * zld + i % D];
    }
    wg_bar(1 + G.id);
  }
  // a warpgroup that gave up waits once more for its MMAs before the columns are freed
  if (G.failed) mbar_wait(G.mbar, G.phase ^ 1u, kTcWaitPolls);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tbase, S::tmem_cols);
}

// ---------------------------------------------------------------------------
// Up to 16 axes: more tiles in flight.  A tile's activations U are 128 x 64
// (16 KB) instead of 128 x 80: the bias k-step of the second and third GEMMs
// takes its A operand from one shared 128 x 16 tile of ones (columns 0-2 one,
// the rest zero) against the bias columns 64-79 of the weights.  The shared
// memory this frees holds more warpgroups, each on its own tile.
// ---------------------------------------------------------------------------
constexpr int kU64 = kFlowHidden;  // columns of U

template <int D>
struct U64Shape {
  using S = TcShape<D>;  // the staged weights are the same
  static_assert(D <= 16 && S::K1 == 16 && S::N3 == 16, "up to 16 axes");
  static constexpr int G = kU64Groups;
  static constexpr int threads = 128 * G;
  static constexpr uint32_t tmem_cols = G * kTcColsPerGroup <= 256 ? 256 : 512;
  static constexpr uint32_t ONES = 128 * 16 * 2, U = 128 * kU64 * 2;
  static constexpr uint32_t ones_off = S::weights, u_off = S::weights + ONES;
  static constexpr uint32_t misc = u_off + G * U;
  static constexpr uint32_t total = misc + 8 * G + 16;
  static_assert(128 * S::ZLD * 4 <= U, "staging fits in U");
  static_assert(total <= 232448, "shared memory of one CTA");
  static_assert(G * kTcColsPerGroup <= 512, "tensor memory");
};

// the MMAs of one GEMM, issued by one thread: nks k-steps from U, then (bias) one from the ones tile
__device__ __forceinline__ void u64_gemm(uint32_t tcol, const unsigned char* U, const unsigned char* ones,
                                         const unsigned char* B, int kb, int nks, bool bias, uint32_t idesc) {
  const uint64_t ad = tc_desc(tc_smem_u32(U), kTcLbo, (uint32_t)kU64 * 16);
  const uint64_t bd = tc_desc(tc_smem_u32(B), kTcLbo, (uint32_t)kb * 16);
  for (int s = 0; s < nks; ++s) tc_mma(tcol, ad + 16u * s, bd + 16u * s, idesc, s > 0);
  if (bias) tc_mma(tcol, tc_desc(tc_smem_u32(ones), kTcLbo, 16 * 16), bd + 16u * nks, idesc, 1u);
}

// operands written: vote barrier, thread 0 issues and commits, every thread waits (bounded);
// false on every thread of the warpgroup once a wait ran out
__device__ __forceinline__ bool u64_run(TcGroup& G, const unsigned char* U, const unsigned char* ones,
                                        const unsigned char* B, int kb, int nks, bool bias, uint32_t idesc) {
  tc_fence_proxy();
  tc_fence_before();
  if (wg_bar_any(1 + G.id, G.failed)) return false;
  if (G.t == 0) {
    tc_fence_after();
    u64_gemm(G.tacc & 0xFFFFu, U, ones, B, kb, nks, bias, idesc);
    tc_commit(G.mbar);
  }
  if (!mbar_wait(G.mbar, G.phase, kTcWaitPolls)) {
    G.failed = true;
    atomicOr(&g_flow_tc_status, 4);
  }
  G.phase ^= 1u;
  tc_fence_after();
  return true;
}

template <int D, int PAR>
__device__ __forceinline__ bool u64_layer(const unsigned char* wl, const unsigned char* ones, unsigned char* U,
                                          TcGroup& G, int dir, float (&z)[D], float& ld) {
  using T = TcShape<D>;
  constexpr int a = PAR == 0 ? (D + 1) / 2 : D / 2, b = D - a;
  const int t = G.t;
#pragma unroll
  for (int q = 0; q < 2; ++q) {  // H: the first 16 columns of U
    float hv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = 8 * q + e;
      hv[e] = c < a ? z[2 * c + PAR] : (c < a + 3 ? 1.0f : 0.0f);
    }
    st_shared_v4(U + tc_off(t, 8 * q, kU64), bf16x2(hv[0], hv[1]), bf16x2(hv[2], hv[3]), bf16x2(hv[4], hv[5]),
                 bf16x2(hv[6], hv[7]));
  }
  const unsigned char* w1 = wl;
  const unsigned char* w2 = wl + T::W1;
  const unsigned char* w3 = w2 + T::W2;
  if (!u64_run(G, U, ones, w1, 16, 1, false, tc_idesc_bf16(128, 64))) return false;
  tc_hidden_epilogue(G.tacc, U, t, kU64);
  tc_fence_before();
  if (!u64_run(G, U, ones, w2, kTcK2, 4, true, tc_idesc_bf16(128, 64))) return false;
  tc_hidden_epilogue(G.tacc, U, t, kU64);
  tc_fence_before();
  if (!u64_run(G, U, ones, w3, kTcK2, 4, true, tc_idesc_bf16(128, 16))) return false;
  float o[16];
  tc_ld16(G.tacc, o);
  tc_fence_before();
#pragma unroll
  for (int m = 0; m < b; ++m) {
    const int k = 2 * m + 1 - PAR;
    const float s = flow_soft_clamp(o[2 * m]), tt = o[2 * m + 1];
    if (dir > 0) {
      z[k] = fmaf(z[k], __expf(s), tt);
      ld += s;
    } else {
      z[k] = (z[k] - tt) * __expf(-s);
      ld -= s;
    }
  }
  return true;
}

template <int D>
__global__ void __launch_bounds__(U64Shape<D>::threads, 1)
    flow_apply_u64_kernel(const __grid_constant__ FlowArgs fa, int dir, const float* __restrict__ xin,
                          float* __restrict__ xout, float* __restrict__ logdet, int64_t n) {
  using P = U64Shape<D>;
  constexpr int zld = D | 1;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int warp = threadIdx.x >> 5;
  uint64_t* mbars = reinterpret_cast<uint64_t*>(sm + P::misc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + P::misc + 8 * P::G);
  unsigned char* ones = sm + P::ones_off;
  tc_stage_weights<D>(fa, sm);
  for (int i = threadIdx.x; i < 128 * 16; i += blockDim.x) {
    const int r = i >> 4, c = i & 15;
    *reinterpret_cast<__nv_bfloat16*>(ones + tc_off(r, c, 16)) = __float2bfloat16_rn(c < 3 ? 1.0f : 0.0f);
  }
  if (warp == 0) tc_alloc(tslot, P::tmem_cols);
  if (threadIdx.x == 0) {
    for (int g = 0; g < P::G; ++g) mbar_init(mbars + g, 1);
    mbar_fence_init();
  }
  tc_fence_proxy();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  TcGroup G;
  G.id = threadIdx.x >> 7;
  G.t = threadIdx.x & 127;
  G.tacc = tbase + (uint32_t)(G.id * kTcColsPerGroup) + ((uint32_t)((warp & 3) * 32) << 16);
  G.mbar = mbars + G.id;
  G.phase = 0;
  G.failed = false;
  unsigned char* U = sm + P::u_off + G.id * P::U;
  float* stg = reinterpret_cast<float*>(U);
  const int t = G.t;
  const int64_t ntiles = (n + 127) / 128;
  for (int64_t tile = (int64_t)blockIdx.x * P::G + G.id; tile < ntiles; tile += (int64_t)gridDim.x * P::G) {
    const int64_t r0 = tile * 128;
    const int rows = (int)min((int64_t)128, n - r0);
    {  // the tile's x, coalesced, into rows of stride zld (odd: conflict-free row reads); all loads first
      float xl[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int i = t + 128 * j;
        xl[j] = i < rows * D ? xin[r0 * D + i] : 0.5f;
      }
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int i = t + 128 * j;
        stg[(i / D) * zld + i % D] = xl[j];
      }
    }
    wg_bar(1 + G.id);
    float z[D];
    float ld = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      z[k] = flow_logit(stg[t * zld + k]);
      ld -= flow_log_sig_prime(z[k]);
    }
    wg_bar(1 + G.id);
    bool ok = true;
    for (int i = 0; i < kFlowLayers && ok; ++i) {
      const int l = dir > 0 ? i : kFlowLayers - 1 - i;
      const unsigned char* wl = sm + l * TcShape<D>::layer;
      ok = (l & 1) ? u64_layer<D, 1>(wl, ones, U, G, dir, z, ld) : u64_layer<D, 0>(wl, ones, U, G, dir, z, ld);
    }
    if (!ok || wg_bar_any(1 + G.id, G.failed)) break;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ld += flow_log_sig_prime(z[k]);
      stg[t * zld + k] = flow_sigmoid(z[k]);
    }
    if (t < rows) logdet[r0 + t] = ld;
    wg_bar(1 + G.id);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int i = t + 128 * j;
      if (i < rows * D) xout[r0 * D + i] = stg[(i / D) * zld + i % D];
    }
    wg_bar(1 + G.id);
  }
  // a warpgroup that gave up waits once more for its MMAs before the columns are freed
  if (G.failed) mbar_wait(G.mbar, G.phase ^ 1u, kTcWaitPolls);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tbase, P::tmem_cols);
}

// f(std::integral_constant<int, d>) for d in 2..32
template <int D = 2, typename F>
int dispatch_d(int d, F&& f) {
  if constexpr (D > kFlowMaxDim) {
    return VEGAS_EINVAL;
  } else {
    return d == D ? f(std::integral_constant<int, D>{}) : dispatch_d<D + 1>(d, f);
  }
}

int num_sms_tc() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

template <int D>
int launch_apply_tc(const FlowArgs& fa, int dir, const float* xin, float* xout, float* logdet, int64_t n,
                    cudaStream_t s) {
  if constexpr (D <= 16) {
    using P = U64Shape<D>;
    auto k = flow_apply_u64_kernel<D>;
    VG_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::total));
    const int64_t ntiles = (n + 127) / 128;
    const int sms = num_sms_tc();
    if (sms < 1) return VEGAS_ECUDA;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (ntiles + P::G - 1) / P::G));
    k<<<grid, P::threads, P::total, s>>>(fa, dir, xin, xout, logdet, n);
    return cuda_status(cudaGetLastError());
  } else {
    using S = TcShape<D>;
    auto k = flow_apply_tc_kernel<D>;
    VG_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total));
    const int64_t ntiles = (n + 127) / 128;
    const int sms = num_sms_tc();
    if (sms < 1) return VEGAS_ECUDA;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (ntiles + S::G - 1) / S::G));
    k<<<grid, S::threads, S::total, s>>>(fa, dir, xin, xout, logdet, n);
    return cuda_status(cudaGetLastError());
  }
}

}  // namespace

int flow_apply(int d, int direction, const float* d_params, const float* d_xin, float* d_xout, float* d_logdet,
               int64_t n, cudaStream_t s) {
  FlowArgs fa{};
  if (flow_layout(d, fa) != VEGAS_OK) return VEGAS_EINVAL;
  if (n == 0) return VEGAS_OK;
  fa.params = d_params;
  const int dir = direction == VEGAS_FLOW_NORMALISE ? 1 : -1;
  return dispatch_d(d, [&](auto D) { return launch_apply_tc<decltype(D)::value>(fa, dir, d_xin, d_xout, d_logdet, n, s); });
}

// The bounded wait on its own: an mbarrier of one expected arrival, waited
// on for `polls` polls.  With arrive = 0 nothing arrives, the wait runs out
// and the status word records it, as a stalled MMA would; with arrive = 1 one
// thread arrives first and the wait completes.
__global__ void tc_wait_selftest_kernel(int polls, int arrive) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(tc_smem_u32(&mbar))
                 : "memory");
  if (!mbar_wait(&mbar, 0, polls)) atomicOr(&g_flow_tc_status, 4);
}

int flow_tc_wait_selftest(int polls, int arrive, cudaStream_t s) {
  tc_wait_selftest_kernel<<<1, 32, 0, s>>>(polls, arrive);
  return cuda_status(cudaGetLastError());
}

int flow_tc_status(bool reset) {
  int v = 0;
  VG_CHECK(cudaMemcpyFromSymbol(&v, g_flow_tc_status, sizeof(int)));
  if (reset && v) {
    const int zero = 0;
    VG_CHECK(cudaMemcpyToSymbol(g_flow_tc_status, &zero, sizeof(int)));
  }
  return (v & 4) ? VEGAS_ETIMEOUT : VEGAS_OK;
}

}  // namespace vg
