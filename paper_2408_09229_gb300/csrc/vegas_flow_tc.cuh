// vegas_flow_tc.cuh -- pieces shared by the coupling flow's tensor-core
// kernels (the batched transform in vegas_flow_tc.cu, the training gradient
// in vegas_flow_grad_tc.cu): the shapes of a dimension, the staging of the
// weights in the tcgen05 core-matrix layout with the bias as a bf16 triple,
// warpgroup barriers, and the GEMM issue of one thread.
#pragma once
#include <cuda_bf16.h>

#include "vegas_flow.cuh"
#include "vegas_internal.h"
#include "vegas_tc.cuh"

namespace vg {
namespace {

constexpr int kTcK2 = kFlowHidden + 16;        // K of the second and third GEMMs: 64 + bias block
constexpr int kTcColsPerGroup = 64;            // tensor-memory columns of one warpgroup's accumulator
constexpr int kTcWaitPolls = 1 << 22;          // bound of every mbarrier wait
constexpr int kU64Groups = 8;                  // warpgroups a CTA up to 16 axes (measured: 8 beats 7 and 6)

// The shapes for d = D axes (every D in 2..32 is its own instantiation: the
// column selections, the moved axes and the row arithmetic of the staging are
// then compile-time).
template <int D>
struct TcShape {
  static constexpr int G = 4;  // warpgroups a CTA (shared memory): this kernel serves 17..32 axes
  static constexpr int threads = 128 * G;
  static constexpr uint32_t tmem_cols = G * kTcColsPerGroup <= 256 ? 256 : 512;  // a power of two
  static constexpr int A0 = (D + 1) / 2;                // conditioning axes of even layers (the larger a)
  static constexpr int K1 = A0 + 3 <= 16 ? 16 : 32;     // K of the first GEMM: a inputs + 3 bias columns
  static constexpr int N3 = 2 * A0 <= 16 ? 16 : 32;     // N of the third GEMM: 2 b outputs, padded
  static constexpr int ZLD = D | 1;                     // staging row stride (odd: conflict-free)
  static constexpr uint32_t W1 = 64 * K1 * 2, W2 = 64 * kTcK2 * 2, W3 = N3 * kTcK2 * 2;
  static constexpr uint32_t layer = W1 + W2 + W3;
  static constexpr uint32_t weights = kFlowLayers * layer;
  static constexpr uint32_t U = 128 * kTcK2 * 2;  // activations; also H (first K1 columns) and the x staging
  static constexpr uint32_t misc = weights + G * U;
  static constexpr uint32_t total = misc + 8 * G + 4 * G + 16;
  static_assert(128 * ZLD * 4 <= U, "staging fits in U");
  static_assert(K1 <= kFlowHidden, "H fits in U's hidden columns");
  static_assert(total <= 232448, "shared memory of one CTA");
};

__device__ __forceinline__ void bias3(float b, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(b);
  const float r = b - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}

// weights of every layer in the core-matrix layout, biases in columns (k, k+1, k+2)
template <int D>
__device__ void tc_stage_weights(const FlowArgs& fa, unsigned char* sm) {
  using S = TcShape<D>;
  const int kTcThreads = blockDim.x;
  const float* P = fa.params;
  for (int l = 0; l < kFlowLayers; ++l) {
    const FlowLayer& L = fa.lay[l];
    unsigned char* w1 = sm + l * S::layer;
    unsigned char* w2 = w1 + S::W1;
    unsigned char* w3 = w2 + S::W2;
    for (int i = threadIdx.x; i < 64 * S::K1; i += kTcThreads) {
      const int j = i / S::K1, c = i - j * S::K1;
      __nv_bfloat16 v = __float2bfloat16_rn(0.0f), h, m, lo;
      if (c < L.a) v = __float2bfloat16_rn(P[L.oW1 + j * L.a + c]);
      else if (c < L.a + 3) {
        bias3(P[L.ob1 + j], h, m, lo);
        v = c == L.a ? h : (c == L.a + 1 ? m : lo);
      }
      *reinterpret_cast<__nv_bfloat16*>(w1 + tc_off(j, c, S::K1)) = v;
    }
    for (int i = threadIdx.x; i < 64 * kTcK2; i += kTcThreads) {
      const int j = i / kTcK2, c = i - j * kTcK2;
      __nv_bfloat16 v = __float2bfloat16_rn(0.0f), h, m, lo;
      if (c < kFlowHidden) v = __float2bfloat16_rn(P[L.oW2 + j * kFlowHidden + c]);
      else if (c < kFlowHidden + 3) {
        bias3(P[L.ob2 + j], h, m, lo);
        v = c == kFlowHidden ? h : (c == kFlowHidden + 1 ? m : lo);
      }
      *reinterpret_cast<__nv_bfloat16*>(w2 + tc_off(j, c, kTcK2)) = v;
    }
    for (int i = threadIdx.x; i < S::N3 * kTcK2; i += kTcThreads) {
      const int j = i / kTcK2, c = i - j * kTcK2;
      __nv_bfloat16 v = __float2bfloat16_rn(0.0f), h, m, lo;
      if (j < 2 * L.b) {
        if (c < kFlowHidden) v = __float2bfloat16_rn(P[L.oW3 + j * kFlowHidden + c]);
        else if (c < kFlowHidden + 3) {
          bias3(P[L.ob3 + j], h, m, lo);
          v = c == kFlowHidden ? h : (c == kFlowHidden + 1 ? m : lo);
        }
      }
      *reinterpret_cast<__nv_bfloat16*>(w3 + tc_off(j, c, kTcK2)) = v;
    }
  }
}

__device__ __forceinline__ void wg_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ void st_shared_v4(unsigned char* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc_smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// row t of U (ku columns) from the 64 accumulator columns: ReLU, bf16 (16 columns at a time: registers)
__device__ __forceinline__ void tc_hidden_epilogue(uint32_t tacc, unsigned char* U, int t, int ku = kTcK2) {
#pragma unroll
  for (int cb = 0; cb < 64; cb += 16) {
    float v[16];
    tc_ld16(tacc + cb, v);
#pragma unroll
    for (int q = 0; q < 2; ++q)
      st_shared_v4(U + tc_off(t, cb + 8 * q, ku), bf16x2_relu(v[8 * q], v[8 * q + 1]),
                   bf16x2_relu(v[8 * q + 2], v[8 * q + 3]), bf16x2_relu(v[8 * q + 4], v[8 * q + 5]),
                   bf16x2_relu(v[8 * q + 6], v[8 * q + 7]));
  }
}

// the MMAs of one GEMM, issued by one thread: D = A B^T over K / 16 k-steps;
// A is a tile of KA columns (its row-group stride), B one of K columns
__device__ __forceinline__ void tc_gemm(uint32_t tacc, const unsigned char* A, const unsigned char* B, int KA, int K,
                                        uint32_t idesc) {
  // a k-step moves both start addresses by 256 bytes: 16 in the descriptors' address field, which cannot
  // carry out of its 14 bits (shared addresses stay below 2^18)
  const uint64_t ad = tc_desc(tc_smem_u32(A), kTcLbo, (uint32_t)KA * 16);
  const uint64_t bd = tc_desc(tc_smem_u32(B), kTcLbo, (uint32_t)K * 16);
  for (int s = 0; s < K / 16; ++s) tc_mma(tacc, ad + 16u * s, bd + 16u * s, idesc, s > 0);
}

struct TcGroup {
  int id, t;             // warpgroup, thread in it
  uint32_t tacc;         // its accumulator columns, lane base of this warp
  uint64_t* mbar;
  uint32_t phase;
  bool failed;           // this thread's last wait ran out
};

// the warpgroup's barrier; true on every thread when any thread arrived with `bad`
__device__ __forceinline__ bool wg_bar_any(int id, bool bad) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbarrier.red.or.pred q, %2, 128, p;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)bad), "r"(id)
      : "memory");
  return r != 0;
}

}  // namespace
}  // namespace vg
