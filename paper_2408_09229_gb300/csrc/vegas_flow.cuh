// vegas_flow.cuh -- the learned proposal's coupling flow on the tensor cores.
//
// Not part of cuVegas (arXiv 2408.09229): the VEGAS+ map M of Sec. 2.1.1
// samples x' = M(y), and the flow F maps x' to the point x = F(x') where the
// integrand is evaluated; the estimator then integrates
// g(x') = f(F(x')) |det dF/dx'|, whose integral equals that of f, so the
// iteration of Algorithms 1-2 runs unchanged on g.  F is a stack of affine
// coupling layers (RealNVP, Dinh et al., ICLR 2017) between a logit and a
// sigmoid:
//   z = clamp(logit(x), -Z, Z);  layer l conditions on the axes k = l (mod 2)
//   and moves the others: s, t = MLP_l(z[A_l]) with s soft-clamped to
//   S tanh(./S); normalising direction z[B] = z[B] e^s + t, sampling
//   direction z[B] = (z[B] - t) e^-s; then x = sigmoid(z).  The
//   log-determinant is sum s plus the two wrap terms log sigmoid'(z).
// MLP_l: a_l -> 64 -> 64 -> 2 b_l with ReLU; output row 2j is s_j, 2j+1 t_j.
//
// The batched transform (vegas_flow_apply) runs on tcgen05 with the
// accumulators in tensor memory (vegas_flow_tc.cu), and so does the training
// gradient up to 16 axes (vegas_flow_grad_tc.cu).  Wider flows train with the
// layer below on mma.sync m16n8k16 (bf16 operands, FP32 accumulation): a
// warp owns 16 samples, and the accumulator fragment of one GEMM is, after
// ReLU and conversion, the A fragment of the next, so the hidden activations
// never leave registers.  Weights are bf16 in shared memory, rows padded so
// that the fragment loads of a warp hit 32 distinct banks.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "vegas_internal.h"

namespace vg {

constexpr int kFlowLayers = 6;
constexpr int kFlowHidden = 64;
constexpr float kFlowSClamp = 2.0f;
constexpr float kFlowZClamp = 20.0f;
constexpr int kFlowMaxDim = 32;
constexpr int kFlowGradTcMaxDim = 16;  // the training gradient runs on tcgen05 up to this many axes

struct FlowArgs;
// the tensor-core training gradient (vegas_flow_grad_tc.cu): per 128 samples one partial gradient and loss, from
// a bf16 weight image of flow_grad_tc_image_bytes(d) bytes that it builds in img
int flow_grad_tc(const FlowArgs& fa, unsigned char* img, const float* x, const float* w, const double* wsum,
                 int64_t n, float* gpart, float* lpart, cudaStream_t s);
size_t flow_grad_tc_image_bytes(int d);
// shared-memory leading dimensions (bf16 elements): 12, 36 and 20 words
constexpr int kLdK16 = 24, kLdK64 = 72, kLdK32 = 40;

struct FlowLayer {
  int a, b, no;                        // conditioning axes, moved axes, outputs padded to 8 (2b <= no)
  int oW1, ob1, oW2, ob2, oW3, ob3;    // offsets in the FP32 parameter vector
  int sW1, sb1, sW2, sb2, sW3, sb3;    // byte offsets of the layer's bf16 / f32 copies in shared memory
};

struct FlowArgs {
  int d, nparams, smem_weights;  // bytes of the staged weights (all layers)
  FlowLayer lay[kFlowLayers];
  const float* params;
};

// ---- mma.sync helpers ------------------------------------------------------
__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// B fragment of a [n][k] row-major bf16 matrix (k contiguous), tile at (n0, k0)
__device__ __forceinline__ void load_b(const __nv_bfloat16* __restrict__ B, int ld, int n0, int k0, uint32_t& b0,
                                       uint32_t& b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* p = B + (n0 + g) * ld + k0 + 2 * t;
  b0 = *reinterpret_cast<const uint32_t*>(p);
  b1 = *reinterpret_cast<const uint32_t*>(p + 8);
}

// B fragments of two adjacent n-tiles (n0 and n0 + 8) at k0 with one
// ldmatrix.x4: lanes 0-7 address rows n0..n0+7 at k0, lanes 8-15 the same
// rows at k0 + 8, lanes 16-31 rows n0+8..n0+15; each 8x8 tile lands in the
// B-fragment layout of m16n8k16 (thread i holds row i/4, columns 2(i%4)+{0,1}).
// Row pitches are multiples of 16 bytes and k0 a multiple of 8.
__device__ __forceinline__ void load_b2(const __nv_bfloat16* __restrict__ B, int ld, int n0, int k0, uint32_t& b00,
                                        uint32_t& b01, uint32_t& b10, uint32_t& b11) {
  const int lane = threadIdx.x & 31;
  const int row = n0 + (lane & 7) + ((lane >> 4) << 3), col = k0 + ((lane >> 3) & 1) * 8;
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(B + row * ld + col);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(b00), "=r"(b01), "=r"(b10), "=r"(b11)
               : "r"(addr));
}

// A fragment of a [m][k] row-major bf16 matrix, tile at (m0, k0)
__device__ __forceinline__ void load_a(const __nv_bfloat16* __restrict__ A, int ld, int m0, int k0, uint32_t (&a)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* p = A + (m0 + g) * ld + k0 + 2 * t;
  a[0] = *reinterpret_cast<const uint32_t*>(p);
  a[1] = *reinterpret_cast<const uint32_t*>(p + 8 * ld);
  a[2] = *reinterpret_cast<const uint32_t*>(p + 8);
  a[3] = *reinterpret_cast<const uint32_t*>(p + 8 * ld + 8);
}

// The element-wise functions use the hardware approximations (__logf,
// __expf): their errors are absolute errors of ~1e-7 in z and in the
// log-determinant, below the FP32 rounding of the map itself.  Exactness of
// the change of variables does not depend on them: each layer's s enters the
// transform and the log-determinant as the same value.
__device__ __forceinline__ float flow_logit(float x) {
  const float z = __logf(x) - __logf(1.0f - x);  // 1 - x is exact for x >= 1/2
  return fminf(fmaxf(z, -kFlowZClamp), kFlowZClamp);
}
// log sigmoid'(z) = -|z| - 2 log(1 + e^-|z|)
__device__ __forceinline__ float flow_log_sig_prime(float z) {
  const float az = fabsf(z);
  return -az - 2.0f * __logf(1.0f + __expf(-az));
}
// sigmoid from e^-|z| <= 1: finite for every z
__device__ __forceinline__ float flow_sigmoid(float z) {
  const float e = __expf(-fabsf(z)), r = __fdividef(1.0f, 1.0f + e);  // 1 + e in [1, 2]
  return z >= 0.0f ? r : e * r;
}
// s = S tanh(o / S) = sign(o) S (1 - 2 e / (1 + e)), e = e^(-2 |o| / S) <= 1: finite for every o
__device__ __forceinline__ float flow_soft_clamp(float o) {
  const float e = __expf(fabsf(o) * (-2.0f / kFlowSClamp));
  return copysignf(kFlowSClamp * __fdividef(1.0f - e, 1.0f + e), o);
}

// The conditioner of layer L on the warp's 16 rows: from the A fragments of
// h (one k-step: a <= 16), the output fragments o[nt][4] for nt < no/8.
// u1 and u2 stay in registers.
template <int NT3>
__device__ __forceinline__ void flow_mlp(const FlowLayer& L, const unsigned char* sm, const uint32_t (&ha)[4],
                                         float (&o)[NT3][4]) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(sm + L.sW1);
  const __nv_bfloat16* W2 = reinterpret_cast<const __nv_bfloat16*>(sm + L.sW2);
  const __nv_bfloat16* W3 = reinterpret_cast<const __nv_bfloat16*>(sm + L.sW3);
  const float* b1 = reinterpret_cast<const float*>(sm + L.sb1);
  const float* b2 = reinterpret_cast<const float*>(sm + L.sb2);
  const float* b3 = reinterpret_cast<const float*>(sm + L.sb3);
  float acc[8][4];
  // layer 1: h (16 x 16) W1^T -> 16 x 64
#pragma unroll
  for (int nt = 0; nt < 8; nt += 2) {
    const float2 bb = *reinterpret_cast<const float2*>(b1 + nt * 8 + 2 * t);
    const float2 bc = *reinterpret_cast<const float2*>(b1 + nt * 8 + 8 + 2 * t);
    acc[nt][0] = bb.x; acc[nt][1] = bb.y; acc[nt][2] = bb.x; acc[nt][3] = bb.y;
    acc[nt + 1][0] = bc.x; acc[nt + 1][1] = bc.y; acc[nt + 1][2] = bc.x; acc[nt + 1][3] = bc.y;
    uint32_t b00, b01, b10, b11;
    load_b2(W1, kLdK16, nt * 8, 0, b00, b01, b10, b11);
    mma16816(acc[nt], ha[0], ha[1], ha[2], ha[3], b00, b01);
    mma16816(acc[nt + 1], ha[0], ha[1], ha[2], ha[3], b10, b11);
  }
  // ReLU, bf16: the A fragments of u1 (4 k-steps of 16)
  uint32_t ua[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    ua[ks][0] = pack_bf16(fmaxf(acc[2 * ks][0], 0.0f), fmaxf(acc[2 * ks][1], 0.0f));
    ua[ks][1] = pack_bf16(fmaxf(acc[2 * ks][2], 0.0f), fmaxf(acc[2 * ks][3], 0.0f));
    ua[ks][2] = pack_bf16(fmaxf(acc[2 * ks + 1][0], 0.0f), fmaxf(acc[2 * ks + 1][1], 0.0f));
    ua[ks][3] = pack_bf16(fmaxf(acc[2 * ks + 1][2], 0.0f), fmaxf(acc[2 * ks + 1][3], 0.0f));
  }
  // layer 2: u1 (16 x 64) W2^T -> 16 x 64
#pragma unroll
  for (int nt = 0; nt < 8; nt += 2) {
    const float2 bb = *reinterpret_cast<const float2*>(b2 + nt * 8 + 2 * t);
    const float2 bc = *reinterpret_cast<const float2*>(b2 + nt * 8 + 8 + 2 * t);
    acc[nt][0] = bb.x; acc[nt][1] = bb.y; acc[nt][2] = bb.x; acc[nt][3] = bb.y;
    acc[nt + 1][0] = bc.x; acc[nt + 1][1] = bc.y; acc[nt + 1][2] = bc.x; acc[nt + 1][3] = bc.y;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      uint32_t b00, b01, b10, b11;
      load_b2(W2, kLdK64, nt * 8, ks * 16, b00, b01, b10, b11);
      mma16816(acc[nt], ua[ks][0], ua[ks][1], ua[ks][2], ua[ks][3], b00, b01);
      mma16816(acc[nt + 1], ua[ks][0], ua[ks][1], ua[ks][2], ua[ks][3], b10, b11);
    }
  }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    ua[ks][0] = pack_bf16(fmaxf(acc[2 * ks][0], 0.0f), fmaxf(acc[2 * ks][1], 0.0f));
    ua[ks][1] = pack_bf16(fmaxf(acc[2 * ks][2], 0.0f), fmaxf(acc[2 * ks][3], 0.0f));
    ua[ks][2] = pack_bf16(fmaxf(acc[2 * ks + 1][0], 0.0f), fmaxf(acc[2 * ks + 1][1], 0.0f));
    ua[ks][3] = pack_bf16(fmaxf(acc[2 * ks + 1][2], 0.0f), fmaxf(acc[2 * ks + 1][3], 0.0f));
  }
  // layer 3: u2 (16 x 64) W3^T -> 16 x no
  // (W3 is staged with a multiple of 16 rows, zero past 2b, so the n-tiles go in pairs)
#pragma unroll
  for (int nt = 0; nt < NT3; nt += 2) {
    if (nt * 8 < L.no) {
      const float2 bb = *reinterpret_cast<const float2*>(b3 + nt * 8 + 2 * t);
      const float2 bc = *reinterpret_cast<const float2*>(b3 + nt * 8 + 8 + 2 * t);
      o[nt][0] = bb.x; o[nt][1] = bb.y; o[nt][2] = bb.x; o[nt][3] = bb.y;
      o[nt + 1][0] = bc.x; o[nt + 1][1] = bc.y; o[nt + 1][2] = bc.x; o[nt + 1][3] = bc.y;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        uint32_t b00, b01, b10, b11;
        load_b2(W3, kLdK64, nt * 8, ks * 16, b00, b01, b10, b11);
        mma16816(o[nt], ua[ks][0], ua[ks][1], ua[ks][2], ua[ks][3], b00, b01);
        mma16816(o[nt + 1], ua[ks][0], ua[ks][1], ua[ks][2], ua[ks][3], b10, b11);
      }
    }
  }
}

// One coupling layer on the warp's 16 rows held in z (row-major [16][zld]
// FP32, shared memory).  dir = +1 normalising, -1 sampling.  ld0 / ld1
// accumulate sum s of rows g and g+8 (g = lane / 4) over this lane's pairs.
template <int NT3>
__device__ __forceinline__ void flow_layer(const FlowLayer& L, int l, const unsigned char* sm, float* z, int zld,
                                           int dir, float& ld0, float& ld1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int par = l & 1;
  // h = z[A]: column c of h is axis 2c + par; columns >= a are zero
  uint32_t ha[4];
  {
    const int c0 = 2 * t, c1 = 2 * t + 1, c2 = 2 * t + 8, c3 = 2 * t + 9;
    auto hv = [&](int row, int c) { return c < L.a ? z[row * zld + 2 * c + par] : 0.0f; };
    ha[0] = pack_bf16(hv(g, c0), hv(g, c1));
    ha[1] = pack_bf16(hv(g + 8, c0), hv(g + 8, c1));
    ha[2] = pack_bf16(hv(g, c2), hv(g, c3));
    ha[3] = pack_bf16(hv(g + 8, c2), hv(g + 8, c3));
  }
  float o[NT3][4];
  flow_mlp<NT3>(L, sm, ha, o);
  __syncwarp();
  // pair m = 4 nt + t holds (s_m, t_m) for rows g and g+8; it moves axis 2m + 1 - par
#pragma unroll
  for (int nt = 0; nt < NT3; ++nt) {
    const int m = 4 * nt + t;
    if (nt * 8 < L.no && m < L.b) {
      const int k = 2 * m + 1 - par;
      const float s0 = flow_soft_clamp(o[nt][0]), t0 = o[nt][1];
      const float s1 = flow_soft_clamp(o[nt][2]), t1 = o[nt][3];
      float& z0 = z[g * zld + k];
      float& z1 = z[(g + 8) * zld + k];
      if (dir > 0) {
        z0 = fmaf(z0, __expf(s0), t0);
        z1 = fmaf(z1, __expf(s1), t1);
        ld0 += s0;
        ld1 += s1;
      } else {
        z0 = (z0 - t0) * __expf(-s0);
        z1 = (z1 - t1) * __expf(-s1);
        ld0 -= s0;
        ld1 -= s1;
      }
    }
  }
  __syncwarp();
}

int flow_layout(int d, FlowArgs& fa);

}  // namespace vg
