// vegas_flow_grad_tc.cu -- the gradient of the learned proposal's training
// loss (vegas_flow_grad) on the fifth-generation tensor cores, for 2..16 axes:
// tcgen05.mma with bf16 operands in shared memory and FP32 accumulators in
// tensor memory.  The flow and the loss are defined in vegas_flow.cuh and
// vegas_flow.cu; the wider flows keep the warp-level path of vegas_flow.cu.
//
// One CTA is one warpgroup on a tile of 128 samples; thread t owns sample t.
// It holds the sample's z and dL/dz in registers and reads row t of every
// accumulator (tensor-memory lane t).
//   Forward (normalising direction), per layer as the transform runs it:
//     H = [bf16 z_A | 1 1 1 | 0], D = H W1'^T, U1 = bf16 relu D,
//     D = [U1 | ones] W2'^T, U2 = bf16 relu D, o = [U2 | ones] W3'^T,
//     z_B = z_B e^s + t;  the primed weights carry the bias as a bf16 triple.
//   Backward, last layer first.  z before the layer comes back by inverting
//   it (z_A is unchanged, so the conditioner recomputes exactly; then
//   z_B = (z_B - t) e^-s), so nothing is stored per layer.  With
//   GO = dL/d(s, t) (bf16), GA2, GA1 the gradients of the hidden
//   pre-activations (bf16, ReLU-masked):
//     gU2 = GO W3      and  dW3 = GO^T [U2 | 1]   (one round trip: both MMAs, one commit)
//     gU1 = GA2 W2     and  dW2 = GA2^T [U1 | 1]
//     gH  = GA1 W1     and  dW1 = GA1^T H
//   The ones rows of the transposed activations give the bias gradients as
//   the extra accumulator column (H already holds its ones).  The transposed
//   operands (samples along K) are written beside the natural ones by the
//   epilogue of the GEMM that produces them.  A weight gradient has at most 64
//   rows, the MMA 128: its A operand reads 128 rows, the last ones from the
//   tiles that follow in shared memory, into accumulator lanes nobody reads.
// Per CTA the gradient is written as one partial vector; vegas_flow.cu sums
// the partials in a fixed order.  Every mbarrier wait is bounded; one that
// runs out sets bit 2 of the status word, and the warpgroup stops at its next
// barrier vote, waits once more (bounded) for its MMAs and frees its tensor
// memory.
#include <algorithm>

#include "vegas_flow_tc.cuh"

namespace vg {

namespace {

__device__ int g_flow_grad_status;  // bit 2: a bounded wait ran out

template <int D>
struct GradTcShape {
  using S = TcShape<D>;
  static constexpr int K1 = S::K1, N3 = S::N3;
  static_assert(D <= 16 && K1 == 16 && N3 == 16, "the tensor-core gradient serves up to 16 axes");
  // the current layer's weights transposed (B operands of the input-gradient GEMMs):
  // W3T [64][N3] (element (h, o) = W3[o][h]), W2T [64][64] ((i, j) = W2[j][i]), W1T [K1][64] ((c, h) = W1[h][c])
  static constexpr uint32_t W3T = 64 * N3 * 2, W2T = 64 * 64 * 2, W1T = K1 * 64 * 2;
  static constexpr uint32_t w3t_off = S::weights, w2t_off = w3t_off + W3T, w1t_off = w2t_off + W2T;
  // natural activations (A operands, K-major, rows of kTcK2 = 80 columns, the last 16 the ones block)
  static constexpr uint32_t P = 128 * kTcK2 * 2;
  static constexpr uint32_t p0_off = w1t_off + W1T, p1_off = p0_off + P;
  // transposed activations, samples along K (= 128): GA^T [64][128] (GA2, then GA1), GO^T [N3][128],
  // H^T [K1][128], [U1 | 1]^T and [U2 | 1]^T [80][128]
  static constexpr uint32_t GAT = 64 * 128 * 2, GOT = N3 * 128 * 2, HT = K1 * 128 * 2, UT = kTcK2 * 128 * 2;
  static constexpr uint32_t gat_off = p1_off + P, got_off = gat_off + GAT, ht_off = got_off + GOT;
  static constexpr uint32_t u1t_off = ht_off + HT, u2t_off = u1t_off + UT;
  static constexpr uint32_t misc = u2t_off + UT;  // mbarrier, tensor-memory slot, warp sums
  // the bf16 weight image in global memory, built once a call: the natural weights of every layer exactly as they
  // sit in shared memory, then each layer's transposed block (W3T, W2T, W1T, as at w3t_off)
  static constexpr uint32_t WTL = W3T + W2T + W1T;
  static constexpr uint32_t image = S::weights + kFlowLayers * WTL;
  static constexpr uint32_t total = misc + 64;
  static constexpr uint32_t kM128 = 128 * 128 * 2;  // the bytes an M = 128 A operand of K = 128 spans
  static_assert(gat_off + kM128 <= misc && got_off + kM128 <= misc, "padded A reads stay in the activations");
  static_assert(total <= 232448, "shared memory of one CTA");
};

constexpr uint32_t kGradTmemCols = 256;  // [0, 64): forward and input gradients; [64, 144): weight gradients

__device__ __forceinline__ void st_bf16_at(unsigned char* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// operands written: vote barrier, thread 0 issues the MMAs (issue()), commits them to the mbarrier, every thread
// waits (bounded); false on every thread once a wait ran out
template <typename Issue>
__device__ __forceinline__ bool grad_run(TcGroup& G, Issue&& issue) {
  tc_fence_proxy();
  tc_fence_before();
  if (wg_bar_any(1, G.failed)) return false;
  if (G.t == 0) {
    tc_fence_after();
    issue();
    tc_commit(G.mbar);
  }
  if (!mbar_wait(G.mbar, G.phase, kTcWaitPolls)) {
    G.failed = true;
    atomicOr(&g_flow_grad_status, 4);
  }
  G.phase ^= 1u;
  tc_fence_after();
  return true;
}

// D (tensor memory) = A B^T over K / 16 k-steps, accumulate from the first; A rows of KA columns, B of KB
__device__ __forceinline__ void grad_gemm(uint32_t tcol, const unsigned char* A, int KA, const unsigned char* B, int KB,
                                          int K, uint32_t idesc) {
  const uint64_t ad = tc_desc(tc_smem_u32(A), kTcLbo, (uint32_t)KA * 16);
  const uint64_t bd = tc_desc(tc_smem_u32(B), kTcLbo, (uint32_t)KB * 16);
  for (int s = 0; s < K / 16; ++s) tc_mma(tcol, ad + 16u * s, bd + 16u * s, idesc, s > 0);
}

// row t of the 64 accumulator columns: ReLU, bf16 into the natural tile (row t) and the transposed one
// (column t); the ReLU mask of the row as 64 bits
__device__ __forceinline__ uint64_t grad_hidden_epilogue(uint32_t tacc, unsigned char* U, unsigned char* UT, int t) {
  uint64_t mask = 0;
#pragma unroll
  for (int cb = 0; cb < 64; cb += 16) {
    float v[16];
    tc_ld16(tacc + cb, v);
#pragma unroll
    for (int q = 0; q < 2; ++q)
      st_shared_v4(U + tc_off(t, cb + 8 * q, kTcK2), bf16x2_relu(v[8 * q], v[8 * q + 1]),
                   bf16x2_relu(v[8 * q + 2], v[8 * q + 3]), bf16x2_relu(v[8 * q + 4], v[8 * q + 5]),
                   bf16x2_relu(v[8 * q + 6], v[8 * q + 7]));
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float r = v[j] > 0.0f ? v[j] : 0.0f;
      if (v[j] > 0.0f) mask |= 1ull << (cb + j);
      st_bf16_at(UT, tc_off(cb + j, t, 128), r);
    }
  }
  return mask;
}

// row t of a 64-column gradient accumulator, masked by the ReLU of its pre-activation, in bf16 into the natural
// tile and the transposed one
__device__ __forceinline__ void grad_masked_epilogue(uint32_t tacc, uint64_t mask, unsigned char* G_, unsigned char* GT,
                                                     int t) {
#pragma unroll
  for (int cb = 0; cb < 64; cb += 16) {
    float v[16];
    tc_ld16(tacc + cb, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = ((mask >> (cb + j)) & 1ull) ? v[j] : 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q)
      st_shared_v4(G_ + tc_off(t, cb + 8 * q, kTcK2), bf16x2(v[8 * q], v[8 * q + 1]), bf16x2(v[8 * q + 2], v[8 * q + 3]),
                   bf16x2(v[8 * q + 4], v[8 * q + 5]), bf16x2(v[8 * q + 6], v[8 * q + 7]));
#pragma unroll
    for (int j = 0; j < 16; ++j) st_bf16_at(GT, tc_off(cb + j, t, 128), v[j]);
  }
}

// rows 0..nrows-1 of a weight-gradient accumulator of ncols columns (<= 80) to the partial gradient: row r goes to
// W[r][0..nw-1] at offset ow (row stride nw) and, from column bcol, to the bias at ob + r.  Warp w reads lanes
// 32w..32w+31; the warps past nrows do not take part.
__device__ __forceinline__ void grad_store_rows(uint32_t taccB, int nrows, int nw, int bcol, float* __restrict__ gp,
                                                int ow, int ob, int t) {
  const int warp = t >> 5;
  if (warp * 32 >= nrows) return;
  float v[80];
  {
    float a[32];
    tc_ld32(taccB, a);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = a[j];
    tc_ld32(taccB + 32, a);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[32 + j] = a[j];
    float c[16];
    tc_ld16(taccB + 64, c);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[64 + j] = c[j];
  }
  if (t < nrows) {
#pragma unroll
    for (int c = 0; c < kFlowHidden; ++c)
      if (c < nw) gp[ow + t * nw + c] = v[c];
    gp[ob + t] = v[bcol];
  }
}

// The weight image: element i of layer blockIdx.y's natural (tc_stage_weights' layout) and transposed blocks,
// bf16 from the FP32 parameters, grid-stride over the layer's elements
template <int D>
__global__ void flow_grad_image_kernel(const __grid_constant__ FlowArgs fa, unsigned char* __restrict__ img) {
  using S = TcShape<D>;
  using Q = GradTcShape<D>;
  const int l = blockIdx.y;
  const FlowLayer& L = fa.lay[l];
  const float* P = fa.params;
  unsigned char* w1 = img + l * S::layer;
  unsigned char* w2 = w1 + S::W1;
  unsigned char* w3 = w2 + S::W2;
  unsigned char* wt = img + S::weights + (size_t)l * Q::WTL;
  unsigned char* w3t = wt;
  unsigned char* w2t = wt + Q::W3T;
  unsigned char* w1t = w2t + Q::W2T;
  const int n1 = 64 * S::K1, n2 = 64 * kTcK2, n3 = S::N3 * kTcK2, n4 = 64 * S::N3, n5 = 64 * 64, n6 = S::K1 * 64;
  const int total = n1 + n2 + n3 + n4 + n5 + n6;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int e = i;
    __nv_bfloat16 h, m, lo;
    if (e < n1) {  // W1' [64][K1]: W1, then the bias triple
      const int j = e / S::K1, c = e - j * S::K1;
      float v = 0.0f;
      if (c < L.a) v = P[L.oW1 + j * L.a + c];
      __nv_bfloat16 b = __float2bfloat16_rn(v);
      if (c >= L.a && c < L.a + 3) {
        bias3(P[L.ob1 + j], h, m, lo);
        b = c == L.a ? h : (c == L.a + 1 ? m : lo);
      }
      *reinterpret_cast<__nv_bfloat16*>(w1 + tc_off(j, c, S::K1)) = b;
      continue;
    }
    e -= n1;
    if (e < n2) {  // W2' [64][80]
      const int j = e / kTcK2, c = e - j * kTcK2;
      __nv_bfloat16 b = __float2bfloat16_rn(c < kFlowHidden ? P[L.oW2 + j * kFlowHidden + c] : 0.0f);
      if (c >= kFlowHidden && c < kFlowHidden + 3) {
        bias3(P[L.ob2 + j], h, m, lo);
        b = c == kFlowHidden ? h : (c == kFlowHidden + 1 ? m : lo);
      }
      *reinterpret_cast<__nv_bfloat16*>(w2 + tc_off(j, c, kTcK2)) = b;
      continue;
    }
    e -= n2;
    if (e < n3) {  // W3' [N3][80]
      const int j = e / kTcK2, c = e - j * kTcK2;
      __nv_bfloat16 b = __float2bfloat16_rn(0.0f);
      if (j < 2 * L.b) {
        if (c < kFlowHidden) b = __float2bfloat16_rn(P[L.oW3 + j * kFlowHidden + c]);
        else if (c < kFlowHidden + 3) {
          bias3(P[L.ob3 + j], h, m, lo);
          b = c == kFlowHidden ? h : (c == kFlowHidden + 1 ? m : lo);
        }
      }
      *reinterpret_cast<__nv_bfloat16*>(w3 + tc_off(j, c, kTcK2)) = b;
      continue;
    }
    e -= n3;
    if (e < n4) {  // W3T [64][N3]: element (hh, o) is W3[o][hh]; the loop runs along the rows of W3
      const int o = e >> 6, hh = e & 63;
      *reinterpret_cast<__nv_bfloat16*>(w3t + tc_off(hh, o, S::N3)) =
          __float2bfloat16_rn(o < 2 * L.b ? P[L.oW3 + o * kFlowHidden + hh] : 0.0f);
      continue;
    }
    e -= n4;
    if (e < n5) {  // W2T [64][64]: element (r, c) is W2[c][r]
      const int c = e >> 6, r = e & 63;
      *reinterpret_cast<__nv_bfloat16*>(w2t + tc_off(r, c, 64)) = __float2bfloat16_rn(P[L.oW2 + c * kFlowHidden + r]);
      continue;
    }
    e -= n5;
    {  // W1T [K1][64]: element (c, hh) is W1[hh][c]
      const int hh = e / S::K1, c = e - hh * S::K1;
      *reinterpret_cast<__nv_bfloat16*>(w1t + tc_off(c, hh, 64)) =
          __float2bfloat16_rn(c < L.a ? P[L.oW1 + hh * L.a + c] : 0.0f);
    }
  }
}

// 16-byte asynchronous copies of `bytes` (a multiple of 16) from global to shared memory by the CTA; completed
// by cp_async_wait_all and a barrier
__device__ __forceinline__ void copy_async(unsigned char* dst, const unsigned char* __restrict__ src, uint32_t bytes) {
  for (uint32_t o = threadIdx.x * 16u; o < bytes; o += blockDim.x * 16u)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc_smem_u32(dst + o)), "l"(src + o) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// H row t into the natural tile (first K1 columns) and, with `transposed`, column t of H^T
template <int D, int PAR>
__device__ __forceinline__ void grad_write_h(const float (&z)[D], unsigned char* Pn, unsigned char* HT, int t,
                                             bool transposed) {
  using S = TcShape<D>;
  constexpr int a = PAR == 0 ? (D + 1) / 2 : D / 2;
  float hv[S::K1];
#pragma unroll
  for (int c = 0; c < S::K1; ++c) hv[c] = c < a ? z[2 * c + PAR] : (c < a + 3 ? 1.0f : 0.0f);
#pragma unroll
  for (int q = 0; q < S::K1 / 8; ++q)
    st_shared_v4(Pn + tc_off(t, 8 * q, kTcK2), bf16x2(hv[8 * q], hv[8 * q + 1]), bf16x2(hv[8 * q + 2], hv[8 * q + 3]),
                 bf16x2(hv[8 * q + 4], hv[8 * q + 5]), bf16x2(hv[8 * q + 6], hv[8 * q + 7]));
  if (transposed) {
#pragma unroll
    for (int c = 0; c < S::K1; ++c) st_bf16_at(HT, tc_off(c, t, 128), hv[c]);
  }
}

// The conditioner of layer l on the tile: GEMM1-3 with H in P0, U1 in P1, U2 in P0; o (row t, N3 columns) out.
// With `keep` the transposed activations and the ReLU masks are kept for the backward pass.
template <int D, int PAR>
__device__ __forceinline__ bool grad_conditioner(const unsigned char* wl, unsigned char* sm, TcGroup& G,
                                                 const float (&z)[D], bool keep, float (&o)[TcShape<D>::N3],
                                                 uint64_t& m1, uint64_t& m2) {
  using S = TcShape<D>;
  using Q = GradTcShape<D>;
  const int t = G.t;
  unsigned char* P0 = sm + Q::p0_off;
  unsigned char* P1 = sm + Q::p1_off;
  const unsigned char* w1 = wl;
  const unsigned char* w2 = wl + S::W1;
  const unsigned char* w3 = w2 + S::W2;
  const uint32_t tcol = G.tacc & 0xFFFFu;
  grad_write_h<D, PAR>(z, P0, sm + Q::ht_off, t, keep);
  if (!grad_run(G, [&] { grad_gemm(tcol, P0, kTcK2, w1, S::K1, S::K1, tc_idesc_bf16(128, 64)); })) return false;
  if (keep) m1 = grad_hidden_epilogue(G.tacc, P1, sm + Q::u1t_off, t);
  else tc_hidden_epilogue(G.tacc, P1, t);
  tc_fence_before();
  if (!grad_run(G, [&] { grad_gemm(tcol, P1, kTcK2, w2, kTcK2, kTcK2, tc_idesc_bf16(128, 64)); })) return false;
  if (keep) m2 = grad_hidden_epilogue(G.tacc, P0, sm + Q::u2t_off, t);
  else tc_hidden_epilogue(G.tacc, P0, t);
  tc_fence_before();
  if (!grad_run(G, [&] { grad_gemm(tcol, P0, kTcK2, w3, kTcK2, kTcK2, tc_idesc_bf16(128, S::N3)); })) return false;
  tc_ld16(G.tacc, o);
  tc_fence_before();
  return true;
}

template <int D, int PAR>
__device__ __forceinline__ bool grad_forward_layer(const unsigned char* wl, unsigned char* sm, TcGroup& G,
                                                   float (&z)[D], float& ld) {
  constexpr int a = PAR == 0 ? (D + 1) / 2 : D / 2, b = D - a;
  float o[TcShape<D>::N3];
  uint64_t m1 = 0, m2 = 0;
  if (!grad_conditioner<D, PAR>(wl, sm, G, z, false, o, m1, m2)) return false;
#pragma unroll
  for (int m = 0; m < b; ++m) {
    const int k = 2 * m + 1 - PAR;
    const float s = flow_soft_clamp(o[2 * m]);
    z[k] = fmaf(z[k], __expf(s), o[2 * m + 1]);
    ld += s;
  }
  return true;
}

// The backward pass through layer l: on entry z is the output of the layer and gz = dL/dz there; on exit z is
// its input and gz = dL/dz before the layer.  The layer's weight gradients go to gp.
template <int D, int PAR>
__device__ __forceinline__ bool grad_backward_layer(const FlowLayer& L, const unsigned char* __restrict__ wt_img,
                                                    const unsigned char* wl, unsigned char* sm, TcGroup& G,
                                                    float (&z)[D], float (&gz)[D], float wn, float* __restrict__ gp) {
  using S = TcShape<D>;
  using Q = GradTcShape<D>;
  constexpr int a = PAR == 0 ? (D + 1) / 2 : D / 2, b = D - a;
  const int t = G.t;
  unsigned char* P0 = sm + Q::p0_off;
  unsigned char* P1 = sm + Q::p1_off;
  unsigned char* GAT = sm + Q::gat_off;
  unsigned char* GOT = sm + Q::got_off;
  const uint32_t tcolA = G.tacc & 0xFFFFu, tcolB = tcolA + 64;
  const uint32_t taccB = G.tacc + 64;
  // the layer's transposed weights: asynchronous copies, complete before the first MMA that reads them (the
  // conditioner's barriers come after the wait)
  copy_async(sm + Q::w3t_off, wt_img, Q::WTL);
  copy_async_wait();
  float o[S::N3];
  uint64_t m1 = 0, m2 = 0;
  if (!grad_conditioner<D, PAR>(wl, sm, G, z, true, o, m1, m2)) return false;
  // GO = dL/d(s, t) of the sample; z and gz back through the affine update
  float go[S::N3];
#pragma unroll
  for (int j = 0; j < S::N3; ++j) go[j] = 0.0f;
#pragma unroll
  for (int m = 0; m < b; ++m) {
    const int k = 2 * m + 1 - PAR;
    const float s = flow_soft_clamp(o[2 * m]), tt = o[2 * m + 1];
    const float es = __expf(s);
    const float zin = (z[k] - tt) * __expf(-s);
    const float gs = -wn + gz[k] * zin * es;  // the log-determinant term and z_out = z_in e^s + t
    go[2 * m] = gs * (1.0f - (s / kFlowSClamp) * (s / kFlowSClamp));
    go[2 * m + 1] = gz[k];
    gz[k] *= es;
    z[k] = zin;
  }
#pragma unroll
  for (int q = 0; q < S::N3 / 8; ++q)
    st_shared_v4(P1 + tc_off(t, 8 * q, kTcK2), bf16x2(go[8 * q], go[8 * q + 1]), bf16x2(go[8 * q + 2], go[8 * q + 3]),
                 bf16x2(go[8 * q + 4], go[8 * q + 5]), bf16x2(go[8 * q + 6], go[8 * q + 7]));
#pragma unroll
  for (int j = 0; j < S::N3; ++j) st_bf16_at(GOT, tc_off(j, t, 128), go[j]);
  // gU2 = GO W3 and dW3 = GO^T [U2 | 1]
  if (!grad_run(G, [&] {
        grad_gemm(tcolA, P1, kTcK2, sm + Q::w3t_off, S::N3, S::N3, tc_idesc_bf16(128, 64));
        grad_gemm(tcolB, GOT, 128, sm + Q::u2t_off, 128, 128, tc_idesc_bf16(128, kTcK2));
      }))
    return false;
  grad_masked_epilogue(G.tacc, m2, P0, GAT, t);  // GA2
  grad_store_rows(taccB, 2 * b, kFlowHidden, kFlowHidden, gp, L.oW3, L.ob3, t);
  tc_fence_before();
  // gU1 = GA2 W2 and dW2 = GA2^T [U1 | 1]
  if (!grad_run(G, [&] {
        grad_gemm(tcolA, P0, kTcK2, sm + Q::w2t_off, 64, 64, tc_idesc_bf16(128, 64));
        grad_gemm(tcolB, GAT, 128, sm + Q::u1t_off, 128, 128, tc_idesc_bf16(128, kTcK2));
      }))
    return false;
  grad_masked_epilogue(G.tacc, m1, P1, GAT, t);  // GA1
  grad_store_rows(taccB, 64, kFlowHidden, kFlowHidden, gp, L.oW2, L.ob2, t);
  tc_fence_before();
  // gH = GA1 W1 and dW1 = GA1^T H (H's ones give the bias)
  if (!grad_run(G, [&] {
        grad_gemm(tcolA, P1, kTcK2, sm + Q::w1t_off, 64, 64, tc_idesc_bf16(128, S::K1));
        grad_gemm(tcolB, GAT, 128, sm + Q::ht_off, 128, 128, tc_idesc_bf16(128, S::K1));
      }))
    return false;
  {
    float gh[16];
    tc_ld16(G.tacc, gh);
#pragma unroll
    for (int c = 0; c < a; ++c) gz[2 * c + PAR] += gh[c];
  }
  {
    const int warp = t >> 5;
    if (warp < 2) {  // rows 0..63
      float v[16];
      tc_ld16(taccB, v);
      for (int c = 0; c < a; ++c) gp[L.oW1 + t * a + c] = v[c];
      gp[L.ob1 + t] = v[a];
    }
  }
  tc_fence_before();
  return true;
}

template <int D>
__global__ void __launch_bounds__(128, 1)
    flow_grad_tc_kernel(const __grid_constant__ FlowArgs fa, const unsigned char* __restrict__ img,
                        const float* __restrict__ x, const float* __restrict__ w, const double* __restrict__ wsum,
                        int64_t n, float* __restrict__ gpart, float* __restrict__ lpart) {
  using S = TcShape<D>;
  using Q = GradTcShape<D>;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + Q::misc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + Q::misc + 8);
  float* red = reinterpret_cast<float*>(sm + Q::misc + 16);
  copy_async(sm, img, S::weights);  // the natural weights of every layer
  // the constant parts of the activations: ones blocks of the natural tiles (columns 64..79: 1 1 1 0 ...) and
  // of the transposed ones (rows 64..79)
  for (unsigned char* Pn : {sm + Q::p0_off, sm + Q::p1_off}) {
    st_shared_v4(Pn + tc_off(t, kFlowHidden, kTcK2), 0x3F803F80u, 0x00003F80u, 0u, 0u);
    st_shared_v4(Pn + tc_off(t, kFlowHidden + 8, kTcK2), 0u, 0u, 0u, 0u);
  }
  for (int r = kFlowHidden; r < kTcK2; ++r) {
    const float v = r < kFlowHidden + 3 ? 1.0f : 0.0f;
    st_bf16_at(sm + Q::u1t_off, tc_off(r, t, 128), v);
    st_bf16_at(sm + Q::u2t_off, tc_off(r, t, 128), v);
  }
  if (warp == 0) tc_alloc(tslot, kGradTmemCols);
  if (t == 0) {
    mbar_init(mbar, 1);
    mbar_fence_init();
  }
  copy_async_wait();
  tc_fence_proxy();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  TcGroup G;
  G.id = 0;
  G.t = t;
  G.tacc = tbase + ((uint32_t)(warp * 32) << 16);
  G.mbar = mbar;
  G.phase = 0;
  G.failed = false;

  // the sample and its normalised weight (weights that are negative or not finite count as 0)
  const int64_t row = (int64_t)blockIdx.x * 128 + t;
  const bool live = row < n;
  const double ws = *wsum;
  const float inv = (ws > 0.0 && ws < INFINITY) ? (float)(1.0 / ws) : 0.0f;
  const float wr = live ? w[row] : 0.0f;
  const float wn = (isfinite(wr) && wr > 0.0f) ? wr * inv : 0.0f;
  float z[D], gz[D];
  float ld = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    z[k] = flow_logit(live ? x[row * D + k] : 0.5f);
    ld -= flow_log_sig_prime(z[k]);
  }
  bool ok = true;
#pragma unroll 1
  for (int l = 0; l < kFlowLayers; ++l) {
    if (!ok) break;
    const unsigned char* wl = sm + l * S::layer;
    ok = (l & 1) ? grad_forward_layer<D, 1>(wl, sm, G, z, ld) : grad_forward_layer<D, 0>(wl, sm, G, z, ld);
  }
  // loss of the sample and the gradient from the output wrap: d/dz log sigmoid'(z) = 1 - 2 sigmoid(z)
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ld += flow_log_sig_prime(z[k]);
    gz[k] = -wn * (1.0f - 2.0f * flow_sigmoid(z[k]));
  }
  {
    float part = -wn * ld;
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (lane == 0) red[warp] = part;
  }
  float* gp = gpart + (size_t)blockIdx.x * fa.nparams;
#pragma unroll 1
  for (int l = kFlowLayers - 1; l >= 0; --l) {
    if (!ok) break;
    const unsigned char* wl = sm + l * S::layer;
    const unsigned char* wt = img + S::weights + (size_t)l * Q::WTL;
    ok = (l & 1) ? grad_backward_layer<D, 1>(fa.lay[l], wt, wl, sm, G, z, gz, wn, gp)
                 : grad_backward_layer<D, 0>(fa.lay[l], wt, wl, sm, G, z, gz, wn, gp);
  }
  // a warpgroup that gave up waits once more for its MMAs before the columns are freed
  if (G.failed) mbar_wait(G.mbar, G.phase ^ 1u, kTcWaitPolls);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (t == 0) lpart[blockIdx.x] = red[0] + red[1] + red[2] + red[3];  // the partial loss
  if (warp == 0) tc_dealloc(tbase, kGradTmemCols);
}

template <int D>
int launch_grad_tc(const FlowArgs& fa, unsigned char* img, const float* x, const float* w, const double* wsum,
                   int64_t n, float* gpart, float* lpart, cudaStream_t s) {
  using Q = GradTcShape<D>;
  flow_grad_image_kernel<D><<<dim3(8, kFlowLayers), 256, 0, s>>>(fa, img);
  VG_CHECK(cudaGetLastError());
  auto k = flow_grad_tc_kernel<D>;
  VG_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::total));
  const int64_t nblk = (n + 127) / 128;
  k<<<(unsigned)nblk, 128, Q::total, s>>>(fa, img, x, w, wsum, n, gpart, lpart);
  return cuda_status(cudaGetLastError());
}

template <typename F>
int dispatch_grad_d(int d, F&& f) {
  switch (d) {
#define VG_D(N) \
  case N: return f(std::integral_constant<int, N>{});
    VG_D(2) VG_D(3) VG_D(4) VG_D(5) VG_D(6) VG_D(7) VG_D(8) VG_D(9) VG_D(10) VG_D(11) VG_D(12) VG_D(13) VG_D(14)
    VG_D(15) VG_D(16)
#undef VG_D
    default: return VEGAS_EINVAL;
  }
}

}  // namespace

// the tensor-core gradient: the weight image (flow_grad_tc_image_bytes(d) bytes, 16-byte aligned), then one CTA
// (128 threads) per 128 samples; gpart [ceil(n/128)][nparams], lpart likewise
int flow_grad_tc(const FlowArgs& fa, unsigned char* img, const float* x, const float* w, const double* wsum,
                 int64_t n, float* gpart, float* lpart, cudaStream_t s) {
  return dispatch_grad_d(fa.d, [&](auto D) {
    return launch_grad_tc<decltype(D)::value>(fa, img, x, w, wsum, n, gpart, lpart, s);
  });
}

size_t flow_grad_tc_image_bytes(int d) {
  if (d < 2 || d > kFlowGradTcMaxDim) return 0;
  return dispatch_grad_d(d, [&](auto D) { return (int)GradTcShape<decltype(D)::value>::image; });
}

int flow_grad_tc_status(bool reset) {
  int v = 0;
  VG_CHECK(cudaMemcpyFromSymbol(&v, g_flow_grad_status, sizeof(int)));
  if (reset && v) {
    const int zero = 0;
    VG_CHECK(cudaMemcpyToSymbol(g_flow_grad_status, &zero, sizeof(int)));
  }
  return (v & 4) ? VEGAS_ETIMEOUT : VEGAS_OK;
}

}  // namespace vg
