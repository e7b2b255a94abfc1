// vegas_flow.cu -- the learned proposal's coupling flow: parameter layout,
// the batched transform in either direction, the gradient of the training
// loss and the Adam update (vegas_flow_* of the C ABI).  The flow itself is
// described in vegas_flow.cuh.
#include <algorithm>
#include <cmath>

#include "vegas_flow.cuh"
#include "vegas_internal.h"

namespace vg {

namespace {
constexpr size_t kAl = 16;
size_t al16(size_t x) { return (x + kAl - 1) / kAl * kAl; }
}  // namespace

// Offsets of every layer's blocks in the parameter vector (W1 [64][a], b1,
// W2 [64][64], b2, W3 [2b][64], b3, in that order, layer after layer) and in
// the shared-memory copy.
int flow_layout(int d, FlowArgs& fa) {
  if (d < 2 || d > kFlowMaxDim) return VEGAS_EINVAL;
  fa.d = d;
  int off = 0;
  size_t so = 0;
  for (int l = 0; l < kFlowLayers; ++l) {
    FlowLayer& L = fa.lay[l];
    L.a = (l % 2 == 0) ? (d + 1) / 2 : d / 2;
    L.b = d - L.a;
    L.no = (2 * L.b + 15) / 16 * 16;  // outputs padded to 16: the n-tiles of W3 load in pairs
    L.oW1 = off; off += kFlowHidden * L.a;
    L.ob1 = off; off += kFlowHidden;
    L.oW2 = off; off += kFlowHidden * kFlowHidden;
    L.ob2 = off; off += kFlowHidden;
    L.oW3 = off; off += 2 * L.b * kFlowHidden;
    L.ob3 = off; off += 2 * L.b;
    L.sW1 = (int)so; so = al16(so + sizeof(__nv_bfloat16) * kFlowHidden * kLdK16);
    L.sb1 = (int)so; so = al16(so + sizeof(float) * kFlowHidden);
    L.sW2 = (int)so; so = al16(so + sizeof(__nv_bfloat16) * kFlowHidden * kLdK64);
    L.sb2 = (int)so; so = al16(so + sizeof(float) * kFlowHidden);
    L.sW3 = (int)so; so = al16(so + sizeof(__nv_bfloat16) * L.no * kLdK64);
    L.sb3 = (int)so; so = al16(so + sizeof(float) * L.no);
  }
  fa.nparams = off;
  fa.smem_weights = (int)so;
  return VEGAS_OK;
}

namespace {

__host__ __device__ inline int flow_zld(int d) { return d | 1; }  // odd row stride: fewer bank conflicts

int num_sms_flow() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace

}  // namespace vg

using namespace vg;

extern "C" int64_t vegas_flow_param_count(int32_t dim) {
  FlowArgs fa{};
  return flow_layout(dim, fa) == VEGAS_OK ? fa.nparams : 0;
}

extern "C" int vegas_flow_apply(int32_t dim, int32_t direction, const float* d_params, const float* d_x_in,
                                float* d_x_out, float* d_logdet, int64_t n, void* stream) {
  if (dim < 2 || dim > kFlowMaxDim || n < 0 || !d_params || (n > 0 && (!d_x_in || !d_x_out || !d_logdet)))
    return VEGAS_EINVAL;
  if (direction != VEGAS_FLOW_NORMALISE && direction != VEGAS_FLOW_SAMPLE) return VEGAS_EINVAL;
  if (n == 0) return VEGAS_OK;
  return flow_apply(dim, direction, d_params, d_x_in, d_x_out, d_logdet, n, (cudaStream_t)stream);
}

extern "C" int vegas_flow_check(void* stream) {
  VG_CHECK(cudaStreamSynchronize((cudaStream_t)stream));
  const int a = flow_tc_status(true), b = flow_grad_tc_status(true);
  return a != VEGAS_OK ? a : b;
}

extern "C" int vegas_flow_wait_selftest(int32_t polls, int32_t arrive, void* stream) {
  if (polls < 1 || polls > (1 << 24)) return VEGAS_EINVAL;
  const int rc = flow_tc_wait_selftest(polls, arrive != 0, (cudaStream_t)stream);
  if (rc != VEGAS_OK) return rc;
  return vegas_flow_check(stream);
}

// ===========================================================================
// Training: loss = - sum_i w_i log|det dN/dx(x_i)| / sum_i w_i and its
// gradient.  A CTA of 2 warps takes 32 samples, so a minibatch of 4096
// spreads over 128 CTAs; the bf16 weights, natural and transposed, are built
// once a call (flow_image_kernel) and copied by every CTA.  The forward pass in
// the normalising direction keeps z before every layer; the backward pass
// recomputes each layer's conditioner and runs its six GEMMs on the tensor
// cores (bf16 operands, FP32 accumulation):
//   dW3 = GO^T U2,  gU2 = GO W3,  dW2 = GA2^T U1,  gU1 = GA2 W2,
//   dW1 = GA1^T H,  gH = GA1 W1,
// with GO the gradient of the layer's (s, t) outputs, GA2 / GA1 those of the
// hidden pre-activations.  Each CTA writes its partial gradient; a second
// kernel sums the partials in a fixed order.
// ===========================================================================
namespace vg {
namespace {

// W warps a CTA, 16 W samples.  W = 2: a minibatch of 4096 samples then spreads over 128 CTAs (with W = 4,
// 64 CTAs left most SMs idle), and above 16 axes shared memory allows no more.
__host__ __device__ constexpr int grad_rows(int W) { return 16 * W; }
__host__ __device__ constexpr int grad_ldr(int W) { return 16 * W + 8; }  // sample-major tiles: 20 or 36 words
inline int grad_warps(int) { return 2; }

struct GradLayout {
  int wnat;               // natural weights of all layers (the layout of flow_layout, built by flow_image_kernel)
  int w1t, w2t, w3t;      // transposed weights of the current layer
  int zs;                 // z before each layer [L][R][zld] f32, then z after the last
  int gz;                 // [R][zld] f32
  int wn;                 // [R] f32 normalised weights
  int H, HT, U1, U1T, U2, U2T, GO, GOT;
  int bias;               // [64 + 64 + 32] f32 bias-gradient accumulators
  int red;                // [W] f32
  int total;
  int ldo;                // leading dimension of GO (no padded to 16 or 32, + 8)
  // the weight image in global memory: the staged natural weights (smem_weights bytes), then per layer
  // the transposed block W1T, W2T, W3T exactly as laid out in shared memory from w1t on (img_tsz bytes)
  int img_t, img_tsz, img_total;
};

GradLayout grad_layout(const FlowArgs& fa, int W) {
  GradLayout G{};
  const int kGradRows = grad_rows(W), kLdR = grad_ldr(W);
  const int zld = flow_zld(fa.d);
  int nomax = 8;
  for (int l = 0; l < kFlowLayers; ++l) nomax = std::max(nomax, fa.lay[l].no);
  const int kpad = nomax <= 16 ? 16 : 32;
  G.ldo = kpad + 8;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = al16(o + bytes);
    return (int)at;
  };
  G.wnat = take(fa.smem_weights);
  G.w1t = take(sizeof(__nv_bfloat16) * 16 * kLdK64);
  G.w2t = take(sizeof(__nv_bfloat16) * 64 * kLdK64);
  G.w3t = take(sizeof(__nv_bfloat16) * 64 * G.ldo);
  G.zs = take(sizeof(float) * (kFlowLayers + 1) * kGradRows * zld);
  G.gz = take(sizeof(float) * kGradRows * zld);
  G.wn = take(sizeof(float) * kGradRows);
  G.H = take(sizeof(__nv_bfloat16) * kGradRows * kLdK16);
  G.HT = take(sizeof(__nv_bfloat16) * 16 * kLdR);
  G.U1 = take(sizeof(__nv_bfloat16) * kGradRows * kLdK64);
  G.U1T = take(sizeof(__nv_bfloat16) * 64 * kLdR);
  G.U2 = take(sizeof(__nv_bfloat16) * kGradRows * kLdK64);
  G.U2T = take(sizeof(__nv_bfloat16) * 64 * kLdR);
  G.GO = take(sizeof(__nv_bfloat16) * kGradRows * G.ldo);
  G.GOT = take(sizeof(__nv_bfloat16) * 32 * kLdR);
  G.bias = take(sizeof(float) * (64 + 64 + 32));
  G.red = take(sizeof(float) * W);
  G.total = (int)o;
  G.img_t = (int)al16((size_t)fa.smem_weights);
  G.img_tsz = G.zs - G.w1t;
  G.img_total = G.img_t + kFlowLayers * G.img_tsz;
  return G;
}

// The weight image of one gradient call: blockIdx.y = layer; the CTAs of a layer share its elements.
__global__ void flow_image_kernel(const __grid_constant__ FlowArgs fa, GradLayout G, unsigned char* __restrict__ img) {
  const int l = blockIdx.y;
  const FlowLayer& L = fa.lay[l];
  const float* P = fa.params;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, step = gridDim.x * blockDim.x;
  __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(img + L.sW1);
  __nv_bfloat16* W2 = reinterpret_cast<__nv_bfloat16*>(img + L.sW2);
  __nv_bfloat16* W3 = reinterpret_cast<__nv_bfloat16*>(img + L.sW3);
  float* b1 = reinterpret_cast<float*>(img + L.sb1);
  float* b2 = reinterpret_cast<float*>(img + L.sb2);
  float* b3 = reinterpret_cast<float*>(img + L.sb3);
  unsigned char* T = img + G.img_t + (size_t)l * G.img_tsz;
  __nv_bfloat16* W1T = reinterpret_cast<__nv_bfloat16*>(T);
  __nv_bfloat16* W2T = reinterpret_cast<__nv_bfloat16*>(T + (G.w2t - G.w1t));
  __nv_bfloat16* W3T = reinterpret_cast<__nv_bfloat16*>(T + (G.w3t - G.w1t));
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  // natural layout (offsets sW1.. of flow_layout): rows padded, zero padding; the transposes beside them
  for (int i = i0; i < kFlowHidden * kLdK16; i += step) {
    const int r = i / kLdK16, c = i - r * kLdK16;
    const __nv_bfloat16 v = c < L.a ? __float2bfloat16_rn(P[L.oW1 + r * L.a + c]) : zero;
    W1[i] = v;
    if (c < 16) W1T[c * kLdK64 + r] = v;  // W1T [16][64 + pad]: column c of W1
  }
  for (int i = i0; i < kFlowHidden * kLdK64; i += step) {
    const int r = i / kLdK64, c = i - r * kLdK64;
    const __nv_bfloat16 v = c < kFlowHidden ? __float2bfloat16_rn(P[L.oW2 + r * kFlowHidden + c]) : zero;
    W2[i] = v;
    if (c < kFlowHidden) W2T[c * kLdK64 + r] = v;
  }
  for (int i = i0; i < L.no * kLdK64; i += step) {
    const int r = i / kLdK64, c = i - r * kLdK64;
    W3[i] = (r < 2 * L.b && c < kFlowHidden) ? __float2bfloat16_rn(P[L.oW3 + r * kFlowHidden + c]) : zero;
  }
  for (int i = i0; i < kFlowHidden * G.ldo; i += step) {  // W3T [64][ldo]: zero past 2 b
    const int c = i / G.ldo, o = i - c * G.ldo;
    W3T[i] = o < 2 * L.b ? __float2bfloat16_rn(P[L.oW3 + o * kFlowHidden + c]) : zero;
  }
  for (int i = i0; i < kFlowHidden; i += step) {
    b1[i] = P[L.ob1 + i];
    b2[i] = P[L.ob2 + i];
  }
  for (int i = i0; i < L.no; i += step) b3[i] = i < 2 * L.b ? P[L.ob3 + i] : 0.0f;
}

template <typename T>
__device__ __forceinline__ T* at(unsigned char* sm, int off) {
  return reinterpret_cast<T*>(sm + off);
}

// C[M x N] = A[M x K] B^T with A [M][lda] and B [N][ldb] bf16 row-major (K
// contiguous); the 16 x 8 tiles are dealt to the CTA's warps; epi(row, col,
// v0, v1) receives each thread's pairs (col, col + 1).
template <int W, typename Epi>
__device__ __forceinline__ void cta_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
                                         int N, int K, Epi&& epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt = M / 16, nt = N / 8;
  for (int tile = warp; tile < mt * nt; tile += W) {
    const int m0 = (tile / nt) * 16, n0 = (tile % nt) * 8;
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k0 = 0; k0 < K; k0 += 16) {
      uint32_t a[4], b0, b1;
      load_a(A, lda, m0, k0, a);
      load_b(B, ldb, n0, k0, b0, b1);
      mma16816(c, a[0], a[1], a[2], a[3], b0, b1);
    }
    epi(m0 + g, n0 + 2 * t, c[0], c[1]);
    epi(m0 + g + 8, n0 + 2 * t, c[2], c[3]);
  }
}

// sum over the 8 lanes that share t (lane bits 2-4)
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

__device__ __forceinline__ void st_bf16(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// 16-byte copy of `bytes` (a multiple of 16) from global to shared memory by the CTA
__device__ __forceinline__ void copy16(unsigned char* dst, const unsigned char* __restrict__ src, int bytes) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d4[i] = s4[i];
}

template <int W>
__global__ void __launch_bounds__(W * 32) flow_grad_kernel(const __grid_constant__ FlowArgs fa,
                                                                   GradLayout G, const float* __restrict__ x,
                                                                   const float* __restrict__ w,
                                                                   const double* __restrict__ wsum, int64_t n,
                                                                   const unsigned char* __restrict__ img,
                                                                   float* __restrict__ gpart,
                                                                   float* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  constexpr int R = grad_rows(W), kLdR = grad_ldr(W);
  const int d = fa.d, zld = flow_zld(d);
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rows = (int)min((int64_t)R, n - r0);
  unsigned char* wsm = sm + G.wnat;
  copy16(wsm, img, fa.smem_weights);  // the staged weights, built once for all CTAs (flow_image_kernel)
  float* zs = at<float>(sm, G.zs);
  float* gz = at<float>(sm, G.gz);
  float* wn = at<float>(sm, G.wn);
  // weights that are not finite count as 0; with no positive weight every gradient is 0
  const double ws = *wsum;
  const float inv = (ws > 0.0 && ws < INFINITY) ? (float)(1.0 / ws) : 0.0f;
  for (int i = tid; i < R * d; i += blockDim.x) {
    const int r = i / d, k = i - r * d;
    zs[r * zld + k] = flow_logit(r < rows ? x[(r0 + r) * d + k] : 0.5f);
  }
  for (int r = tid; r < R; r += blockDim.x) {
    const float wr = r < rows ? w[r0 + r] : 0.0f;
    wn[r] = (isfinite(wr) && wr > 0.0f) ? wr * inv : 0.0f;
  }
  __syncthreads();
  // ---- forward (normalising): keep z before every layer ----
  float lsum0 = 0.0f, lsum1 = 0.0f;  // sum s of this lane's pairs, rows g and g+8 of its warp
  for (int l = 0; l < kFlowLayers; ++l) {
    float* zi = zs + l * R * zld;
    float* zo = zs + (l + 1) * R * zld;
    for (int i = tid; i < R * zld; i += blockDim.x) zo[i] = zi[i];
    __syncthreads();
    float a0 = 0.0f, a1 = 0.0f;
    if (d <= 16) flow_layer<2>(fa.lay[l], l, wsm, zo + warp * 16 * zld, zld, 1, a0, a1);
    else flow_layer<4>(fa.lay[l], l, wsm, zo + warp * 16 * zld, zld, 1, a0, a1);
    lsum0 += a0;
    lsum1 += a1;
    __syncthreads();
  }
  // ---- loss: - sum wn logdet; initial gradient from the output wrap ----
  {
    float part = 0.0f;
    const float* zf = zs + kFlowLayers * R * zld;
    const float* z0 = zs;
    // coupling part: lane (g, t) holds the pairs of rows warp*16+g and +8
    float c0 = lsum0, c1 = lsum1;
    c0 += __shfl_xor_sync(0xffffffffu, c0, 1);
    c0 += __shfl_xor_sync(0xffffffffu, c0, 2);
    c1 += __shfl_xor_sync(0xffffffffu, c1, 1);
    c1 += __shfl_xor_sync(0xffffffffu, c1, 2);
    if (t == 0) part -= wn[warp * 16 + g] * c0 + wn[warp * 16 + g + 8] * c1;
    if (lane < 16) {
      const int r = warp * 16 + lane;
      float wraps = 0.0f;
      for (int k = 0; k < d; ++k) wraps += flow_log_sig_prime(zf[r * zld + k]) - flow_log_sig_prime(z0[r * zld + k]);
      part -= wn[r] * wraps;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    float* red = at<float>(sm, G.red);
    if (lane == 0) red[warp] = part;
    for (int i = tid; i < R * zld; i += blockDim.x) {
      const int r = i / zld, k = i - r * zld;
      gz[i] = k < d ? -wn[r] * (1.0f - 2.0f * flow_sigmoid(zf[i])) : 0.0f;
    }
    __syncthreads();
    if (tid == 0) {
      float s = 0.0f;
      for (int k = 0; k < W; ++k) s += red[k];
      lpart[blockIdx.x] = s;
    }
  }
  float* gp = gpart + (size_t)blockIdx.x * fa.nparams;
  // ---- backward, last layer first ----
  for (int l = kFlowLayers - 1; l >= 0; --l) {
    const FlowLayer& L = fa.lay[l];
    const int par = l & 1;
    const float* zi = zs + l * R * zld;  // z before layer l
    __nv_bfloat16* H = at<__nv_bfloat16>(sm, G.H);
    __nv_bfloat16* HT = at<__nv_bfloat16>(sm, G.HT);
    __nv_bfloat16* U1 = at<__nv_bfloat16>(sm, G.U1);
    __nv_bfloat16* U1T = at<__nv_bfloat16>(sm, G.U1T);
    __nv_bfloat16* U2 = at<__nv_bfloat16>(sm, G.U2);
    __nv_bfloat16* U2T = at<__nv_bfloat16>(sm, G.U2T);
    __nv_bfloat16* GO = at<__nv_bfloat16>(sm, G.GO);
    __nv_bfloat16* GOT = at<__nv_bfloat16>(sm, G.GOT);
    __nv_bfloat16* W1T = at<__nv_bfloat16>(sm, G.w1t);
    __nv_bfloat16* W2T = at<__nv_bfloat16>(sm, G.w2t);
    __nv_bfloat16* W3T = at<__nv_bfloat16>(sm, G.w3t);
    float* gb = at<float>(sm, G.bias);  // [0,64) b1, [64,128) b2, [128,160) b3
    const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(wsm + L.sW1);
    const __nv_bfloat16* W2 = reinterpret_cast<const __nv_bfloat16*>(wsm + L.sW2);
    const __nv_bfloat16* W3 = reinterpret_cast<const __nv_bfloat16*>(wsm + L.sW3);
    const float* b1 = reinterpret_cast<const float*>(wsm + L.sb1);
    const float* b2 = reinterpret_cast<const float*>(wsm + L.sb2);
    const float* b3 = reinterpret_cast<const float*>(wsm + L.sb3);
    const int kpad = G.ldo - 8;
    // transposed weights of this layer (from the image); H and its transpose; zero the padding of GO / GOT
    copy16(sm + G.w1t, img + G.img_t + (size_t)l * G.img_tsz, G.img_tsz);
    for (int i = tid; i < R * 16; i += blockDim.x) {
      const int r = i / 16, c = i - r * 16;
      const __nv_bfloat16 v = __float2bfloat16_rn(c < L.a ? zi[r * zld + 2 * c + par] : 0.0f);
      H[r * kLdK16 + c] = v;
      HT[c * kLdR + r] = v;
    }
    for (int i = tid; i < R * kpad; i += blockDim.x) {
      const int r = i / kpad, o = i - r * kpad;
      GO[r * G.ldo + o] = __float2bfloat16_rn(0.0f);
      if (o < 32) GOT[o * kLdR + r] = __float2bfloat16_rn(0.0f);
    }
    for (int i = tid; i < 160; i += blockDim.x) gb[i] = 0.0f;
    __syncthreads();
    // recompute the conditioner on the warp's rows: U1, U2 (and transposes), o
    float o[4][4];
    {
      const int m0 = warp * 16;
      uint32_t ha[4];
      load_a(H, kLdK16, m0, 0, ha);
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float2 bb = *reinterpret_cast<const float2*>(b1 + nt * 8 + 2 * t);
        acc[nt][0] = bb.x; acc[nt][1] = bb.y; acc[nt][2] = bb.x; acc[nt][3] = bb.y;
        uint32_t b0, bq;
        load_b(W1, kLdK16, nt * 8, 0, b0, bq);
        mma16816(acc[nt], ha[0], ha[1], ha[2], ha[3], b0, bq);
      }
      uint32_t ua[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float v0 = fmaxf(acc[nt][0], 0.0f), v1 = fmaxf(acc[nt][1], 0.0f);
        const float v2 = fmaxf(acc[nt][2], 0.0f), v3 = fmaxf(acc[nt][3], 0.0f);
        st_bf16(U1 + (m0 + g) * kLdK64 + col, v0); st_bf16(U1 + (m0 + g) * kLdK64 + col + 1, v1);
        st_bf16(U1 + (m0 + g + 8) * kLdK64 + col, v2); st_bf16(U1 + (m0 + g + 8) * kLdK64 + col + 1, v3);
        st_bf16(U1T + col * kLdR + m0 + g, v0); st_bf16(U1T + (col + 1) * kLdR + m0 + g, v1);
        st_bf16(U1T + col * kLdR + m0 + g + 8, v2); st_bf16(U1T + (col + 1) * kLdR + m0 + g + 8, v3);
        const int ks = nt >> 1, hi = nt & 1;
        ua[ks][hi * 2 + 0] = pack_bf16(v0, v1);
        ua[ks][hi * 2 + 1] = pack_bf16(v2, v3);
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float2 bb = *reinterpret_cast<const float2*>(b2 + nt * 8 + 2 * t);
        acc[nt][0] = bb.x; acc[nt][1] = bb.y; acc[nt][2] = bb.x; acc[nt][3] = bb.y;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          uint32_t b0, bq;
          load_b(W2, kLdK64, nt * 8, ks * 16, b0, bq);
          mma16816(acc[nt], ua[ks][0], ua[ks][1], ua[ks][2], ua[ks][3], b0, bq);
        }
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float v0 = fmaxf(acc[nt][0], 0.0f), v1 = fmaxf(acc[nt][1], 0.0f);
        const float v2 = fmaxf(acc[nt][2], 0.0f), v3 = fmaxf(acc[nt][3], 0.0f);
        st_bf16(U2 + (m0 + g) * kLdK64 + col, v0); st_bf16(U2 + (m0 + g) * kLdK64 + col + 1, v1);
        st_bf16(U2 + (m0 + g + 8) * kLdK64 + col, v2); st_bf16(U2 + (m0 + g + 8) * kLdK64 + col + 1, v3);
        st_bf16(U2T + col * kLdR + m0 + g, v0); st_bf16(U2T + (col + 1) * kLdR + m0 + g, v1);
        st_bf16(U2T + col * kLdR + m0 + g + 8, v2); st_bf16(U2T + (col + 1) * kLdR + m0 + g + 8, v3);
        const int ks = nt >> 1, hi = nt & 1;
        ua[ks][hi * 2 + 0] = pack_bf16(v0, v1);
        ua[ks][hi * 2 + 1] = pack_bf16(v2, v3);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        if (nt * 8 < L.no) {
          const float2 bb = *reinterpret_cast<const float2*>(b3 + nt * 8 + 2 * t);
          o[nt][0] = bb.x; o[nt][1] = bb.y; o[nt][2] = bb.x; o[nt][3] = bb.y;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            uint32_t b0, bq;
            load_b(W3, kLdK64, nt * 8, ks * 16, b0, bq);
            mma16816(o[nt], ua[ks][0], ua[ks][1], ua[ks][2], ua[ks][3], b0, bq);
          }
        }
      }
      // GO from (s, t) and the incoming gradient; gz of the moved axes
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int m = 4 * nt + t;
        float gs0 = 0.0f, gt0 = 0.0f, gs1 = 0.0f, gt1 = 0.0f;
        if (nt * 8 < L.no && m < L.b) {
          const int k = 2 * m + 1 - par;
          const int ra = m0 + g, rb = m0 + g + 8;
          const float s0 = flow_soft_clamp(o[nt][0]);
          const float s1 = flow_soft_clamp(o[nt][2]);
          const float e0 = __expf(s0), e1 = __expf(s1);
          const float gza = gz[ra * zld + k], gzb = gz[rb * zld + k];
          const float dsa = -wn[ra] + gza * zi[ra * zld + k] * e0;
          const float dsb = -wn[rb] + gzb * zi[rb * zld + k] * e1;
          gs0 = dsa * (1.0f - (s0 / kFlowSClamp) * (s0 / kFlowSClamp));
          gs1 = dsb * (1.0f - (s1 / kFlowSClamp) * (s1 / kFlowSClamp));
          gt0 = gza;
          gt1 = gzb;
          gz[ra * zld + k] = gza * e0;
          gz[rb * zld + k] = gzb * e1;
          st_bf16(GO + ra * G.ldo + 2 * m, gs0); st_bf16(GO + ra * G.ldo + 2 * m + 1, gt0);
          st_bf16(GO + rb * G.ldo + 2 * m, gs1); st_bf16(GO + rb * G.ldo + 2 * m + 1, gt1);
          st_bf16(GOT + (2 * m) * kLdR + ra, gs0); st_bf16(GOT + (2 * m + 1) * kLdR + ra, gt0);
          st_bf16(GOT + (2 * m) * kLdR + rb, gs1); st_bf16(GOT + (2 * m + 1) * kLdR + rb, gt1);
        }
        // bias gradient of b3: sum over the rows of the warp
        const float sb = sum_over_g(gs0 + gs1), tb = sum_over_g(gt0 + gt1);
        if (g == 0 && nt * 8 < L.no && m < L.b) {
          atomicAdd(gb + 128 + 2 * m, sb);
          atomicAdd(gb + 128 + 2 * m + 1, tb);
        }
      }
    }
    __syncthreads();
    // dW3 = GO^T U2: [no x R] [R x 64]
    cta_gemm<W>(GOT, kLdR, U2T, kLdR, (L.no + 15) / 16 * 16, 64, R, [&](int r, int c, float v0, float v1) {
      if (r < 2 * L.b) {
        gp[L.oW3 + r * 64 + c] = v0;
        gp[L.oW3 + r * 64 + c + 1] = v1;
      }
    });
    __syncthreads();
    // gU2 = GO W3: [R x kpad] [kpad x 64] (the warp's own rows); GA2 = gU2 * (U2 > 0) into U2 / U2T
    cta_gemm<W>(GO, G.ldo, W3T, G.ldo, R, 64, kpad, [&](int r, int c, float v0, float v1) {
      const float m0v = __bfloat162float(U2[r * kLdK64 + c]) > 0.0f ? v0 : 0.0f;
      const float m1v = __bfloat162float(U2[r * kLdK64 + c + 1]) > 0.0f ? v1 : 0.0f;
      st_bf16(U2 + r * kLdK64 + c, m0v); st_bf16(U2 + r * kLdK64 + c + 1, m1v);
      st_bf16(U2T + c * kLdR + r, m0v); st_bf16(U2T + (c + 1) * kLdR + r, m1v);
      atomicAdd(gb + 64 + c, m0v);
      atomicAdd(gb + 64 + c + 1, m1v);
    });
    __syncthreads();
    // dW2 = GA2^T U1: [64 x R] [R x 64]
    cta_gemm<W>(U2T, kLdR, U1T, kLdR, 64, 64, R, [&](int r, int c, float v0, float v1) {
      gp[L.oW2 + r * 64 + c] = v0;
      gp[L.oW2 + r * 64 + c + 1] = v1;
    });
    __syncthreads();
    // gU1 = GA2 W2: [R x 64] [64 x 64]; GA1 = gU1 * (U1 > 0) into U1 / U1T
    cta_gemm<W>(U2, kLdK64, W2T, kLdK64, R, 64, 64, [&](int r, int c, float v0, float v1) {
      const float m0v = __bfloat162float(U1[r * kLdK64 + c]) > 0.0f ? v0 : 0.0f;
      const float m1v = __bfloat162float(U1[r * kLdK64 + c + 1]) > 0.0f ? v1 : 0.0f;
      st_bf16(U1 + r * kLdK64 + c, m0v); st_bf16(U1 + r * kLdK64 + c + 1, m1v);
      st_bf16(U1T + c * kLdR + r, m0v); st_bf16(U1T + (c + 1) * kLdR + r, m1v);
      atomicAdd(gb + c, m0v);
      atomicAdd(gb + c + 1, m1v);
    });
    __syncthreads();
    // dW1 = GA1^T H: [64 x R] [R x 16]
    cta_gemm<W>(U1T, kLdR, HT, kLdR, 64, 16, R, [&](int r, int c, float v0, float v1) {
      if (c < L.a) gp[L.oW1 + r * L.a + c] = v0;
      if (c + 1 < L.a) gp[L.oW1 + r * L.a + c + 1] = v1;
    });
    // gH = GA1 W1: [R x 64] [64 x 16]; the conditioning axes take it
    cta_gemm<W>(U1, kLdK64, W1T, kLdK64, R, 16, 64, [&](int r, int c, float v0, float v1) {
      if (c < L.a) gz[r * zld + 2 * c + par] += v0;
      if (c + 1 < L.a) gz[r * zld + 2 * (c + 1) + par] += v1;
    });
    __syncthreads();
    for (int i = tid; i < 64; i += blockDim.x) {
      gp[L.ob1 + i] = gb[i];
      gp[L.ob2 + i] = gb[64 + i];
    }
    for (int i = tid; i < 2 * L.b; i += blockDim.x) gp[L.ob3 + i] = gb[128 + i];
    __syncthreads();
  }
}

// sum of the weights, one CTA, fixed order
__global__ void flow_wsum_kernel(const float* __restrict__ w, int64_t n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float wi = w[i];
    if (isfinite(wi) && wi > 0.0f) s += (double)wi;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    *out = t;
  }
}

// grad[p] = sum over CTAs of the partials, in CTA order; loss likewise
__global__ void flow_reduce_kernel(const float* __restrict__ gpart, const float* __restrict__ lpart, int nblk,
                                   int np, float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += gpart[(size_t)b * np + p];
    grad[p] = s;
  }
  if (p == 0 && loss) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += lpart[b];
    *loss = s;
  }
}

__global__ void flow_adam_kernel(int64_t np, float* __restrict__ theta, const float* __restrict__ grad,
                                 float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                                 float eps, float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct GradScratch {
  size_t wsum, lpart, gpart, img, img_tc, total;
  int nblk;
};
GradScratch grad_scratch(const FlowArgs& fa, int64_t n) {
  GradScratch S{};
  const int W = grad_warps(fa.d);
  const int R = grad_rows(W);
  S.nblk = (int)((n + R - 1) / R);
  size_t o = 0;
  S.wsum = o; o = al16(o + sizeof(double));
  S.lpart = o; o = al16(o + sizeof(float) * S.nblk);
  S.gpart = o; o = al16(o + sizeof(float) * (size_t)S.nblk * fa.nparams);
  S.img = o; o = al16(o + (size_t)grad_layout(fa, W).img_total);
  S.img_tc = o; o = al16(o + flow_grad_tc_image_bytes(fa.d));
  S.total = o;
  return S;
}

}  // namespace
}  // namespace vg

extern "C" size_t vegas_flow_grad_scratch_bytes(int32_t dim, int64_t n) {
  FlowArgs fa{};
  if (flow_layout(dim, fa) != VEGAS_OK || n < 1) return 0;
  return grad_scratch(fa, n).total;
}

extern "C" int vegas_flow_grad(int32_t dim, const float* d_params, const float* d_x, const float* d_w, int64_t n,
                               float* d_grad, float* d_loss, void* d_scratch, size_t scratch_bytes, void* stream) {
  FlowArgs fa{};
  if (flow_layout(dim, fa) != VEGAS_OK || n < 1 || n > (int64_t(1) << 31) || !d_params || !d_x || !d_w || !d_grad ||
      !d_scratch)
    return VEGAS_EINVAL;
  fa.params = d_params;
  const GradScratch S = grad_scratch(fa, n);
  if (scratch_bytes < S.total) return VEGAS_ENOSPACE;
  const int W = grad_warps(dim);
  const GradLayout G = grad_layout(fa, W);
  if (G.total > 227 * 1024) return VEGAS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* sc = (unsigned char*)d_scratch;
  double* wsum = (double*)(sc + S.wsum);
  float* lpart = (float*)(sc + S.lpart);
  float* gpart = (float*)(sc + S.gpart);
  unsigned char* img = sc + S.img;
  flow_wsum_kernel<<<1, 1024, 0, s>>>(d_w, n, wsum);
  VG_CHECK(cudaGetLastError());
  if (dim <= kFlowGradTcMaxDim) {  // tcgen05: one CTA per 128 samples
    const int rc = flow_grad_tc(fa, sc + S.img_tc, d_x, d_w, wsum, n, gpart, lpart, s);
    if (rc != VEGAS_OK) return rc;
    const int nblk = (int)((n + 127) / 128);
    flow_reduce_kernel<<<(fa.nparams + 255) / 256, 256, 0, s>>>(gpart, lpart, nblk, fa.nparams, d_grad, d_loss);
    return cuda_status(cudaGetLastError());
  }
  flow_image_kernel<<<dim3(4, kFlowLayers), 256, 0, s>>>(fa, G, img);
  VG_CHECK(cudaGetLastError());
  static_assert(grad_rows(2) == 32, "two-warp CTAs");
  VG_CHECK(cudaFuncSetAttribute(flow_grad_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, G.total));
  flow_grad_kernel<2><<<S.nblk, 2 * 32, G.total, s>>>(fa, G, d_x, d_w, wsum, n, img, gpart, lpart);
  VG_CHECK(cudaGetLastError());
  flow_reduce_kernel<<<(fa.nparams + 255) / 256, 256, 0, s>>>(gpart, lpart, S.nblk, fa.nparams, d_grad, d_loss);
  return cuda_status(cudaGetLastError());
}

extern "C" int vegas_flow_adam(int64_t nparams, float* d_params, const float* d_grad, float* d_m, float* d_v,
                               int32_t step, float lr, float beta1, float beta2, float eps, void* stream) {
  if (nparams < 1 || !d_params || !d_grad || !d_m || !d_v || step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f) ||
      !(beta1 < 1.0f) || !(beta2 >= 0.0f) || !(beta2 < 1.0f) || !(eps >= 0.0f))
    return VEGAS_EINVAL;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  flow_adam_kernel<<<(unsigned)((nparams + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      nparams, d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps, c1, c2);
  return cuda_status(cudaGetLastError());
}

// ===========================================================================
// The integrand at the flow's points: values[j] = f(x_j) |det dF/dx'| with
// the log-determinant of the sampling direction; the fill then integrates
// these tabulated values over the VEGAS+ map (kIntegrandTabulated).
// ===========================================================================
#include "vegas_fill.cuh"

namespace vg {
namespace {

template <int ID, int DMAX>
__global__ void __launch_bounds__(256) flow_eval_kernel(const float* __restrict__ X, const float* __restrict__ logdet,
                                                        float* __restrict__ values, int64_t n, int d,
                                                        const double* __restrict__ raw, int np_raw, int np_derived) {
  extern __shared__ __align__(16) unsigned char esm[];
  float* prm = reinterpret_cast<float*>(esm);
  prep_params<ID, float, DMAX>(raw, np_raw, d, prm);
  __syncthreads();
  const float s0 = prm[0], s1 = prm[1];
  const int K = ID == VEGAS_GAUSS_SUM ? (int)prm[2] : 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    float x[DMAX];
    if ((d & 3) == 0) {  // 16-byte aligned rows: four coordinates a load
#pragma unroll
      for (int k = 0; k < DMAX; k += 4) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (k < d) v = *reinterpret_cast<const float4*>(X + j * d + k);
        x[k] = v.x;
        x[k + 1] = v.y;
        x[k + 2] = v.z;
        x[k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < DMAX; ++k) x[k] = k < d ? X[j * d + k] : 0.0f;
    }
    const float f = integrand<ID, float, DMAX>(x, d, prm, np_derived, s0, s1, K);
    values[j] = f * __expf(logdet[j]);
  }
}

template <int ID, int DMAX>
int launch_eval(const float* X, const float* logdet, float* values, int64_t n, int d, const double* raw, int np_raw,
                int np_derived, cudaStream_t s) {
  const int nprm = std::max(4, derived_smem_count(ID, d, DMAX, np_raw));
  const size_t smem = sizeof(float) * (size_t)nprm;
  auto k = flow_eval_kernel<ID, DMAX>;
  if (smem > 48 * 1024) VG_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * std::max(1, num_sms_flow())));
  k<<<grid, 256, smem, s>>>(X, logdet, values, n, d, raw, np_raw, np_derived);
  return cuda_status(cudaGetLastError());
}

template <int DMAX>
int eval_id(int integrand, const float* X, const float* logdet, float* values, int64_t n, int d, const double* raw,
            int np_raw, int np_derived, cudaStream_t s) {
  switch (integrand) {
#define VG_EVAL(ID) \
  case ID: return launch_eval<ID, DMAX>(X, logdet, values, n, d, raw, np_raw, np_derived, s);
    VG_EVAL(VEGAS_GAUSS_SUM)
    VG_EVAL(VEGAS_PRODUCT_PEAK)
    VG_EVAL(VEGAS_OSCILLATORY)
    VG_EVAL(VEGAS_SIN_EXP)
    VG_EVAL(VEGAS_LINEAR)
    VG_EVAL(VEGAS_COSINE)
    VG_EVAL(VEGAS_EXPONENTIAL)
    VG_EVAL(VEGAS_ROOS_ARNOLD)
    VG_EVAL(VEGAS_MOROKOFF_CAFLISCH)
#undef VG_EVAL
    default: return VEGAS_EINVAL;
  }
}

}  // namespace

int flow_eval(int integrand, int d, const double* d_params, int64_t nparams, const float* X, const float* logdet,
              float* values, int64_t n, cudaStream_t s) {
  const int npd = derived_param_count(integrand, d, nullptr, nparams);
  if (npd < 0) return VEGAS_EINVAL;
  const int dm = dmax_for(d);
  if (dm == 4) return eval_id<4>(integrand, X, logdet, values, n, d, d_params, (int)nparams, npd, s);
  if (dm == 8) return eval_id<8>(integrand, X, logdet, values, n, d, d_params, (int)nparams, npd, s);
  if (dm == 16) return eval_id<16>(integrand, X, logdet, values, n, d, d_params, (int)nparams, npd, s);
  return eval_id<32>(integrand, X, logdet, values, n, d, d_params, (int)nparams, npd, s);
}

// training rows: xs[i] = X[i * stride]
// The training set of one iteration: rows r = 0 .. rows-1 in a period of P.
// Row r with r mod P < P-1 is sample i = (r / P)(P-1) + r mod P, the point of
// evaluation i * stride and its weight w_i (zero weight past the last sample);
// with a floor lambda > 0 row r with r mod P = P-1 is uniform point u = r / P,
// a Philox4x32-10 draw keyed by (seed, iteration), with weight
// lambda (P-1) mean(w).  Every window of consecutive rows then carries floor
// weight lambda times its data weight, on average, spread over the whole cube.
__global__ void flow_gather_kernel(const float* __restrict__ X, int d, int64_t stride, int64_t m,
                                   const float* __restrict__ w, const double* __restrict__ wsum, float lambda, int P,
                                   uint32_t k0, uint32_t k1, int64_t rows, float* __restrict__ xs,
                                   float* __restrict__ ws) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t q = r / P, ph = r - q * P;
  if (lambda > 0.0f && ph == P - 1) {
    const double wbar = m > 0 ? *wsum / (double)m : 0.0;
    ws[r] = (float)((double)lambda * (double)(P - 1) * wbar);
    for (int k0c = 0; k0c < d; k0c += 4) {
      const uint4 b = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)k0c, 0x464C4F57u), k0, k1);
      const uint32_t u[4] = {b.x, b.y, b.z, b.w};
      for (int t = 0; t < 4 && k0c + t < d; ++t)
        xs[r * d + k0c + t] = ((float)(u[t] >> 8) + 0.5f) * 0x1p-24f;  // in (0, 1)
    }
    return;
  }
  const int64_t i = lambda > 0.0f ? q * (P - 1) + ph : r;
  if (i < m) {
    ws[r] = w[i];
    for (int k = 0; k < d; ++k) xs[r * d + k] = X[i * stride * d + k];
  } else {
    ws[r] = 0.0f;
    for (int k = 0; k < d; ++k) xs[r * d + k] = 0.5f;
  }
}

int64_t flow_train_rows(int64_t m, float lambda) {
  if (!(lambda > 0.0f)) return m;
  return (m + kFloorPeriod - 2) / (kFloorPeriod - 1) * kFloorPeriod;
}

int flow_gather(const float* X, int d, int64_t stride, int64_t m, const float* w, float lambda, uint64_t seed,
                uint32_t iter, double* wsum, float* xs, float* ws, cudaStream_t s) {
  const int64_t rows = flow_train_rows(m, lambda);
  if (lambda > 0.0f) {
    flow_wsum_kernel<<<1, 1024, 0, s>>>(w, m, wsum);
    VG_CHECK(cudaGetLastError());
  }
  const uint32_t k0 = (uint32_t)seed ^ 0x3C6EF372u, k1 = (uint32_t)(seed >> 32) ^ iter;
  flow_gather_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(X, d, stride, m, w, wsum, lambda, kFloorPeriod,
                                                                    k0, k1, rows, xs, ws);
  return cuda_status(cudaGetLastError());
}

}  // namespace vg
