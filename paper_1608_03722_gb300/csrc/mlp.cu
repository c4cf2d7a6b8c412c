// mlp.cu -- BF16 tensor-core MLP surrogate 4 -> 64 -> 64 -> 3 (GELU) of the
// sweep observables (mean extension / contour length, excess twist,
// denatured fraction) as a function of (force, torque, length, kT).
//
// Weights are kept as FP32 masters and BF16 copies; every contraction runs on
// the tensor cores (warp-level mma.sync m16n8k16, BF16 operands, FP32
// accumulation), one warp per 16-row tile of the batch.  Small dimensions (4
// inputs, 3 outputs) are zero-padded to the MMA shape.  The forward pass keeps
// the pre-activations for the backward pass; the backward pass forms the mean
// squared error on normalised targets and accumulates the weight gradients in
// FP32; Adam updates the masters and refreshes the BF16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dsdna.h"

namespace {

constexpr int NI = 4, NH = 64, NO = 3;
// parameter layout (FP32 and BF16 copies): W1[NH][NI] b1[NH] W2[NH][NH] b2[NH] W3[NO][NH] b3[NO]
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NO * NH;
constexpr int NP = OB3 + NO;
constexpr int TILE = 16;       // batch rows per warp
constexpr int WARPS = 2;

struct Norm {
  float in_mean[NI], in_scale[NI], out_mean[NO], out_scale[NO];
};

__device__ __forceinline__ unsigned pack2(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}

// D(16x8) += A(16x16, row) * B(16x8, col); BF16 operands, FP32 accumulate
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragments of the m16n8k16 shape, lane = 4 g + t:
//   A: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
//   B: (k = 2t..2t+1, n = g), (k = 2t+8.., n = g)
//   D: (g, 2t..2t+1), (g+8, 2t..2t+1)
template <class FA>
__device__ __forceinline__ void frag_a(unsigned* a, FA A, int r0, int c0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  a[0] = pack2(A(r0 + g, c0 + 2 * t), A(r0 + g, c0 + 2 * t + 1));
  a[1] = pack2(A(r0 + g + 8, c0 + 2 * t), A(r0 + g + 8, c0 + 2 * t + 1));
  a[2] = pack2(A(r0 + g, c0 + 2 * t + 8), A(r0 + g, c0 + 2 * t + 9));
  a[3] = pack2(A(r0 + g + 8, c0 + 2 * t + 8), A(r0 + g + 8, c0 + 2 * t + 9));
}
template <class FB>
__device__ __forceinline__ void frag_b(unsigned* b, FB B, int k0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  b[0] = pack2(B(k0 + 2 * t, n0 + g), B(k0 + 2 * t + 1, n0 + g));
  b[1] = pack2(B(k0 + 2 * t + 8, n0 + g), B(k0 + 2 * t + 9, n0 + g));
}
template <class FS>
__device__ __forceinline__ void frag_d_store(const float* d, FS S, int r0, int c0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  S(r0 + g, c0 + 2 * t, d[0]);
  S(r0 + g, c0 + 2 * t + 1, d[1]);
  S(r0 + g + 8, c0 + 2 * t, d[2]);
  S(r0 + g + 8, c0 + 2 * t + 1, d[3]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct MlpDev {
  float* P;             // FP32 masters [NP]
  __nv_bfloat16* Pb;    // BF16 copies [NP]
  float* G;             // gradients [NP]
  float* M;             // Adam first moment [NP]
  float* V;             // Adam second moment [NP]
  float* Xn;            // cached normalised inputs [max_batch][NI]
  float* Z1;            // cached pre-activations [max_batch][NH]
  float* Z2;            // [max_batch][NH]
  float* Yn;            // normalised outputs [max_batch][NO]
  float* loss;          // [1]
  Norm norm;
};

// per-warp shared staging: activations of one 16-row tile
struct WarpSmem {
  float x[TILE][NI];
  float h1[TILE][NH];
  float h2[TILE][NH];
  float t[TILE][NH];   // scratch: gradients of the current layer
};

__global__ void k_mlp_forward(MlpDev m, const float* X, int B, float* Y) {
  __shared__ __nv_bfloat16 w[NP];
  __shared__ WarpSmem ws[WARPS];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = m.Pb[i];
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& s = ws[wid];
  const int r0 = (blockIdx.x * WARPS + wid) * TILE;
  if (r0 >= B) return;
  for (int i = lane; i < TILE * NI; i += 32) {
    const int r = i / NI, c = i % NI;
    const float v = (r0 + r < B) ? (X[(size_t)(r0 + r) * NI + c] - m.norm.in_mean[c]) / m.norm.in_scale[c] : 0.0f;
    s.x[r][c] = v;
    if (r0 + r < B) m.Xn[(size_t)(r0 + r) * NI + c] = v;
  }
  __syncwarp();
  // layer 1: Z1 = Xn W1^T + b1 (K = 4 padded to 16)
  for (int n0 = 0; n0 < NH; n0 += 8) {
    unsigned a[4], b[2];
    float d[4] = {0, 0, 0, 0};
    frag_a(a, [&](int r, int c) { return c < NI ? s.x[r][c] : 0.0f; }, 0, 0);
    frag_b(b, [&](int k, int n) { return k < NI ? __bfloat162float(w[OW1 + n * NI + k]) : 0.0f; }, 0, n0);
    mma16816(d, a, b);
    frag_d_store(d, [&](int r, int c, float v) {
      v += m.P[OB1 + c];
      if (r0 + r < B) m.Z1[(size_t)(r0 + r) * NH + c] = v;
      s.h1[r][c] = gelu(v);
    }, 0, n0);
  }
  __syncwarp();
  // layer 2: Z2 = H1 W2^T + b2
  for (int n0 = 0; n0 < NH; n0 += 8) {
    float d[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < NH; k0 += 16) {
      unsigned a[4], b[2];
      frag_a(a, [&](int r, int c) { return s.h1[r][c]; }, 0, k0);
      frag_b(b, [&](int k, int n) { return __bfloat162float(w[OW2 + n * NH + k]); }, k0, n0);
      mma16816(d, a, b);
    }
    frag_d_store(d, [&](int r, int c, float v) {
      v += m.P[OB2 + c];
      if (r0 + r < B) m.Z2[(size_t)(r0 + r) * NH + c] = v;
      s.h2[r][c] = gelu(v);
    }, 0, n0);
  }
  __syncwarp();
  // layer 3: Y = H2 W3^T + b3 (N = 3 padded to 8)
  float d[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < NH; k0 += 16) {
    unsigned a[4], b[2];
    frag_a(a, [&](int r, int c) { return s.h2[r][c]; }, 0, k0);
    frag_b(b, [&](int k, int n) { return n < NO ? __bfloat162float(w[OW3 + n * NH + k]) : 0.0f; }, k0, 0);
    mma16816(d, a, b);
  }
  frag_d_store(d, [&](int r, int c, float v) {
    if (c < NO && r0 + r < B) {
      v += m.P[OB3 + c];
      m.Yn[(size_t)(r0 + r) * NO + c] = v;
      Y[(size_t)(r0 + r) * NO + c] = m.norm.out_mean[c] + m.norm.out_scale[c] * v;
    }
  }, 0, 0);
}

// Mean squared error over B x 3 normalised outputs and its gradient.
__global__ void k_mlp_backward(MlpDev m, const float* T, int B) {
  __shared__ __nv_bfloat16 w[NP];
  __shared__ WarpSmem ws[WARPS];
  __shared__ float dy[WARPS][TILE][8];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = m.Pb[i];
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& s = ws[wid];
  const int r0 = (blockIdx.x * WARPS + wid) * TILE;
  if (r0 >= B) return;
  const float inv = 1.0f / (float)(B * NO);
  float lsum = 0.0f;
  for (int i = lane; i < TILE * 8; i += 32) {
    const int r = i / 8, c = i % 8;
    float g = 0.0f;
    if (c < NO && r0 + r < B) {
      const float tn = (T[(size_t)(r0 + r) * NO + c] - m.norm.out_mean[c]) / m.norm.out_scale[c];
      const float e = m.Yn[(size_t)(r0 + r) * NO + c] - tn;
      lsum += e * e;
      g = 2.0f * e * inv;
    }
    dy[wid][r][c] = g;
  }
  for (int i = lane; i < TILE * NI; i += 32) {
    const int r = i / NI, c = i % NI;
    s.x[r][c] = (r0 + r < B) ? m.Xn[(size_t)(r0 + r) * NI + c] : 0.0f;
  }
  for (int i = lane; i < TILE * NH; i += 32) {
    const int r = i / NH, c = i % NH;
    const bool ok = r0 + r < B;
    s.h1[r][c] = ok ? gelu(m.Z1[(size_t)(r0 + r) * NH + c]) : 0.0f;
    s.h2[r][c] = ok ? gelu(m.Z2[(size_t)(r0 + r) * NH + c]) : 0.0f;
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) atomicAdd(m.loss, lsum * inv);
  __syncwarp();
  // dW3 = dY^T H2 (M = 3 padded to 16, K = batch tile), db3
  for (int n0 = 0; n0 < NH; n0 += 8) {
    unsigned a[4], b[2];
    float d[4] = {0, 0, 0, 0};
    frag_a(a, [&](int r, int c) { return r < NO ? dy[wid][c][r] : 0.0f; }, 0, 0);
    frag_b(b, [&](int k, int n) { return s.h2[k][n]; }, 0, n0);
    mma16816(d, a, b);
    frag_d_store(d, [&](int r, int c, float v) { if (r < NO) atomicAdd(&m.G[OW3 + r * NH + c], v); }, 0, n0);
  }
  if (lane < NO) {
    float sum = 0.0f;
    for (int r = 0; r < TILE; ++r) sum += dy[wid][r][lane];
    atomicAdd(&m.G[OB3 + lane], sum);
  }
  // dH2 = dY W3 (K = 3 padded to 16); dZ2 = dH2 * gelu'(Z2) -> s.t
  for (int n0 = 0; n0 < NH; n0 += 8) {
    unsigned a[4], b[2];
    float d[4] = {0, 0, 0, 0};
    frag_a(a, [&](int r, int c) { return c < NO ? dy[wid][r][c] : 0.0f; }, 0, 0);
    frag_b(b, [&](int k, int n) { return k < NO ? __bfloat162float(w[OW3 + k * NH + n]) : 0.0f; }, 0, n0);
    mma16816(d, a, b);
    frag_d_store(d, [&](int r, int c, float v) {
      s.t[r][c] = (r0 + r < B) ? v * gelu_d(m.Z2[(size_t)(r0 + r) * NH + c]) : 0.0f;
    }, 0, n0);
  }
  __syncwarp();
  // dW2 = dZ2^T H1, db2
  for (int m0 = 0; m0 < NH; m0 += 16)
    for (int n0 = 0; n0 < NH; n0 += 8) {
      unsigned a[4], b[2];
      float d[4] = {0, 0, 0, 0};
      frag_a(a, [&](int r, int c) { return s.t[c][r]; }, m0, 0);
      frag_b(b, [&](int k, int n) { return s.h1[k][n]; }, 0, n0);
      mma16816(d, a, b);
      frag_d_store(d, [&](int r, int c, float v) { atomicAdd(&m.G[OW2 + r * NH + c], v); }, m0, n0);
    }
  for (int c = lane; c < NH; c += 32) {
    float sum = 0.0f;
    for (int r = 0; r < TILE; ++r) sum += s.t[r][c];
    atomicAdd(&m.G[OB2 + c], sum);
  }
  // dH1 = dZ2 W2; dZ1 = dH1 * gelu'(Z1) -> s.h2 (H2 no longer needed)
  for (int n0 = 0; n0 < NH; n0 += 8) {
    float d[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < NH; k0 += 16) {
      unsigned a[4], b[2];
      frag_a(a, [&](int r, int c) { return s.t[r][c]; }, 0, k0);
      frag_b(b, [&](int k, int n) { return __bfloat162float(w[OW2 + k * NH + n]); }, k0, n0);
      mma16816(d, a, b);
    }
    frag_d_store(d, [&](int r, int c, float v) {
      s.h2[r][c] = (r0 + r < B) ? v * gelu_d(m.Z1[(size_t)(r0 + r) * NH + c]) : 0.0f;
    }, 0, n0);
  }
  __syncwarp();
  // dW1 = dZ1^T Xn (N = 4 padded to 8), db1
  for (int m0 = 0; m0 < NH; m0 += 16) {
    unsigned a[4], b[2];
    float d[4] = {0, 0, 0, 0};
    frag_a(a, [&](int r, int c) { return s.h2[c][r]; }, m0, 0);
    frag_b(b, [&](int k, int n) { return n < NI ? s.x[k][n] : 0.0f; }, 0, 0);
    mma16816(d, a, b);
    frag_d_store(d, [&](int r, int c, float v) { if (c < NI) atomicAdd(&m.G[OW1 + r * NI + c], v); }, m0, 0);
  }
  for (int c = lane; c < NH; c += 32) {
    float sum = 0.0f;
    for (int r = 0; r < TILE; ++r) sum += s.h2[r][c];
    atomicAdd(&m.G[OB1 + c], sum);
  }
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t) and decoupled
// weight decay wd on the weight matrices (not the biases):
// p <- p - lr (m_hat / (sqrt(v_hat) + eps) + wd p).
__global__ void k_mlp_adam(MlpDev m, float lr, float b1, float b2, float eps, float c1, float c2, float wd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float g = m.G[i];
  const float mm = b1 * m.M[i] + (1.0f - b1) * g;
  const float vv = b2 * m.V[i] + (1.0f - b2) * g * g;
  m.M[i] = mm;
  m.V[i] = vv;
  const bool weight = i < OB1 || (i >= OW2 && i < OB2) || (i >= OW3 && i < OB3);
  const float p0 = m.P[i];
  const float p = p0 - lr * ((mm / c1) / (sqrtf(vv / c2) + eps) + (weight ? wd * p0 : 0.0f));
  m.P[i] = p;
  m.Pb[i] = __float2bfloat16_rn(p);
}

__global__ void k_mlp_refresh_bf16(MlpDev m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NP) m.Pb[i] = __float2bfloat16_rn(m.P[i]);
}

}  // namespace

struct dsdna_mlp {
  MlpDev d{};
  int max_batch = 0;
  cudaStream_t st = nullptr;
  dsdna_allocator alloc{};
  bool have_alloc = false;
  std::vector<void*> bufs;
  int64_t adam_t = 0;
};

static void* mlp_alloc(dsdna_mlp* m, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (m->have_alloc) p = m->alloc.alloc(bytes, m->alloc.user);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (p) m->bufs.push_back(p);
  return p;
}

extern "C" void dsdna_mlp_destroy(dsdna_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->st);
  for (void* p : m->bufs) {
    if (m->have_alloc) m->alloc.release(p, m->alloc.user);
    else cudaFree(p);
  }
  delete m;
}

extern "C" int dsdna_mlp_create(int max_batch, const dsdna_allocator* alloc, void* cuda_stream, dsdna_mlp** out) {
  if (!out || max_batch < 1) return DSDNA_EINVAL;
  *out = nullptr;
  dsdna_mlp* m = new dsdna_mlp();
  m->max_batch = ((max_batch + TILE - 1) / TILE) * TILE;
  m->st = (cudaStream_t)cuda_stream;
  if (alloc && alloc->alloc && alloc->release) { m->alloc = *alloc; m->have_alloc = true; }
  MlpDev& d = m->d;
  d.P = (float*)mlp_alloc(m, sizeof(float) * NP);
  d.Pb = (__nv_bfloat16*)mlp_alloc(m, sizeof(__nv_bfloat16) * NP);
  d.G = (float*)mlp_alloc(m, sizeof(float) * NP);
  d.M = (float*)mlp_alloc(m, sizeof(float) * NP);
  d.V = (float*)mlp_alloc(m, sizeof(float) * NP);
  d.Xn = (float*)mlp_alloc(m, sizeof(float) * NI * m->max_batch);
  d.Z1 = (float*)mlp_alloc(m, sizeof(float) * NH * m->max_batch);
  d.Z2 = (float*)mlp_alloc(m, sizeof(float) * NH * m->max_batch);
  d.Yn = (float*)mlp_alloc(m, sizeof(float) * NO * m->max_batch);
  d.loss = (float*)mlp_alloc(m, sizeof(float) * 4);
  if (!d.P || !d.Pb || !d.G || !d.M || !d.V || !d.Xn || !d.Z1 || !d.Z2 || !d.Yn || !d.loss) {
    dsdna_mlp_destroy(m);
    return DSDNA_ENOMEM;
  }
  for (int c = 0; c < NI; ++c) { d.norm.in_mean[c] = 0.0f; d.norm.in_scale[c] = 1.0f; }
  for (int c = 0; c < NO; ++c) { d.norm.out_mean[c] = 0.0f; d.norm.out_scale[c] = 1.0f; }
  cudaMemsetAsync(d.P, 0, sizeof(float) * NP, m->st);
  cudaMemsetAsync(d.G, 0, sizeof(float) * NP, m->st);
  cudaMemsetAsync(d.M, 0, sizeof(float) * NP, m->st);
  cudaMemsetAsync(d.V, 0, sizeof(float) * NP, m->st);
  k_mlp_refresh_bf16<<<(NP + 255) / 256, 256, 0, m->st>>>(d);
  if (cudaStreamSynchronize(m->st) != cudaSuccess) { dsdna_mlp_destroy(m); return DSDNA_ECUDA; }
  *out = m;
  return DSDNA_OK;
}

extern "C" int dsdna_mlp_num_params(void) { return NP; }

extern "C" int dsdna_mlp_set_params(dsdna_mlp* m, const float* params, const float* in_mean, const float* in_scale,
                                    const float* out_mean, const float* out_scale) {
  if (!m) return DSDNA_EINVAL;
  if (params) {
    if (cudaMemcpyAsync(m->d.P, params, sizeof(float) * NP, cudaMemcpyHostToDevice, m->st) != cudaSuccess) return DSDNA_ECUDA;
    k_mlp_refresh_bf16<<<(NP + 255) / 256, 256, 0, m->st>>>(m->d);
    cudaMemsetAsync(m->d.M, 0, sizeof(float) * NP, m->st);
    cudaMemsetAsync(m->d.V, 0, sizeof(float) * NP, m->st);
    m->adam_t = 0;
  }
  for (int c = 0; c < NI; ++c) {
    if (in_mean) m->d.norm.in_mean[c] = in_mean[c];
    if (in_scale) m->d.norm.in_scale[c] = in_scale[c];
  }
  for (int c = 0; c < NO; ++c) {
    if (out_mean) m->d.norm.out_mean[c] = out_mean[c];
    if (out_scale) m->d.norm.out_scale[c] = out_scale[c];
  }
  return cudaStreamSynchronize(m->st) == cudaSuccess ? DSDNA_OK : DSDNA_ECUDA;
}

extern "C" int dsdna_mlp_get_params(dsdna_mlp* m, float* params, float* grads) {
  if (!m) return DSDNA_EINVAL;
  if (params && cudaMemcpyAsync(params, m->d.P, sizeof(float) * NP, cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
    return DSDNA_ECUDA;
  if (grads && cudaMemcpyAsync(grads, m->d.G, sizeof(float) * NP, cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
    return DSDNA_ECUDA;
  return cudaStreamSynchronize(m->st) == cudaSuccess ? DSDNA_OK : DSDNA_ECUDA;
}

extern "C" int dsdna_mlp_forward(dsdna_mlp* m, const float* X, int B, float* Y) {
  if (!m || !X || !Y || B < 1 || B > m->max_batch) return DSDNA_EINVAL;
  const int tiles = (B + TILE - 1) / TILE;
  k_mlp_forward<<<(tiles + WARPS - 1) / WARPS, 32 * WARPS, 0, m->st>>>(m->d, X, B, Y);
  return cudaGetLastError() == cudaSuccess ? DSDNA_OK : DSDNA_ECUDA;
}

extern "C" int dsdna_mlp_backward(dsdna_mlp* m, const float* T, int B, float* loss_host) {
  if (!m || !T || B < 1 || B > m->max_batch) return DSDNA_EINVAL;
  cudaMemsetAsync(m->d.G, 0, sizeof(float) * NP, m->st);
  cudaMemsetAsync(m->d.loss, 0, sizeof(float), m->st);
  const int tiles = (B + TILE - 1) / TILE;
  k_mlp_backward<<<(tiles + WARPS - 1) / WARPS, 32 * WARPS, 0, m->st>>>(m->d, T, B);
  if (cudaGetLastError() != cudaSuccess) return DSDNA_ECUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, m->d.loss, sizeof(float), cudaMemcpyDeviceToHost, m->st) != cudaSuccess) return DSDNA_ECUDA;
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return DSDNA_ECUDA;
  }
  return DSDNA_OK;
}

extern "C" int dsdna_mlp_adam_step(dsdna_mlp* m, float lr, float beta1, float beta2, float eps, float weight_decay) {
  if (!m || weight_decay < 0.0f) return DSDNA_EINVAL;
  ++m->adam_t;
  const float c1 = (float)(1.0 - std::pow((double)beta1, (double)m->adam_t));
  const float c2 = (float)(1.0 - std::pow((double)beta2, (double)m->adam_t));
  k_mlp_adam<<<(NP + 255) / 256, 256, 0, m->st>>>(m->d, lr, beta1, beta2, eps, c1, c2, weight_decay);
  return cudaGetLastError() == cudaSuccess ? DSDNA_OK : DSDNA_ECUDA;
}
