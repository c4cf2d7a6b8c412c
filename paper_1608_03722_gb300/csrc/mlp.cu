// mlp.cu -- BF16 tensor-core MLP surrogate 4 -> 64 -> 64 -> 3 (GELU) of the
// sweep observables (mean extension / contour length, excess twist,
// denatured fraction) as a function of (force, torque, length, kT).
//
// Weights are kept as FP32 masters and BF16 copies.  The contractions run on
// the fifth-generation tensor cores: tcgen05.mma (kind::f16, BF16 operands in
// shared memory, FP32 accumulators in tensor memory), one 128-row batch tile
// per CTA, issued by one thread and completed through an mbarrier; epilogues
// read the accumulators with tcgen05.ld.  Small dimensions (4 inputs, 3
// outputs) are zero-padded to the MMA shape; the 3- and 4-wide weight
// gradients are FP32 warp reductions.  The forward pass keeps the
// pre-activations for the backward pass; the backward pass forms the mean
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

struct Norm {
  float in_mean[NI], in_scale[NI], out_mean[NO], out_scale[NO];
};

// ---------------------------------------------------------------- tcgen05 helpers
// Operands live in shared memory in the K-major, no-swizzle core-matrix layout:
// a core matrix is 8 rows x 16 bytes (8 BF16 along K); core matrices follow
// each other along K (128 bytes apart, the leading byte offset), and groups of
// 8 rows are K * 16 bytes apart (the stride byte offset).
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor of a K-major operand with K columns whose
// current 16-column chunk starts at shared address `addr`: start >> 4 (bits
// 0-13), leading byte offset >> 4 (16-29), stride byte offset >> 4 (32-45),
// descriptor version 1 (bit 46), no swizzle (bits 61-63 zero).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int K) {
  const uint64_t lbo = 128, sbo = (uint64_t)K * 16;
  return (uint64_t)((addr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFu) << 16) | (((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// D[128 x N] (+)= A[128 x K] B[N x K]^T: K / 16 MMAs issued by the calling thread.
__device__ __forceinline__ void umma_128xN(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, int K, int N,
                                           bool accumulate) {
  const uint32_t idesc = mma_idesc(128, N);
  for (int kc = 0; kc < K / 16; ++kc) {
    const uint64_t ad = smem_desc(a_addr + kc * 256, K), bd = smem_desc(b_addr + kc * 256, K);
    const uint32_t acc = (accumulate || kc > 0) ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// Wait for phase `parity` of the mbarrier, at most ~2^22 polls; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 FP32 accumulator columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int TC_COLS = 128;   // TMEM columns per CTA (two 64-column accumulators)

// Warp 0 allocates TC_COLS TMEM columns; the base address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_COLS) : "memory");
}

__device__ __forceinline__ void put_bf16(unsigned char* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
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
  unsigned* err;        // [1] set when a tensor-core wait gave up
  Norm norm;
};

// ---------------------------------------------------------------- forward
// One CTA of 128 threads per 128-row batch tile; thread t owns row t, which
// is also TMEM lane t of every accumulator (M = 128, warp w reads lanes
// 32w..32w+31).  Every contraction is a tcgen05.mma (BF16 operands from shared
// memory, FP32 accumulator in TMEM) issued by thread 0 and completed through
// an mbarrier; epilogues read the accumulators with tcgen05.ld.
constexpr int TC_ROWS = 128;
constexpr size_t F_AX = 0;                          // A  Xn  [128 x 16] (K = 4 padded)
constexpr size_t F_BW1 = F_AX + 128 * 16 * 2;       // B  W1  [64 x 16]
constexpr size_t F_AH1 = F_BW1 + 64 * 16 * 2;       // A  H1  [128 x 64]
constexpr size_t F_BW2 = F_AH1 + 128 * 64 * 2;      // B  W2  [64 x 64]
constexpr size_t F_AH2 = F_BW2 + 64 * 64 * 2;       // A  H2  [128 x 64]
constexpr size_t F_BW3 = F_AH2 + 128 * 64 * 2;      // B  W3  [16 x 64] (rows 3..15 zero)
constexpr size_t F_BYTES = F_BW3 + 16 * 64 * 2;

// Issue (thread 0) and complete (every thread) one batch of MMAs; ok turns
// false for the whole CTA if the mbarrier wait gives up.
struct TcSync {
  uint32_t mbar;
  uint32_t phase;
  bool ok;
  __device__ void start() {   // operands written by threads -> visible to the tensor core
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  __device__ void finish() {
    if (ok) ok = mbar_wait(mbar, phase);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
  }
};

__global__ void __launch_bounds__(TC_ROWS) k_mlp_forward(MlpDev m, const float* X, int B, float* Y) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  const int row = blockIdx.x * TC_ROWS + t;
  const bool live = row < B;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int i = t; i < 64 * 16; i += TC_ROWS) {
    const int n = i / 16, k = i % 16;
    *reinterpret_cast<__nv_bfloat16*>(sm + F_BW1 + cm_off(n, k, 16)) = k < NI ? m.Pb[OW1 + n * NI + k] : zero;
  }
  for (int i = t; i < 64 * 64; i += TC_ROWS) {
    const int n = i / 64, k = i % 64;
    *reinterpret_cast<__nv_bfloat16*>(sm + F_BW2 + cm_off(n, k, 64)) = m.Pb[OW2 + n * NH + k];
  }
  for (int i = t; i < 16 * 64; i += TC_ROWS) {
    const int n = i / 64, k = i % 64;
    *reinterpret_cast<__nv_bfloat16*>(sm + F_BW3 + cm_off(n, k, 64)) = n < NO ? m.Pb[OW3 + n * NH + k] : zero;
  }
  for (int k = 0; k < 16; ++k) {
    float v = 0.0f;
    if (live && k < NI) {
      v = (X[(size_t)row * NI + k] - m.norm.in_mean[k]) / m.norm.in_scale[k];
      m.Xn[(size_t)row * NI + k] = v;
    }
    put_bf16(sm + F_AX, cm_off(t, k, 16), v);
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  tmem_alloc(&tslot);
  TcSync sy{smem_u32(&mbar), 0u, true};
  sy.start();
  const uint32_t tmem = tslot;
  const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16);
  // layer 1: Z1 = Xn W1^T + b1 -> TMEM columns 0..63
  if (t == 0) {
    umma_128xN(tmem, smem_u32(sm + F_AX), smem_u32(sm + F_BW1), 16, 64, false);
    umma_commit(sy.mbar);
  }
  sy.finish();
  if (sy.ok)
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(lanes + c0, v);
      for (int j = 0; j < 16; ++j) {
        const float z = v[j] + m.P[OB1 + c0 + j];
        if (live) m.Z1[(size_t)row * NH + c0 + j] = z;
        put_bf16(sm + F_AH1, cm_off(t, c0 + j, 64), gelu(z));
      }
    }
  // layer 2: Z2 = H1 W2^T + b2 -> columns 64..127
  sy.start();
  if (t == 0 && sy.ok) {
    umma_128xN(tmem + 64, smem_u32(sm + F_AH1), smem_u32(sm + F_BW2), 64, 64, false);
    umma_commit(sy.mbar);
  }
  sy.finish();
  if (sy.ok)
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(lanes + 64 + c0, v);
      for (int j = 0; j < 16; ++j) {
        const float z = v[j] + m.P[OB2 + c0 + j];
        if (live) m.Z2[(size_t)row * NH + c0 + j] = z;
        put_bf16(sm + F_AH2, cm_off(t, c0 + j, 64), gelu(z));
      }
    }
  // layer 3: Y = H2 W3^T + b3 -> columns 0..15 (N = 3 padded to 16)
  sy.start();
  if (t == 0 && sy.ok) {
    umma_128xN(tmem, smem_u32(sm + F_AH2), smem_u32(sm + F_BW3), 64, 16, false);
    umma_commit(sy.mbar);
  }
  sy.finish();
  if (sy.ok) {
    float v[16];
    tmem_ld16(lanes, v);
    if (live)
      for (int c = 0; c < NO; ++c) {
        const float yn = v[c] + m.P[OB3 + c];
        m.Yn[(size_t)row * NO + c] = yn;
        Y[(size_t)row * NO + c] = m.norm.out_mean[c] + m.norm.out_scale[c] * yn;
      }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tmem_free(tmem);
  if (!sy.ok && t == 0) atomicOr(m.err, 1u);
}

// ---------------------------------------------------------------- backward
// Mean squared error over the B x 3 normalised outputs and its gradient, one
// 128-row tile per CTA.  dH2 = dY W3, dH1 = dZ2 W2 and dW2 = dZ2^T H1 (K = the
// tile's 128 rows; M = 64 output rows padded to 128) run on the tensor cores;
// the 3- and 4-wide gradients dW3 = dY^T H2, dW1 = dZ1^T Xn and the biases are
// FP32 warp reductions.  Weight gradients are added to G with atomics.
constexpr size_t B_ADY = 0;                          // A  dY    [128 x 16] (K = 3 padded)
constexpr size_t B_BW3T = B_ADY + 128 * 16 * 2;      // B  W3^T  [64 x 16]: (f, o) = W3[o][f]
constexpr size_t B_ADZ2 = B_BW3T + 64 * 16 * 2;      // A  dZ2   [128 x 64]
constexpr size_t B_BW2T = B_ADZ2 + 128 * 64 * 2;     // B  W2^T  [64 x 64]: (i, o) = W2[o][i]
constexpr size_t B_ADZ2T = B_BW2T + 64 * 64 * 2;     // A  dZ2^T [128 x 128]: (o, b) = dZ2[b][o]; rows 64.. zero
constexpr size_t B_BH1T = B_ADZ2T + 128 * 128 * 2;   // B  H1^T  [64 x 128]: (i, b) = H1[b][i]
constexpr size_t B_BYTES = B_BH1T + 64 * 128 * 2;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(TC_ROWS) k_mlp_backward(MlpDev m, const float* T, int B) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int row = blockIdx.x * TC_ROWS + t;
  const bool live = row < B;
  const float inv = 1.0f / (float)(B * NO);
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int i = t; i < 64 * 16; i += TC_ROWS) {
    const int n = i / 16, k = i % 16;
    *reinterpret_cast<__nv_bfloat16*>(sm + B_BW3T + cm_off(n, k, 16)) = k < NO ? m.Pb[OW3 + k * NH + n] : zero;
  }
  for (int i = t; i < 64 * 64; i += TC_ROWS) {
    const int n = i / 64, k = i % 64;
    *reinterpret_cast<__nv_bfloat16*>(sm + B_BW2T + cm_off(n, k, 64)) = m.Pb[OW2 + k * NH + n];
  }
  for (int i = t; i < 64 * 128 * 2 / 16; i += TC_ROWS)   // rows 64..127 of dZ2^T: the second half of the buffer
    reinterpret_cast<uint4*>(sm + B_ADZ2T + 64 * 128 * 2)[i] = make_uint4(0u, 0u, 0u, 0u);
  // dY of this row and the loss
  float dy[NO], lsum = 0.0f;
  for (int c = 0; c < NO; ++c) {
    dy[c] = 0.0f;
    if (live) {
      const float tn = (T[(size_t)row * NO + c] - m.norm.out_mean[c]) / m.norm.out_scale[c];
      const float e = m.Yn[(size_t)row * NO + c] - tn;
      lsum += e * e;
      dy[c] = 2.0f * e * inv;
    }
  }
  for (int k = 0; k < 16; ++k) put_bf16(sm + B_ADY, cm_off(t, k, 16), k < NO ? dy[k] : 0.0f);
  lsum = warp_sum(lsum);
  if (lane == 0) atomicAdd(m.loss, lsum * inv);
  // dW3 = dY^T H2 and db3 (CUDA cores); H1^T operand
  for (int f = 0; f < NH; ++f) {
    const float h2 = live ? gelu(m.Z2[(size_t)row * NH + f]) : 0.0f;
    const float h1 = live ? gelu(m.Z1[(size_t)row * NH + f]) : 0.0f;
    put_bf16(sm + B_BH1T, cm_off(f, t, 128), h1);
    for (int o = 0; o < NO; ++o) {
      const float g = warp_sum(dy[o] * h2);
      if (lane == 0) atomicAdd(&m.G[OW3 + o * NH + f], g);
    }
  }
  for (int o = 0; o < NO; ++o) {
    const float g = warp_sum(dy[o]);
    if (lane == 0) atomicAdd(&m.G[OB3 + o], g);
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  tmem_alloc(&tslot);
  TcSync sy{smem_u32(&mbar), 0u, true};
  sy.start();
  const uint32_t tmem = tslot;
  const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16);
  // dH2 = dY W3 -> columns 0..63
  if (t == 0) {
    umma_128xN(tmem, smem_u32(sm + B_ADY), smem_u32(sm + B_BW3T), 16, 64, false);
    umma_commit(sy.mbar);
  }
  sy.finish();
  // dZ2 = dH2 gelu'(Z2): A operand, its transpose, db2
  if (sy.ok)
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(lanes + c0, v);
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j;
        const float dz = live ? v[j] * gelu_d(m.Z2[(size_t)row * NH + c]) : 0.0f;
        put_bf16(sm + B_ADZ2, cm_off(t, c, 64), dz);
        put_bf16(sm + B_ADZ2T, cm_off(c, t, 128), dz);
        const float g = warp_sum(dz);
        if (lane == 0) atomicAdd(&m.G[OB2 + c], g);
      }
    }
  // dH1 = dZ2 W2 -> columns 64..127; dW2 = dZ2^T H1 -> columns 0..63 (lanes 0..63)
  sy.start();
  if (t == 0 && sy.ok) {
    umma_128xN(tmem + 64, smem_u32(sm + B_ADZ2), smem_u32(sm + B_BW2T), 64, 64, false);
    umma_128xN(tmem, smem_u32(sm + B_ADZ2T), smem_u32(sm + B_BH1T), 128, 64, false);
    umma_commit(sy.mbar);
  }
  sy.finish();
  if (sy.ok) {
    if (warp < 2)   // output rows o = t < 64 of dW2
      for (int c0 = 0; c0 < NH; c0 += 16) {
        float v[16];
        tmem_ld16(lanes + c0, v);
        for (int j = 0; j < 16; ++j) atomicAdd(&m.G[OW2 + t * NH + c0 + j], v[j]);
      }
    // dZ1 = dH1 gelu'(Z1); dW1 = dZ1^T Xn and db1 (CUDA cores)
    float xn[NI];
    for (int i = 0; i < NI; ++i) xn[i] = live ? m.Xn[(size_t)row * NI + i] : 0.0f;
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tmem_ld16(lanes + 64 + c0, v);
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j;
        const float dz = live ? v[j] * gelu_d(m.Z1[(size_t)row * NH + c]) : 0.0f;
        const float gb = warp_sum(dz);
        if (lane == 0) atomicAdd(&m.G[OB1 + c], gb);
        for (int i = 0; i < NI; ++i) {
          const float g = warp_sum(dz * xn[i]);
          if (lane == 0) atomicAdd(&m.G[OW1 + c * NI + i], g);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tmem_free(tmem);
  if (!sy.ok && t == 0) atomicOr(m.err, 1u);
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
  m->max_batch = ((max_batch + 127) / 128) * 128;
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
  d.err = reinterpret_cast<unsigned*>(d.loss + 1);
  if (!d.P || !d.Pb || !d.G || !d.M || !d.V || !d.Xn || !d.Z1 || !d.Z2 || !d.Yn || !d.loss) {
    dsdna_mlp_destroy(m);
    return DSDNA_ENOMEM;
  }
  for (int c = 0; c < NI; ++c) { d.norm.in_mean[c] = 0.0f; d.norm.in_scale[c] = 1.0f; }
  for (int c = 0; c < NO; ++c) { d.norm.out_mean[c] = 0.0f; d.norm.out_scale[c] = 1.0f; }
  if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_BYTES) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B_BYTES) != cudaSuccess) {
    dsdna_mlp_destroy(m);
    return DSDNA_ECUDA;
  }
  cudaMemsetAsync(d.loss, 0, sizeof(float) * 4, m->st);
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
  unsigned err = 0;
  if (cudaMemcpyAsync(&err, m->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, m->st) != cudaSuccess) return DSDNA_ECUDA;
  if (cudaStreamSynchronize(m->st) != cudaSuccess) return DSDNA_ECUDA;
  return err ? DSDNA_ETIMEOUT : DSDNA_OK;
}

extern "C" int dsdna_mlp_forward(dsdna_mlp* m, const float* X, int B, float* Y) {
  if (!m || !X || !Y || B < 1 || B > m->max_batch) return DSDNA_EINVAL;
  k_mlp_forward<<<(B + TC_ROWS - 1) / TC_ROWS, TC_ROWS, F_BYTES, m->st>>>(m->d, X, B, Y);
  return cudaGetLastError() == cudaSuccess ? DSDNA_OK : DSDNA_ECUDA;
}

extern "C" int dsdna_mlp_backward(dsdna_mlp* m, const float* T, int B, float* loss_host) {
  if (!m || !T || B < 1 || B > m->max_batch) return DSDNA_EINVAL;
  cudaMemsetAsync(m->d.G, 0, sizeof(float) * NP, m->st);
  cudaMemsetAsync(m->d.loss, 0, sizeof(float), m->st);
  k_mlp_backward<<<(B + TC_ROWS - 1) / TC_ROWS, TC_ROWS, B_BYTES, m->st>>>(m->d, T, B);
  if (cudaGetLastError() != cudaSuccess) return DSDNA_ECUDA;
  if (loss_host) {
    float lw[2];
    if (cudaMemcpyAsync(lw, m->d.loss, sizeof(lw), cudaMemcpyDeviceToHost, m->st) != cudaSuccess) return DSDNA_ECUDA;
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return DSDNA_ECUDA;
    *loss_host = lw[0];
    unsigned err;
    std::memcpy(&err, &lw[1], sizeof(err));                   // the error word follows the loss
    if (err) return DSDNA_ETIMEOUT;
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
