// mcx_mlp.cu -- the learned direction proposal: a 4 -> 3x128 (SiLU) -> 40
// network whose outputs parametrise an 8-component Gaussian mixture over the
// normalised aim point, trained on ray histories with a weighted negative
// log-likelihood, and the importance sampler that draws ray starts from the
// defensive mixture alpha U(window) + (1 - alpha) GMM.
//
// The hidden and output layers, forward and backward, are BF16 products on
// the 5th-generation tensor cores (tcgen05.mma, FP32 accumulators in tensor
// memory); the 4-input layer, the mixture head, the loss and Adam run on the
// CUDA cores.  A training step is one fused kernel per 128-row tile (the
// forward pass, the loss and the input-gradient chain, with activations in
// shared and tensor memory) and three split-K weight-gradient products.
//
// Parameters are one flat FP32 vector (the master copy), in the order
// W1 [4,128], b1, W2 [128,128], b2, W3 [128,128], b3, W4 [128,40], b4, with
// y = x W + b per layer; BF16 copies of W2..W4 feed the tensor cores.
#include <cuda.h>   // CUtensorMap and its encoder's types (the encoder comes from the runtime)
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "mcx_host.h"
#include "mcx_tracer.cuh"

namespace mcx {

using bf16 = __nv_bfloat16;

constexpr int kHid = 128;
constexpr int kComp = 8;
constexpr int kOut = 5 * kComp;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 4 * kHid;
constexpr int kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kHid * kOut;
constexpr int kNParams = kOffB4 + kOut;
static_assert(kNParams == 38824, "parameter count");
constexpr float kLsC = 2.5f, kLsM = -2.5f;
constexpr float kLog2Pi = 1.8378770664093453f;

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + expf(-z)); }
// Inference form: z sigmoid(z) = h + h tanh(h) with h = z / 2, on the
// hardware tanh (one MUFU instruction, relative error ~5e-4, below the BF16
// rounding the activations receive next).  The sampler's importance weight
// uses the same network outputs that drew the sample, so the estimator stays
// unbiased whatever the activation's rounding.
__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
  return fmaf(h, t, h);
}
// The same of z = v + b with the halved bias hb = b / 2 given: h = v / 2 + hb
// in one fused multiply-add.
__device__ __forceinline__ float silu_fast_hb(float v, float hb) {
  const float h = fmaf(v, 0.5f, hb);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
  return fmaf(h, t, h);
}
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.f / (1.f + expf(-z));
  return s * (1.f + z * (1.f - s));
}

// ------------------------------------------------------------------ GEMM arguments
// C[M, N] = A[M, K] B[K, N] in BF16 with FP32 accumulation for the training
// steps (tc_gemm_kernel, below the tcgen05 helpers).  A is read as stored
// row-major [M, lda] or, with a_t, as the transpose of a row-major [K, lda]
// matrix; likewise B ([K, ldb] or, with b_t, [N, ldb] transposed).  Split-K
// runs along gridDim.z in chunks of k_chunk; gridDim.y runs up to three
// independent products of one launch (GemmGroup).
enum Epi { EPI_FWD = 0, EPI_HEAD = 1, EPI_WGRAD = 3 };

struct GemmArgs {
  const bf16* A;
  int lda, a_t;
  const bf16* B;
  int ldb, b_t;
  int M, N, K, k_chunk;
  const float* bias;      // FWD, HEAD: [N]
  float* of;              // FWD: z (may be null); HEAD: o; WGRAD: dW (added)
  int ldo;
  bf16* ob;               // FWD: silu(z) (may be null)
  int ldob;
  int* err;               // set when a tensor-core wait gave up
  uint32_t spin;          // polls of a tensor-core wait before it gives up
  int mn;                 // A as row-major [K, lda] (M contiguous) and B as row-major
                          // [K, ldb] (N contiguous), both staged MN-major
};
struct GemmGroup {
  GemmArgs g[3];          // product blockIdx.y
};

// ------------------------------------------------------------------ SIMT layers
// z1 = x W1 + b1 (FP32), h1 = silu(z1) as BF16; one thread per hidden unit.
__global__ void __launch_bounds__(128) layer1_kernel(const float* __restrict__ x, int n,
                                                     const float* __restrict__ P, bf16* __restrict__ h1) {
  const int j = threadIdx.x;
  const float w0 = P[kOffW1 + j], w1 = P[kOffW1 + kHid + j], w2 = P[kOffW1 + 2 * kHid + j],
              w3 = P[kOffW1 + 3 * kHid + j], b = P[kOffB1 + j];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const float4 xi = reinterpret_cast<const float4*>(x)[i];
    const float z = ((xi.x * w0 + xi.y * w1) + (xi.z * w2 + xi.w * w3)) + b;
    h1[(size_t)i * kHid + j] = __float2bfloat16(silu_f(z));
  }
}

// ------------------------------------------------------------------ mixture head
struct Mix {
  float logpi[kComp], mu[kComp], mv[kComp], lsu[kComp], lsv[kComp];
};

// Fast forms for the mixture head (sampler and training loss): exponential
// and logarithm on the hardware approximations (relative error ~1e-6 over the
// head's ranges), and tanh(y) = 1 - 2 / (exp(2y) + 1) on the same exponential
// (absolute error ~1e-7; it enters the log-scales C tanh(r / C) + M
// additively).  Sampling and weighting read the same mixture, so the
// importance weights stay exact for the density that drew the sample.
__device__ __forceinline__ float tanh_e(float y) { return 1.f - __fdividef(2.f, __expf(2.f * y) + 1.f); }

__device__ __forceinline__ void mixture_of(const float* o, Mix& m) {
  float amax = -CUDART_INF_F;
#pragma unroll
  for (int k = 0; k < kComp; ++k) amax = fmaxf(amax, o[5 * k]);
  float se = 0.f;
#pragma unroll
  for (int k = 0; k < kComp; ++k) se += __expf(o[5 * k] - amax);
  const float lse = amax + __logf(se);
#pragma unroll
  for (int k = 0; k < kComp; ++k) {
    m.logpi[k] = o[5 * k] - lse;
    m.mu[k] = o[5 * k + 1];
    m.mv[k] = o[5 * k + 2];
    m.lsu[k] = kLsC * tanh_e(o[5 * k + 3] / kLsC) + kLsM;
    m.lsv[k] = kLsC * tanh_e(o[5 * k + 4] / kLsC) + kLsM;
  }
}

// log q_gmm(tu, tv) and the per-component log terms
__device__ __forceinline__ float log_mix(const Mix& m, float tu, float tv, float ell[kComp]) {
  float mx = -CUDART_INF_F;
#pragma unroll
  for (int k = 0; k < kComp; ++k) {
    const float zu = (tu - m.mu[k]) * __expf(-m.lsu[k]);
    const float zv = (tv - m.mv[k]) * __expf(-m.lsv[k]);
    ell[k] = m.logpi[k] - 0.5f * zu * zu - m.lsu[k] - 0.5f * zv * zv - m.lsv[k] - kLog2Pi;
    mx = fmaxf(mx, ell[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kComp; ++k) s += __expf(ell[k] - mx);
  return mx + __logf(s);
}

__global__ void sum_kernel(const float* __restrict__ v, int n, float* __restrict__ out) {
  float s = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += v[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Adam on the FP32 master parameters, then the BF16 copies of W2..W4.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, float lr, float b1, float b2, float eps, float c1,
                            float c2, bf16* __restrict__ w2, bf16* __restrict__ w3,
                            bf16* __restrict__ w4) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    P[i] = p;
    if (i >= kOffW2 && i < kOffB2) w2[i - kOffW2] = __float2bfloat16(p);
    else if (i >= kOffW3 && i < kOffB3) w3[i - kOffW3] = __float2bfloat16(p);
    else if (i >= kOffW4 && i < kOffB4) w4[i - kOffW4] = __float2bfloat16(p);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ P, bf16* __restrict__ w2, bf16* __restrict__ w3,
                               bf16* __restrict__ w4) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    if (i >= kOffW2 && i < kOffB2) w2[i - kOffW2] = __float2bfloat16(P[i]);
    else if (i >= kOffW3 && i < kOffB3) w3[i - kOffW3] = __float2bfloat16(P[i]);
    else if (i >= kOffW4 && i < kOffB4) w4[i - kOffW4] = __float2bfloat16(P[i]);
  }
}

// ------------------------------------------------------------------ sampler
struct PropConst {
  float alpha, hu, hv;
  float shift[4], scale[4];
  float angle;
  uint32_t spin;          // polls of a tensor-core wait before it gives up
};

// Network inputs of rays [begin, begin + n): the learned path makes the plain
// sampler's draws (source point, aim point, energy) and keeps all but the aim.
__global__ void __launch_bounds__(256) prop_inputs_kernel(const DevInstrument I, uint64_t begin,
                                                          int n, uint64_t seed, PropConst pc,
                                                          float* __restrict__ x) {
  __shared__ DevComp S;
  if (threadIdx.x == 0) S = I.comps[0];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  RayStream rs;
  rs.init(begin + i, (uint32_t)I.instr_id, seed);
  float sx, sy, tx, ty, E;
  sample_start<float>(S, rs, sx, sy, tx, ty, E);   // the plain aim point is not used
  float4 xi;
  xi.x = (sx - pc.shift[0]) * pc.scale[0];
  xi.y = (sy - pc.shift[1]) * pc.scale[1];
  xi.z = (E - pc.shift[2]) * pc.scale[2];
  xi.w = (pc.angle - pc.shift[3]) * pc.scale[3];
  reinterpret_cast<float4*>(x)[i] = xi;
}

__device__ __forceinline__ void write_mixture_start(const DevComp& S, const PropConst& pc, RayStream& rs,
                                                    const float* o, float sx, float sy, float E,
                                                    float* __restrict__ st, uint64_t ld, uint64_t i);

// Starts of rays [begin, begin + n) from the defensive mixture: the draws of
// prop_inputs_kernel, then a selector and two more uniforms (Box-Muller for a
// Gaussian component).  Aim points outside the window get weight 0.
__global__ void __launch_bounds__(256) prop_sample_kernel(const DevInstrument I, uint64_t begin,
                                                          int n, uint64_t seed, PropConst pc,
                                                          const float* __restrict__ o,
                                                          float* __restrict__ st, uint64_t ld) {
  __shared__ DevComp S;
  if (threadIdx.x == 0) S = I.comps[0];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  RayStream rs;
  rs.init(begin + i, (uint32_t)I.instr_id, seed);
  float sx, sy, tx, ty, E;
  sample_start<float>(S, rs, sx, sy, tx, ty, E);
  float oi[kOut];
#pragma unroll
  for (int c = 0; c < kOut; ++c) oi[c] = o[(size_t)i * kOut + c];
  write_mixture_start(S, pc, rs, oi, sx, sy, E, st, ld, i);
}

// Draws the aim point of one ray from the defensive mixture (network outputs
// o) with the stream's next three uniforms and writes its start (row i).
__device__ __forceinline__ void write_mixture_start(const DevComp& S, const PropConst& pc, RayStream& rs,
                                                    const float* o, float sx, float sy, float E,
                                                    float* __restrict__ st, uint64_t ld, uint64_t i) {
  const float u_sel = Uniform<float>::draw(rs);
  const float u_a = Uniform<float>::draw(rs);
  const float u_b = Uniform<float>::draw(rs);
  Mix m;
  mixture_of(o, m);
  float tu, tv;
  if (u_sel < pc.alpha) {
    tu = 2.f * u_a - 1.f;
    tv = 2.f * u_b - 1.f;
  } else {
    const float v = (u_sel - pc.alpha) / (1.f - pc.alpha);
    int k = 0;
    float c = 0.f;
#pragma unroll
    for (int j = 0; j < kComp; ++j) {
      c += __expf(m.logpi[j]);
      if (c <= v) k = j + 1;
    }
    k = k < kComp ? k : kComp - 1;
    const float rad = sqrtf(-2.f * logf(1.f - u_a));
    float sn, cs;
    sincospif(2.f * u_b, &sn, &cs);
    float muk = 0.f, mvk = 0.f, lsuk = 0.f, lsvk = 0.f;
#pragma unroll
    for (int j = 0; j < kComp; ++j)
      if (j == k) { muk = m.mu[j]; mvk = m.mv[j]; lsuk = m.lsu[j]; lsvk = m.lsv[j]; }
    tu = muk + __expf(lsuk) * rad * cs;
    tv = mvk + __expf(lsvk) * rad * sn;
  }
  float w = 0.f;
  if (fabsf(tu) <= 1.f && fabsf(tv) <= 1.f) {
    float ell[kComp];
    const float qa = pc.alpha * 0.25f + (1.f - pc.alpha) * __expf(log_mix(m, tu, tv, ell));
    w = (0.25f / qa) * source_weight<float>(S, sx, sy, tu * pc.hu, tv * pc.hv, E);
  }
  st[i] = sx;
  st[ld + i] = sy;
  st[2 * ld + i] = E;
  st[3 * ld + i] = tu * pc.hu;
  st[4 * ld + i] = tv * pc.hv;
  st[5 * ld + i] = w;
}

// ------------------------------------------------------------------ shared helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// ------------------------------------------------------------------ tcgen05 sampler
// The same computation on the 5th-generation tensor cores.  One CTA per SM,
// kTcGroups warpgroups of 128 threads; each warpgroup takes 128-ray tiles
// (one ray per thread, which is also one TMEM lane) independently of the
// others, so one group's MMAs overlap another's epilogue:
//   layer 1 (4 -> 128) on the CUDA cores, each thread writing its ray's row
//     of BF16 activations into the group's shared-memory tile;
//   layers 2, 3 (128 -> 128) and the head (128 -> 40, padded to N = 48) as
//     tcgen05.mma kind::f16 (BF16 operands from shared memory, FP32
//     accumulator in the group's 128 TMEM columns), issued by one thread and
//     committed to the group's mbarrier;
//   each epilogue reads the thread's own accumulator row (tcgen05.ld
//     32x32b), adds the bias, applies SiLU and writes the next layer's
//     activations in place; after the head it samples the mixture.
// Operands use the no-swizzle K-major core-matrix layout: 8 x 8 BF16 blocks
// of 128 contiguous bytes, block (row/8, k/8) at ((row/8) * 16 + k/8) * 128,
// so a K = 16 step is two blocks 128 B apart (leading offset) and successive
// 8-row groups are 2048 B apart (stride offset).
constexpr int kTcGroups = 4;
constexpr int kHeadN = 48;                                     // kOut rounded up to 16
constexpr size_t kTcTile = (size_t)kHid * kHid * sizeof(bf16); // 128 x 128 BF16 = 32 KB
constexpr size_t kTcWeightBytes = 2 * kTcTile + (size_t)kHeadN * kHid * sizeof(bf16) +
                                  (size_t)(4 * kHid + 3 * kHid + kOut) * sizeof(float);
constexpr size_t kTcTilesOff = (kTcWeightBytes + 1023) & ~(size_t)1023;
constexpr size_t kTcSmem = 1024 + kTcTilesOff + kTcGroups * kTcTile;
constexpr int kTcSpinLimit = 1 << 24;                         // bounded mbarrier wait

__device__ __forceinline__ int core_off(int row, int k) {
  return (((row >> 3) * (kHid / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// tcgen05 shared-memory matrix descriptor: start, leading and stride byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// The same with A and B MN-major (bits 15, 16): each 8 x 8 core matrix holds
// 8 K rows of 8 contiguous M (N) elements; the descriptor's leading offset is
// then the stride between core matrices adjacent in K, its stride offset the
// stride between those adjacent in M (N) (measured on GB300 against a CPU
// product; the other reading gives wrong sums).
__device__ __forceinline__ uint32_t tc_idesc_mn(int m, int n) { return tc_idesc(m, n) | (1u << 15) | (1u << 16); }

// D[tmem] (+)= A[128 x 128] B^T over K = 128 in eight K = 16 steps, then a
// commit that arrives on `mbar` when the MMAs have completed.
__device__ __forceinline__ void tc_layer(uint32_t tmem, uint32_t a_smem, uint32_t b_smem, int n,
                                         uint32_t mbar) {
  const uint32_t idesc = tc_idesc(128, n);
#pragma unroll
  for (int kk = 0; kk < kHid / 16; ++kk) {
    const uint64_t da = tc_desc(a_smem + kk * 256, 128, 2048);
    const uint64_t db = tc_desc(b_smem + kk * 256, 128, 2048);
    const uint32_t acc = kk > 0 ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(mbar));
}

// Waits for the mbarrier phase with the given parity; false after `limit`
// polls (the caller reports it instead of waiting forever).  A wait that gave
// up is followed by a drain wait with the full limit (kTcSpinLimit) on the
// same phase, so that no tensor-core operation still writes the TMEM the
// kernel then frees.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, uint32_t limit = kTcSpinLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// true on every thread of the group iff v holds on all of them (a barrier
// with an AND reduction), so the group leaves its loop together.
__device__ __forceinline__ bool tc_group_all(int group, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r) : "r"((uint32_t)v), "r"(1 + group) : "memory");
  return r != 0;
}

// The group's 128 threads (named barrier 1 + group), with the tcgen05 fences
// that order TMEM reads and shared-memory writes before the next MMA.
__device__ __forceinline__ void tc_group_sync(int group) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("bar.sync %0, 128;" :: "r"(1 + group) : "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ------------------------------------------------------------------ tcgen05 training GEMM
// One 128-row tile of C per CTA (all N <= 128 columns at once), eight warps:
//   K in chunks of kGk, each staged by all threads into shared memory in the
//     no-swizzle K-major core-matrix layout (8 x 8 BF16 blocks of 128 B; a
//     K-contiguous source with 16-byte vector loads, a K-strided one gathered
//     eight K values at a time, consecutive threads on consecutive rows), two
//     stage buffers so that the threads stage chunk c + 1 while the tensor
//     cores run chunk c;
//   one thread issues the chunk's kGk / 16 tcgen05.mma kind::f16 steps
//     (BF16 x BF16 -> FP32 in TMEM) and commits them to the buffer's
//     mbarrier, which the threads wait on before restaging that buffer;
//   after the last chunk the warps read the accumulator rows (TMEM lanes)
//     into a shared-memory tile, and the epilogue runs over it in row-major
//     order (coalesced global accesses): bias and SiLU (forward), bias (head),
//     or an atomic add into the weight gradient (split-K over the batch rows
//     along gridDim.z).
// Every wait is bounded; a wait that gives up sets *err, waits once more
// (bounded) for the MMAs in flight, frees the TMEM and skips the epilogue.
constexpr int kGk = 64;                                   // K per staged chunk
constexpr int kGm = 128;                                  // rows per tile (TMEM lanes)

template <int BN>
struct TcGemmSmem {
  static constexpr size_t a_bytes = (size_t)kGm * kGk * sizeof(bf16);
  static constexpr size_t stage = a_bytes + (size_t)BN * kGk * sizeof(bf16);
  static constexpr int ldc = BN + 4;                   // FP32 tile row stride (no bank conflicts)
  static constexpr size_t c_bytes = (size_t)kGm * ldc * sizeof(float);
  static constexpr size_t bytes = (2 * stage > c_bytes ? 2 * stage : c_bytes) + 1024;   // + alignment
  static constexpr uint32_t tmem_cols = BN <= 32 ? 32 : (BN <= 64 ? 64 : 128);
};

// byte offset of element (row, k) in a kGk-wide K-major core-matrix tile
__device__ __forceinline__ int core_off_chunk(int row, int k) {
  return (((row >> 3) * (kGk / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// Rows [0, nrows) of one operand tile for K indices [kc0, kc0 + kGk): element
// (r, k) comes from src[(r0 + r) * ld + kc0 + k] (kcontig) or
// src[(kc0 + k) * ld + r0 + r]; rows >= rmax and K indices >= kend are zero.
__device__ __forceinline__ void stage_tile(unsigned char* dst, const bf16* __restrict__ src, int ld, bool kcontig,
                                           int r0, int rmax, int nrows, int kc0, int kend) {
  constexpr int groups = kGk / 8;
  for (int g = threadIdx.x; g < nrows * groups; g += blockDim.x) {
    int r, j;
    if (kcontig) { r = g / groups; j = g % groups; }
    else { r = g % nrows; j = g / nrows; }   // consecutive threads: consecutive rows
    const int gr = r0 + r, gk = kc0 + 8 * j;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < rmax && gk < kend) {
      if (kcontig && gk + 8 <= kend) {
        // 16 bytes straight into shared memory (cp.async): every load of the
        // tile is in flight at once; the caller waits for them (cp_async_wait)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                     :: "r"(smem_u32(dst + core_off_chunk(r, 8 * j))), "l"(src + (size_t)gr * ld + gk)
                     : "memory");
        continue;
      } else {
        uint16_t e[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const bool in = gk + q < kend;
          const bf16 x = in ? (kcontig ? src[(size_t)gr * ld + gk + q] : src[(size_t)(gk + q) * ld + gr])
                            : __float2bfloat16(0.f);
          e[q] = *reinterpret_cast<const uint16_t*>(&x);
        }
        v = make_uint4(e[0] | ((uint32_t)e[1] << 16), e[2] | ((uint32_t)e[3] << 16),
                       e[4] | ((uint32_t)e[5] << 16), e[6] | ((uint32_t)e[7] << 16));
      }
    }
    *reinterpret_cast<uint4*>(dst + core_off_chunk(r, 8 * j)) = v;
  }
}

// Rows k in [kc0, kc0 + kGk) of a row-major [K, ld] operand, columns
// [c0, c0 + ncols) (zero at or beyond cmax, and for k >= kend), as an
// MN-major core-matrix tile: element (k, c) at
// ((k / 8) (ncols / 8) + c / 8) 128 + (k mod 8) 16 + (c mod 8) 2 bytes, so K
// groups are (ncols / 8) 128 bytes apart and column groups 128.  Each 16-byte
// piece (8 columns of one row) is one cp.async (ld a multiple of 8 elements).
__device__ __forceinline__ void stage_tile_mn(unsigned char* dst, const bf16* __restrict__ src, int ld, int c0,
                                              int cmax, int ncols, int kc0, int kend) {
  const int groups = ncols / 8;
  for (int g = threadIdx.x; g < kGk * groups; g += blockDim.x) {
    const int k = g / groups, cb = g % groups;
    const int gk = kc0 + k, gc = c0 + 8 * cb;
    unsigned char* d = dst + (((k >> 3) * groups + cb) << 7) + ((k & 7) << 4);
    if (gk < kend && gc + 8 <= cmax) {
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                   :: "r"(smem_u32(d)), "l"(src + (size_t)gk * ld + gc) : "memory");
    } else {
      uint16_t e[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bf16 x = (gk < kend && gc + q < cmax) ? src[(size_t)gk * ld + gc + q] : __float2bfloat16(0.f);
        e[q] = *reinterpret_cast<const uint16_t*>(&x);
      }
      *reinterpret_cast<uint4*>(d) = make_uint4(e[0] | ((uint32_t)e[1] << 16), e[2] | ((uint32_t)e[3] << 16),
                                                e[4] | ((uint32_t)e[5] << 16), e[6] | ((uint32_t)e[7] << 16));
    }
  }
}

constexpr int kGemmThreads = 256;   // two warps per TMEM lane quarter

template <int BN, int EPI>
__global__ void __launch_bounds__(kGemmThreads) tc_gemm_kernel(const __grid_constant__ GemmGroup gg) {
  const GemmArgs& g = gg.g[blockIdx.y];
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char* gsm = gsm_raw + ((1024 - (smem_u32(gsm_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  using L = TcGemmSmem<BN>;
  const int m0 = blockIdx.x * kGm;
  const int k_begin = blockIdx.z * g.k_chunk;
  const int k_end = min(g.K, k_begin + g.k_chunk);
  const int n_chunks = k_end > k_begin ? (k_end - k_begin + kGk - 1) / kGk : 0;
  // B tile width: BN, or N rounded up to 16 for the MN-major products
  const int nb = g.mn ? min(BN, (g.N + 15) & ~15) : BN;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[b])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(L::tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  auto stage = [&](int c) {
    unsigned char* a_s = gsm + (size_t)(c & 1) * L::stage;
    const int kc0 = k_begin + c * kGk;
    if (g.mn) {
      stage_tile_mn(a_s, g.A, g.lda, m0, g.M, kGm, kc0, k_end);
      stage_tile_mn(a_s + L::a_bytes, g.B, g.ldb, 0, g.N, nb, kc0, k_end);
    } else {
      stage_tile(a_s, g.A, g.lda, !g.a_t, m0, g.M, kGm, kc0, k_end);
      stage_tile(a_s + L::a_bytes, g.B, g.ldb, g.b_t != 0, 0, g.N, BN, kc0, k_end);
    }
  };
  if (n_chunks > 0) stage(0);
  cp_async_wait();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = g.mn ? tc_idesc_mn(kGm, nb) : tc_idesc(kGm, BN);
  bool ok = true;
  int last = -1;   // last chunk whose MMAs were issued (the same on every thread)
  for (int c = 0; c < n_chunks; ++c) {
    const uint32_t buf = (uint32_t)(c & 1);
    last = c;
    if (threadIdx.x == 0) {
      const uint32_t a_s = smem_u32(gsm + buf * L::stage), b_s = a_s + (uint32_t)L::a_bytes;
#pragma unroll
      for (int kk = 0; kk < kGk / 16; ++kk) {
        // K-major: a K = 16 step is two core matrices 128 B apart; MN-major:
        // two K groups, (width / 8) 128 B apart
        const uint64_t da = g.mn ? tc_desc(a_s + kk * 2 * (kGm / 8) * 128, (kGm / 8) * 128, 128)
                                 : tc_desc(a_s + kk * 256, 128, (kGk / 8) * 128);
        const uint64_t db = g.mn ? tc_desc(b_s + kk * 2 * (nb / 8) * 128, (nb / 8) * 128, 128)
                                 : tc_desc(b_s + kk * 256, 128, (kGk / 8) * 128);
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
            :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar[buf])));
    }
    if (c + 1 < n_chunks) {
      // the other buffer was read by chunk c - 1: wait for its MMAs first
      if (c >= 1) ok = __syncthreads_and(tc_wait(smem_u32(&mbar[buf ^ 1u]), (uint32_t)(((c - 1) >> 1) & 1), g.spin));
      if (!ok) break;
      stage(c + 1);
      cp_async_wait();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
  // the last commit covers every MMA issued before it
  if (ok && last >= 0)
    ok = __syncthreads_and(tc_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), g.spin));
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(g.err, 1);
    if (last >= 0) tc_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // each thread's accumulator row (its TMEM lane) into an FP32 tile in the
  // operand buffers (the MMAs reading them have completed), then the
  // epilogue in row-major order, so that global loads, stores and atomics
  // coalesce across the threads
  float* cs = reinterpret_cast<float*>(gsm);
  // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its sub-partition); the
  // two warps of a lane quarter take alternate 16-column groups
  const int quarter = (threadIdx.x >> 5) & 3, half = threadIdx.x >> 7;
  const int trow = quarter * 32 + (threadIdx.x & 31);
  const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16);
  if (ok) {
#pragma unroll 1
    for (int c0 = 16 * half; c0 < nb; c0 += 32) {
      float v[16];
      if (n_chunks > 0) tc_ld16(tlane + c0, v);
      else for (int j = 0; j < 16; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(cs + (size_t)trow * L::ldc + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
  __syncthreads();
  if (ok && EPI == EPI_WGRAD && (g.N & 3) == 0 && (g.ldo & 3) == 0 &&
      (reinterpret_cast<uintptr_t>(g.of) & 15) == 0) {
    // four adjacent columns per vector atomic (16-byte aligned rows)
    const int nq = g.N >> 2;
    for (int e = threadIdx.x; e < kGm * nq; e += blockDim.x) {
      const int r = e / nq, gn = 4 * (e % nq), gm = m0 + r;
      if (gm >= g.M) continue;
      const float4 v = *reinterpret_cast<const float4*>(cs + (size_t)r * L::ldc + gn);
      if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
        atomicAdd(reinterpret_cast<float4*>(g.of + (size_t)gm * g.ldo + gn), v);
    }
  } else if (ok) {
    for (int e = threadIdx.x; e < kGm * BN; e += blockDim.x) {
      const int r = e / BN, gn = e % BN, gm = m0 + r;
      if (gm >= g.M || gn >= g.N) continue;
      const float a = cs[(size_t)r * L::ldc + gn];
      if (EPI == EPI_FWD) {
        const float z = a + g.bias[gn];
        if (g.of) g.of[(size_t)gm * g.ldo + gn] = z;
        g.ob[(size_t)gm * g.ldob + gn] = __float2bfloat16(silu_f(z));
      } else if (EPI == EPI_HEAD) {
        g.of[(size_t)gm * g.ldo + gn] = a + g.bias[gn];
      } else {
        if (a != 0.f) atomicAdd(&g.of[(size_t)gm * g.ldo + gn], a);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(L::tmem_cols));
}

// `count` products of equal M and K in one launch (gridDim.y = count).
template <int BN, int EPI>
static cudaError_t gemm_group(const GemmArgs* g, int count, int splits, cudaStream_t s) {
  GemmGroup gg{};
  for (int i = 0; i < count; ++i) {
    if (g[i].N > BN || g[i].M != g[0].M || g[i].K != g[0].K) return cudaErrorInvalidValue;
    gg.g[i] = g[i];
  }
  constexpr size_t smem = TcGemmSmem<BN>::bytes;
  cudaFuncSetAttribute(tc_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((g[0].M + kGm - 1) / kGm, count, splits);
  tc_gemm_kernel<BN, EPI><<<grid, kGemmThreads, smem, s>>>(gg);
  return cudaGetLastError();
}

template <int BN, int EPI>
static cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t s) {
  return gemm_group<BN, EPI>(&g, 1, splits, s);
}

// ------------------------------------------------------------------ weight gradients through TMA
// The three weight-gradient products dW = A^T B of a training step (A: h3,
// h2, h1; B: dO, dz3, dz2; both row-major [row][feature], K = rows), as one
// launch of (1, 3 products, row chunks) CTAs like tc_gemm_kernel's grouped
// WGRAD launch, with the operands brought in by the tensor memory
// accelerator: per 64-row K chunk, one thread issues 2-D tiled loads of
// 8 features x 64 rows (16 bytes x 64 rows, 1 KB each) into the chunk's
// stage buffer, completing on the stage's mbarrier by transaction bytes;
// rows past the batch and features past B's width (40 -> 48) arrive as
// zeros.  Feature group g lands at g x 1 KB, so core matrix (K group kg,
// feature group g) sits at g x 1024 + kg x 128: MN-major operands whose K
// groups are 128 bytes apart and feature groups 1024.  Two stages: chunk
// c + 2 is loaded once the MMAs of chunk c have completed (their commit's
// mbarrier).  Every wait is bounded; a wait that gives up sets *err, waits
// once more (bounded) for the loads and MMAs in flight, frees the TMEM and
// skips the epilogue.  The epilogue is tc_gemm_kernel's: accumulator rows
// through shared memory, added to dW with 16-byte vector atomics.
struct alignas(64) WgradTma {
  CUtensorMap a[3];   // h3, h2, h1: [rows][128]
  CUtensorMap b[3];   // dO [rows][40], dz3, dz2 [rows][128]
  float* of[3];       // dW4 [128][40], dW3, dW2 [128][128] (added to)
  int n[3];           // columns of B (and of dW)
  int K;              // rows
  int k_chunk;        // rows per CTA (a multiple of 64)
  int* err;
  uint32_t spin;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar) : "memory");
}

__global__ void __launch_bounds__(kGemmThreads) tc_wgrad_tma_kernel(const __grid_constant__ WgradTma p) {
  using L = TcGemmSmem<128>;
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char* gsm = gsm_raw + ((1024 - (smem_u32(gsm_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t full[2], mdone[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok, s_last;
  const int y = blockIdx.y;
  const CUtensorMap* ta = &p.a[y];
  const CUtensorMap* tb = &p.b[y];
  const int N = p.n[y];
  const int nb = min(128, (N + 15) & ~15);   // B tile width (a multiple of 16 for M = 128)
  const int nbg = nb / 8;
  const uint32_t bytes = (uint32_t)(kGm / 8 + nbg) * 1024u;
  const int k_begin = blockIdx.z * p.k_chunk;
  const int k_end = min(p.K, k_begin + p.k_chunk);
  const int n_chunks = k_end > k_begin ? (k_end - k_begin + kGk - 1) / kGk : 0;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mdone[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(L::tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc_idesc_mn(kGm, nb);
    int issued = 0, last = -1;
    bool ok = true;
    auto load = [&](int c) {
      const uint32_t buf = (uint32_t)(c & 1);
      const uint32_t a_s = smem_u32(gsm + buf * L::stage), b_s = a_s + (uint32_t)L::a_bytes;
      const uint32_t fb = smem_u32(&full[buf]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"(bytes) : "memory");
      const int row = k_begin + c * kGk;
      for (int g = 0; g < kGm / 8; ++g) tma_load_2d(a_s + 1024u * g, ta, 8 * g, row, fb);
      for (int g = 0; g < nbg; ++g) tma_load_2d(b_s + 1024u * g, tb, 8 * g, row, fb);
      issued = c + 1;
    };
    for (int c = 0; c < n_chunks && c < 2; ++c) load(c);
    for (int c = 0; c < n_chunks; ++c) {
      const uint32_t buf = (uint32_t)(c & 1);
      if (!(ok = tc_wait(smem_u32(&full[buf]), (uint32_t)((c >> 1) & 1), p.spin))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_s = smem_u32(gsm + buf * L::stage), b_s = a_s + (uint32_t)L::a_bytes;
#pragma unroll
      for (int kk = 0; kk < kGk / 16; ++kk) {
        // a K = 16 step is two K groups, 128 bytes apart; feature groups 1024
        const uint64_t da = tc_desc(a_s + kk * 256, 128, 1024);
        const uint64_t db = tc_desc(b_s + kk * 256, 128, 1024);
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
            :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mdone[buf])));
      last = c;
      if (c + 2 < n_chunks) {
        // the buffer is free once chunk c's MMAs have read it
        if (!(ok = tc_wait(smem_u32(&mdone[buf]), (uint32_t)((c >> 1) & 1), p.spin))) break;
        load(c + 2);
      }
    }
    if (!ok) {
      // drain: the loads issued and not consumed, then the MMAs issued
      for (int c = last + 1; c < issued; ++c) tc_wait(smem_u32(&full[c & 1]), (uint32_t)((c >> 1) & 1));
    }
    s_ok = ok ? 1 : 0;
    s_last = last;
  }
  __syncthreads();
  bool ok = s_ok != 0;
  const int last = s_last;
  // the last commit covers every MMA issued before it
  if (last >= 0) ok = __syncthreads_and(ok && tc_wait(smem_u32(&mdone[last & 1]), (uint32_t)((last >> 1) & 1), p.spin));
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(p.err, 1);
    if (last >= 0) tc_wait(smem_u32(&mdone[last & 1]), (uint32_t)((last >> 1) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float* cs = reinterpret_cast<float*>(gsm);
  const int quarter = (threadIdx.x >> 5) & 3, half = threadIdx.x >> 7;
  const int trow = quarter * 32 + (threadIdx.x & 31);
  const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16);
  if (ok) {
#pragma unroll 1
    for (int c0 = 16 * half; c0 < nb; c0 += 32) {
      float v[16];
      if (n_chunks > 0) tc_ld16(tlane + c0, v);
      else for (int j = 0; j < 16; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(cs + (size_t)trow * L::ldc + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
  __syncthreads();
  if (ok) {
    // four adjacent columns per vector atomic (N a multiple of 4, rows of dW 16-byte aligned)
    const int nq = N >> 2;
    float* of = p.of[y];
    for (int e = threadIdx.x; e < kGm * nq; e += blockDim.x) {
      const int r = e / nq, gn = 4 * (e % nq);
      const float4 v = *reinterpret_cast<const float4*>(cs + (size_t)r * L::ldc + gn);
      if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
        atomicAdd(reinterpret_cast<float4*>(of + (size_t)r * N + gn), v);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(L::tmem_cols));
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// A row-major [rows][cols] BF16 array as a 2-D tensor map with 8 x 64 boxes
// (16 bytes of a row, 64 rows), no swizzle, zeros outside.
static bool encode_rows(CUtensorMap* m, const bf16* base, int cols, int rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || rows < 1 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || (cols * sizeof(bf16)) % 16 != 0)
    return false;
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)cols * sizeof(bf16)};
  const cuuint32_t box[2] = {8, (cuuint32_t)kGk};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Bias + SiLU of this thread's accumulator row, written back as its BF16
// activation row (core-matrix layout) for the next layer; `hbias` holds the
// halved biases (silu_fast_hb).
__device__ __forceinline__ void tc_hidden_epilogue(uint32_t taddr, const float* hbias, unsigned char* H,
                                                   int row) {
#pragma unroll 1
  for (int c0 = 0; c0 < kHid; c0 += 16) {
    float v[16], hb[16];
    tc_ld16(taddr + c0, v);
#pragma unroll
    for (int q = 0; q < 4; ++q)   // 16-byte loads of the halved biases (hbias 16-byte aligned)
      *reinterpret_cast<float4*>(hb + 4 * q) = *reinterpret_cast<const float4*>(hbias + c0 + 4 * q);
    uint32_t p[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      p[j] = pack_bf16(silu_fast_hb(v[2 * j], hb[2 * j]), silu_fast_hb(v[2 * j + 1], hb[2 * j + 1]));
    *reinterpret_cast<uint4*>(H + core_off(row, c0)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4*>(H + core_off(row, c0 + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
  }
}

__global__ void __launch_bounds__(kTcGroups * 128, 1)
    prop_tc_kernel(const DevInstrument I, uint64_t begin, uint64_t n, uint64_t seed, PropConst pc,
                   const float* __restrict__ P, const bf16* __restrict__ gw2, const bf16* __restrict__ gw3,
                   const bf16* __restrict__ gw4, float* __restrict__ st, uint64_t ld, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the operand tiles
  unsigned char* smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* W2t = smem;
  unsigned char* W3t = W2t + kTcTile;
  unsigned char* W4t = W3t + kTcTile;
  float* W1 = reinterpret_cast<float*>(W4t + (size_t)kHeadN * kHid * sizeof(bf16));
  float* B1 = W1 + 4 * kHid;
  float* B2 = B1 + kHid;
  float* B3 = B2 + kHid;
  float* B4 = B3 + kHid;
  unsigned char* tiles = smem + kTcTilesOff;
  __shared__ __align__(8) uint64_t mbar[kTcGroups];
  __shared__ uint32_t tmem_base;
  __shared__ DevComp S;

  // weights, transposed to [out][in] in the core-matrix layout; head rows
  // kOut..kHeadN-1 are zero
  for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
    const int k = i / kHid, j = i % kHid;   // W[k][j]: input k, output j
    *reinterpret_cast<bf16*>(W2t + core_off(j, k)) = gw2[i];
    *reinterpret_cast<bf16*>(W3t + core_off(j, k)) = gw3[i];
  }
  for (int i = threadIdx.x; i < kHeadN * kHid; i += blockDim.x) {
    const int j = i / kHid, k = i % kHid;
    *reinterpret_cast<bf16*>(W4t + core_off(j, k)) =
        j < kOut ? gw4[k * kOut + j] : __float2bfloat16(0.f);
  }
  for (int i = threadIdx.x; i < 4 * kHid; i += blockDim.x) W1[i] = P[kOffW1 + i];
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    B1[i] = P[kOffB1 + i];
    B2[i] = 0.5f * P[kOffB2 + i];   // halved: silu_fast_hb
    B3[i] = 0.5f * P[kOffB3 + i];
  }
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) B4[i] = P[kOffB4 + i];
  if (threadIdx.x == 0) {
    S = I.comps[0];
    for (int g = 0; g < kTcGroups; ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[g])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {   // warp 0 allocates every group's 128 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(kTcGroups * 128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const int group = threadIdx.x >> 7, row = threadIdx.x & 127, warp_q = (threadIdx.x >> 5) & 3;
  const uint32_t tmem = tmem_base + (uint32_t)(group * 128);
  const uint32_t tlane = tmem + ((uint32_t)(warp_q * 32) << 16);   // this warp's TMEM lanes
  unsigned char* H = tiles + (size_t)group * kTcTile;
  const uint32_t h_smem = smem_u32(H), mb = smem_u32(&mbar[group]);
  const uint32_t w2s = smem_u32(W2t), w3s = smem_u32(W3t), w4s = smem_u32(W4t);
  uint32_t phase = 0;
  bool ok = true;
  const uint64_t n_tiles = (n + 127) / 128;
  for (uint64_t tile = (uint64_t)blockIdx.x * kTcGroups + group; tile < n_tiles && ok;
       tile += (uint64_t)gridDim.x * kTcGroups) {
    const uint64_t r = tile * 128 + row;
    RayStream rs;
    float sx, sy, tx, ty, E;
    rs.init(begin + r, (uint32_t)I.instr_id, seed);
    sample_start<float>(S, rs, sx, sy, tx, ty, E);
    const float x0 = (sx - pc.shift[0]) * pc.scale[0], x1 = (sy - pc.shift[1]) * pc.scale[1];
    const float x2 = (E - pc.shift[2]) * pc.scale[2], x3 = (pc.angle - pc.shift[3]) * pc.scale[3];
    // layer 1 on the CUDA cores: this ray's 128 hidden units, the weights of
    // four units per 16-byte shared-memory load
#pragma unroll 1
    for (int j0 = 0; j0 < kHid; j0 += 8) {
      float h[8];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int j = j0 + 4 * q;
        const float4 a0 = *reinterpret_cast<const float4*>(W1 + j);
        const float4 a1 = *reinterpret_cast<const float4*>(W1 + kHid + j);
        const float4 a2 = *reinterpret_cast<const float4*>(W1 + 2 * kHid + j);
        const float4 a3 = *reinterpret_cast<const float4*>(W1 + 3 * kHid + j);
        const float4 b = *reinterpret_cast<const float4*>(B1 + j);
        // weight-only arithmetic (the network's output is no count): fused
        h[4 * q + 0] = silu_fast(fmaf(x3, a3.x, fmaf(x2, a2.x, fmaf(x1, a1.x, fmaf(x0, a0.x, b.x)))));
        h[4 * q + 1] = silu_fast(fmaf(x3, a3.y, fmaf(x2, a2.y, fmaf(x1, a1.y, fmaf(x0, a0.y, b.y)))));
        h[4 * q + 2] = silu_fast(fmaf(x3, a3.z, fmaf(x2, a2.z, fmaf(x1, a1.z, fmaf(x0, a0.z, b.z)))));
        h[4 * q + 3] = silu_fast(fmaf(x3, a3.w, fmaf(x2, a2.w, fmaf(x1, a1.w, fmaf(x0, a0.w, b.w)))));
      }
      uint32_t p[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) p[q] = pack_bf16(h[2 * q], h[2 * q + 1]);
      *reinterpret_cast<uint4*>(H + core_off(row, j0)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
    // layers 2 and 3
#pragma unroll 1
    for (int layer = 0; layer < 2 && ok; ++layer) {
      tc_group_sync(group);
      if (row == 0) tc_layer(tmem, h_smem, layer == 0 ? w2s : w3s, kHid, mb);
      ok = tc_group_all(group, tc_wait(mb, phase, pc.spin));
      if (!ok) tc_wait(mb, phase);   // drain: the layer's MMAs finish before TMEM is freed
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) tc_hidden_epilogue(tlane, layer == 0 ? B2 : B3, H, row);
    }
    if (!ok) break;
    // head, then the mixture sample of this thread's ray
    tc_group_sync(group);
    if (row == 0) tc_layer(tmem, h_smem, w4s, kHeadN, mb);
    ok = tc_group_all(group, tc_wait(mb, phase, pc.spin));
    if (!ok) tc_wait(mb, phase);     // drain, as above
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;
    float o[kHeadN];
#pragma unroll
    for (int c0 = 0; c0 < kHeadN; c0 += 16) tc_ld16(tlane + c0, o + c0);
#pragma unroll
    for (int c = 0; c < kOut; ++c) o[c] += B4[c];
    if (r < n) write_mixture_start(S, pc, rs, o, sx, sy, E, st, ld, r);
  }
  if (!ok && row == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_base), "r"(kTcGroups * 128));
}

// ------------------------------------------------------------------ fused training tile
// One training step's row-parallel work, fused per 128-row tile (one row
// per TMEM lane, four warps per lane quarter splitting the columns, one CTA
// per SM, persistent over tiles):
//   layer 1 on the CUDA cores -> BF16 h1 in shared memory;
//   layers 2, 3 and the head as tcgen05.mma (FP32 accumulators kept in TMEM:
//     the backward pass rereads the pre-activations z2, z3 from there);
//   the mixture loss and its output gradient dO on the CUDA cores, the four
//     warps of a lane quarter taking two mixture components each;
//   the input-gradient chain dz3 = (dO W4^T) silu'(z3), dz2 = (dz3 W3^T)
//     silu'(z2), dz1 = (dz2 W2^T) silu'(z1) as tcgen05.mma, z1 recomputed
//     from the four inputs;
//   the bias gradients of layers 1-3 and the first layer's weight gradient
//     as tcgen05.mma over the tile's rows: [x, 1]^T dz for dz3, dz2 (their
//     ones column gives the b3, b2 gradients) and dz1 (W1 and b1).  Both
//     operands are read MN-major: dz in H is [row][unit] with the units
//     contiguous, so read as its transpose it is MN-major for M = unit,
//     K = row; likewise the [row][x0..x3, 1, 0 ..] tile for N = 16.  The
//     products accumulate in TMEM over all of the CTA's tiles;
//   the head-bias gradient reduced over rows in registers (a warp-transposing
//     butterfly) and summed per CTA in shared memory.
// Each weight matrix W[in][out] is held once in shared memory, as the
// core-matrix tile of its row-major layout: the forward products read it as
// an MN-major B operand (N = out, K = in), the backward ones as a K-major
// B operand (N = in, K = out).
// Activations and output gradients that the weight-gradient GEMMs contract
// over the rows (h1, h2, h3, dO, dz3, dz2, BF16) go to global memory
// row-major ([row][feature]) straight from the epilogues.
// TMEM columns (512): z2 [0, 128), z3 [128, 256), head [256, 304); then
// dz3 [256, 384), dz2 [128, 256), dz1 [0, 128) as each earlier value is used;
// for the whole kernel [x, 1]^T dz1 [384, 400), [x, 1]^T dz3 [400, 416) and
// [x, 1]^T dz2 [416, 432).
constexpr int kDoK = 48;                                              // head width padded to 16
constexpr int kXaN = 16;                                              // [x0..x3, 1, 0 ...]
constexpr size_t kTrW2 = 0, kTrW3 = kTrW2 + kTcTile, kTrW4 = kTrW3 + kTcTile;
constexpr size_t kTrH = kTrW4 + (size_t)kHid * kDoK * sizeof(bf16);
constexpr size_t kTrDo = kTrH + kTcTile;
constexpr size_t kTrXa = kTrDo + (size_t)kHid * kDoK * sizeof(bf16);
constexpr size_t kTrF = kTrXa + (size_t)128 * kXaN * sizeof(bf16);    // floats from here
constexpr int kTrNF = 4 * kHid + 3 * kHid + kDoK;                      // W1, b1..b3, b4
constexpr int kTrNR = kDoK;                                            // per-CTA b4 gradient
constexpr size_t kTrSmem = 1024 + kTrF + (size_t)(kTrNF + kTrNR) * sizeof(float);
static_assert(kTrH % 1024 == 0 && kTrDo % 1024 == 0 && kTrXa % 1024 == 0 && kTrF % 16 == 0,
              "operand tiles 1024-aligned, floats 16-aligned");
static_assert(kOut == 5 * kComp && kComp == 8, "four warps of a lane quarter, two components each");

// byte offset of element (row, k) in a K = 48 K-major core-matrix tile
__device__ __forceinline__ int core_off48(int row, int k) {
  return (((row >> 3) * (kDoK / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// Issue D[tmem] = A B^T over `ksteps` K = 16 steps (the caller commits): A a
// 128-row K-major core-matrix tile whose 8-row groups are a_sbo bytes apart;
// B K-major (b_mn false: its 8-row groups b_stride apart) or MN-major (b_mn:
// core matrices adjacent in K b_stride apart, in N 128 B).
__device__ __forceinline__ void tc_issue(uint32_t tmem, uint32_t a, uint32_t a_sbo, uint32_t b, uint32_t b_stride,
                                         bool b_mn, int n, int ksteps) {
  const uint32_t idesc = tc_idesc(128, n) | (b_mn ? (1u << 16) : 0u);
  for (int kk = 0; kk < ksteps; ++kk) {
    const uint64_t da = tc_desc(a + kk * 256, 128, a_sbo);
    const uint64_t db = b_mn ? tc_desc(b + kk * 2 * b_stride, b_stride, 128) : tc_desc(b + kk * 256, 128, b_stride);
    const uint32_t acc = kk > 0 ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
  }
}

// Issue D[tmem] (+)= A^T B over the tile's 128 rows, A = the [row][unit] H
// tile (M = 128 units), B = the [row][16] XA tile (N = 16), both read
// MN-major: core matrices adjacent in K (rows) are 16 x 128 B (A) and
// 2 x 128 B (B) apart, those adjacent in M (N) 128 B.  acc = 0 on the first
// K step of the CTA's first tile only.
__device__ __forceinline__ void tc_issue_xt(uint32_t tmem, uint32_t a, uint32_t b, bool first) {
  const uint32_t idesc = tc_idesc_mn(128, kXaN);
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t da = tc_desc(a + kk * 2 * 2048, 2048, 128);
    const uint64_t db = tc_desc(b + kk * 2 * (kXaN / 8) * 128, (kXaN / 8) * 128, 128);
    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar));
}

// Lane l of the warp receives the sum over the warp's lanes of v[l mod N]
// (N = 32 or 16): a butterfly that halves the vector at each step, then for
// N = 16 one exchange between the two half-warps.
template <int N>
__device__ __forceinline__ float warp_transpose_sum(float v[N]) {
  static_assert(N == 32 || N == 16, "N = 32 or 16");
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int s = N / 2; s >= 1; s >>= 1) {
    const bool up = (lane & (unsigned)s) != 0u;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return N == 32 ? v[0] : v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Layer-1 pre-activations of units j0 .. j0 + 7 (j0 a multiple of 4) for
// input x, from W1 [4][kHid] and b1 in shared memory, 16-byte loads.
__device__ __forceinline__ void z1_of8(const float4 x, const float* W1, const float* B1, int j0, float z[8]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = j0 + 4 * h;
    const float4 w0 = *reinterpret_cast<const float4*>(W1 + j);
    const float4 w1 = *reinterpret_cast<const float4*>(W1 + kHid + j);
    const float4 w2 = *reinterpret_cast<const float4*>(W1 + 2 * kHid + j);
    const float4 w3 = *reinterpret_cast<const float4*>(W1 + 3 * kHid + j);
    const float4 b = *reinterpret_cast<const float4*>(B1 + j);
    z[4 * h + 0] = ((x.x * w0.x + x.y * w1.x) + (x.z * w2.x + x.w * w3.x)) + b.x;
    z[4 * h + 1] = ((x.x * w0.y + x.y * w1.y) + (x.z * w2.y + x.w * w3.y)) + b.y;
    z[4 * h + 2] = ((x.x * w0.z + x.y * w1.z) + (x.z * w2.z + x.w * w3.z)) + b.z;
    z[4 * h + 3] = ((x.x * w0.w + x.y * w1.w) + (x.z * w2.w + x.w * w3.w)) + b.w;
  }
}

struct TrainArgs {
  const float* x;          // [n][4] normalised inputs
  const float* t;          // [n][2] normalised aim points
  const float* w;          // [n] history weights
  const float* wsum;       // sum of w (device)
  int n;
  const float* P;          // FP32 parameters
  const bf16 *w2, *w3, *w4;
  // row-major operands of the weight-gradient GEMMs
  bf16 *h1, *h2, *h3;      // [n][128]
  bf16* dO;                // [n][40]
  bf16 *dz3, *dz2;         // [n][128]
  float* G;                // gradient (biases and W1 added here)
  double* loss;
  int* err;
  uint32_t spin;
};

// Eight BF16 values of row gr at column c of a row-major [n][ld] output
// (valid rows only; ld and c multiples of 8).
__device__ __forceinline__ void put8(bf16* dst, int ld, int c, int gr, bool valid, const uint32_t p[4]) {
  if (valid) *reinterpret_cast<uint4*>(dst + (size_t)gr * ld + c) = make_uint4(p[0], p[1], p[2], p[3]);
}

__device__ __forceinline__ void tr_sync_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// SiLU and its derivative for training on the fast exponential and division
// (relative error ~1e-6, far below the BF16 rounding of the activations).
__device__ __forceinline__ float silu_t(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu_t(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

constexpr int kTrThreads = 512;                      // four warps per TMEM lane quarter,
constexpr int kTrCols = kHid / (kTrThreads / 128);   // each a quarter of the columns

__global__ void __launch_bounds__(kTrThreads, 1) train_tile_kernel(const TrainArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char* sm = tsm_raw + ((1024 - (smem_u32(tsm_raw) & 1023)) & 1023);
  unsigned char* H = sm + kTrH;
  unsigned char* DO = sm + kTrDo;
  unsigned char* XA = sm + kTrXa;
  float* W1 = reinterpret_cast<float*>(sm + kTrF);
  float* B1 = W1 + 4 * kHid;
  float* B2 = B1 + kHid;
  float* B3 = B2 + kHid;
  float* B4 = B3 + kHid;                   // kDoK entries, 40.. zero
  float* R4 = B4 + kDoK;                   // per-CTA b4 gradient [kDoK]
  float* ELL = reinterpret_cast<float*>(H);   // loss stage: [row][kComp] log terms (H is free then)
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;

  // weights W[in][out] as the core-matrix tiles of their row-major layouts,
  // 8 outputs (16 bytes) per copy; the DO tile zeroed (columns 40.. stay 0)
  for (int i = threadIdx.x; i < kHid * (kHid / 8); i += blockDim.x) {
    const int k = i / (kHid / 8), j = 8 * (i % (kHid / 8));
    *reinterpret_cast<uint4*>(sm + kTrW2 + core_off(k, j)) = *reinterpret_cast<const uint4*>(a.w2 + k * kHid + j);
    *reinterpret_cast<uint4*>(sm + kTrW3 + core_off(k, j)) = *reinterpret_cast<const uint4*>(a.w3 + k * kHid + j);
  }
  for (int i = threadIdx.x; i < kHid * (kDoK / 8); i += blockDim.x) {
    const int k = i / (kDoK / 8), j = 8 * (i % (kDoK / 8));
    const uint4 v = j < kOut ? *reinterpret_cast<const uint4*>(a.w4 + k * kOut + j) : make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sm + kTrW4 + core_off48(k, j)) = v;
    *reinterpret_cast<uint4*>(DO + core_off48(k, j)) = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int i = threadIdx.x; i < 4 * kHid; i += blockDim.x) W1[i] = a.P[kOffW1 + i];
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    B1[i] = a.P[kOffB1 + i];
    B2[i] = a.P[kOffB2 + i];
    B3[i] = a.P[kOffB3 + i];
  }
  for (int i = threadIdx.x; i < kDoK; i += blockDim.x) {
    B4[i] = i < kOut ? a.P[kOffB4 + i] : 0.f;
    R4[i] = 0.f;
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tr_sync_to_async();
  const uint32_t tmem = tmem_base;
  // warp w reads TMEM lanes 32 (w mod 4) ..: row = its lane there; the four
  // warps of a lane quarter take the column slices [kTrCols part, + kTrCols)
  const int lane = threadIdx.x & 31, quarter = (threadIdx.x >> 5) & 3, part = threadIdx.x >> 7;
  const int row = quarter * 32 + lane, cb = part * kTrCols;
  const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t h_s = smem_u32(H), do_s = smem_u32(DO), xa_s = smem_u32(XA), mb = smem_u32(&mbar);
  const uint32_t w2s = smem_u32(sm + kTrW2), w3s = smem_u32(sm + kTrW3), w4s = smem_u32(sm + kTrW4);
  constexpr uint32_t kZ2 = 0, kZ3 = 128, kHd = 256, kD3 = 256, kD2 = 128, kD1 = 0;
  constexpr uint32_t kX1 = 384, kX3 = 400, kX2 = 416;
  const float wsum = *a.wsum;
  uint32_t phase = 0;
  bool ok = true;
  double loss = 0.0;
  // wait for the MMAs just committed; on a wait that gives up, drain them
  // with the full limit (so that TMEM is not freed under them) and stop
  auto wait_mma = [&]() {
    const bool done = tc_wait(mb, phase, a.spin);
    if (!done) tc_wait(mb, phase);
    ok = __syncthreads_and(done) != 0;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  };
  const int n_tiles = (a.n + 127) / 128;
  // this thread's row inputs, loaded one tile ahead
  float4 xn = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 tn = make_float2(0.f, 0.f);
  float wn = 0.f;
  auto fetch = [&](int tile) {
    const int g = tile * 128 + row;
    if (tile < n_tiles && g < a.n) {
      xn = reinterpret_cast<const float4*>(a.x)[g];
      tn = reinterpret_cast<const float2*>(a.t)[g];
      wn = a.w[g];
    }
  };
  fetch(blockIdx.x);
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const bool first = tile == (int)blockIdx.x;
    const int r0 = tile * 128, gr = r0 + row;
    const bool valid = gr < a.n;
    const float4 x = valid ? xn : make_float4(0.f, 0.f, 0.f, 0.f);
    const float tu = tn.x, tv = tn.y, wr = wn;
    fetch(tile + gridDim.x);
    if (part == 0) {
      // row `row` of the MN-major [row][16] tile [x0..x3, 1, 0 ..] (zero for
      // rows past n): columns 0..7, then 8..15
      unsigned char* xr = XA + (((row >> 3) * (kXaN / 8)) << 7) + ((row & 7) << 4);
      const float one = valid ? 1.f : 0.f;
      *reinterpret_cast<uint4*>(xr) = make_uint4(pack_bf16(x.x, x.y), pack_bf16(x.z, x.w), pack_bf16(one, 0.f), 0u);
      *reinterpret_cast<uint4*>(xr + 128) = make_uint4(0u, 0u, 0u, 0u);
    }
    // layer 1 (the expression of layer1_kernel), this thread's kTrCols units
#pragma unroll 1
    for (int j0 = cb; j0 < cb + kTrCols; j0 += 8) {
      float h[8];
      z1_of8(x, W1, B1, j0, h);
      uint32_t p[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) p[q] = pack_bf16(silu_t(h[2 * q]), silu_t(h[2 * q + 1]));
      put8(a.h1, kHid, j0, gr, valid, p);
      *reinterpret_cast<uint4*>(H + core_off(row, j0)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
    // layers 2 and 3: z in TMEM, h in place in H
#pragma unroll 1
    for (int layer = 0; layer < 2 && ok; ++layer) {
      tr_sync_to_async();
      if (threadIdx.x == 0) {
        tc_issue(tmem + (layer == 0 ? kZ2 : kZ3), h_s, 2048, layer == 0 ? w2s : w3s, 2048, true, kHid, 8);
        tc_commit(mb);
      }
      wait_mma();
      if (!ok) break;
      const float* bias = layer == 0 ? B2 : B3;
#pragma unroll 1
      for (int c0 = 0; c0 < kTrCols; c0 += 16) {
        float v[16];
        tc_ld16(tl + (layer == 0 ? kZ2 : kZ3) + cb + c0, v);
        const int c = cb + c0;
        uint32_t p[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          p[j] = pack_bf16(silu_t(v[2 * j] + bias[c + 2 * j]), silu_t(v[2 * j + 1] + bias[c + 2 * j + 1]));
        put8(layer == 0 ? a.h2 : a.h3, kHid, c, gr, valid, p);
        put8(layer == 0 ? a.h2 : a.h3, kHid, c + 8, gr, valid, p + 4);
        *reinterpret_cast<uint4*>(H + core_off(row, c)) = make_uint4(p[0], p[1], p[2], p[3]);
        *reinterpret_cast<uint4*>(H + core_off(row, c + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
      }
    }
    if (!ok) break;
    // head
    tr_sync_to_async();
    if (threadIdx.x == 0) {
      tc_issue(tmem + kHd, h_s, 2048, w4s, (kDoK / 8) * 128, true, kDoK, 8);
      tc_commit(mb);
    }
    wait_mma();
    if (!ok) break;
    // loss and dO: every thread takes its row's log-softmax of the mixture
    // weights and the log terms of its part's two components k = 2 part,
    // 2 part + 1; the log terms are exchanged through ELL, then each thread
    // writes its components' output gradients
    {
      float o[kDoK];
#pragma unroll
      for (int c0 = 0; c0 < kDoK; c0 += 16) tc_ld16(tl + kHd + c0, o + c0);
#pragma unroll
      for (int c = 0; c < kOut; ++c) o[c] += B4[c];
      float amax = -CUDART_INF_F;
#pragma unroll
      for (int k = 0; k < kComp; ++k) amax = fmaxf(amax, o[5 * k]);
      float se = 0.f;
#pragma unroll
      for (int k = 0; k < kComp; ++k) se += __expf(o[5 * k] - amax);
      const float lse = amax + __logf(se);
      float lsu[2] = {0.f, 0.f}, lsv[2] = {0.f, 0.f}, ellk[2] = {0.f, 0.f};
#pragma unroll
      for (int k = 0; k < kComp; ++k) {
        if ((k >> 1) != part) continue;
        const int kk = k & 1;
        lsu[kk] = kLsC * tanh_e(o[5 * k + 3] / kLsC) + kLsM;
        lsv[kk] = kLsC * tanh_e(o[5 * k + 4] / kLsC) + kLsM;
        const float zu = (tu - o[5 * k + 1]) * __expf(-lsu[kk]);
        const float zv = (tv - o[5 * k + 2]) * __expf(-lsv[kk]);
        ellk[kk] = (o[5 * k] - lse) - 0.5f * zu * zu - lsu[kk] - 0.5f * zv * zv - lsv[kk] - kLog2Pi;
        ELL[row * (kComp + 1) + k] = ellk[kk];
      }
      __syncthreads();
      float mx = -CUDART_INF_F, e8[kComp];
#pragma unroll
      for (int k = 0; k < kComp; ++k) {
        e8[k] = ELL[row * (kComp + 1) + k];
        mx = fmaxf(mx, e8[k]);
      }
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kComp; ++k) s += __expf(e8[k] - mx);
      const float lq = mx + __logf(s);
      float d[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) d[c] = 0.f;
      if (valid) {
        const float om = wr / wsum;
        if (part == 0) loss += (double)(-om * lq);
#pragma unroll
        for (int k = 0; k < kComp; ++k) {
          if ((k >> 1) != part) continue;
          const int kk = k & 1;
          const float r = __expf(ellk[kk] - lq);
          const float su = __expf(lsu[kk]), sv = __expf(lsv[kk]);
          const float zu = (tu - o[5 * k + 1]) / su, zv = (tv - o[5 * k + 2]) / sv;
          const float tu_ = tanh_e(o[5 * k + 3] / kLsC), tv_ = tanh_e(o[5 * k + 4] / kLsC);
          d[5 * kk + 0] = -om * (r - __expf(o[5 * k] - lse));
          d[5 * kk + 1] = -om * (r * zu / su);
          d[5 * kk + 2] = -om * (r * zv / sv);
          d[5 * kk + 3] = -om * (r * (zu * zu - 1.f) * (1.f - tu_ * tu_));
          d[5 * kk + 4] = -om * (r * (zv * zv - 1.f) * (1.f - tv_ * tv_));
        }
      }
      // columns 10 part .. 10 part + 9, two per 4-byte store (never across
      // an 8-column group)
      const int c0 = 10 * part;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const uint32_t pr = pack_bf16(d[2 * q], d[2 * q + 1]);
        *reinterpret_cast<uint32_t*>(DO + core_off48(row, c0 + 2 * q)) = pr;
        if (valid) *reinterpret_cast<uint32_t*>(a.dO + (size_t)gr * kOut + c0 + 2 * q) = pr;
      }
      const float col = warp_transpose_sum<16>(d);
      if (lane < 10) atomicAdd(&R4[c0 + lane], col);
    }
    // dz3 = (dO W4^T) silu'(z3)
    tr_sync_to_async();
    if (threadIdx.x == 0) {
      tc_issue(tmem + kD3, do_s, (kDoK / 8) * 128, w4s, (kDoK / 8) * 128, false, kHid, kDoK / 16);
      tc_commit(mb);
    }
    wait_mma();
    if (!ok) break;
    // the backward chain through layers 3 and 2: dz = (prev) silu'(acc + b)
#pragma unroll 1
    for (int layer = 0; layer < 2 && ok; ++layer) {
      const uint32_t dcol = layer == 0 ? kD3 : kD2, zcol = layer == 0 ? kZ3 : kZ2;
      const float* bias = layer == 0 ? B3 : B2;
#pragma unroll 1
      for (int c0 = 0; c0 < kTrCols; c0 += 16) {
        float g[16], z[16];
        tc_ld16(tl + dcol + cb + c0, g);
        tc_ld16(tl + zcol + cb + c0, z);
        const int c = cb + c0;
        uint32_t p[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2)
          p[j / 2] = pack_bf16(valid ? g[j] * dsilu_t(z[j] + bias[c + j]) : 0.f,
                               valid ? g[j + 1] * dsilu_t(z[j + 1] + bias[c + j + 1]) : 0.f);
        put8(layer == 0 ? a.dz3 : a.dz2, kHid, c, gr, valid, p);
        put8(layer == 0 ? a.dz3 : a.dz2, kHid, c + 8, gr, valid, p + 4);
        *reinterpret_cast<uint4*>(H + core_off(row, c)) = make_uint4(p[0], p[1], p[2], p[3]);
        *reinterpret_cast<uint4*>(H + core_off(row, c + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
      }
      // the next input gradient (dz in H times the layer's weights
      // transposed) and [x, 1]^T dz, under one commit
      tr_sync_to_async();
      if (threadIdx.x == 0) {
        tc_issue(tmem + (layer == 0 ? kD2 : kD1), h_s, 2048, layer == 0 ? w3s : w2s, 2048, false, kHid, 8);
        tc_issue_xt(tmem + (layer == 0 ? kX3 : kX2), h_s, xa_s, first);
        tc_commit(mb);
      }
      wait_mma();
    }
    if (!ok) break;
    // dz1 = (dz2 W2^T) silu'(z1) into H (BF16)
#pragma unroll 1
    for (int c0 = 0; c0 < kTrCols; c0 += 16) {
      float g[16], z[16];
      tc_ld16(tl + kD1 + cb + c0, g);
      const int c = cb + c0;
      z1_of8(x, W1, B1, c, z);
      z1_of8(x, W1, B1, c + 8, z + 8);
      uint32_t p[8];
#pragma unroll
      for (int j = 0; j < 16; j += 2)
        p[j / 2] = pack_bf16(valid ? g[j] * dsilu_t(z[j]) : 0.f, valid ? g[j + 1] * dsilu_t(z[j + 1]) : 0.f);
      *reinterpret_cast<uint4*>(H + core_off(row, c)) = make_uint4(p[0], p[1], p[2], p[3]);
      *reinterpret_cast<uint4*>(H + core_off(row, c + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
    }
    // [x, 1]^T dz1 added in TMEM; the next tile rewrites H and XA only after
    // this product has completed (wait_mma's barrier)
    tr_sync_to_async();
    if (threadIdx.x == 0) {
      tc_issue_xt(tmem + kX1, h_s, xa_s, first);
      tc_commit(mb);
    }
    wait_mma();
  }
  if (!ok && threadIdx.x == 0) atomicExch(a.err, 1);
  // per-CTA sums into the gradient, the loss
  __syncthreads();
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) atomicAdd(&a.G[kOffB4 + i], R4[i]);
  if (ok && part < 3) {
    // TMEM lane `row` = unit `row` of the [x, 1]^T dz products: part 0 reads
    // the W1 gradient (columns 0..3, from x0..x3) and b1's (column 4), parts
    // 1 and 2 the b3 and b2 gradients (column 4); every CTA ran a tile
    float v[16];
    tc_ld16(tl + (part == 0 ? kX1 : (part == 1 ? kX3 : kX2)), v);
    if (part == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) atomicAdd(&a.G[kOffW1 + i * kHid + row], v[i]);
    }
    atomicAdd(&a.G[(part == 0 ? kOffB1 : (part == 1 ? kOffB3 : kOffB2)) + row], v[4]);
  }
  const double ls = warp_sum(loss);
  if (lane == 0) atomicAdd(a.loss, ls);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// Training rows from a history: x from the starts (the angle input from
// angle[i] when given, else pc.angle), t = (u/hu, v/hv), w = det; the sum of
// w added to *wsum (one atomic per block of 256).
__global__ void __launch_bounds__(256) history_rows_kernel(const float* __restrict__ st, uint64_t ld,
                                                           const float* __restrict__ det,
                                                           const float* __restrict__ angle, int n, PropConst pc,
                                                           float* __restrict__ x, float* __restrict__ t,
                                                           float* __restrict__ w, float* __restrict__ wsum) {
  __shared__ float part[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float wi = i < n ? det[i] : 0.f;
  const float ws = warp_sum(wi);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += part[k];
    atomicAdd(wsum, b);
  }
  if (i >= n) return;
  float4 xi;
  xi.x = (st[i] - pc.shift[0]) * pc.scale[0];
  xi.y = (st[ld + i] - pc.shift[1]) * pc.scale[1];
  xi.z = (st[2 * ld + i] - pc.shift[2]) * pc.scale[2];
  xi.w = ((angle ? angle[i] : pc.angle) - pc.shift[3]) * pc.scale[3];
  reinterpret_cast<float4*>(x)[i] = xi;
  t[2 * i] = st[3 * ld + i] / pc.hu;
  t[2 * i + 1] = st[4 * ld + i] / pc.hv;
  w[i] = wi;
}

}  // namespace mcx

using namespace mcx;

struct mcx_proposal {
  int device = 0;
  cudaStream_t stream = nullptr;
  PropConst pc{};
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  bf16 *w2 = nullptr, *w3 = nullptr, *w4 = nullptr;
  int adam_t = 0;
  // workspace for up to `cap` rows: inputs, outputs; activations h1..h3
  // and the output and hidden gradients of training, all row-major
  // [row][feature]
  int cap = 0;
  float *x = nullptr, *t = nullptr, *w = nullptr;
  bf16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
  float *o = nullptr, *wsum = nullptr;
  bf16 *dob = nullptr, *dzb = nullptr, *dzb2 = nullptr;
  double* dloss = nullptr;
  int* err = nullptr;        // set by the sampler when a tensor-core wait gave up
  // tensor maps of the weight-gradient operands, encoded for tma_rows rows
  // of the current workspace (0: none yet)
  WgradTma tma{};
  int tma_rows = 0;
};

static void prop_free_ws(mcx_proposal* Q) {
  void* bufs[] = {Q->x, Q->t, Q->w, Q->h1, Q->h2, Q->h3, Q->o, Q->wsum, Q->dob, Q->dzb, Q->dzb2, Q->dloss};
  for (void* b : bufs)
    if (b) cudaFree(b);
  Q->x = Q->t = Q->w = Q->o = Q->wsum = nullptr;
  Q->h1 = Q->h2 = Q->h3 = Q->dob = Q->dzb = Q->dzb2 = nullptr;
  Q->dloss = nullptr;
  Q->cap = 0;
  Q->tma_rows = 0;
}

static mcx_status prop_ws(mcx_proposal* Q, int n) {
  if (n <= Q->cap) return MCX_OK;
  prop_free_ws(Q);
  const size_t N = (size_t)n;
  cudaError_t e = cudaSuccess;
  auto fa = [&](float** p, size_t cnt) { if (e == cudaSuccess) e = cudaMalloc(p, cnt * sizeof(float)); };
  auto ba = [&](bf16** p, size_t cnt) { if (e == cudaSuccess) e = cudaMalloc(p, cnt * sizeof(bf16)); };
  fa(&Q->x, 4 * N); fa(&Q->t, 2 * N); fa(&Q->w, N);
  ba(&Q->h1, kHid * N); ba(&Q->h2, kHid * N); ba(&Q->h3, kHid * N);
  fa(&Q->o, kOut * N);
  fa(&Q->wsum, 64);
  ba(&Q->dob, kOut * N); ba(&Q->dzb, kHid * N); ba(&Q->dzb2, kHid * N);
  if (e == cudaSuccess) e = cudaMalloc(&Q->dloss, 64);
  if (e != cudaSuccess) {
    prop_free_ws(Q);
    return cuda_fail(e, "proposal workspace");
  }
  Q->cap = n;
  return MCX_OK;
}

// Network outputs o [n, 40] for inputs Q->x (forward through all layers).
static mcx_status prop_forward(mcx_proposal* Q, int n) {
  cudaStream_t s = Q->stream;
  const int g1 = n < 4096 ? n : 4096;
  layer1_kernel<<<g1 > 0 ? g1 : 1, 128, 0, s>>>(Q->x, n, Q->P, Q->h1);
  GemmArgs a{};
  a.err = Q->err;
  a.spin = Q->pc.spin;
  a.M = n; a.K = kHid; a.k_chunk = kHid;
  a.A = Q->h1; a.lda = kHid; a.B = Q->w2; a.ldb = kHid; a.N = kHid;
  a.bias = Q->P + kOffB2; a.of = nullptr; a.ldo = kHid; a.ob = Q->h2; a.ldob = kHid;
  cudaError_t e = gemm<128, EPI_FWD>(a, 1, s);
  a.A = Q->h2; a.B = Q->w3; a.bias = Q->P + kOffB3; a.of = nullptr; a.ob = Q->h3;
  if (e == cudaSuccess) e = gemm<128, EPI_FWD>(a, 1, s);
  GemmArgs h{};
  h.err = Q->err;
  h.spin = Q->pc.spin;
  h.M = n; h.K = kHid; h.k_chunk = kHid; h.N = kOut;
  h.A = Q->h3; h.lda = kHid; h.B = Q->w4; h.ldb = kOut; h.bias = Q->P + kOffB4; h.of = Q->o; h.ldo = kOut;
  if (e == cudaSuccess) e = gemm<48, EPI_HEAD>(h, 1, s);
  if (e != cudaSuccess) return cuda_fail(e, "proposal forward");
  return MCX_OK;
}

// Loss and gradient (into Q->G, zeroed first) of the weighted NLL on the
// rows Q->x, Q->t, Q->w; the loss is left in *Q->dloss (device).  The
// row-parallel work (forward, loss, input gradients, bias and first-layer
// gradients) runs fused per 128-row tile (train_tile_kernel); the three
// products over the rows, dW4 = h3^T dO, dW3 = h2^T dz3 and dW2 = h1^T dz2,
// are split-K tcgen05 GEMMs (K = rows in 256-row chunks, atomically added).
static cudaError_t prop_loss_grad(mcx_proposal* Q, int n, bool wsum_ready) {
  cudaStream_t s = Q->stream;
  cudaError_t e = cudaSuccess;
  if (!wsum_ready) {
    e = cudaMemsetAsync(Q->wsum, 0, sizeof(float), s);
    if (e == cudaSuccess) sum_kernel<<<64, 256, 0, s>>>(Q->w, n, Q->wsum);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->dloss, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->G, 0, sizeof(float) * kNParams, s);
  if (e != cudaSuccess) return e;
  TrainArgs ta{};
  ta.x = Q->x; ta.t = Q->t; ta.w = Q->w; ta.wsum = Q->wsum; ta.n = n;
  ta.P = Q->P; ta.w2 = Q->w2; ta.w3 = Q->w3; ta.w4 = Q->w4;
  ta.h1 = Q->h1; ta.h2 = Q->h2; ta.h3 = Q->h3; ta.dO = Q->dob; ta.dz3 = Q->dzb; ta.dz2 = Q->dzb2;
  ta.G = Q->G; ta.loss = Q->dloss; ta.err = Q->err; ta.spin = Q->pc.spin;
  e = cudaFuncSetAttribute(train_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrSmem);
  if (e != cudaSuccess) return e;
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, Q->device);
  const int tiles = (n + 127) / 128;
  train_tile_kernel<<<tiles < n_sm ? tiles : n_sm, kTrThreads, kTrSmem, s>>>(ta);
  e = cudaGetLastError();
  // weight gradients over the rows: K (= rows) split into 512-row chunks, so
  // that a batch of 65536 rows gives 128 CTAs per product (measured on the
  // 1e8-history epoch: 256-row chunks 0.238 s, 512 0.234 s, 1024 0.245 s);
  // both operands row-major [row][feature], brought in by TMA (tensor maps
  // encoded once per workspace and row count)
  const int kc = 512, splits = (n + kc - 1) / kc;
  if (e == cudaSuccess && Q->tma_rows != n) {
    const bool enc = encode_rows(&Q->tma.a[0], Q->h3, kHid, n) && encode_rows(&Q->tma.a[1], Q->h2, kHid, n) &&
                     encode_rows(&Q->tma.a[2], Q->h1, kHid, n) && encode_rows(&Q->tma.b[0], Q->dob, kOut, n) &&
                     encode_rows(&Q->tma.b[1], Q->dzb, kHid, n) && encode_rows(&Q->tma.b[2], Q->dzb2, kHid, n);
    if (!enc) return cudaErrorNotSupported;
    Q->tma_rows = n;
  }
  Q->tma.of[0] = Q->G + kOffW4;
  Q->tma.of[1] = Q->G + kOffW3;
  Q->tma.of[2] = Q->G + kOffW2;
  Q->tma.n[0] = kOut;
  Q->tma.n[1] = Q->tma.n[2] = kHid;
  Q->tma.K = n;
  Q->tma.k_chunk = kc;
  Q->tma.err = Q->err;
  Q->tma.spin = Q->pc.spin;
  if (e == cudaSuccess) {
    constexpr size_t smem = TcGemmSmem<128>::bytes;
    e = cudaFuncSetAttribute(tc_wgrad_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // the three products in one launch (gridDim.y = 3), so that they share the GPU
    if (e == cudaSuccess) tc_wgrad_tma_kernel<<<dim3(1, 3, splits), kGemmThreads, smem, s>>>(Q->tma);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  return e;
}

// MCX_ERR_TIMEOUT when a tensor-core wait of this proposal gave up (the flag
// stays set: the proposal's device state is no longer trusted).
static mcx_status tc_status(mcx_proposal* Q) {
  int bad = 0;
  cudaError_t e = cudaMemcpyAsync(&bad, Q->err, sizeof(int), cudaMemcpyDeviceToHost, Q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(Q->stream);
  if (e != cudaSuccess) return cuda_fail(e, "proposal status");
  if (bad) return fail(MCX_ERR_TIMEOUT, "a tensor-core wait of the proposal timed out");
  return MCX_OK;
}

static mcx_status check_rows(uint64_t n) {
  if (n > (1u << 24)) return fail(MCX_ERR_INVALID, "at most 2^24 rows per call");
  return MCX_OK;
}

extern "C" mcx_status mcx_proposal_create(const mcx_proposal_desc* d, const float* params,
                                          mcx_proposal** out) {
  if (!out || !d) return fail(MCX_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (!(d->alpha > 0.f && d->alpha <= 1.f)) return fail(MCX_ERR_INVALID, "alpha must be in (0, 1]");
  if (!(d->half_u > 0.f && d->half_v > 0.f)) return fail(MCX_ERR_INVALID, "window half sizes must be positive");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(d->x_shift[i]) || !std::isfinite(d->x_scale[i]))
      return fail(MCX_ERR_INVALID, "non-finite input normalisation");
  DeviceGuard guard(d->device);
  if (!guard.ok) return fail(MCX_ERR_CUDA, "cannot select device %d", d->device);
  mcx_proposal* Q = new mcx_proposal();
  Q->device = d->device;
  Q->stream = (cudaStream_t)d->stream;
  Q->pc.spin = (uint32_t)kTcSpinLimit;
  Q->pc.alpha = d->alpha;
  Q->pc.hu = d->half_u;
  Q->pc.hv = d->half_v;
  for (int i = 0; i < 4; ++i) { Q->pc.shift[i] = d->x_shift[i]; Q->pc.scale[i] = d->x_scale[i]; }
  cudaError_t e = cudaMalloc(&Q->P, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&Q->G, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&Q->Mo, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&Q->Vo, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMalloc(&Q->w2, sizeof(bf16) * kHid * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&Q->w3, sizeof(bf16) * kHid * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&Q->w4, sizeof(bf16) * kHid * kOut);
  if (e == cudaSuccess) e = cudaMalloc(&Q->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->err, 0, sizeof(int), Q->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->Mo, 0, sizeof(float) * kNParams, Q->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->Vo, 0, sizeof(float) * kNParams, Q->stream);
  if (e == cudaSuccess) {
    if (params) e = cudaMemcpyAsync(Q->P, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, Q->stream);
    else e = cudaMemsetAsync(Q->P, 0, sizeof(float) * kNParams, Q->stream);
  }
  if (e == cudaSuccess) {
    to_bf16_kernel<<<64, 256, 0, Q->stream>>>(Q->P, Q->w2, Q->w3, Q->w4);
    e = cudaStreamSynchronize(Q->stream);
  }
  if (e != cudaSuccess) {
    mcx_status st = cuda_fail(e, "proposal create");
    mcx_proposal_destroy(Q);
    return st;
  }
  *out = Q;
  return MCX_OK;
}

extern "C" void mcx_proposal_destroy(mcx_proposal* Q) {
  if (!Q) return;
  DeviceGuard guard(Q->device);
  cudaStreamSynchronize(Q->stream);
  prop_free_ws(Q);
  void* bufs[] = {Q->P, Q->G, Q->Mo, Q->Vo, Q->w2, Q->w3, Q->w4, Q->err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete Q;
}

extern "C" mcx_status mcx_proposal_set_params(mcx_proposal* Q, const float* params) {
  if (!Q || !params) return fail(MCX_ERR_INVALID, "NULL argument");
  DeviceGuard guard(Q->device);
  cudaError_t e = cudaMemcpyAsync(Q->P, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, Q->stream);
  if (e == cudaSuccess) {
    to_bf16_kernel<<<64, 256, 0, Q->stream>>>(Q->P, Q->w2, Q->w3, Q->w4);
    cudaMemsetAsync(Q->Mo, 0, sizeof(float) * kNParams, Q->stream);
    cudaMemsetAsync(Q->Vo, 0, sizeof(float) * kNParams, Q->stream);
    Q->adam_t = 0;
    e = cudaStreamSynchronize(Q->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "set params");
  return MCX_OK;
}

extern "C" mcx_status mcx_proposal_get_params(mcx_proposal* Q, float* params) {
  if (!Q || !params) return fail(MCX_ERR_INVALID, "NULL argument");
  DeviceGuard guard(Q->device);
  cudaError_t e = cudaMemcpyAsync(params, Q->P, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, Q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(Q->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get params");
  return MCX_OK;
}

extern "C" mcx_status mcx_proposal_forward(mcx_proposal* Q, const float* d_x, uint64_t n, float* d_out) {
  if (!Q || ((!d_x || !d_out) && n)) return fail(MCX_ERR_INVALID, "NULL argument");
  if (check_rows(n) != MCX_OK) return MCX_ERR_INVALID;
  if (n == 0) return MCX_OK;
  DeviceGuard guard(Q->device);
  mcx_status st = prop_ws(Q, (int)n);
  if (st != MCX_OK) return st;
  cudaMemcpyAsync(Q->x, d_x, sizeof(float) * 4 * n, cudaMemcpyDeviceToDevice, Q->stream);
  st = prop_forward(Q, (int)n);
  if (st != MCX_OK) return st;
  cudaError_t e = cudaMemcpyAsync(d_out, Q->o, sizeof(float) * kOut * n, cudaMemcpyDeviceToDevice, Q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(Q->stream);
  if (e != cudaSuccess) return cuda_fail(e, "proposal forward");
  return tc_status(Q);
}

extern "C" mcx_status mcx_proposal_loss_grad(mcx_proposal* Q, const float* d_x, const float* d_t,
                                             const float* d_w, uint64_t n, double* loss, float* grad) {
  if (!Q || !d_x || !d_t || !d_w || n == 0) return fail(MCX_ERR_INVALID, "NULL argument or n = 0");
  if (check_rows(n) != MCX_OK) return MCX_ERR_INVALID;
  DeviceGuard guard(Q->device);
  mcx_status st = prop_ws(Q, (int)n);
  if (st != MCX_OK) return st;
  cudaMemcpyAsync(Q->x, d_x, sizeof(float) * 4 * n, cudaMemcpyDeviceToDevice, Q->stream);
  cudaMemcpyAsync(Q->t, d_t, sizeof(float) * 2 * n, cudaMemcpyDeviceToDevice, Q->stream);
  cudaMemcpyAsync(Q->w, d_w, sizeof(float) * n, cudaMemcpyDeviceToDevice, Q->stream);
  cudaError_t e = prop_loss_grad(Q, (int)n, false);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, Q->dloss, sizeof(double), cudaMemcpyDeviceToHost, Q->stream);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, Q->G, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, Q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(Q->stream);
  if (e != cudaSuccess) return cuda_fail(e, "proposal loss/grad");
  return tc_status(Q);
}

// Adam over mini-batches of `batch` consecutive rows of a history (a
// trailing partial batch is skipped); per-row angles when d_angle is given.
static mcx_status prop_train(mcx_proposal* Q, const float* d_starts, const float* d_det, const float* d_angle,
                             uint64_t n, float angle, const mcx_train_opts* o, double* last_loss) {
  if (!Q || !d_starts || !d_det || !o || n == 0) return fail(MCX_ERR_INVALID, "NULL argument or n = 0");
  if (o->batch < 128 || o->batch > (1u << 20)) return fail(MCX_ERR_INVALID, "batch must be in [128, 2^20]");
  if (!(o->lr > 0.f)) return fail(MCX_ERR_INVALID, "lr must be positive");
  DeviceGuard guard(Q->device);
  const int B = (int)o->batch;
  mcx_status st = prop_ws(Q, B);
  if (st != MCX_OK) return st;
  PropConst pc = Q->pc;
  pc.angle = angle;
  cudaError_t e = cudaSuccess;
  for (uint32_t ep = 0; ep < o->epochs && e == cudaSuccess; ++ep) {
    for (uint64_t b0 = 0; b0 + (uint64_t)B <= n && e == cudaSuccess; b0 += B) {
      e = cudaMemsetAsync(Q->wsum, 0, sizeof(float), Q->stream);
      if (e != cudaSuccess) break;
      history_rows_kernel<<<(B + 255) / 256, 256, 0, Q->stream>>>(d_starts + b0, n, d_det + b0,
                                                                  d_angle ? d_angle + b0 : nullptr, B, pc,
                                                                  Q->x, Q->t, Q->w, Q->wsum);
      e = prop_loss_grad(Q, B, true);
      if (e != cudaSuccess) break;
      ++Q->adam_t;
      const float c1 = 1.f - powf(o->beta1, (float)Q->adam_t);
      const float c2 = 1.f - powf(o->beta2, (float)Q->adam_t);
      adam_kernel<<<64, 256, 0, Q->stream>>>(Q->P, Q->G, Q->Mo, Q->Vo, o->lr, o->beta1, o->beta2, o->eps,
                                             c1, c2, Q->w2, Q->w3, Q->w4);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && last_loss) e = cudaMemcpyAsync(last_loss, Q->dloss, sizeof(double), cudaMemcpyDeviceToHost, Q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(Q->stream);
  if (e != cudaSuccess) return cuda_fail(e, "proposal train");
  return tc_status(Q);
}

extern "C" mcx_status mcx_proposal_train(mcx_proposal* Q, const float* d_starts, const float* d_det,
                                         uint64_t n, float angle, const mcx_train_opts* o,
                                         double* last_loss) {
  return prop_train(Q, d_starts, d_det, nullptr, n, angle, o, last_loss);
}

extern "C" mcx_status mcx_proposal_train_angles(mcx_proposal* Q, const float* d_starts, const float* d_det,
                                                const float* d_angle, uint64_t n, const mcx_train_opts* o,
                                                double* last_loss) {
  if (!d_angle) return fail(MCX_ERR_INVALID, "d_angle is NULL");
  return prop_train(Q, d_starts, d_det, d_angle, n, 0.f, o, last_loss);
}

cudaError_t mcx::proposal_sample_async(mcx_proposal* Q, const DevInstrument& d, uint64_t begin, uint64_t n,
                                       uint64_t seed, float angle, float* d_starts, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  PropConst pc = Q->pc;
  pc.angle = angle;
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, Q->device);
  cudaError_t e = cudaFuncSetAttribute(prop_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = (n + 127) / 128;
  const uint64_t blocks = (tiles + kTcGroups - 1) / kTcGroups;
  const unsigned grid = (unsigned)(blocks < (uint64_t)n_sm ? blocks : (uint64_t)n_sm);
  prop_tc_kernel<<<grid, kTcGroups * 128, kTcSmem, s>>>(d, begin, n, seed, pc, Q->P, Q->w2, Q->w3, Q->w4,
                                                        d_starts, n, Q->err);
  return cudaGetLastError();
}

mcx_status mcx::proposal_check(mcx_proposal* Q, cudaStream_t s) {
  int bad = 0;
  cudaError_t e = cudaMemcpyAsync(&bad, Q->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "proposal status");
  if (bad) return fail(MCX_ERR_TIMEOUT, "an earlier proposal sample timed out waiting for the tensor cores");
  return MCX_OK;
}

extern "C" mcx_status mcx_proposal_set_wait_limit(mcx_proposal* Q, int64_t polls) {
  if (!Q) return fail(MCX_ERR_INVALID, "proposal is NULL");
  Q->pc.spin = polls < 0 ? (uint32_t)kTcSpinLimit : (uint32_t)(polls < kTcSpinLimit ? polls : kTcSpinLimit);
  return MCX_OK;
}

extern "C" mcx_status mcx_proposal_attach(mcx_instrument* I, mcx_proposal* Q, float angle) {
  if (!I) return fail(MCX_ERR_INVALID, "instrument is NULL");
  if (!Q) {
    I->prop = nullptr;
    return MCX_OK;
  }
  if (I->precision != MCX_PREC_MIXED) return fail(MCX_ERR_UNSUPPORTED, "the proposal feeds the mixed form");
  if (I->scatter)
    return fail(MCX_ERR_UNSUPPORTED, "a scattering phantom draws from the ray's own stream, which given starts lack");
  if (I->device != Q->device) return fail(MCX_ERR_INVALID, "proposal and instrument on different devices");
  if (!(angle == angle)) return fail(MCX_ERR_INVALID, "angle is not a number");
  DeviceGuard guard(I->device);
  if (!I->prop_buf) {
    I->prop_buf = (float*)instrument_alloc(I, sizeof(float) * 6 * kPropChunk);
    if (!I->prop_buf) return fail(MCX_ERR_OOM, "proposal start buffer");
  }
  I->prop = Q;
  I->prop_angle = angle;
  return MCX_OK;
}

extern "C" mcx_status mcx_proposal_sample(mcx_proposal* Q, mcx_instrument* I, uint64_t ray_begin,
                                          uint64_t n, uint64_t seed, float angle, float* d_starts) {
  if (!Q || !I || (!d_starts && n)) return fail(MCX_ERR_INVALID, "NULL argument");
  if (I->precision != MCX_PREC_MIXED) return fail(MCX_ERR_UNSUPPORTED, "the proposal feeds the mixed form");
  if (I->device != Q->device) return fail(MCX_ERR_INVALID, "proposal and instrument on different devices");
  if (ray_begin + n < ray_begin || ray_begin + n > (1ull << 62))
    return fail(MCX_ERR_INVALID, "ray ids must stay below 2^62");
  if (n == 0) return MCX_OK;
  DeviceGuard guard(Q->device);
  PropConst pc = Q->pc;
  pc.angle = angle;
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, Q->device);
  // a tensor-core wait that gave up in an earlier call is reported here
  int bad = 0;
  cudaError_t e = cudaMemcpyAsync(&bad, Q->err, sizeof(int), cudaMemcpyDeviceToHost, I->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return cuda_fail(e, "proposal sample");
  if (bad) return fail(MCX_ERR_TIMEOUT, "an earlier proposal sample timed out waiting for the tensor cores");
  cudaFuncSetAttribute(prop_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  const uint64_t tiles = (n + 127) / 128;
  const uint64_t blocks = (tiles + kTcGroups - 1) / kTcGroups;
  const unsigned grid = (unsigned)(blocks < (uint64_t)n_sm ? blocks : (uint64_t)n_sm);
  prop_tc_kernel<<<grid, kTcGroups * 128, kTcSmem, I->stream>>>(
      I->dev, ray_begin, n, seed, pc, Q->P, Q->w2, Q->w3, Q->w4, d_starts, n, Q->err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "proposal sample");
  return MCX_OK;
}
