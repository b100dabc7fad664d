// The learned cost predictor / surrogate network: a multilayer perceptron
// n_in -> 256 -> 256 -> 256 -> n_out with SiLU, trained and run on the GPU by
// the kernels below. Every contraction runs on the fifth-generation tensor
// cores (tcgen05.mma, kind::f16) in BF16 with the FP32 accumulator in tensor
// memory: inference as one whole-network kernel per 128-row tile, training
// layer by layer (FP32 master weights and activations are rounded to BF16
// when a tile is staged in shared memory); the MSE gradient, bias gradients
// and Adam are FP32 element kernels.
//
// Inputs of the network for one cell: x = [T/1000, ln p, Y_1..Y_nsp, ln dt];
// outputs: [ln(attempted steps), dT, dY_1..dY_nsp]. Both are normalised by
// stored means and standard deviations.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dlbchem.h"
#include "dlb_common.cuh"
#include "dlb_ctx.h"

namespace dlb {

// SiLU z sigma(z) through sigma(z) = (1 + tanh(z/2)) / 2, with the hardware
// tanh on a pair of half-precision values (tanh.approx.f16x2: one
// special-function operation for two activations instead of an exponential
// and a reciprocal for each; the fused forward's epilogue is bound by that
// unit). z/2 rounded to FP16 and the approximate tanh put an error of order
// 1e-3 into sigma, below the BF16 rounding the activations get next; |z/2|
// beyond the FP16 range gives tanh = +-1, the limits of sigma. Training uses
// the same sigma, so the layer-by-layer and fused passes agree.
__device__ __forceinline__ float2 tanh2_half(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  uint32_t y;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<const uint32_t*>(&h)));
  return __half22float2(*reinterpret_cast<const __half2*>(&y));
}
__device__ __forceinline__ float2 silu2_f(float z0, float z1) {
  const float h0 = 0.5f * z0, h1 = 0.5f * z1;
  const float2 t = tanh2_half(h0, h1);
  return make_float2(fmaf(h0, t.x, h0), fmaf(h1, t.y, h1));
}
__device__ __forceinline__ float silu_f(float z) { return silu2_f(z, 0.0f).x; }
// d/dz z sigma(z) = sigma (1 + z (1 - sigma)), with the same sigma
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = fmaf(0.5f, tanh2_half(0.5f * z, 0.0f).x, 0.5f);
  return s * fmaf(z, 1.0f - s, 1.0f);
}

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[n]); optional pre-activation
// copy Z and SiLU. A: TA ? A[k*lda + m] : A[m*lda + k]; B: TB ? B[n*ldb + k]
// : B[k*ldb + n]. On the fifth-generation tensor cores: BF16 operands (FP32
// rounded while staged) in shared memory in the canonical K-major layout
// without swizzle (8 x 8 core matrices of 128 B, the K-groups of a row group
// contiguous), FP32 accumulator in tensor memory. One CTA of 128 threads
// computes a 128 x 64 tile: every thread stages, one thread issues the MMAs of
// a k-tile (K = 16 each) and commits them to an mbarrier, all wait (bounded),
// then each warp reads its 32 accumulator rows from tensor memory for the
// epilogue. A wait that gives up sets *status, writes NaN and still frees the
// tensor memory.
constexpr int kTM = 128, kTN = 64, kTK = 64;
constexpr uint32_t kTmemCols = 64;
constexpr int kWaitLimit = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start, leading-dimension byte offset (between
// core matrices along K), stride byte offset (between 8-row groups), version 1
// (the sm_100 family), no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// byte offset of (row, k) in a tile of rows x kTK BF16 values
__device__ __forceinline__ int tile_off(int row, int k) {
  return ((row >> 3) * (kTK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                      const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                      int ldc, const float* __restrict__ bias, float* __restrict__ Z,
                                                      int act, int* __restrict__ status) {
  __shared__ __align__(1024) unsigned char sop[(kTM + kTN) * kTK * 2];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  unsigned char* sA = sop;
  unsigned char* sB = sop + kTM * kTK * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N and M
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kTN >> 3) << 17) | (uint32_t(kTM >> 4) << 24);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K && ok; k0 += kTK) {
    // stage the k-tile (zero outside the matrices)
    for (int e = tid; e < kTM * kTK; e += 128) {
      int mm, kk;
      if (TA) { kk = e / kTM; mm = e % kTM; } else { mm = e / kTK; kk = e % kTK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.0f;
      if (gm < M && gk < K) v = TA ? A[int64_t(gk) * lda + gm] : A[int64_t(gm) * lda + gk];
      *reinterpret_cast<__nv_bfloat16*>(sA + tile_off(mm, kk)) = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < kTN * kTK; e += 128) {
      int nn, kk;
      if (TB) { nn = e / kTK; kk = e % kTK; } else { kk = e / kTN; nn = e % kTN; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.0f;
      if (gn < N && gk < K) v = TB ? B[int64_t(gn) * ldb + gk] : B[int64_t(gk) * ldb + gn];
      *reinterpret_cast<__nv_bfloat16*>(sB + tile_off(nn, kk)) = __float2bfloat16_rn(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy stores -> tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < kTK / 16; ++kk) {
        const uint64_t ad = umma_desc(smem_u32(sA) + kk * 256, 128, (kTK / 8) * 128);
        const uint64_t bd = umma_desc(smem_u32(sB) + kk * 256, 128, (kTK / 8) * 128);
        const uint32_t acc = (k0 > 0 || kk > 0) ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar))
                   : "memory");
    }
    // every thread waits for this k-tile's MMAs before the tile is overwritten (bounded)
    uint32_t done = 0;
    for (int it = 0; it < kWaitLimit && !done; ++it)
      asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                   : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase) : "memory");
    phase ^= 1u;
    ok = __syncthreads_and(done != 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0 && status) atomicExch(status, 1);
  // epilogue: warp w holds rows 32w .. 32w + 31 of the tile, 16 columns per load
  const int gm = m0 + 32 * warp + lane;
  for (int c0 = 0; c0 < kTN; c0 += 16) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(tmem + (uint32_t(32 * warp) << 16) + uint32_t(c0)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (gm < M) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int gn = n0 + c0 + j;
        if (gn < N) {
          float v = ok ? __uint_as_float(r[j]) + (bias ? bias[gn] : 0.0f) : __int_as_float(0x7fc00000);
          if (Z) Z[int64_t(gm) * ldc + gn] = v;
          if (act) v = silu_f(v);
          C[int64_t(gm) * ldc + gn] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// Whole-network forward pass for inference: one persistent CTA per SM, three
// roles in warps of their own. The weights, packed once into BF16 k-tiles of
// 64 (four MMAs of K = 16 each) in exactly the shared-memory layout the MMA
// reads, stream through a two-deep ring of 32 KB buffers filled by bulk
// copies (cp.async.bulk, the TMA engine, completing on mbarriers) from a
// producer warp; an output layer of at most 16 KB is copied once and stays. An MMA warp issues tcgen05.mma (kind::f16, BF16 operands,
// FP32 accumulator in tensor memory) and commits each k-tile to free its
// buffer. Eight epilogue warps (two per tensor-memory lane quarter, 32 rows
// each, alternate 16-column chunks) read the accumulator, add the bias, apply
// SiLU and write the activations back to shared memory as BF16: the next
// layer's A operand. Activations never leave shared memory; only the network
// input and output cross HBM. The CTA keeps two 128-row tiles in flight, each
// with its own activation tile and accumulator, and alternates them layer by
// layer, so the epilogue of one tile runs while the tensor cores work on the
// other. Arithmetic per element is that of the layered path above: BF16
// operands, FP32 accumulation over k-tiles of 64, FP32 bias and SiLU,
// activations rounded to BF16 as the next layer's operand. Supported shapes:
// hidden widths multiples of 64 up to 256, n_in and n_out up to 256, at most
// kFusedMaxLayers layers.
// ---------------------------------------------------------------------------
constexpr int kFusedMaxLayers = 8;
constexpr int kFusedMaxN = 256;
constexpr int kFK = 64;                                       // k-tile of the weight stream
constexpr int kFusedStages = 2;                               // weight ring depth
constexpr int kFusedSmemH = kTM * kFusedMaxN * 2;             // 64 KB per activation tile
constexpr int kFusedSmemW = kFusedMaxN * kFK * 2;             // 32 KB per weight buffer
constexpr int kFusedBias = kFusedMaxLayers * kFusedMaxN * 4;  // every layer's bias
// the output layer's packed weights stay in shared memory when they fit here
// (a narrow output: they then skip the ring and its per-k-tile round trips)
constexpr int kFusedResident = 16 * 1024;
constexpr int kFusedSmem = 2 * kFusedSmemH + kFusedStages * kFusedSmemW + kFusedBias + kFusedResident + 1024;
constexpr int kFusedEpiWarps = 8;                             // two per tensor-memory lane quarter
constexpr int kFusedThreads = 32 * (kFusedEpiWarps + 2);      // + producer warp + MMA warp

struct FusedNet {
  int nl;                                       // layers
  int fi[kFusedMaxLayers], fo[kFusedMaxLayers];
  int kp[kFusedMaxLayers], np[kFusedMaxLayers];  // fan-in padded to kFK, fan-out padded to 16
  int64_t woff[kFusedMaxLayers];                // byte offset of the layer's packed weights
  const float* bias[kFusedMaxLayers];
  const unsigned char* wpk;
  uint32_t res_bytes;                           // output layer resident in shared memory (0: streamed)
};

// byte offset of (row, k) in a tile of rows x kext BF16 values (kext a multiple of 8)
__device__ __forceinline__ int core_off(int row, int k, int kext) {
  return ((row >> 3) * (kext >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Layer weights W [fi][fo] (FP32, row-major) as BF16 k-tiles for the fused
// pass: k-tile t holds rows n < np and k in [kFK t, kFK t + kFK) of W^T in
// core matrices (the B operand, K-major), zero outside W.
__global__ void pack_weights_kernel(int fi, int fo, int kp, int np, const float* __restrict__ W,
                                    unsigned char* __restrict__ dst) {
  const int64_t total = int64_t(kp) * np;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int n = int(e % np), k = int(e / np);
    const float v = (n < fo && k < fi) ? W[int64_t(k) * fo + n] : 0.0f;
    const int kt = k / kFK;
    *reinterpret_cast<__nv_bfloat16*>(dst + int64_t(kt) * np * kFK * 2 + core_off(n, k - kt * kFK, kFK)) =
        __float2bfloat16_rn(v);
  }
}

// bounded mbarrier wait on the phase of the given parity; true once it completed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a in the low half (lower k)
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Work order of one CTA: its row tiles in pairs; within a pair, unit
// (tile, layer) in the order (t0, 0), (t1, 0), (t0, 1), (t1, 1), ...; tile j of
// the pair uses slot j (activation tile and accumulator). All three roles walk
// this order.
struct FusedOrder {
  int64_t ntiles, first, stride, mine;   // row tiles, this CTA's first, grid stride, count
  int nl;
  // unit u -> (local tile index, layer); units per pair = nl * tiles in the pair
  __device__ void unit(int64_t u, int64_t& lt, int& l) const {
    const int64_t per_pair = 2 * int64_t(nl);
    const int64_t pair = u / per_pair;
    int64_t r = u - pair * per_pair;
    const int64_t in_pair = mine - 2 * pair >= 2 ? 2 : 1;
    l = int(r / in_pair);
    lt = 2 * pair + (r - int64_t(l) * in_pair);
  }
  __device__ int64_t units() const { return mine * nl; }
};

__global__ void __launch_bounds__(kFusedThreads, 1) mlp_fused_forward_kernel(int64_t B, const float* __restrict__ X,
                                                                             float* __restrict__ out,
                                                                             const FusedNet net,
                                                                             int* __restrict__ status) {
  extern __shared__ unsigned char fused_smem_raw[];
  unsigned char* sH0 =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(fused_smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sW = sH0 + 2 * kFusedSmemH;                               // kFusedStages buffers
  float* sbias = reinterpret_cast<float*>(sW + kFusedStages * kFusedSmemW);  // [layer][kFusedMaxN]
  unsigned char* sR = reinterpret_cast<unsigned char*>(sbias) + kFusedBias;    // resident output layer
  __shared__ __align__(8) unsigned long long full[kFusedStages], empty[kFusedStages], acc_full[2], h_ready[2], res_bar, drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  FusedOrder ord;
  ord.ntiles = (B + kTM - 1) / kTM;
  ord.first = blockIdx.x;
  ord.stride = gridDim.x;
  ord.mine = ord.first < ord.ntiles ? (ord.ntiles - 1 - ord.first) / ord.stride + 1 : 0;
  ord.nl = net.nl;
  const int64_t nunits = ord.units();
  if (tid == 0) {
    for (int b = 0; b < kFusedStages; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&res_bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain_bar)) : "memory");
    for (int j = 0; j < 2; ++j) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[j])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&h_ready[j])), "r"(kFusedEpiWarps)
                   : "memory");
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int l = 0; l < net.nl; ++l)
    for (int n = tid; n < net.np[l]; n += kFusedThreads) sbias[l * kFusedMaxN + n] = n < net.fo[l] ? net.bias[l][n] : 0.0f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(uint32_t(2 * kFusedMaxN)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // a wait that gives up stops every role: the others skip their later waits
  auto wait = [&](unsigned long long* bar, uint32_t parity) {
    if (abort_flag) return false;
    if (mbar_wait(smem_u32(bar), parity)) return true;
    abort_flag = 1;
    return false;
  };
  if (warp == kFusedEpiWarps) {
    // producer: weight k-tile g of the stream into buffer g % kFusedStages
    if (lane == 0) {
      int64_t g = 0;
      for (int64_t u = 0; u < nunits && !abort_flag; ++u) {
        int64_t lt;
        int l;
        ord.unit(u, lt, l);
        if (l + 1 == net.nl && net.res_bytes) continue;   // resident: not streamed
        const uint32_t bytes = uint32_t(net.np[l]) * kFK * 2;
        for (int kt = 0; kt < net.kp[l] / kFK; ++kt, ++g) {
          const int st = int(g % kFusedStages);
          if (g >= kFusedStages && !wait(&empty[st], uint32_t(g / kFusedStages - 1) & 1u)) break;
          const uint32_t bar = smem_u32(&full[st]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           smem_u32(sW + st * kFusedSmemW)),
                       "l"(net.wpk + net.woff[l] + size_t(kt) * bytes), "r"(bytes), "r"(bar)
                       : "memory");
        }
      }
      // on a give-up, let the copies in flight land before the CTA leaves
      if (abort_flag && g > 0) mbar_wait(smem_u32(&full[(g - 1) % kFusedStages]), uint32_t((g - 1) / kFusedStages) & 1u);
    }
  } else if (warp == kFusedEpiWarps + 1) {
    // MMA issuer
    if (lane == 0) {
      int64_t g = 0, done_units[2] = {0, 0};
      bool res_ready = false;
      if (net.res_bytes && nunits > 0) {   // the output layer's weights, once
        const uint32_t bar = smem_u32(&res_bar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(net.res_bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(sR)),
                     "l"(net.wpk + net.woff[net.nl - 1]), "r"(net.res_bytes), "r"(bar)
                     : "memory");
      }
      for (int64_t u = 0; u < nunits && !abort_flag; ++u) {
        int64_t lt;
        int l;
        ord.unit(u, lt, l);
        const int slot = int(lt & 1);
        const int kp = net.kp[l], np = net.np[l];
        // the slot's activations are written and its accumulator drained
        if (!wait(&h_ready[slot], uint32_t(done_units[slot]) & 1u)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc =
            (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(np >> 3) << 17) | (uint32_t(kTM >> 4) << 24);
        const uint32_t hbase = smem_u32(sH0 + slot * kFusedSmemH);
        const uint32_t dtm = tmem + uint32_t(slot * kFusedMaxN);
        bool ok = true;
        if (l + 1 == net.nl && net.res_bytes) {
          // resident output layer: no ring, one commit for the whole unit
          if (!res_ready) {
            if (!wait(&res_bar, 0u)) break;
            res_ready = true;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int kt = 0; kt < kp / kFK; ++kt) {
#pragma unroll
            for (int kk = 0; kk < kFK / 16; ++kk) {
              const uint64_t ad = umma_desc(hbase + uint32_t(kt * (kFK / 8) + kk * 2) * 128u, 128, uint32_t(kp) * 16u);
              const uint64_t bd = umma_desc(smem_u32(sR) + uint32_t(kt) * uint32_t(np) * (kFK * 2) + uint32_t(kk) * 256u,
                                            128, (kFK / 8) * 128);
              const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
              asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                           "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
                           "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&acc_full[slot]))
                       : "memory");
          ++done_units[slot];
          continue;
        }
        for (int kt = 0; kt < kp / kFK; ++kt, ++g) {
          const int st = int(g % kFusedStages);
          if (!wait(&full[st], uint32_t(g / kFusedStages) & 1u)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int kk = 0; kk < kFK / 16; ++kk) {
            const uint64_t ad = umma_desc(hbase + uint32_t(kt * (kFK / 8) + kk * 2) * 128u, 128, uint32_t(kp) * 16u);
            const uint64_t bd = umma_desc(smem_u32(sW + st * kFusedSmemW) + uint32_t(kk) * 256u, 128, (kFK / 8) * 128);
            const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
                         "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
          }
          // the buffer is free once these MMAs complete
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty[st]))
                       : "memory");
        }
        if (!ok) break;
        // the unit's accumulator is complete when its MMAs are
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&acc_full[slot]))
                     : "memory");
        ++done_units[slot];
      }
      // on a give-up, let the copy and the MMAs in flight finish before tensor
      // memory is freed: one more commit covers every MMA issued so far
      if (abort_flag) {
        if (net.res_bytes && nunits > 0 && !res_ready) mbar_wait(smem_u32(&res_bar), 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&drain_bar))
                     : "memory");
        mbar_wait(smem_u32(&drain_bar), 0u);
      }
    }
  } else {
    // epilogue warps: warp w reads tensor-memory lane quarter w % 4 (rows
    // 32 (w % 4) + lane of each tile) and the 16-column chunks of parity w / 4
    const int quarter = warp & 3, half = warp >> 2;
    const int row = 32 * quarter + lane;
    auto stage_input = [&](int64_t lt) {
      const int slot = int(lt & 1);
      unsigned char* sH = sH0 + slot * kFusedSmemH;
      const int64_t r0 = (ord.first + lt * ord.stride) * kTM;
      const int kp = net.kp[0], fi = net.fi[0];
      const float* x = X + (r0 + row) * fi;
      const bool in = r0 + row < B;
      for (int k0 = 8 * half; k0 < kp; k0 += 16) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (in && k0 + j < fi) ? x[k0 + j] : 0.0f;
        *reinterpret_cast<uint4*>(sH + core_off(row, k0, kp)) = make_uint4(
            pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&h_ready[slot])) : "memory");
    };
    if (ord.mine > 0) stage_input(0);
    if (ord.mine > 1) stage_input(1);
    int64_t seen[2] = {0, 0};
    for (int64_t u = 0; u < nunits; ++u) {
      int64_t lt;
      int l;
      ord.unit(u, lt, l);
      const int slot = int(lt & 1);
      // warp-uniform, since the tensor-memory loads below are warp-collective
      const bool ok = __all_sync(0xffffffffu, wait(&acc_full[slot], uint32_t(seen[slot]) & 1u));
      ++seen[slot];
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int np = net.np[l], fo = net.fo[l];
      const bool last = l + 1 == net.nl;
      const float* bias = sbias + l * kFusedMaxN;
      const int64_t gr = (ord.first + lt * ord.stride) * kTM + row;
      unsigned char* sH = sH0 + slot * kFusedSmemH;
      const int kpn = last ? 0 : net.kp[l + 1];
      if (ok) {
        // this warp's 16-column chunks c0 = 16 half + 32 i; four tensor-memory
        // loads in flight per wait
        const int nch = (np - 16 * half + 31) / 32;
        for (int i0 = 0; i0 < nch; i0 += 4) {
          uint32_t r[4][16];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (i0 + q < nch)
              tmem_ld16(tmem + (uint32_t(32 * quarter) << 16) + uint32_t(slot * kFusedMaxN + 16 * half + 32 * (i0 + q)),
                        r[q]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (i0 + q >= nch) break;
            const int c0 = 16 * half + 32 * (i0 + q);
            float b[16];
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              *reinterpret_cast<float4*>(b + j) = *reinterpret_cast<const float4*>(bias + c0 + j);
            if (last) {
              if (gr < B) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  if (c0 + j < fo) out[gr * fo + c0 + j] = __uint_as_float(r[q][j]) + b[j];
              }
            } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                  const int n = c0 + 8 * h + j;
                  const float2 a = silu2_f(__uint_as_float(r[q][8 * h + j]) + b[8 * h + j],
                                           __uint_as_float(r[q][8 * h + j + 1]) + b[8 * h + j + 1]);
                  w[j / 2] = pack_bf16x2(n < fo ? a.x : 0.0f, n + 1 < fo ? a.y : 0.0f);
                }
                *reinterpret_cast<uint4*>(sH + core_off(row, c0 + 8 * h, kpn)) = make_uint4(w[0], w[1], w[2], w[3]);
              }
            }
          }
        }
      } else if (last && gr < B) {
        for (int n = half; n < fo; n += 2) out[gr * fo + n] = __int_as_float(0x7fc00000);
      }
      if (!last) {
        for (int k0 = np + 8 * half; k0 < kpn; k0 += 16)
          *reinterpret_cast<uint4*>(sH + core_off(row, k0, kpn)) = make_uint4(0, 0, 0, 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&h_ready[slot])) : "memory");
      } else if (lt + 2 < ord.mine) {
        // this slot's next tile (its accumulator has been read)
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        stage_input(lt + 2);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_flag && status) atomicExch(status, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(2 * kFusedMaxN)) : "memory");
}

// dZ = dH * silu'(Z), in place on dH.
__global__ void silu_back_kernel(int64_t n, float* __restrict__ dH, const float* __restrict__ Z) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dH[i] *= dsilu_f(Z[i]);
}

// MSE: dOut = 2 (out - y) / (B n_out); loss += sum (out - y)^2 / (B n_out).
__global__ void mse_kernel(int64_t n, float scale, const float* __restrict__ out, const float* __restrict__ y,
                           float* __restrict__ dout, float* __restrict__ loss) {
  float s = 0.0f;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float d = out[i] - y[i];
    dout[i] = 2.0f * d * scale;
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, s * scale);
}

// db[n] = sum_m dZ[m][n].
__global__ void bias_grad_kernel(int M, int N, const float* __restrict__ dZ, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int m = 0; m < M; ++m) s += dZ[int64_t(m) * N + n];
  db[n] = s;
}

// Adam (Kingma & Ba 2015, Algorithm 1), bias-corrected, FP32.
__global__ void adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Normalised network input of cell i from the species-major FP64 state.
__global__ void features_kernel(int64_t n, int nsp, const double* __restrict__ T, const double* __restrict__ p,
                                const double* __restrict__ Y, double dt, const float* __restrict__ mu,
                                const float* __restrict__ isd, float* __restrict__ X) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int nin = nsp + 3;
  float* x = X + i * nin;
  x[0] = (float(T[i] * 1e-3) - mu[0]) * isd[0];
  x[1] = (float(log(p[i])) - mu[1]) * isd[1];
  for (int k = 0; k < nsp; ++k) x[2 + k] = (float(Y[int64_t(k) * n + i]) - mu[2 + k]) * isd[2 + k];
  x[nin - 1] = (float(log(dt)) - mu[nin - 1]) * isd[nin - 1];
}

// Physical predictions from the normalised network output: ln steps, dT,
// dY (species-major, FP64).
__global__ void predictions_kernel(int64_t n, int nsp, const float* __restrict__ out, const float* __restrict__ mu,
                                   const float* __restrict__ sd, float* __restrict__ lnsteps,
                                   double* __restrict__ dT, double* __restrict__ dY) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int nout = nsp + 2;
  const float* o = out + i * nout;
  lnsteps[i] = o[0] * sd[0] + mu[0];
  dT[i] = double(o[1] * sd[1] + mu[1]);
  for (int k = 0; k < nsp; ++k) dY[int64_t(k) * n + i] = double(o[2 + k] * sd[2 + k] + mu[2 + k]);
}

}  // namespace dlb

struct dlbchem_mlp {
  int n_in = 0, n_hidden = 256, n_out = 0, n_layers = 3;
  int64_t nparams = 0;
  float* d_params = nullptr;   // [W1 b1 W2 b2 W3 b3 W4 b4], W row-major [fan_in, fan_out]
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_grad = nullptr;
  float* d_norm = nullptr;     // mu_x, isd_x, mu_y, sd_y
  int* d_status = nullptr;     // set to 1 by a GEMM whose tensor-core wait gave up
  int adam_t = 0;
  // fused forward (inference): BF16 weights packed as the fused kernel's
  // k-tiles, repacked after every parameter change
  bool fused_ok = false;       // the shape is one the fused kernel takes
  bool fused_on = true;        // dlbchem_mlp_set_fused
  bool packed_dirty = true;
  unsigned char* d_wpk = nullptr;
  dlb::FusedNet fnet{};
  int num_sms = 0;
  // activations for the largest batch seen
  int64_t cap = 0;
  float* d_act = nullptr;
  std::string err;
};

namespace {

int mfail(dlbchem_mlp* m, int code, const std::string& msg) {
  if (m) m->err = msg;
  return code;
}

struct LayerOff {
  int64_t w, b;
  int fi, fo;
};

std::vector<LayerOff> layers_of(const dlbchem_mlp* m) {
  std::vector<int> dims = {m->n_in};
  for (int i = 0; i < m->n_layers; ++i) dims.push_back(m->n_hidden);
  dims.push_back(m->n_out);
  std::vector<LayerOff> L;
  int64_t o = 0;
  for (size_t i = 0; i + 1 < dims.size(); ++i) {
    LayerOff l;
    l.fi = dims[i];
    l.fo = dims[i + 1];
    l.w = o;
    o += int64_t(l.fi) * l.fo;
    l.b = o;
    o += l.fo;
    L.push_back(l);
  }
  return L;
}

cudaError_t gemm(bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, const float* bias, float* Z, int act, int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;   // nothing to contract
  dim3 grid((N + dlb::kTN - 1) / dlb::kTN, (M + dlb::kTM - 1) / dlb::kTM);
  if (!ta && !tb) dlb::gemm_tc_kernel<false, false><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, act, status);
  else if (ta && !tb) dlb::gemm_tc_kernel<true, false><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, act, status);
  else if (!ta && tb) dlb::gemm_tc_kernel<false, true><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, act, status);
  else dlb::gemm_tc_kernel<true, true><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, act, status);
  return cudaGetLastError();
}

// activation workspace: per hidden layer Z and H [cap x n_hidden], output
// [cap x n_out], two gradient buffers [cap x max(n_hidden, n_out)].
int ensure_act(dlbchem_mlp* m, int64_t batch) {
  if (batch <= m->cap) return DLBCHEM_OK;
  if (m->d_act) cudaFree(m->d_act);
  m->d_act = nullptr;
  m->cap = 0;
  const int64_t wmax = std::max(m->n_hidden, m->n_out);
  const int64_t per = 2 * int64_t(m->n_layers) * m->n_hidden + m->n_out + 2 * wmax;
  if (cudaMalloc(&m->d_act, size_t(batch) * per * 4) != cudaSuccess) {
    m->d_act = nullptr;
    return mfail(m, DLBCHEM_OOM, "network activation allocation failed");
  }
  m->cap = batch;
  return DLBCHEM_OK;
}

// Fused-forward tables of the network (weights still to pack); false if the
// shape is not one the fused kernel takes.
bool plan_fused(dlbchem_mlp* m) {
  const auto L = layers_of(m);
  if (int(L.size()) > dlb::kFusedMaxLayers) return false;
  if (m->n_hidden % 64 != 0 || m->n_hidden > dlb::kFusedMaxN || m->n_in > dlb::kFusedMaxN ||
      m->n_out > dlb::kFusedMaxN)
    return false;
  dlb::FusedNet& f = m->fnet;
  f.nl = int(L.size());
  int64_t off = 0;
  for (int l = 0; l < f.nl; ++l) {
    f.fi[l] = L[l].fi;
    f.fo[l] = L[l].fo;
    f.kp[l] = (L[l].fi + dlb::kFK - 1) / dlb::kFK * dlb::kFK;
    f.np[l] = (L[l].fo + 15) / 16 * 16;
    f.woff[l] = off;
    off += int64_t(f.kp[l]) * f.np[l] * 2;
  }
  if (cudaMalloc(&m->d_wpk, size_t(off)) != cudaSuccess) {
    m->d_wpk = nullptr;
    return false;
  }
  f.wpk = m->d_wpk;
  for (int l = 0; l < f.nl; ++l) f.bias[l] = m->d_params + L[l].b;
  const int64_t last_bytes = int64_t(f.kp[f.nl - 1]) * f.np[f.nl - 1] * 2;
  f.res_bytes = last_bytes <= dlb::kFusedResident ? uint32_t(last_bytes) : 0u;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  return cudaFuncSetAttribute(dlb::mlp_fused_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              dlb::kFusedSmem) == cudaSuccess;
}

cudaError_t forward_fused(dlbchem_mlp* m, int64_t B, const float* X, float* out, cudaStream_t s) {
  const auto L = layers_of(m);
  cudaError_t e = cudaSuccess;
  if (m->packed_dirty) {
    for (int l = 0; l < m->fnet.nl && e == cudaSuccess; ++l) {
      const int64_t tot = int64_t(m->fnet.kp[l]) * m->fnet.np[l];
      dlb::pack_weights_kernel<<<unsigned(std::min<int64_t>((tot + 255) / 256, 1024)), 256, 0, s>>>(
          L[l].fi, L[l].fo, m->fnet.kp[l], m->fnet.np[l], m->d_params + L[l].w, m->d_wpk + m->fnet.woff[l]);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    m->packed_dirty = false;
  }
  // persistent: one CTA per SM (its two accumulators fill tensor memory)
  const int64_t tiles = (B + dlb::kTM - 1) / dlb::kTM;
  const int64_t grid = std::min<int64_t>(tiles, int64_t(m->num_sms));
  dlb::mlp_fused_forward_kernel<<<unsigned(grid), dlb::kFusedThreads, dlb::kFusedSmem, s>>>(B, X, out, m->fnet,
                                                                                           m->d_status);
  return cudaGetLastError();
}

// Forward; with keep the pre-activations are stored for the backward pass.
// Without keep (inference) the fused whole-network kernel runs where the
// shape allows it.
cudaError_t forward(dlbchem_mlp* m, int64_t B, const float* X, float* out, bool keep, cudaStream_t s) {
  if (!keep && m->fused_ok && m->fused_on) return forward_fused(m, B, X, out, s);
  const auto L = layers_of(m);
  const int64_t H = m->n_hidden;
  float* Zs = m->d_act;                                  // n_layers x [B x H]
  float* Hs = Zs + int64_t(m->n_layers) * B * H;         // n_layers x [B x H]
  const float* in = X;
  cudaError_t e = cudaSuccess;
  for (int li = 0; li < int(L.size()) && e == cudaSuccess; ++li) {
    const bool last = li + 1 == int(L.size());
    float* dst = last ? out : Hs + int64_t(li) * B * H;
    float* z = (!last && keep) ? Zs + int64_t(li) * B * H : nullptr;
    e = gemm(false, false, int(B), L[li].fo, L[li].fi, in, L[li].fi, m->d_params + L[li].w, L[li].fo, dst, L[li].fo,
             m->d_params + L[li].b, z, last ? 0 : 1, m->d_status, s);
    in = dst;
  }
  return e;
}

}  // namespace

extern "C" {

int dlbchem_mlp_create(int n_in, int n_hidden, int n_out, dlbchem_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1) return DLBCHEM_BAD_ARG;
  *out = nullptr;
  auto* m = new dlbchem_mlp;
  m->n_in = n_in; m->n_hidden = n_hidden; m->n_out = n_out;
  const auto L = layers_of(m);
  m->nparams = L.back().b + L.back().fo;
  const size_t bytes = size_t(m->nparams) * 4;
  if (cudaMalloc(&m->d_params, bytes) != cudaSuccess || cudaMalloc(&m->d_m, bytes) != cudaSuccess ||
      cudaMalloc(&m->d_v, bytes) != cudaSuccess || cudaMalloc(&m->d_grad, bytes) != cudaSuccess ||
      cudaMalloc(&m->d_norm, size_t(2 * (n_in + n_out)) * 4) != cudaSuccess ||
      cudaMalloc(&m->d_status, sizeof(int)) != cudaSuccess) {
    dlbchem_mlp_destroy(m);
    return DLBCHEM_OOM;
  }
  cudaMemset(m->d_params, 0, bytes);
  cudaMemset(m->d_status, 0, sizeof(int));
  cudaMemset(m->d_m, 0, bytes);
  cudaMemset(m->d_v, 0, bytes);
  std::vector<float> norm(2 * (n_in + n_out), 0.0f);
  for (int i = 0; i < n_in; ++i) norm[n_in + i] = 1.0f;
  for (int i = 0; i < n_out; ++i) norm[2 * n_in + n_out + i] = 1.0f;
  cudaMemcpy(m->d_norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice);
  m->fused_ok = plan_fused(m);
  *out = m;
  return DLBCHEM_OK;
}

int64_t dlbchem_mlp_nparams(const dlbchem_mlp* m) { return m ? m->nparams : -1; }

int dlbchem_mlp_set_params(dlbchem_mlp* m, const float* params, void* stream) {
  if (!m || !params) return DLBCHEM_BAD_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  m->packed_dirty = true;
  cudaError_t e = cudaMemcpyAsync(m->d_params, params, size_t(m->nparams) * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_m, 0, size_t(m->nparams) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_v, 0, size_t(m->nparams) * 4, s);
  m->adam_t = 0;
  return e == cudaSuccess ? DLBCHEM_OK : mfail(m, DLBCHEM_CUDA, cudaGetErrorString(e));
}

int dlbchem_mlp_get_params(dlbchem_mlp* m, float* params, void* stream) {
  if (!m || !params) return DLBCHEM_BAD_ARG;
  const cudaError_t e = cudaMemcpyAsync(params, m->d_params, size_t(m->nparams) * 4, cudaMemcpyDeviceToDevice,
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DLBCHEM_OK : mfail(m, DLBCHEM_CUDA, cudaGetErrorString(e));
}

int dlbchem_mlp_set_norm(dlbchem_mlp* m, const float* mu_x, const float* sd_x, const float* mu_y, const float* sd_y) {
  if (!m || !mu_x || !sd_x || !mu_y || !sd_y) return DLBCHEM_BAD_ARG;
  std::vector<float> norm;
  for (int i = 0; i < m->n_in; ++i) norm.push_back(mu_x[i]);
  for (int i = 0; i < m->n_in; ++i) {
    if (!(sd_x[i] > 0)) return mfail(m, DLBCHEM_BAD_ARG, "input scales must be positive");
    norm.push_back(1.0f / sd_x[i]);
  }
  for (int i = 0; i < m->n_out; ++i) norm.push_back(mu_y[i]);
  for (int i = 0; i < m->n_out; ++i) norm.push_back(sd_y[i]);
  const cudaError_t e = cudaMemcpy(m->d_norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? DLBCHEM_OK : mfail(m, DLBCHEM_CUDA, cudaGetErrorString(e));
}

int dlbchem_mlp_forward(dlbchem_mlp* m, int64_t batch, const float* X, float* out, void* stream) {
  if (!m || batch < 0 || (batch > 0 && (!X || !out))) return DLBCHEM_BAD_ARG;
  if (batch == 0) return DLBCHEM_OK;
  int rc = ensure_act(m, batch);
  if (rc != DLBCHEM_OK) return rc;
  const cudaError_t e = forward(m, batch, X, out, false, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DLBCHEM_OK : mfail(m, DLBCHEM_CUDA, cudaGetErrorString(e));
}

// Loss and gradient of the MSE on one batch (X [B x n_in], Y [B x n_out],
// normalised). grad: device [nparams] or NULL (internal buffer); loss:
// device float or NULL.
int dlbchem_mlp_grad(dlbchem_mlp* m, int64_t B, const float* X, const float* Y, float* grad, float* loss, void* stream) {
  if (!m || B < 1 || !X || !Y) return DLBCHEM_BAD_ARG;
  int rc = ensure_act(m, B);
  if (rc != DLBCHEM_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* g = grad ? grad : m->d_grad;
  const auto L = layers_of(m);
  const int64_t H = m->n_hidden, wmax = std::max(m->n_hidden, m->n_out);
  float* Zs = m->d_act;
  float* Hs = Zs + int64_t(m->n_layers) * B * H;
  float* out = Hs + int64_t(m->n_layers) * B * H;
  float* dA = out + B * m->n_out;
  float* dB = dA + B * wmax;
  cudaError_t e = forward(m, B, X, out, true, s);
  if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, 4, s);
  if (e == cudaSuccess) {
    const int64_t n = B * m->n_out;
    dlb::mse_kernel<<<unsigned(std::min<int64_t>((n + 255) / 256, 1024)), 256, 0, s>>>(n, 1.0f / float(n), out, Y, dA,
                                                                                     loss);
    e = cudaGetLastError();
  }
  float* dcur = dA;
  float* dnext = dB;
  for (int li = int(L.size()) - 1; li >= 0 && e == cudaSuccess; --li) {
    const float* hin = li == 0 ? X : Hs + int64_t(li - 1) * B * H;
    // dW = hin^T dZ  (M = fan_in, N = fan_out, K = B)
    e = gemm(true, false, L[li].fi, L[li].fo, int(B), hin, L[li].fi, dcur, L[li].fo, g + L[li].w, L[li].fo, nullptr,
             nullptr, 0, m->d_status, s);
    if (e == cudaSuccess) {
      dlb::bias_grad_kernel<<<(L[li].fo + 127) / 128, 128, 0, s>>>(int(B), L[li].fo, dcur, g + L[li].b);
      e = cudaGetLastError();
    }
    if (li == 0 || e != cudaSuccess) break;
    // dH_prev = dZ W^T  (M = B, N = fan_in, K = fan_out), then through SiLU
    e = gemm(false, true, int(B), L[li].fi, L[li].fo, dcur, L[li].fo, m->d_params + L[li].w, L[li].fo, dnext,
             L[li].fi, nullptr, nullptr, 0, m->d_status, s);
    if (e == cudaSuccess) {
      const int64_t n = B * H;
      dlb::silu_back_kernel<<<unsigned(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, s>>>(
          n, dnext, Zs + int64_t(li - 1) * B * H);
      e = cudaGetLastError();
    }
    float* t = dcur; dcur = dnext; dnext = t;
  }
  return e == cudaSuccess ? DLBCHEM_OK : mfail(m, DLBCHEM_CUDA, cudaGetErrorString(e));
}

int dlbchem_mlp_adam(dlbchem_mlp* m, const float* grad, float lr, void* stream) {
  if (!m || !(lr > 0)) return DLBCHEM_BAD_ARG;
  m->adam_t += 1;
  m->packed_dirty = true;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, float(m->adam_t)), c2 = 1.0f - std::pow(b2, float(m->adam_t));
  dlb::adam_kernel<<<unsigned(std::min<int64_t>((m->nparams + 255) / 256, 2048)), 256, 0,
                     static_cast<cudaStream_t>(stream)>>>(m->nparams, m->d_params, grad ? grad : m->d_grad, m->d_m,
                                                          m->d_v, lr, b1, b2, 1e-8f, c1, c2);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DLBCHEM_OK : mfail(m, DLBCHEM_CUDA, cudaGetErrorString(e));
}

int dlbchem_mlp_train_step(dlbchem_mlp* m, int64_t B, const float* X, const float* Y, float lr, float* loss,
                           void* stream) {
  int rc = dlbchem_mlp_grad(m, B, X, Y, nullptr, loss, stream);
  return rc == DLBCHEM_OK ? dlbchem_mlp_adam(m, nullptr, lr, stream) : rc;
}

int dlbchem_mlp_set_fused(dlbchem_mlp* m, int enable) {
  if (!m || (enable != 0 && enable != 1)) return DLBCHEM_BAD_ARG;
  m->fused_on = enable != 0;
  return DLBCHEM_OK;
}

int dlbchem_mlp_fused(const dlbchem_mlp* m) { return m ? int(m->fused_ok && m->fused_on) : -1; }

const char* dlbchem_mlp_last_error(const dlbchem_mlp* m) { return m ? m->err.c_str() : ""; }

void dlbchem_mlp_destroy(dlbchem_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  for (float* p : {m->d_params, m->d_m, m->d_v, m->d_grad, m->d_norm, m->d_act})
    if (p) cudaFree(p);
  if (m->d_status) cudaFree(m->d_status);
  if (m->d_wpk) cudaFree(m->d_wpk);
  delete m;
}

}  // extern "C"

namespace dlb {

// Network predictions for n cells of one context's field (used by
// dlbchem_integrate when the predictor or the surrogate is on): features ->
// forward -> physical ln steps, dT, dY. X, out, lnsteps, dT, dY are caller
// workspace.
cudaError_t mlp_predict(dlbchem_mlp* m, int64_t n, int nsp, const double* T, const double* p, const double* Y,
                        double dt, float* X, float* out, float* lnsteps, double* dT, double* dY, cudaStream_t s) {
  if (ensure_act(m, std::min<int64_t>(n, 65536)) != DLBCHEM_OK) return cudaErrorMemoryAllocation;
  const float* mu_x = m->d_norm;
  const float* isd_x = mu_x + m->n_in;
  const float* mu_y = isd_x + m->n_in;
  const float* sd_y = mu_y + m->n_out;
  features_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, nsp, T, p, Y, dt, mu_x, isd_x, X);
  cudaError_t e = cudaGetLastError();
  for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += 65536) {
    const int64_t b = std::min<int64_t>(65536, n - b0);
    e = forward(m, b, X + b0 * m->n_in, out + b0 * m->n_out, false, s);
  }
  if (e == cudaSuccess) {
    predictions_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, nsp, out, mu_y, sd_y, lnsteps, dT, dY);
    e = cudaGetLastError();
  }
  return e;
}

int mlp_shape(const dlbchem_mlp* m, int* n_in, int* n_out) {
  *n_in = m->n_in;
  *n_out = m->n_out;
  return 0;
}

}  // namespace dlb
