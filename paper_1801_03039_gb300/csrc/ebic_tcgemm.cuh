// The surrogate's training GEMMs on the fifth-generation tensor cores
// (tcgen05.mma, bf16 operands, fp32 accumulators in tensor memory).
//
// D[M x N] = op(A)[M x K] . op(B)[K x N] for the six products of one Adam
// step (forward: x W1, h1 W2; reverse: h1^T dh2, dh2 W2^T, x^T dh1, dh1 W1^T).
// A CTA owns a 128-row tile of D with every one of its N <= 256 columns; one
// thread issues the MMAs, M = 128, K = 16 each; the eight warps read the
// accumulators back with tcgen05.ld (warp w: TMEM lanes 32 (w % 4) ..,
// columns of half w / 4) and apply the epilogue.
//
// Two kernels, by how the operands sit in global memory:
//   k_gemm_tc_full   both operands K-major (k contiguous): the whole K (80 or
//                    256) is brought into shared memory at once, A by the
//                    tensor-memory-access engine (cp.async.bulk.tensor, one
//                    box of 8 k x R rows per group of eight k; rows past the
//                    matrix arrive as zeros), B the same way or, for the
//                    forward weights, by one bulk copy of the pre-packed W^T
//                    that the scoring kernel also reads.
//   k_gemm_tc_split  both operands MN-major (the weight gradients, K = the
//                    batch): K is split across gridDim.z; each split walks its
//                    range in chunks of 64, and the threads load 8 x 8 blocks
//                    with 16-byte loads, transpose them in registers and store
//                    them K-major; split z writes its partial product to slice
//                    z, summed afterwards in split order.
//
// Shared-memory operand layouts (no swizzle, 8 x 8 core matrices of 128
// bytes, element (r, k) of an R x K operand):
//   "group-major", written by the tensor copies and the split loader:
//       (k / 8) * R * 8 + r * 8 + k % 8          (bf16 units)
//     K-adjacent core matrices R * 16 bytes apart, 8-row groups 128 bytes.
//   "row-major" (the packed weights): ((r / 8) * (K / 8) + k / 8) * 64 +
//       (r % 8) * 8 + k % 8; K-adjacent 128 bytes, 8-row groups K * 16.
// Every wait is bounded; a wait that gives up sets *err, and the CTA lets
// its copies land, frees its tensor memory and stores nothing.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ebic_async.cuh"
#include "ebic_tcmlp.cuh"

namespace ebic {

namespace tcg {

constexpr int kTM = 128;           // rows of a D tile (TMEM lanes)
constexpr int kKC = 64;            // K elements per chunk of the split kernel
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 256;
// both kernels ask for at least this much shared memory, so that no more than
// two CTAs share an SM and their tensor-memory allocations (256 columns each)
// always fit; the operands start at the first 1024-byte boundary of the
// dynamic shared memory, so every request adds 1 KB
constexpr int kMinSmem = 100 * 1024;
constexpr int kAlignSlack = 1024;

enum { EPI_BIAS_RELU_BF16 = 0, EPI_MASK_BF16 = 1, EPI_F32 = 2, EPI_F32_SPLIT = 3 };
enum { B_TMA = 0, B_PACKED = 1 };

// one box of a 2-D tensor map: inner coordinate x (elements), row y
__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* map, int x, int y,
                                      unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
               "r"(kTmemCols)
               : "memory");
}

}  // namespace tcg

namespace tcg {

// a plain bulk copy onto a barrier whose byte count was already announced
__device__ __forceinline__ void bulk_nc(void* dst, const void* src, uint32_t bytes,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// The epilogue of a 128 x N tile held in TMEM columns [0, N): warp w reads
// lanes 32 (w % 4) .. + 31 (rows of the tile) and the 16-column groups of its
// half (w / 4) in turn; `zero` stores zeros instead (a split with no K).
template <int EPI>
__device__ __forceinline__ void epilogue(uint32_t tmem, int warp, int lane, int m0, int M, int N,
                                         bool zero, const float* __restrict__ bias,
                                         const __nv_bfloat16* __restrict__ mask, int ldm,
                                         float* __restrict__ Cf, __nv_bfloat16* __restrict__ Cb,
                                         int ldc) {
  typedef __nv_bfloat16 bf;
  const int q = warp & 3, cg = warp >> 2;
  const int m = m0 + 32 * q + lane;
  for (int c = 16 * cg; c < N; c += 32) {
    float v[16];
    if (zero) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    } else {
      ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
    }
    if (m >= M) continue;
    if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
      __align__(16) bf o[16];
      if (EPI == EPI_BIAS_RELU_BF16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[c + i], 0.f));
      } else {
        __align__(16) bf mk[16];
        const uint4* mp = reinterpret_cast<const uint4*>(mask + (size_t)m * ldm + c);
        *reinterpret_cast<uint4*>(mk) = mp[0];
        *reinterpret_cast<uint4*>(mk + 8) = mp[1];
#pragma unroll
        for (int i = 0; i < 16; ++i)
          o[i] = __float2bfloat16_rn(__bfloat162float(mk[i]) > 0.f ? v[i] : 0.f);
      }
      uint4* dst = reinterpret_cast<uint4*>(Cb + (size_t)m * ldc + c);
      dst[0] = *reinterpret_cast<const uint4*>(o);
      dst[1] = *reinterpret_cast<const uint4*>(o + 8);
    } else {
      float4* dst = reinterpret_cast<float4*>(Cf + (size_t)m * ldc + c);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
  }
}

// 8 x 8 bf16 block transpose: in[i] holds elements (i, 0..7), out[j] gets
// elements (0..7, j).
__device__ __forceinline__ void transpose8(const uint4 (&in)[8], uint4 (&out)[8]) {
  uint32_t w[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    w[i][0] = in[i].x;
    w[i][1] = in[i].y;
    w[i][2] = in[i].z;
    w[i][3] = in[i].w;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t sel = (j & 1) ? 0x7632u : 0x5410u;
    uint32_t o[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) o[p] = __byte_perm(w[2 * p][j >> 1], w[2 * p + 1][j >> 1], sel);
    out[j] = make_uint4(o[0], o[1], o[2], o[3]);
  }
}

}  // namespace tcg

// D = op(A) op(B) with both operands K-major, the whole K in shared memory.
// A (M x K, row pitch set in tmA) arrives by tensor copies; B (N x K) by
// tensor copies (BSRC = B_TMA, tmB) or as the packed row-major W^T at
// Bpacked (B_PACKED).  K and N are multiples of 16, N <= 256, K <= 256.
// grid.x = M tiles of 128.
template <int BSRC, int EPI>
__global__ void __launch_bounds__(tcg::kThreads, 1)
k_gemm_tc_full(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __nv_bfloat16* __restrict__ Bpacked, int M, int N, int K,
               const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, int ldm,
               float* __restrict__ Cf, __nv_bfloat16* __restrict__ Cb, int ldc,
               int* __restrict__ err) {
  using namespace tcg;
  typedef __nv_bfloat16 bf;
  extern __shared__ __align__(16) unsigned char gsm_full[];
  unsigned char* gsm = gsm_full + ((1024u - (smem_addr(gsm_full) & 1023u)) & 1023u);
  bf* sA = reinterpret_cast<bf*>(gsm);                       // 128 x K, group-major
  bf* sB = sA + kTM * K;                                     // N x K
  __shared__ __align__(8) unsigned long long lbar, mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM;
  if (tid == 0) {
    mbar_init(&lbar, 1);
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes_b = (uint32_t)N * (uint32_t)K * 2u;
    expect_tx(&lbar, (uint32_t)kTM * (uint32_t)K * 2u + bytes_b);
    for (int g = 0; g < K / 8; ++g) tma2d(sA + (size_t)g * kTM * 8, &tmA, 8 * g, m0, &lbar);
    if (BSRC == B_TMA) {
      for (int g = 0; g < K / 8; ++g) tma2d(sB + (size_t)g * N * 8, &tmB, 8 * g, 0, &lbar);
    } else {
      bulk_nc(sB, Bpacked, bytes_b, &lbar);
    }
  }
  if (warp == 0) tmem_alloc(&tslot);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const bool landed = mbar_wait(&lbar, 0);
  bool ok = __syncthreads_and(landed) != 0;
  if (ok) {
    if (tid == 0) {
      const uint32_t aA = smem_addr(sA), aB = smem_addr(sB);
      const uint32_t id = tc::idesc(kTM, N);
      for (int k0 = 0; k0 < K; k0 += 16) {
        const uint64_t da = tc::sdesc(aA + (uint32_t)(k0 / 8) * kTM * 16, kTM * 16, 128);
        const uint64_t db = BSRC == B_TMA
                                ? tc::sdesc(aB + (uint32_t)(k0 / 8) * (uint32_t)N * 16,
                                            (uint32_t)N * 16, 128)
                                : tc::sdesc(aB + (uint32_t)(k0 / 8) * 128, 128, (uint32_t)K * 16);
        tc::mma(tmem, da, db, id, k0 > 0);
      }
      tc::commit(&mbar);
    }
    ok = __syncthreads_and(mbar_wait(&mbar, 0)) != 0;
    tc::fence_after();
    if (ok) {
      epilogue<EPI>(tmem, warp, lane, m0, M, N, false, bias, mask, ldm, Cf, Cb, ldc);
    } else {
      mbar_wait(&mbar, 0);                          // let the MMAs finish before freeing
    }
  } else if (!landed) {
    mbar_wait(&lbar, 0);                            // let the copies land before leaving
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem);
}

// Split-K D slices with both operands MN-major: op(A)(m, k) = A[k * lda + m],
// op(B)(k, n) = B[k * ldb + n].  grid = (M tiles of 128, 1, splits); split z
// takes K rows [z * kchunk, min(K, (z + 1) * kchunk)) (kchunk a multiple of
// 64) and writes Cf[z][M][ldc].  M and N are multiples of 8, N <= 256, and
// both leading dimensions give 16-byte aligned rows.
__global__ void __launch_bounds__(tcg::kThreads, 1)
k_gemm_tc_split(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ Cf, int ldc,
                int* __restrict__ err) {
  using namespace tcg;
  typedef __nv_bfloat16 bf;
  extern __shared__ __align__(16) unsigned char gsm_split[];
  unsigned char* gsm = gsm_split + ((1024u - (smem_addr(gsm_split) & 1023u)) & 1023u);
  bf* sA = reinterpret_cast<bf*>(gsm);                       // 128 x 64, group-major
  bf* sB = sA + kTM * kKC;                                   // N x 64, group-major
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM;
  const int splits = gridDim.z;
  const int kchunk = ((K + splits - 1) / splits + kKC - 1) / kKC * kKC;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tslot);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const uint32_t aA = smem_addr(sA), aB = smem_addr(sB);
  const uint32_t id = tc::idesc(kTM, N);
  const int nbA = 8 * (kTM / 8), nb = nbA + 8 * (N / 8);   // 8 x 8 blocks of a chunk
  bool ok = true;
  uint32_t ph = 0;
  for (int k0 = kbeg; k0 < kend && ok; k0 += kKC) {
    for (int blk = tid; blk < nb; blk += kThreads) {
      const bool isA = blk < nbA;
      const int b = isA ? blk : blk - nbA;
      const int rg = isA ? b % (kTM / 8) : b % (N / 8);      // group of 8 rows of the operand
      const int kg = isA ? b / (kTM / 8) : b / (N / 8);      // group of 8 k
      const int col = isA ? m0 + 8 * rg : 8 * rg;            // first m or n of the block
      const int lim = isA ? M : N;
      const bf* src = isA ? A : B;
      const int ld = isA ? lda : ldb;
      uint4 in[8], out[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + 8 * kg + i;
        in[i] = (k < kend && col < lim)
                    ? *reinterpret_cast<const uint4*>(src + (size_t)k * ld + col)
                    : make_uint4(0u, 0u, 0u, 0u);
      }
      transpose8(in, out);
      bf* dst = (isA ? sA + (size_t)kg * kTM * 8 : sB + (size_t)kg * N * 8) + (size_t)(8 * rg) * 8;
#pragma unroll
      for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4*>(dst + j * 8) = out[j];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      for (int kk = 0; kk < kKC; kk += 16)
        tc::mma(tmem, tc::sdesc(aA + (uint32_t)(kk / 8) * kTM * 16, kTM * 16, 128),
                tc::sdesc(aB + (uint32_t)(kk / 8) * (uint32_t)N * 16, (uint32_t)N * 16, 128), id,
                k0 > kbeg || kk > 0);
      tc::commit(&mbar);
    }
    const bool w = mbar_wait(&mbar, ph);
    ph ^= 1u;
    ok = __syncthreads_and(w) != 0;
    tc::fence_after();
  }
  if (ok) {
    epilogue<EPI_F32_SPLIT>(tmem, warp, lane, m0, M, N, kbeg >= kend, nullptr, nullptr, 0,
                            Cf + (size_t)blockIdx.z * M * ldc, nullptr, ldc);
  } else {
    mbar_wait(&mbar, ph ^ 1u);                      // let the MMAs finish before freeing
    if (tid == 0) atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem);
}

}  // namespace ebic
