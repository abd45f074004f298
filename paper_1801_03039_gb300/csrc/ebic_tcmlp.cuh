// The surrogate's scoring pass on the fifth-generation tensor cores
// (tcgen05.mma with fp32 accumulators in tensor memory).
//
// Tiles of 128 series.  Per tile the CTA's eight warps build the features x
// (sixteen series a warp, two embedding dimensions a lane; sums in fp32, in
// column order, rounded to bf16, as every other path does) in shared memory;
// one thread issues the layer-1 MMAs (M = 128, N = 256, K = 80 in five
// K = 16 steps) into tensor-memory columns [0, 256); the epilogue
// reads them back (tcgen05.ld), adds b1, applies ReLU and rounds to bf16 into
// a quarter-width h1 buffer; layer 2 runs as four K-quarters of 64 (four
// K = 16 steps each) into columns [256, 512), accumulating; the last
// epilogue adds b2, applies ReLU, rounds to bf16 and takes the dot product
// with w3 per row.  W1^T (256 x 80) and W2^T (256 x 256) stay in shared memory
// for the whole kernel, brought in by one bulk copy.
//
// Operands sit in shared memory K-major without swizzle, in 8 x 8 core
// matrices of 128 bytes: element (r, k) of an R x K operand is at
// ((r / 8) * (K / 8) + k / 8) * 64 + (r % 8) * 8 + k % 8 (bf16 units).  The
// matrix descriptor of a K = 16 step starting at column k0 points at core
// matrix (0, k0 / 8), with 128 bytes between K-adjacent core matrices and
// K * 16 bytes between 8-row groups.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "ebic_async.cuh"

namespace ebic {

namespace tc {

constexpr int kTT = 128;                          // series per tile (TMEM lanes)
constexpr int kF = 80, kH = 256, kEmb = 64;       // as the surrogate's layers
constexpr size_t kW1 = (size_t)kH * kF * 2;       // W1^T bytes
constexpr size_t kW2 = (size_t)kH * kH * 2;       // W2^T bytes
constexpr int kQ = 64;                            // h1 columns per layer-2 K-quarter
constexpr size_t kX = (size_t)kTT * kF * 2;       // x tile bytes
constexpr size_t kHq = (size_t)kTT * kQ * 2;      // a quarter of an h1 tile
// x and the current h1 quarter share one buffer (x is dead once the layer-1
// MMAs have completed); the total stays below 196 KB, which leaves the SM a
// 60 KB L1 for the embedding rows the feature gather rereads
constexpr size_t kXH = kX > kHq ? kX : kHq;
constexpr size_t kSmem = kW1 + kW2 + kXH + 3 * (size_t)kH * 4 + (size_t)kTT * 2 * 4;
static_assert(kSmem + 1024 + 128 <= 196 * 1024, "shared memory above the 196 KB carve-out");
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 512;

__host__ __device__ constexpr int cm(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// Instruction descriptor of kind::f16: fp32 D, bf16 A and B, both K-major,
// M x N.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address, byte offset
// between K-adjacent core matrices (lbo), between 8-row groups (sbo).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;                                  // descriptor version of tcgen05
  return d;
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id,
                                    bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate ? 1u : 0u)
      : "memory");
}

__device__ __forceinline__ void commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Embedding rows are reread by every tile: ask L1 to keep them.
__device__ __forceinline__ float2 ld_keep(const float2* p) {
  float2 v;
  asm("ld.global.nc.L1::evict_last.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

}  // namespace tc

// W1^T and W2^T in the tcgen05 forward's shared-memory layout (bf16 core
// matrices), from the fp32 masters W1 [kF][kH] and W2 [kH][kH]: one bulk
// copy moves the result into shared memory.
__global__ void k_pack_fwd_tc(const float* __restrict__ W1, const float* __restrict__ W2,
                              __nv_bfloat16* __restrict__ out) {
  using namespace tc;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kH * kF) {
    const int n = i / kF, k = i % kF;
    out[cm(n, k, kF)] = __float2bfloat16_rn(W1[k * kH + n]);
  } else if (i < kH * kF + kH * kH) {
    const int r = i - kH * kF, n = r / kH, k = r % kH;
    out[kH * kF + cm(n, k, kH)] = __float2bfloat16_rn(W2[k * kH + n]);
  }
}

// Scores y[n] of n series (seq [n][stride], len[n]).  One CTA per SM, tiles
// of 128 series in a grid stride.  Every wait is bounded; a wait that gives
// up sets *err and leaves NaN scores for the tiles not done.
__global__ void __launch_bounds__(tc::kThreads, 1)
k_mlp_forward_tc(const uint16_t* __restrict__ seq, const int32_t* __restrict__ len,
                 int32_t stride, int32_t n, int32_t C, const float* __restrict__ emb,
                 const float* __restrict__ cmean, const float* __restrict__ csd, float len_scale,
                 const __nv_bfloat16* __restrict__ wpack, const float* __restrict__ b1,
                 const float* __restrict__ b2, const float* __restrict__ w3,
                 const float* __restrict__ b3, float* __restrict__ y, int* __restrict__ err) {
  using namespace tc;
  typedef __nv_bfloat16 bf;
  extern __shared__ __align__(128) unsigned char tsm[];
  bf* sW1 = reinterpret_cast<bf*>(tsm);                        // [256 x 80] core matrices
  bf* sW2 = sW1 + kH * kF;                                     // [256 x 256]
  bf* sX = sW2 + kH * kH;                                      // [128 x 80]
  bf* sH = sX;                                                 // [128 x 64], aliases x
  float* b1s = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sX) + kXH);
  float* b2s = b1s + kH;
  float* w3s = b2s + kH;
  float* yp = w3s + kH;                                        // [128][2]
  __shared__ __align__(8) unsigned long long wbar, mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntiles = (n + kTT - 1) / kTT;

  if (tid == 0) {
    mbar_init(&wbar, 1);
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) bulk_load(sW1, wpack, (uint32_t)(kW1 + kW2), &wbar);
  for (int i = tid; i < kH; i += kThreads) {
    b1s[i] = b1[i];
    b2s[i] = b2[i];
    w3s[i] = w3[i];
  }
  const float bias3 = b3[0];
  const bool wok = mbar_wait(&wbar, 0);
  if (!__syncthreads_and(wok)) {
    if (!wok) mbar_wait(&wbar, 0);                // let the copy land before leaving
    if (tid == 0) atomicExch(err, 1);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      if (tid < kTT && tile * kTT + tid < n) y[tile * kTT + tid] = __int_as_float(0x7fc00000);
    return;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  const uint32_t id = idesc(kTT, kH);
  const uint32_t aX = smem_addr(sX), aW1 = smem_addr(sW1), aH = smem_addr(sH),
                 aW2 = smem_addr(sW2);
  const int q = warp & 3;                                       // TMEM lane quadrant
  const int cg = warp >> 2;                                     // column half of the epilogues
  const int row = 32 * q + lane;                                // this thread's tile row
  uint32_t ph = 0;
  bool ok = true;
  // one commit of the issuing thread, waited for by every thread
  auto wait_mma = [&]() -> bool {
    const bool w = mbar_wait(&mbar, ph);
    ph ^= 1u;
    fence_after();
    return __syncthreads_and(w) != 0;
  };

  int tile = blockIdx.x;
  for (; tile < ntiles && ok; tile += gridDim.x) {
    const int r0 = tile * kTT;
    // ---- features: warp w builds rows [16 w, 16 w + 16); lane l holds
    // dimensions 2 l and 2 l + 1 of all sixteen, so every embedding load is
    // one 256-byte row for the whole warp; sums run in column order, as in
    // the other paths ----
    {
      const int rb = warp * 16, k = lane & 15, grow = r0 + rb + k;
      const int L = grow < n ? min(max(len[grow], 0), stride) : 0;
      const uint16_t* sp = seq + (size_t)(grow < n ? grow : 0) * stride;
      const int Lmax = __reduce_max_sync(0xffffffffu, L);
      const float2* e2 = reinterpret_cast<const float2*>(emb) + lane;   // 32 float2 a column
      float2 acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
      float m = 0.f, dsum = 0.f;
      // two columns a step (32 loads in flight a lane); the next step's
      // column ids are read one step ahead
      int cn0 = L > 0 ? (int)__ldg(sp) : C, cn1 = L > 1 ? (int)__ldg(sp + 1) : C;
      for (int i = 0; i < Lmax; i += 2) {
        const int c0 = cn0, c1 = cn1;
        cn0 = i + 2 < L ? (int)__ldg(sp + i + 2) : C;
        cn1 = i + 3 < L ? (int)__ldg(sp + i + 3) : C;
        int cc0[16], cc1[16];
        float2 v0[16], v1[16];
        const uint32_t pair = (uint32_t)c0 | ((uint32_t)c1 << 16);   // both ids < 65,536
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t pj = __shfl_sync(0xffffffffu, pair, j);
          cc0[j] = (int)(pj & 0xFFFFu);
          cc1[j] = (int)(pj >> 16);
          v0[j] = cc0[j] < C ? ld_keep(e2 + (size_t)cc0[j] * 32) : make_float2(0.f, 0.f);
          v1[j] = cc1[j] < C ? ld_keep(e2 + (size_t)cc1[j] * 32) : make_float2(0.f, 0.f);
        }
        if (lane < 16) {
          if (c0 < C) {
            m += cmean[c0];
            dsum += csd[c0];
          }
          if (c1 < C) {
            m += cmean[c1];
            dsum += csd[c1];
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (cc0[j] < C) {
            acc[j].x += v0[j].x;
            acc[j].y += v0[j].y;
          }
          if (cc1[j] < C) {
            acc[j].x += v1[j].x;
            acc[j].y += v1[j].y;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        *reinterpret_cast<__nv_bfloat162*>(sX + cm(rb + j, 2 * lane, kF)) =
            __floats2bfloat162_rn(acc[j].x, acc[j].y);
      if (lane < 16) {
        __align__(16) bf o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16_rn(0.f);
        o[0] = __float2bfloat16_rn(L ? m / (float)L : 0.f);
        o[1] = __float2bfloat16_rn(L ? dsum / (float)L : 0.f);
        o[2] = __float2bfloat16_rn((float)L / len_scale);
        *reinterpret_cast<uint4*>(sX + cm(rb + k, 64, kF)) = *reinterpret_cast<const uint4*>(o);
        *reinterpret_cast<uint4*>(sX + cm(rb + k, 72, kF)) = *reinterpret_cast<const uint4*>(o + 8);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    // ---- layer 1 into TMEM columns [0, 256) ----
    if (tid == 0) {
      for (int k0 = 0; k0 < kF; k0 += 16)
        mma(tmem, sdesc(aX + (k0 / 8) * 128, 128, (kF / 8) * 128),
            sdesc(aW1 + (k0 / 8) * 128, 128, (kF / 8) * 128), id, k0 > 0);
      commit(&mbar);
    }
    if (!(ok = wait_mma())) break;
    // ---- h1 by quarters of 64 columns, each followed by its layer-2 MMAs
    // (the first quarter overwrites x, which the completed layer-1 MMAs no
    // longer read) ----
    for (int h = 0; h < kH / kQ && ok; ++h) {
      const int c0 = 32 * cg;                                   // column within the quarter
      float v[32];
      ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kQ * h + c0), v);
#pragma unroll
      for (int g8 = 0; g8 < 4; ++g8) {
        __align__(16) bf o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          o[i] = __float2bfloat16_rn(fmaxf(v[8 * g8 + i] + b1s[kQ * h + c0 + 8 * g8 + i], 0.f));
        *reinterpret_cast<uint4*>(sH + cm(row, c0 + 8 * g8, kQ)) =
            *reinterpret_cast<const uint4*>(o);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        for (int k0 = 0; k0 < kQ; k0 += 16)
          mma(tmem + (uint32_t)kH, sdesc(aH + (k0 / 8) * 128, 128, (kQ / 8) * 128),
              sdesc(aW2 + ((kQ * h + k0) / 8) * 128, 128, (kH / 8) * 128), id, h > 0 || k0 > 0);
        commit(&mbar);
      }
      ok = wait_mma();
    }
    if (!ok) break;
    // ---- y = relu(h1 W2 + b2) . w3 + b3 ----
    float p = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c0 = 128 * cg + 32 * t;
      float v[32];
      ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kH + c0), v);
#pragma unroll
      for (int i = 0; i < 32; ++i)
        p += __bfloat162float(__float2bfloat16_rn(fmaxf(v[i] + b2s[c0 + i], 0.f))) * w3s[c0 + i];
    }
    yp[row * 2 + cg] = p;
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < kTT && r0 + tid < n) y[r0 + tid] = bias3 + yp[tid * 2] + yp[tid * 2 + 1];
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    for (; tile < ntiles; tile += gridDim.x)
      if (tid < kTT && tile * kTT + tid < n) y[tile * kTT + tid] = __int_as_float(0x7fc00000);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace ebic
