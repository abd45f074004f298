// Fitness surrogate: a small MLP that predicts a series' standardised
// log-fitness from sum-pooled column features, trained on (series, exact
// fitness) pairs that EBIC runs log, and used to pre-screen oversampled
// offspring.  Not part of the paper: the exact evaluator (Eq. (1) on exact
// support) still scores every individual that enters a population.
//
//   features  x[0:64] = sum of learned column embeddings, x[64] = mean column
//             mean, x[65] = mean column standard deviation, x[66] = length /
//             len_scale, x[67:80] = 0
//   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 . w3 + b3
//
// Forward and backward are this file's kernels: bf16 operands on the tensor
// cores (mma.sync m16n8k16, fp32 accumulation) with the bias / ReLU / ReLU-mask
// epilogues fused into the GEMM, fp32 master weights, Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ebic_async.cuh"
#include "ebic_internal.cuh"
#include "ebic_tcmlp.cuh"
#include "ebic_tcgemm.cuh"

namespace ebic {

constexpr int kF = 80;     // feature width (67 used, padded to a multiple of 16)
constexpr int kEmb = 64;
constexpr int kH = 256;

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// column statistics of the handle's matrix (mean, population sd; NaN skipped)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_colstats(const float* __restrict__ A_c, int32_t R,
                                                  int32_t R_pad, float* mean, float* sd) {
  const int c = blockIdx.x;
  const float* col = A_c + (size_t)c * R_pad;
  double s = 0.0, s2 = 0.0;
  long long n = 0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const float v = col[r];
    if (v == v) {
      s += v;
      s2 += (double)v * v;
      ++n;
    }
  }
  __shared__ double ss[256], ss2[256];
  __shared__ long long sn[256];
  ss[threadIdx.x] = s;
  ss2[threadIdx.x] = s2;
  sn[threadIdx.x] = n;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      ss2[threadIdx.x] += ss2[threadIdx.x + o];
      sn[threadIdx.x] += sn[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = sn[0] ? ss[0] / (double)sn[0] : 0.0;
    const double var = sn[0] ? ss2[0] / (double)sn[0] - m * m : 0.0;
    mean[c] = (float)m;
    sd[c] = (float)sqrt(var > 0.0 ? var : 0.0);
  }
}

// ---------------------------------------------------------------------------
// features: one warp per series (lanes over the 64 embedding dimensions x 2)
// ---------------------------------------------------------------------------
// (a length outside [0, stride] is clamped and a column >= C skipped, so that
// stale or unused rows read nothing out of bounds)
__global__ void __launch_bounds__(256)
k_features(const uint16_t* __restrict__ seq, const int32_t* __restrict__ len, int32_t stride,
           const int32_t* __restrict__ idx, int32_t n, int32_t C, const float* __restrict__ emb,
           const float* __restrict__ cmean, const float* __restrict__ csd, float len_scale,
           bf16* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= n) return;
  const long long r = idx ? (long long)idx[b] : b;
  const int L = min(max(len[r], 0), stride);
  const uint16_t* s = seq + (size_t)r * stride;
  float e0 = 0.f, e1 = 0.f, m = 0.f, d = 0.f;
  for (int i = 0; i < L; ++i) {
    const int c = s[i];
    if (c >= C) continue;
    e0 += emb[(size_t)c * kEmb + lane];
    e1 += emb[(size_t)c * kEmb + 32 + lane];
    m += cmean[c];
    d += csd[c];
  }
  bf16* o = x + (size_t)b * kF;
  o[lane] = __float2bfloat16_rn(e0);
  o[32 + lane] = __float2bfloat16_rn(e1);
  if (lane < 16) {
    float v = 0.f;
    if (lane == 0) v = L ? m / (float)L : 0.f;
    if (lane == 1) v = L ? d / (float)L : 0.f;
    if (lane == 2) v = (float)L / len_scale;
    o[64 + lane] = __float2bfloat16_rn(v);
  }
}

// ---------------------------------------------------------------------------
// GEMM on the tensor cores: C[M x N] = op(A)[M x K] . op(B)[K x N], bf16
// operands, fp32 accumulation (mma.sync m16n8k16).  op(A)(m, k) = A[m*lda+k]
// (TA: A[k*lda+m]); op(B)(k, n) = B[k*ldb+n] (TB: B[n*ldb+k]).  CTA tile
// 64 x 64 x 32, four warps of 32 x 32.  gridDim.z splits K: with
// EPI_F32_SPLIT split z writes its partial product to slice z of Cf
// ([splits][M][ldc]), summed afterwards in split order (k_sum_splits), so the
// result does not depend on scheduling.  grid = (M tiles, N tiles, K splits).
// ---------------------------------------------------------------------------
enum { EPI_BIAS_RELU_BF16 = 0, EPI_MASK_BF16 = 1, EPI_F32 = 2, EPI_F32_SPLIT = 3 };
constexpr int kBM = 64, kBN = 64, kBK = 32;

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128)
k_gemm_bf16(int M, int N, int K, const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
            int ldb, const float* __restrict__ bias, const bf16* __restrict__ mask, int ldm,
            float* __restrict__ Cf, bf16* __restrict__ Cb, int ldc) {
  __shared__ bf16 As[kBM][kBK + 8];    // (m, k)
  __shared__ bf16 Bs[kBN][kBK + 8];    // (n, k)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;   // M can exceed 65535 tiles
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, tq = lane & 3;
  const int ksplit = gridDim.z;
  const int kchunk = ((K + ksplit - 1) / ksplit + kBK - 1) / kBK * kBK;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const bf16 zero = __float2bfloat16_rn(0.f);
  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
    for (int e = tid; e < kBM * kBK; e += 128) {
      const int mm = TA ? e % kBM : e / kBK, kk = TA ? e / kBM : e % kBK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[mm][kk] = (gm < M && gk < kend) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk])
                                         : zero;
    }
    for (int e = tid; e < kBN * kBK; e += 128) {
      const int nn = TB ? e / kBK : e % kBN, kk = TB ? e % kBK : e / kBN;
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[nn][kk] = (gn < N && gk < kend) ? (TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn])
                                         : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      uint32_t a[2][4], bq[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + g;
        a[i][0] = pack2(As[r][kk + tq * 2], As[r][kk + tq * 2 + 1]);
        a[i][1] = pack2(As[r + 8][kk + tq * 2], As[r + 8][kk + tq * 2 + 1]);
        a[i][2] = pack2(As[r][kk + 8 + tq * 2], As[r][kk + 8 + tq * 2 + 1]);
        a[i][3] = pack2(As[r + 8][kk + 8 + tq * 2], As[r + 8][kk + 8 + tq * 2 + 1]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + g;
        bq[j][0] = pack2(Bs[c][kk + tq * 2], Bs[c][kk + tq * 2 + 1]);
        bq[j][1] = pack2(Bs[c][kk + 8 + tq * 2], Bs[c][kk + 8 + tq * 2 + 1]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
              "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(bq[j][0]),
                "r"(bq[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + tq * 2 + (q & 1);
        if (m >= M || n >= N) continue;
        float v = acc[i][j][q];
        if (EPI == EPI_BIAS_RELU_BF16) {
          v = fmaxf(v + bias[n], 0.f);
          Cb[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
        } else if (EPI == EPI_MASK_BF16) {
          v = __bfloat162float(mask[(size_t)m * ldm + n]) > 0.f ? v : 0.f;
          Cb[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
        } else if (EPI == EPI_F32) {
          Cf[(size_t)m * ldc + n] = v;
        } else {
          Cf[(size_t)blockIdx.z * M * ldc + (size_t)m * ldc + n] = v;
        }
      }
}

// y = h2 . w3 + b3 (warp per row); with targets: dy = 2 (y - t) / B and the
// row's share of the mean squared error, (y - t)^2 / B, in sq (summed later
// in row order)
__global__ void __launch_bounds__(256)
k_out(const bf16* __restrict__ h2, const float* __restrict__ w3, const float* __restrict__ b3,
      int n, float* __restrict__ y, const float* __restrict__ t, const int32_t* __restrict__ idx,
      float* __restrict__ dy, float* __restrict__ sq) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= n) return;
  float s = 0.f;
  for (int j = lane; j < kH; j += 32) s += __bfloat162float(h2[(size_t)b * kH + j]) * w3[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  s += b3[0];
  if (lane == 0) {
    y[b] = s;
    if (t) {
      const float tt = t[idx ? idx[b] : b];
      const float r = s - tt;
      dy[b] = 2.f * r / (float)n;
      sq[b] = r * r / (float)n;
    }
  }
}

// dh2[b][j] = dy[b] w3[j] [h2[b][j] > 0]  (bf16)
__global__ void __launch_bounds__(256) k_dh2(const float* __restrict__ dy,
                                             const float* __restrict__ w3,
                                             const bf16* __restrict__ h2, int n,
                                             bf16* __restrict__ dh2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * kH) return;
  const int b = (int)(i / kH), j = (int)(i % kH);
  const float v = __bfloat162float(h2[i]) > 0.f ? dy[b] * w3[j] : 0.f;
  dh2[i] = __float2bfloat16_rn(v);
}

// Column sums out[j] = sum_b scale[b] * X[b][j] for j < cols (scale =
// nullptr: 1), in two fixed-order levels so that the result does not depend
// on scheduling: CTA (32-column tile, segment of kColSeg rows) has its eight
// warps take every eighth row of the segment, each in row order, adds the
// warps in order and writes part[segment][j]; k_sum_splits then adds the
// segments in order.  X bf16 (or fp32 via Xf).
constexpr int kColSeg = 128;
__global__ void __launch_bounds__(256)
k_colsum_part(const bf16* __restrict__ Xb, const float* __restrict__ Xf, int n, int cols,
              const float* __restrict__ scale, float* __restrict__ part) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r0 = threadIdx.x >> 5;
  const int b_lo = blockIdx.y * kColSeg, b_hi = min(n, b_lo + kColSeg);
  float s = 0.f;
  if (c < cols) {
#pragma unroll 4
    for (int b = b_lo + r0; b < b_hi; b += 8) {
      const float v = Xb ? __bfloat162float(Xb[(size_t)b * cols + c]) : Xf[(size_t)b * cols + c];
      s += scale ? scale[b] * v : v;
    }
  }
  __shared__ float red[8][33];
  red[r0][threadIdx.x & 31] = s;
  __syncthreads();
  if (r0 == 0 && c < cols) {
    float t = 0.f;
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x & 31];
    part[(size_t)blockIdx.y * cols + c] = t;
  }
}

// Embedding gradient without atomics: dEmb[c] = sum over the batch's series
// b of (occurrences of c in series b) * dx[b][0:64].  CTA (column tile of 64,
// series segment) accumulates its segment in series order into
// part[segment][c][64]; k_emb_grad_reduce adds the segments in order.
constexpr int kEmbSeg = 32;     // series per chunk held in shared memory
__global__ void __launch_bounds__(256)
k_emb_grad_part(const uint16_t* __restrict__ seq, const int32_t* __restrict__ len, int32_t stride,
                const int32_t* __restrict__ idx, int32_t B, int32_t C, int32_t seg_len,
                const float* __restrict__ dx, float* __restrict__ part) {
  __shared__ float dxs[kEmbSeg][kEmb];
  __shared__ uint8_t cnt[kEmbSeg][64];
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * 64, seg = blockIdx.y;
  const int cc = tid >> 2, k0 = (tid & 3) * 16;            // column in tile, 16 dims
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  const int b_lo = seg * seg_len, b_hi = min(B, b_lo + seg_len);
  for (int b0 = b_lo; b0 < b_hi; b0 += kEmbSeg) {
    for (int i = tid; i < kEmbSeg * kEmb; i += 256) {
      const int bb = i / kEmb, k = i % kEmb;
      dxs[bb][k] = b0 + bb < b_hi ? dx[(size_t)(b0 + bb) * kF + k] : 0.f;
    }
    for (int i = tid; i < kEmbSeg * 64; i += 256) cnt[i / 64][i % 64] = 0;
    __syncthreads();
    if (tid < kEmbSeg && b0 + tid < b_hi) {                  // one thread per series
      const long long r = idx ? (long long)idx[b0 + tid] : b0 + tid;
      const int L = min(max(len[r], 0), stride);
      const uint16_t* sp = seq + (size_t)r * stride;
      for (int i = 0; i < L; ++i) {
        const int c = sp[i] - c0;
        if (c >= 0 && c < 64 && sp[i] < C) cnt[tid][c] += 1;
      }
    }
    __syncthreads();
    const int nb = min(kEmbSeg, b_hi - b0);
    for (int bb = 0; bb < nb; ++bb) {
      const float w = (float)cnt[bb][cc];
      if (w != 0.f) {
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] += w * dxs[bb][k0 + q];
      }
    }
    __syncthreads();
  }
  const int c = c0 + cc;
  if (c < C) {
    float* o = part + ((size_t)seg * C + c) * kEmb + k0;
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q] = acc[q];
  }
}

__global__ void k_sum_splits(const float* __restrict__ part, int splits, long long count,
                             float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * count + i];
  out[i] = s;
}

// Adam over one flat parameter array; optional bf16 copy of the result
__global__ void __launch_bounds__(256)
k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
       float c2, bf16* __restrict__ copy, const float2* __restrict__ ctab,
       const int32_t* __restrict__ ctr) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (ctab) {                                       // replayed step: its corrections
    const float2 c = ctab[*ctr];
    c1 = c.x;
    c2 = c.y;
  }
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (copy) copy[i] = __float2bfloat16_rn(pi);
}

// The replay index of a captured training step, advanced at its end.
__global__ void k_step_advance(int32_t* ctr) { *ctr += 1; }

__global__ void k_to_bf16(const float* __restrict__ src, bf16* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// W1^T and W2^T in the fused forward's shared-memory layout (bf16, rows of
// kF + 8 / kH + 8 with zero padding), from the fp32 masters W1 [kF][kH] and
// W2 [kH][kH]; one bulk copy moves the result into shared memory.
__global__ void k_pack_fwd(const float* __restrict__ W1, const float* __restrict__ W2,
                           bf16* __restrict__ out) {
  constexpr int ldx = kF + 8, ldh = kH + 8;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kH * ldx) {
    const int nn = i / ldx, k = i % ldx;
    out[i] = __float2bfloat16_rn(k < kF ? W1[k * kH + nn] : 0.f);
  } else if (i < kH * ldx + kH * ldh) {
    const int r = i - kH * ldx, nn = r / ldh, k = r % ldh;
    out[i] = __float2bfloat16_rn(k < kH ? W2[k * kH + nn] : 0.f);
  }
}

// standardised log1p targets: t = (log1p(f) - mean) / sd
__global__ void k_targets(const double* __restrict__ f, long long n, float mean, float sd,
                          float* __restrict__ t) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] = (float)((log1p(f[i]) - (double)mean) / (double)sd);
}

// Sum and sum of squares of log1p(f): block b writes its partial sums to
// out[2 b], out[2 b + 1] (a fixed-order tree inside the block); the host adds
// the blocks in order.
__global__ void __launch_bounds__(256) k_sum_log1p(const double* __restrict__ f, long long n,
                                                  double* __restrict__ out) {
  __shared__ double r1[256], r2[256];
  double s = 0.0, s2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = log1p(f[i]);
    s += v;
    s2 += v * v;
  }
  r1[threadIdx.x] = s;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = r1[0];
    out[2 * blockIdx.x + 1] = r2[0];
  }
}

// minibatch indices: idx[b] = floor(u * n), u from Philox-4x32-10 keyed by (seed, step)
__global__ void k_sample(uint64_t seed, uint32_t step, long long n, int B, int32_t* idx,
                         const int32_t* __restrict__ ctr) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (ctr) step += (uint32_t)*ctr;                  // replayed step: base + replay index
  uint32_t x0 = (uint32_t)b, x1 = step, x2 = 0x5EEDu, x3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    const uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
  }
  idx[b] = (int32_t)((((unsigned long long)x0 << 32 | x1) % (unsigned long long)n));
}

// ---------------------------------------------------------------------------
// Fused forward pass for scoring (no activations kept): a persistent CTA holds
// W1^T and W2^T in shared memory (bf16, padded rows against bank conflicts)
// and loops over tiles of 64 series.  Per tile: features by the 8 warps (one
// series per warp at a time, embedding sums in fp32, rounded to bf16 as in
// k_features), h1 = relu(x W1 + b1) and h2 = relu(h1 W2 + b2) on the tensor
// cores (mma.sync m16n8k16 bf16, fp32 accumulation; warp w owns output
// columns [32 w, 32 w + 32)), and y = h2 . w3 + b3 reduced in the second
// epilogue, so h2 never leaves registers.
// ---------------------------------------------------------------------------
constexpr int kFT = 64;                 // series per tile
constexpr int kLdX = kF + 8;            // row stride (bf16) of x and W1^T
constexpr int kLdH = kH + 8;            // row stride (bf16) of h1 and W2^T
constexpr int kFwdThreads = 256;
constexpr size_t kFwdSmem = (size_t)kH * kLdX * 2 + (size_t)kH * kLdH * 2 +
                            (size_t)kFT * kLdX * 2 + (size_t)kFT * kLdH * 2 +
                            (size_t)kFT * 8 * 4 + 3 * (size_t)kH * 4;

__device__ __forceinline__ uint32_t lds32(const bf16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kFwdThreads, 1)
k_mlp_forward(const uint16_t* __restrict__ seq, const int32_t* __restrict__ len, int32_t stride,
              int32_t n, int32_t C, const float* __restrict__ emb,
              const float* __restrict__ cmean, const float* __restrict__ csd, float len_scale,
              const bf16* __restrict__ wpack, const float* __restrict__ b1,
              const float* __restrict__ b2, const float* __restrict__ w3,
              const float* __restrict__ b3, float* __restrict__ y, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char fsm[];
  bf16* w1t = reinterpret_cast<bf16*>(fsm);                 // [kH][kLdX]
  bf16* w2t = w1t + kH * kLdX;                              // [kH][kLdH]
  bf16* xs = w2t + kH * kLdH;                               // [kFT][kLdX]
  bf16* hs = xs + kFT * kLdX;                               // [kFT][kLdH]
  float* yp = reinterpret_cast<float*>(hs + kFT * kLdH);    // [kFT][8]
  float* b1s = yp + kFT * 8;
  float* b2s = b1s + kH;
  float* w3s = b2s + kH;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;

  // W1^T and W2^T (packed by k_pack_fwd in this layout) by one bulk copy
  __shared__ __align__(8) unsigned long long wbar;
  constexpr uint32_t kWBytes = (uint32_t)((kH * kLdX + kH * kLdH) * sizeof(bf16));
  if (tid == 0) {
    mbar_init(&wbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) bulk_load(w1t, wpack, kWBytes, &wbar);
  for (int i = tid; i < kH; i += kFwdThreads) {
    b1s[i] = b1[i];
    b2s[i] = b2[i];
    w3s[i] = w3[i];
  }
  const float bias3 = b3[0];
  const bool ok = mbar_wait(&wbar, 0);
  if (!__syncthreads_and(ok)) {
    // the copy did not complete in time: wait once more (bounded) for it to
    // land before the CTA exits, flag the error, leave NaN scores
    if (!ok) mbar_wait(&wbar, 0);
    if (tid == 0) atomicExch(err, 1);
    const int ntiles_ = (n + kFT - 1) / kFT;
    for (int tile = blockIdx.x; tile < ntiles_; tile += gridDim.x)
      if (tid < kFT && tile * kFT + tid < n) y[tile * kFT + tid] = __int_as_float(0x7fc00000);
    return;
  }

  const int ntiles = (n + kFT - 1) / kFT;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile * kFT;
    // ---- features: warp w fills rows 8 w .. 8 w + 7 ----
    for (int rr = 0; rr < 8; ++rr) {
      const int lr = warp * 8 + rr, row = r0 + lr;
      float e0 = 0.f, e1 = 0.f, m = 0.f, dsum = 0.f;
      int L = 0;
      if (row < n) {
        L = min(max(len[row], 0), stride);
        const uint16_t* sp = seq + (size_t)row * stride;
        const int cA = lane < L ? (int)sp[lane] : 0;
        const int cB = lane + 32 < L ? (int)sp[lane + 32] : 0;
#pragma unroll 4
        for (int i = 0; i < L; ++i) {
          const int c = __shfl_sync(0xffffffffu, i < 32 ? cA : cB, i & 31);
          if (c >= C) continue;
          e0 += emb[(size_t)c * kEmb + lane];
          e1 += emb[(size_t)c * kEmb + 32 + lane];
          m += cmean[c];
          dsum += csd[c];
        }
      }
      bf16* xr = xs + lr * kLdX;
      xr[lane] = __float2bfloat16_rn(e0);
      xr[32 + lane] = __float2bfloat16_rn(e1);
      if (lane < 16) {
        float v = 0.f;
        if (lane == 0) v = L ? m / (float)L : 0.f;
        if (lane == 1) v = L ? dsum / (float)L : 0.f;
        if (lane == 2) v = (float)L / len_scale;
        xr[64 + lane] = __float2bfloat16_rn(v);
      }
    }
    __syncthreads();
    const int n0 = warp * 32;
    // ---- layer 1: h1 = relu(x W1 + b1), K = 80 ----
    {
      float acc[4][4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll
      for (int k0 = 0; k0 < kF; k0 += 16) {
        uint32_t bq[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bf16* bp = w1t + (n0 + 8 * j + g) * kLdX + k0 + 2 * tq;
          bq[j][0] = lds32(bp);
          bq[j][1] = lds32(bp + 8);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bf16* ap = xs + (16 * i + g) * kLdX + k0 + 2 * tq;
          const uint32_t a0 = lds32(ap), a1 = lds32(ap + 8 * kLdX), a2 = lds32(ap + 8),
                         a3 = lds32(ap + 8 * kLdX + 8);
#pragma unroll
          for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a0, a1, a2, a3, bq[j][0], bq[j][1]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int col = n0 + 8 * j + 2 * tq;
          const int ra = 16 * i + g;
          const float bA = b1s[col], bB = b1s[col + 1];
          __nv_bfloat162 lo, hi;
          lo.x = __float2bfloat16_rn(fmaxf(acc[i][j][0] + bA, 0.f));
          lo.y = __float2bfloat16_rn(fmaxf(acc[i][j][1] + bB, 0.f));
          hi.x = __float2bfloat16_rn(fmaxf(acc[i][j][2] + bA, 0.f));
          hi.y = __float2bfloat16_rn(fmaxf(acc[i][j][3] + bB, 0.f));
          *reinterpret_cast<__nv_bfloat162*>(hs + ra * kLdH + col) = lo;
          *reinterpret_cast<__nv_bfloat162*>(hs + (ra + 8) * kLdH + col) = hi;
        }
    }
    __syncthreads();
    // ---- layer 2 + output: y = relu(h1 W2 + b2) . w3 + b3, K = 256 ----
    {
      float acc[4][4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll 4
      for (int k0 = 0; k0 < kH; k0 += 16) {
        uint32_t bq[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bf16* bp = w2t + (n0 + 8 * j + g) * kLdH + k0 + 2 * tq;
          bq[j][0] = lds32(bp);
          bq[j][1] = lds32(bp + 8);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bf16* ap = hs + (16 * i + g) * kLdH + k0 + 2 * tq;
          const uint32_t a0 = lds32(ap), a1 = lds32(ap + 8 * kLdH), a2 = lds32(ap + 8),
                         a3 = lds32(ap + 8 * kLdH + 8);
#pragma unroll
          for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a0, a1, a2, a3, bq[j][0], bq[j][1]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float pa = 0.f, pb = 0.f;               // rows 16 i + g and 16 i + g + 8
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int col = n0 + 8 * j + 2 * tq;
          const float vA = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[i][j][0] + b2s[col], 0.f)));
          const float vB = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[i][j][1] + b2s[col + 1], 0.f)));
          const float vC = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[i][j][2] + b2s[col], 0.f)));
          const float vD = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[i][j][3] + b2s[col + 1], 0.f)));
          pa += vA * w3s[col] + vB * w3s[col + 1];
          pb += vC * w3s[col] + vD * w3s[col + 1];
        }
        pa += __shfl_xor_sync(0xffffffffu, pa, 1);
        pa += __shfl_xor_sync(0xffffffffu, pa, 2);
        pb += __shfl_xor_sync(0xffffffffu, pb, 1);
        pb += __shfl_xor_sync(0xffffffffu, pb, 2);
        if (tq == 0) {
          yp[(16 * i + g) * 8 + warp] = pa;
          yp[(16 * i + g + 8) * 8 + warp] = pb;
        }
      }
    }
    __syncthreads();
    if (tid < kFT && r0 + tid < n) {
      float t = bias3;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += yp[tid * 8 + w];
      y[r0 + tid] = t;
    }
  }
}

}  // namespace ebic

using namespace ebic;

struct ebic_surrogate_ctx {
  int device = 0;
  int32_t C = 0;
  float len_scale = 64.f;
  float t_mean = 0.f, t_sd = 1.f;
  int32_t steps_done = 0;
  int32_t attached = 0;        // runs screening with this surrogate
  uint64_t seed = 0;
  ebic_handle h = nullptr;
  cudaStream_t stream = nullptr;
  // fp32 master parameters, gradients and Adam moments: one flat buffer each,
  // Emb[C * 64] | W1[80 * 256] | b1[256] | W2[256 * 256] | b2[256] | w3[256] | b3[1]
  long long n_par = 0;
  long long o_emb = 0, o_w1 = 0, o_b1 = 0, o_w2 = 0, o_b2 = 0, o_w3 = 0, o_b3 = 0;
  DevBuf par, grad, mom, vel, w1b, w2b, cmean, csd;
  DevBuf wpack;                // W1^T | W2^T in the fused forward's layout (bf16)
  DevBuf wpack_tc;             // W1^T | W2^T in the tcgen05 forward's layout (bf16)
  int32_t fwd_kind = 0;        // scoring kernel: 0 tcgen05, 1 mma.sync
  int32_t gemm_kind = 0;       // training GEMMs: 0 tcgen05, 1 mma.sync
  int32_t sm_count = 0;
  DevBuf ferr;                 // set by the fused forward on a copy timeout
  // training activations (capacity rows)
  int32_t cap = 0;
  DevBuf act, dh1, dh2, dx, y, dy, idx, loss, tgt, tmp, sq, split, epart, csplit;
  DevBuf ctab, ctr;            // replayed training: Adam corrections per step, replay index
  // training log: series [log_n][kLogStride], lengths, exact fitness
  long long log_n = 0, log_cap = 0;
  DevBuf log_seq, log_len, log_fit;

  // series per segment of the embedding gradient: at most 32 segments and at
  // most 16 MB of partial sums, each segment a multiple of 32 series
  int emb_seg_len(int B) const {
    long long segs = std::min<long long>(32, std::max<long long>(1, (16ll << 20) / ((long long)C * 64 * 4)));
    segs = std::min<long long>(segs, (B + 31) / 32);
    long long len = (B + segs - 1) / segs;
    return (int)((len + 31) / 32 * 32);
  }
};

namespace ebic {

constexpr int kLogStride = EBIC_MAX_EA_LEN;
constexpr int kSumBlocks = 456;     // partial sums of the target statistics

// x [rows][80] | h1 [rows][256] | h2 [rows][256], bf16, each 256-byte aligned
static inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
size_t sur_act_bytes(long long rows) {
  const size_t r = (size_t)rows;
  return round256(r * kF * sizeof(bf16)) + 2 * round256(r * kH * sizeof(bf16));
}
struct ActView {
  bf16 *x, *h1, *h2;
};
static ActView act_view(void* base, long long rows) {
  char* p = static_cast<char*>(base);
  ActView a;
  a.x = reinterpret_cast<bf16*>(p);
  p += round256((size_t)rows * kF * sizeof(bf16));
  a.h1 = reinterpret_cast<bf16*>(p);
  p += round256((size_t)rows * kH * sizeof(bf16));
  a.h2 = reinterpret_cast<bf16*>(p);
  return a;
}

int32_t sur_columns(const ebic_surrogate_ctx* s) { return s->C; }
void sur_attach(ebic_surrogate_ctx* s, int delta) { s->attached += delta; }

static ebic_status sur_reserve(ebic_surrogate_ctx* s, int32_t rows) {
  if (rows <= s->cap) return EBIC_OK;
  const size_t r = (size_t)rows;
  EBIC_TRY(s->act.reserve(sur_act_bytes(rows)));
  EBIC_TRY(s->dh1.reserve(r * kH * sizeof(bf16)));
  EBIC_TRY(s->dh2.reserve(r * kH * sizeof(bf16)));
  EBIC_TRY(s->dx.reserve(r * kF * sizeof(float)));
  EBIC_TRY(s->y.reserve(r * sizeof(float)));
  EBIC_TRY(s->dy.reserve(r * sizeof(float)));
  EBIC_TRY(s->idx.reserve(r * sizeof(int32_t)));
  EBIC_TRY(s->sq.reserve(r * sizeof(float)));
  const int ks = std::max(1, std::min(32, rows / 256));
  EBIC_TRY(s->split.reserve((size_t)ks * kH * kH * sizeof(float)));
  EBIC_TRY(s->csplit.reserve((size_t)((rows + kColSeg - 1) / kColSeg) * kH * sizeof(float)));
  const int seg = s->emb_seg_len(rows);
  EBIC_TRY(s->epart.reserve((size_t)((rows + seg - 1) / seg) * s->C * kEmb * sizeof(float)));
  s->cap = rows;
  return EBIC_OK;
}

template <bool TA, bool TB, int EPI>
static void gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
                 const float* bias, const bf16* mask, int ldm, float* Cf, bf16* Cb, int ldc,
                 int ksplit, cudaStream_t st) {
  dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN), (unsigned)ksplit);
  k_gemm_bf16<TA, TB, EPI><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, bias, mask, ldm, Cf,
                                                  Cb, ldc);
}

// out[0 .. cols) = the column sums of k_colsum_part (2 launches).
static void colsum(ebic_surrogate_ctx* s, const bf16* Xb, const float* Xf, int n, int cols,
                   const float* scale, float* out, cudaStream_t st) {
  const int nseg = (n + kColSeg - 1) / kColSeg;
  k_colsum_part<<<dim3((unsigned)((cols + 31) / 32), (unsigned)nseg), 256, 0, st>>>(
      Xb, Xf, n, cols, scale, s->csplit.as<float>());
  k_sum_splits<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(s->csplit.as<float>(), nseg,
                                                               (long long)cols, out);
}

// ---- the tcgen05 training GEMMs (ebic_tcgemm.cuh) ----

typedef CUresult (*TmapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of a K-major bf16 matrix (rows x cols, row pitch ld elements)
// in boxes of 8 columns x box_rows rows; rows past the end read as zeros.
static ebic_status tmap_kmajor(CUtensorMap* m, const bf16* p, int rows, int cols, int ld,
                               int box_rows) {
  static TmapEncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    EBIC_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn)
      return fail(EBIC_ERR_CUDA, "the CUDA driver API has no tensor-map encoder entry point");
    encode = reinterpret_cast<TmapEncodeFn>(fn);
  }
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t pitch[1] = {(cuuint64_t)ld * sizeof(bf16)};
  const cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
  const cuuint32_t step[2] = {1u, 1u};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(p), dim,
                            pitch, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(EBIC_ERR_CUDA, "tensor-map encoding failed");
  return EBIC_OK;
}

// D[M x N] = A[M x K] . op(B), A K-major (pitch lda); B either K-major as
// N x K (Bk, pitch ldb) or the packed W^T at Bpacked.  One launch.
template <int BSRC, int EPI>
static ebic_status gemm_tc_full(ebic_surrogate_ctx* s, int M, int N, int K, const bf16* A,
                                int lda, const bf16* Bk, int ldb, const bf16* Bpacked,
                                const float* bias, const bf16* mask, int ldm, float* Cf,
                                bf16* Cb, int ldc, cudaStream_t st) {
  CUtensorMap ta, tb;
  std::memset(&tb, 0, sizeof(tb));
  EBIC_TRY(tmap_kmajor(&ta, A, M, K, lda, tcg::kTM));
  if (BSRC == tcg::B_TMA) EBIC_TRY(tmap_kmajor(&tb, Bk, N, K, ldb, N));
  const int smem = std::max(tcg::kMinSmem, (tcg::kTM + N) * K * (int)sizeof(bf16)) +
                   tcg::kAlignSlack;
  EBIC_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_full<BSRC, EPI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_gemm_tc_full<BSRC, EPI><<<(unsigned)((M + tcg::kTM - 1) / tcg::kTM), tcg::kThreads, smem,
                              st>>>(ta, tb, Bpacked, M, N, K, bias, mask, ldm, Cf, Cb, ldc,
                                    s->ferr.as<int>());
  return EBIC_OK;
}

// Split-K slices of op(A) op(B) with both operands MN-major.  One launch.
static ebic_status gemm_tc_split(ebic_surrogate_ctx* s, int M, int N, int K, const bf16* A,
                                 int lda, const bf16* B, int ldb, float* Cf, int ldc, int ksplit,
                                 cudaStream_t st) {
  const int smem = std::max(tcg::kMinSmem, (tcg::kTM + N) * tcg::kKC * (int)sizeof(bf16)) +
                   tcg::kAlignSlack;
  EBIC_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem));
  const dim3 grid((unsigned)((M + tcg::kTM - 1) / tcg::kTM), 1u, (unsigned)ksplit);
  k_gemm_tc_split<<<grid, tcg::kThreads, smem, st>>>(M, N, K, A, lda, B, ldb, Cf, ldc,
                                                     s->ferr.as<int>());
  return EBIC_OK;
}

// Features and both hidden layers of n series (rows idx[b], or 0 .. n - 1):
// 3 launches.
static ebic_status sur_hidden(ebic_surrogate_ctx* s, const uint16_t* seq, const int32_t* len,
                              int32_t stride, const int32_t* idx, int32_t n, const ActView& a,
                              cudaStream_t st) {
  const float* P = s->par.as<float>();
  k_features<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(seq, len, stride, idx, n, s->C,
                                                      P + s->o_emb, s->cmean.as<float>(),
                                                      s->csd.as<float>(), s->len_scale, a.x);
  if (s->gemm_kind == 0) {
    const bf16* wt = s->wpack_tc.as<bf16>();          // W1^T | W2^T, packed row-major
    EBIC_TRY((gemm_tc_full<tcg::B_PACKED, tcg::EPI_BIAS_RELU_BF16>(
        s, n, kH, kF, a.x, kF, nullptr, 0, wt, P + s->o_b1, nullptr, 0, nullptr, a.h1, kH, st)));
    EBIC_TRY((gemm_tc_full<tcg::B_PACKED, tcg::EPI_BIAS_RELU_BF16>(
        s, n, kH, kH, a.h1, kH, nullptr, 0, wt + kH * kF, P + s->o_b2, nullptr, 0, nullptr, a.h2,
        kH, st)));
    return EBIC_OK;
  }
  gemm<false, false, EPI_BIAS_RELU_BF16>(n, kH, kF, a.x, kF, s->w1b.as<bf16>(), kH, P + s->o_b1,
                                         nullptr, 0, nullptr, a.h1, kH, 1, st);
  gemm<false, false, EPI_BIAS_RELU_BF16>(n, kH, kH, a.h1, kH, s->w2b.as<bf16>(), kH, P + s->o_b2,
                                         nullptr, 0, nullptr, a.h2, kH, 1, st);
  return EBIC_OK;
}

ebic_status sur_forward_scores(ebic_surrogate_ctx* s, const uint16_t* seq, const int32_t* len,
                               int32_t stride, int32_t n, void* act, float* y, cudaStream_t st,
                               int* launches) {
  (void)act;
  if (n <= 0) {
    if (launches) *launches = 0;
    return EBIC_OK;
  }
  const float* P = s->par.as<float>();
  if (s->fwd_kind == 0) {
    static_assert(tc::kF == kF && tc::kH == kH && tc::kEmb == kEmb, "layer widths");
    EBIC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward_tc,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc::kSmem));
    const int ntiles = (n + tc::kTT - 1) / tc::kTT;
    const int grid = std::min(ntiles, std::max(s->sm_count, 1));
    k_mlp_forward_tc<<<grid, tc::kThreads, tc::kSmem, st>>>(
        seq, len, stride, n, s->C, P + s->o_emb, s->cmean.as<float>(), s->csd.as<float>(),
        s->len_scale, s->wpack_tc.as<bf16>(), P + s->o_b1, P + s->o_b2, P + s->o_w3,
        P + s->o_b3, y, s->ferr.as<int>());
    if (launches) *launches = 1;
    EBIC_CUDA_TRY(cudaGetLastError());
    return EBIC_OK;
  }
  // opt in to the large shared-memory carve-out (per device; cheap to repeat)
  EBIC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kFwdSmem));
  const int ntiles = (n + kFT - 1) / kFT;
  const int grid = std::min(ntiles, 152);
  k_mlp_forward<<<grid, kFwdThreads, kFwdSmem, st>>>(
      seq, len, stride, n, s->C, P + s->o_emb, s->cmean.as<float>(), s->csd.as<float>(),
      s->len_scale, s->wpack.as<bf16>(), P + s->o_b1, P + s->o_b2, P + s->o_w3, P + s->o_b3, y,
      s->ferr.as<int>());
  if (launches) *launches = 1;
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

// Both packed copies of W1^T | W2^T the scoring kernels read (2 launches).
static void pack_forward(ebic_surrogate_ctx* s, cudaStream_t st) {
  const float* P = s->par.as<float>();
  constexpr int npack = kH * (kF + 8) + kH * (kH + 8);
  k_pack_fwd<<<(npack + 255) / 256, 256, 0, st>>>(P + s->o_w1, P + s->o_w2, s->wpack.as<bf16>());
  constexpr int ntc = kH * kF + kH * kH;
  k_pack_fwd_tc<<<(ntc + 255) / 256, 256, 0, st>>>(P + s->o_w1, P + s->o_w2,
                                                   s->wpack_tc.as<bf16>());
}

// One training step on batch rows idx (device; nullptr: rows 0 .. B - 1);
// gradients are left in s->grad.
// One Adam step (update) or the loss and gradients only.  With ctab/ctr the
// step is being captured for replay: Adam's bias corrections come from
// ctab[*ctr] and the caller counts the steps.
static ebic_status sur_step(ebic_surrogate_ctx* s, const uint16_t* seq, const int32_t* len,
                            int32_t stride, const float* t, const int32_t* idx, int32_t B,
                            float lr, bool update, cudaStream_t st,
                            const float2* ctab = nullptr, const int32_t* ctr = nullptr) {
  EBIC_TRY(sur_reserve(s, B));
  const ActView a = act_view(s->act.ptr, B);
  EBIC_TRY(sur_hidden(s, seq, len, stride, idx, B, a, st));
  float* P = s->par.as<float>();
  float* G = s->grad.as<float>();
  const unsigned wb = (unsigned)((B + 7) / 8);
  k_out<<<wb, 256, 0, st>>>(a.h2, P + s->o_w3, P + s->o_b3, B, s->y.as<float>(), t, idx,
                            s->dy.as<float>(), s->sq.as<float>());
  colsum(s, nullptr, s->sq.as<float>(), B, 1, nullptr, s->loss.as<float>(), st);
  // output layer
  colsum(s, a.h2, nullptr, B, kH, s->dy.as<float>(), G + s->o_w3, st);
  colsum(s, nullptr, s->dy.as<float>(), B, 1, nullptr, G + s->o_b3, st);
  const long long nb = (long long)B * kH;
  k_dh2<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(s->dy.as<float>(), P + s->o_w3, a.h2, B,
                                                      s->dh2.as<bf16>());
  // layer 2: dW2 = h1^T dh2 (split K, partials summed in order), db2,
  // dh1 = (dh2 W2^T) [h1 > 0]
  const int ks = std::max(1, std::min(32, B / 256));
  float* split = s->split.as<float>();
  const bool tcg5 = s->gemm_kind == 0;
  if (tcg5)
    EBIC_TRY(gemm_tc_split(s, kH, kH, B, a.h1, kH, s->dh2.as<bf16>(), kH, split, kH, ks, st));
  else
    gemm<true, false, EPI_F32_SPLIT>(kH, kH, B, a.h1, kH, s->dh2.as<bf16>(), kH, nullptr, nullptr,
                                     0, split, nullptr, kH, ks, st);
  k_sum_splits<<<(kH * kH + 255) / 256, 256, 0, st>>>(split, ks, (long long)kH * kH, G + s->o_w2);
  colsum(s, s->dh2.as<bf16>(), nullptr, B, kH, nullptr, G + s->o_b2, st);
  if (tcg5)
    EBIC_TRY((gemm_tc_full<tcg::B_TMA, tcg::EPI_MASK_BF16>(
        s, B, kH, kH, s->dh2.as<bf16>(), kH, s->w2b.as<bf16>(), kH, nullptr, nullptr, a.h1, kH,
        nullptr, s->dh1.as<bf16>(), kH, st)));
  else
    gemm<false, true, EPI_MASK_BF16>(B, kH, kH, s->dh2.as<bf16>(), kH, s->w2b.as<bf16>(), kH,
                                     nullptr, a.h1, kH, nullptr, s->dh1.as<bf16>(), kH, 1, st);
  // layer 1: dW1 = x^T dh1, db1, dx = dh1 W1^T, then the embedding rows
  if (tcg5)
    EBIC_TRY(gemm_tc_split(s, kF, kH, B, a.x, kF, s->dh1.as<bf16>(), kH, split, kH, ks, st));
  else
    gemm<true, false, EPI_F32_SPLIT>(kF, kH, B, a.x, kF, s->dh1.as<bf16>(), kH, nullptr, nullptr,
                                     0, split, nullptr, kH, ks, st);
  k_sum_splits<<<(kF * kH + 255) / 256, 256, 0, st>>>(split, ks, (long long)kF * kH, G + s->o_w1);
  colsum(s, s->dh1.as<bf16>(), nullptr, B, kH, nullptr, G + s->o_b1, st);
  if (tcg5)
    EBIC_TRY((gemm_tc_full<tcg::B_TMA, tcg::EPI_F32>(s, B, kF, kH, s->dh1.as<bf16>(), kH,
                                                     s->w1b.as<bf16>(), kH, nullptr, nullptr,
                                                     nullptr, 0, s->dx.as<float>(), nullptr, kF,
                                                     st)));
  else
    gemm<false, true, EPI_F32>(B, kF, kH, s->dh1.as<bf16>(), kH, s->w1b.as<bf16>(), kH, nullptr,
                               nullptr, 0, s->dx.as<float>(), nullptr, kF, 1, st);
  {
    const int seg = s->emb_seg_len(B);
    const dim3 eg((unsigned)((s->C + 63) / 64), (unsigned)((B + seg - 1) / seg));
    k_emb_grad_part<<<eg, 256, 0, st>>>(seq, len, stride, idx, B, s->C, seg, s->dx.as<float>(),
                                        s->epart.as<float>());
    const long long ne = (long long)s->C * kEmb;
    k_sum_splits<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(s->epart.as<float>(), (int)eg.y, ne,
                                                              G + s->o_emb);
  }
  count_launches(23);   // 3 + 20 above
  if (update) {
    if (!ctab) s->steps_done += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)s->steps_done));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)s->steps_done));
    struct Seg {
      long long o, n;
      bf16* copy;
    } segs[] = {{s->o_emb, s->o_w1 - s->o_emb, nullptr},
                {s->o_w1, (long long)kF * kH, s->w1b.as<bf16>()},
                {s->o_b1, kH, nullptr},
                {s->o_w2, (long long)kH * kH, s->w2b.as<bf16>()},
                {s->o_b2, kH + kH + 1, nullptr}};   // b2 | w3 | b3 are contiguous
    for (const Seg& g : segs) {
      k_adam<<<(unsigned)((g.n + 255) / 256), 256, 0, st>>>(
          P + g.o, G + g.o, s->mom.as<float>() + g.o, s->vel.as<float>() + g.o, g.n, lr, b1, b2,
          1e-8f, c1, c2, g.copy, ctab, ctr);
    }
    pack_forward(s, st);
    count_launches(7);
  }
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

static ebic_status refresh_copies(ebic_surrogate_ctx* s, cudaStream_t st) {
  const float* P = s->par.as<float>();
  k_to_bf16<<<(kF * kH + 255) / 256, 256, 0, st>>>(P + s->o_w1, s->w1b.as<bf16>(),
                                                   (long long)kF * kH);
  k_to_bf16<<<(kH * kH + 255) / 256, 256, 0, st>>>(P + s->o_w2, s->w2b.as<bf16>(),
                                                   (long long)kH * kH);
  pack_forward(s, st);
  count_launches(4);
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

// Deterministic initial weights: Box-Muller normals on a splitmix64 stream.
static void init_weights(ebic_surrogate_ctx* s, std::vector<float>& p) {
  uint64_t z = s->seed ^ 0x9E3779B97F4A7C15ull;
  auto unif = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t q = z;
    q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
    q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
    q ^= q >> 31;
    return ((double)(q >> 11) + 0.5) * 0x1p-53;
  };
  auto nrm = [&]() {
    const double u1 = unif(), u2 = unif();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  p.assign((size_t)s->n_par, 0.f);
  for (long long i = 0; i < (long long)s->C * kEmb; ++i) p[(size_t)(s->o_emb + i)] = (float)(0.1 * nrm());
  for (int r = 0; r < 67; ++r)
    for (int c = 0; c < kH; ++c)
      p[(size_t)(s->o_w1 + (long long)r * kH + c)] = (float)(nrm() * std::sqrt(2.0 / 67));
  for (long long i = 0; i < (long long)kH * kH; ++i)
    p[(size_t)(s->o_w2 + i)] = (float)(nrm() * std::sqrt(2.0 / kH));
  for (int i = 0; i < kH; ++i) p[(size_t)(s->o_w3 + i)] = (float)(nrm() * std::sqrt(1.0 / kH));
}

static void sur_release(ebic_surrogate_ctx* s) {
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (DevBuf* b : {&s->par, &s->grad, &s->mom, &s->vel, &s->w1b, &s->w2b, &s->wpack,
                    &s->wpack_tc, &s->ferr,
                    &s->cmean, &s->csd,
                    &s->act, &s->dh1, &s->dh2, &s->dx, &s->y, &s->dy, &s->idx, &s->loss,
                    &s->tgt, &s->tmp, &s->sq, &s->split, &s->epart, &s->csplit, &s->ctab, &s->ctr, &s->log_seq,
                    &s->log_len, &s->log_fit})
    b->release();
  if (s->stream) cudaStreamDestroy(s->stream);
  s->stream = nullptr;
}

static ebic_status sur_create(ebic_ctx* h, int32_t len_scale, uint64_t seed,
                              ebic_surrogate_ctx* s) {
  s->device = h->device;
  // the scoring kernel shuffles two column ids (or the end marker C) in one
  // 32-bit word; the loader already keeps C at or below 65,535
  if (h->C > 65535) return fail(EBIC_ERR_ARG, "the surrogate supports at most 65,535 columns");
  s->C = h->C;
  s->h = h;
  s->seed = seed;
  s->len_scale = (float)len_scale;
  EBIC_CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  s->o_emb = 0;
  s->o_w1 = s->o_emb + (long long)s->C * kEmb;
  s->o_b1 = s->o_w1 + (long long)kF * kH;
  s->o_w2 = s->o_b1 + kH;
  s->o_b2 = s->o_w2 + (long long)kH * kH;
  s->o_w3 = s->o_b2 + kH;
  s->o_b3 = s->o_w3 + kH;
  s->n_par = s->o_b3 + 1;
  const size_t pb = (size_t)s->n_par * sizeof(float);
  EBIC_TRY(s->par.reserve(pb));
  EBIC_TRY(s->grad.reserve(pb));
  EBIC_TRY(s->mom.reserve_zeroed(pb, s->stream));
  EBIC_TRY(s->vel.reserve_zeroed(pb, s->stream));
  EBIC_TRY(s->w1b.reserve((size_t)kF * kH * sizeof(bf16)));
  EBIC_TRY(s->w2b.reserve((size_t)kH * kH * sizeof(bf16)));
  EBIC_TRY(s->wpack.reserve((size_t)(kH * (kF + 8) + kH * (kH + 8)) * sizeof(bf16)));
  EBIC_TRY(s->wpack_tc.reserve(tc::kW1 + tc::kW2));
  EBIC_CUDA_TRY(cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device));
  EBIC_TRY(s->ferr.reserve_zeroed(sizeof(int), s->stream));
  EBIC_TRY(s->cmean.reserve((size_t)s->C * sizeof(float)));
  EBIC_TRY(s->csd.reserve((size_t)s->C * sizeof(float)));
  EBIC_TRY(s->loss.reserve(sizeof(float)));
  EBIC_TRY(s->tmp.reserve(2 * kSumBlocks * sizeof(double)));
  std::vector<float> p;
  init_weights(s, p);
  EBIC_CUDA_TRY(cudaMemcpyAsync(s->par.ptr, p.data(), pb, cudaMemcpyHostToDevice, s->stream));
  EBIC_TRY(refresh_copies(s, s->stream));
  k_colstats<<<(unsigned)s->C, 256, 0, s->stream>>>(h->A_c, h->R, h->R_pad, s->cmean.as<float>(),
                                                    s->csd.as<float>());
  count_launches(1);
  EBIC_CUDA_TRY(cudaGetLastError());
  EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return EBIC_OK;
}

static ebic_status sur_train(ebic_surrogate_ctx* s, const uint16_t* seq, const int32_t* len,
                             int32_t stride, const double* fit, long long n, int32_t steps,
                             int32_t batch, float lr, float* out_loss) {
  cudaStream_t st = s->stream;
  // standardised log1p targets over the whole set
  EBIC_TRY(s->tgt.reserve((size_t)n * sizeof(float)));
  k_sum_log1p<<<kSumBlocks, 256, 0, st>>>(fit, n, s->tmp.as<double>());
  double m2[2 * kSumBlocks];
  EBIC_CUDA_TRY(cudaMemcpyAsync(m2, s->tmp.ptr, sizeof(m2), cudaMemcpyDeviceToHost, st));
  EBIC_CUDA_TRY(cudaStreamSynchronize(st));
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < kSumBlocks; ++i) {
    s1 += m2[2 * i];
    s2 += m2[2 * i + 1];
  }
  const double mean = s1 / (double)n;
  const double var = s2 / (double)n - mean * mean;
  s->t_mean = (float)mean;
  s->t_sd = (float)std::sqrt(var > 1e-12 ? var : 1.0);
  k_targets<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(fit, n, s->t_mean, s->t_sd,
                                                         s->tgt.as<float>());
  count_launches(2);
  EBIC_TRY(sur_reserve(s, batch));
  if (steps > 0) {
    // One step (minibatch draw, forward, reverse pass, Adam, weight packing)
    // is captured once and replayed `steps` times.  What changes from step
    // to step comes from the device: the replay index (advanced by the last
    // kernel of the step) picks the Philox step number of the draw and
    // Adam's bias corrections from a table computed here exactly as the
    // eager step computes them.
    const long long base = s->steps_done;
    std::vector<float2> tab((size_t)steps);
    for (int32_t i = 0; i < steps; ++i) {
      const double t = (double)(base + i + 1);
      tab[(size_t)i] = make_float2((float)(1.0 - std::pow(0.9, t)), (float)(1.0 - std::pow(0.999, t)));
    }
    EBIC_TRY(s->ctab.reserve(tab.size() * sizeof(float2)));
    EBIC_TRY(s->ctr.reserve(sizeof(int32_t)));
    EBIC_CUDA_TRY(cudaMemcpyAsync(s->ctab.ptr, tab.data(), tab.size() * sizeof(float2),
                                  cudaMemcpyHostToDevice, st));
    EBIC_CUDA_TRY(cudaMemsetAsync(s->ctr.ptr, 0, sizeof(int32_t), st));
    EBIC_CUDA_TRY(cudaStreamSynchronize(st));        // the table outlives this scope's vector
    const uint64_t c0 = ebic_kernel_launches();
    cudaGraph_t graph = nullptr;
    EBIC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    k_sample<<<(unsigned)((batch + 255) / 256), 256, 0, st>>>(
        s->seed, (uint32_t)(base + 1), n, batch, s->idx.as<int32_t>(), s->ctr.as<int32_t>());
    count_launches(1);
    ebic_status rs = sur_step(s, seq, len, stride, s->tgt.as<float>(), s->idx.as<int32_t>(), batch,
                              lr, true, st, s->ctab.as<float2>(), s->ctr.as<int32_t>());
    k_step_advance<<<1, 1, 0, st>>>(s->ctr.as<int32_t>());
    count_launches(1);
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (rs != EBIC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rs;
    }
    if (ce != cudaSuccess) return fail(EBIC_ERR_CUDA, "training step capture: %s", cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(EBIC_ERR_CUDA, "training step graph: %s", cudaGetErrorString(ie));
    const uint64_t per_step = ebic_kernel_launches() - c0;
    cudaError_t le = cudaSuccess;
    for (int32_t i = 0; i < steps && le == cudaSuccess; ++i) le = cudaGraphLaunch(exec, st);
    cudaGraphExecDestroy(exec);
    if (le != cudaSuccess) return fail(EBIC_ERR_CUDA, "training step replay: %s", cudaGetErrorString(le));
    count_launches(per_step * (uint64_t)(steps - 1));
    s->steps_done += steps;
  }
  float loss = 0.f;
  if (out_loss && steps > 0)
    EBIC_CUDA_TRY(cudaMemcpyAsync(&loss, s->loss.ptr, sizeof(float), cudaMemcpyDeviceToHost, st));
  EBIC_CUDA_TRY(cudaStreamSynchronize(st));
  if (out_loss) *out_loss = loss;
  return EBIC_OK;
}

static ebic_status sur_log(ebic_surrogate_ctx* s, ebic_ctx* h) {
  const uint16_t* seq = nullptr;
  const int32_t* len = nullptr;
  const double* fit = nullptr;
  long long n = 0;
  int32_t stride = 0;
  EBIC_TRY(ea_archive(h, &seq, &len, &fit, &n, &stride));
  if (n == 0) return EBIC_OK;
  const long long need = s->log_n + n;
  if (need > s->log_cap) {
    long long cap = std::max<long long>(need, 2 * s->log_cap);
    DevBuf nseq, nlen, nfit;
    ebic_status rs = nseq.reserve((size_t)cap * kLogStride * sizeof(uint16_t));
    if (rs == EBIC_OK) rs = nlen.reserve((size_t)cap * sizeof(int32_t));
    if (rs == EBIC_OK) rs = nfit.reserve((size_t)cap * sizeof(double));
    if (rs != EBIC_OK) {
      nseq.release();
      nlen.release();
      nfit.release();
      return rs;
    }
    if (s->log_n) {
      EBIC_CUDA_TRY(cudaMemcpyAsync(nseq.ptr, s->log_seq.ptr,
                                    (size_t)s->log_n * kLogStride * sizeof(uint16_t),
                                    cudaMemcpyDeviceToDevice, s->stream));
      EBIC_CUDA_TRY(cudaMemcpyAsync(nlen.ptr, s->log_len.ptr, (size_t)s->log_n * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, s->stream));
      EBIC_CUDA_TRY(cudaMemcpyAsync(nfit.ptr, s->log_fit.ptr, (size_t)s->log_n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s->stream));
      EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
    }
    s->log_seq.release();
    s->log_len.release();
    s->log_fit.release();
    s->log_seq = nseq;
    s->log_len = nlen;
    s->log_fit = nfit;
    nseq.ptr = nlen.ptr = nfit.ptr = nullptr;
    s->log_cap = cap;
  }
  uint16_t* dseq = s->log_seq.as<uint16_t>() + (size_t)s->log_n * kLogStride;
  EBIC_CUDA_TRY(cudaMemcpy2DAsync(dseq, kLogStride * sizeof(uint16_t), seq,
                                  (size_t)stride * sizeof(uint16_t),
                                  (size_t)stride * sizeof(uint16_t), (size_t)n,
                                  cudaMemcpyDeviceToDevice, s->stream));
  EBIC_CUDA_TRY(cudaMemcpyAsync(s->log_len.as<int32_t>() + s->log_n, len, (size_t)n * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, s->stream));
  EBIC_CUDA_TRY(cudaMemcpyAsync(s->log_fit.as<double>() + s->log_n, fit, (size_t)n * sizeof(double),
                                cudaMemcpyDeviceToDevice, s->stream));
  EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->log_n += n;
  return EBIC_OK;
}

}  // namespace ebic

extern "C" {

ebic_status ebic_surrogate_create(ebic_handle h, int32_t len_scale, uint64_t seed,
                                  ebic_surrogate* out) {
  if (!h || !out || len_scale < 1) return fail(EBIC_ERR_ARG, "bad surrogate arguments");
  ebic_surrogate_ctx* s = new ebic_surrogate_ctx();
  const ebic_status st = sur_create(h, len_scale, seed, s);
  if (st != EBIC_OK) {
    sur_release(s);
    delete s;
    return st;
  }
  *out = s;
  return EBIC_OK;
}

ebic_status ebic_surrogate_free(ebic_surrogate s) {
  if (!s) return EBIC_OK;
  if (s->attached > 0)
    return fail(EBIC_ERR_STATE, "the surrogate is screening %d run(s); detach it first",
                s->attached);
  sur_release(s);
  delete s;
  return EBIC_OK;
}

ebic_status ebic_surrogate_params(ebic_surrogate s, float* host_params, int64_t* n_params,
                                  int32_t write) {
  if (!s || !n_params) return fail(EBIC_ERR_ARG, "null pointer");
  const long long n = s->n_par;
  if (host_params) {
    if (*n_params < n)
      return fail(EBIC_ERR_ARG, "buffer holds %lld parameters, %lld needed", (long long)*n_params, n);
    if (write) {
      EBIC_CUDA_TRY(cudaMemcpyAsync(s->par.ptr, host_params, (size_t)n * sizeof(float),
                                    cudaMemcpyHostToDevice, s->stream));
      EBIC_TRY(refresh_copies(s, s->stream));
    } else {
      EBIC_CUDA_TRY(cudaMemcpyAsync(host_params, s->par.ptr, (size_t)n * sizeof(float),
                                    cudaMemcpyDeviceToHost, s->stream));
    }
    EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  *n_params = n;
  return EBIC_OK;
}

ebic_status ebic_surrogate_grads(ebic_surrogate s, float* host_grads, int64_t n) {
  if (!s || !host_grads || n < s->n_par) return fail(EBIC_ERR_ARG, "bad gradient buffer");
  EBIC_CUDA_TRY(cudaMemcpyAsync(host_grads, s->grad.ptr, (size_t)s->n_par * sizeof(float),
                                cudaMemcpyDeviceToHost, s->stream));
  EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return EBIC_OK;
}

ebic_status ebic_surrogate_colstats(ebic_surrogate s, float* host_mean, float* host_sd) {
  if (!s || !host_mean || !host_sd) return fail(EBIC_ERR_ARG, "null pointer");
  EBIC_CUDA_TRY(cudaMemcpyAsync(host_mean, s->cmean.ptr, (size_t)s->C * sizeof(float),
                                cudaMemcpyDeviceToHost, s->stream));
  EBIC_CUDA_TRY(cudaMemcpyAsync(host_sd, s->csd.ptr, (size_t)s->C * sizeof(float),
                                cudaMemcpyDeviceToHost, s->stream));
  EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return EBIC_OK;
}

ebic_status ebic_surrogate_step(ebic_surrogate s, const uint16_t* d_seq, const int32_t* d_len,
                                int32_t stride, const float* d_target, const int32_t* d_idx,
                                int32_t batch, float lr, int32_t update, float* out_loss) {
  if (!s || !d_seq || !d_len || !d_target || batch < 1 || stride < 1)
    return fail(EBIC_ERR_ARG, "bad step arguments");
  const cudaStream_t st = s->stream;
  EBIC_TRY(sur_step(s, d_seq, d_len, stride, d_target, d_idx, batch, lr, update != 0, st));
  float loss = 0.f;
  EBIC_CUDA_TRY(cudaMemcpyAsync(&loss, s->loss.ptr, sizeof(float), cudaMemcpyDeviceToHost, st));
  EBIC_CUDA_TRY(cudaStreamSynchronize(st));
  if (out_loss) *out_loss = loss;
  return EBIC_OK;
}

ebic_status ebic_surrogate_log(ebic_surrogate s, ebic_handle h, int64_t* out_total) {
  if (!s || !h) return fail(EBIC_ERR_ARG, "null pointer");
  if (h->C != s->C) return fail(EBIC_ERR_ARG, "the run's matrix has %d columns, the surrogate %d", h->C, s->C);
  EBIC_TRY(sur_log(s, h));
  if (out_total) *out_total = s->log_n;
  return EBIC_OK;
}

ebic_status ebic_surrogate_train(ebic_surrogate s, const uint16_t* d_seq, const int32_t* d_len,
                                 int32_t stride, const double* d_fitness, int64_t n,
                                 int32_t steps, int32_t batch, float lr, float* out_loss) {
  if (!s || steps < 0 || batch < 1 || batch > (1 << 24))
    return fail(EBIC_ERR_ARG, "bad training arguments");
  if (!d_seq && !d_len && !d_fitness) {
    d_seq = s->log_seq.as<uint16_t>();
    d_len = s->log_len.as<int32_t>();
    d_fitness = s->log_fit.as<double>();
    stride = kLogStride;
    n = s->log_n;
  }
  if (!d_seq || !d_len || !d_fitness || n < 2 || n > (1ll << 31) - 1 || stride < 1)
    return fail(EBIC_ERR_ARG, "training needs at least 2 pairs (%lld given)", (long long)n);
  return sur_train(s, d_seq, d_len, stride, d_fitness, n, steps, batch, lr, out_loss);
}

ebic_status ebic_surrogate_target_norm(ebic_surrogate s, float* mean, float* sd) {
  if (!s) return fail(EBIC_ERR_ARG, "null surrogate");
  if (mean) *mean = s->t_mean;
  if (sd) *sd = s->t_sd;
  return EBIC_OK;
}

ebic_status ebic_surrogate_forward_kernel(ebic_surrogate s, int32_t kind) {
  if (!s) return fail(EBIC_ERR_ARG, "null surrogate");
  if (kind != 0 && kind != 1) return fail(EBIC_ERR_ARG, "forward kernel must be 0 or 1");
  s->fwd_kind = kind;
  return EBIC_OK;
}

ebic_status ebic_surrogate_train_kernel(ebic_surrogate s, int32_t kind) {
  if (!s) return fail(EBIC_ERR_ARG, "null surrogate");
  if (kind != 0 && kind != 1) return fail(EBIC_ERR_ARG, "training kernel must be 0 or 1");
  s->gemm_kind = kind;
  return EBIC_OK;
}

ebic_status ebic_surrogate_predict(ebic_surrogate s, const uint16_t* d_seq, const int32_t* d_len,
                                   int32_t stride, int64_t n, float* d_out, void* stream) {
  if (!s || !d_seq || !d_len || !d_out || n < 0 || n > (1ll << 31) - 1 || stride < 1)
    return fail(EBIC_ERR_ARG, "bad prediction arguments");
  if (n == 0) return EBIC_OK;
  const cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : s->stream;
  const int32_t chunk = 1 << 16;
  const int32_t rows = (int32_t)std::min<int64_t>(chunk, n);
  if (stream) EBIC_CUDA_TRY(cudaStreamSynchronize(s->stream));
  EBIC_TRY(sur_reserve(s, rows));
  for (int64_t b0 = 0; b0 < n; b0 += chunk) {
    const int32_t m = (int32_t)std::min<int64_t>(chunk, n - b0);
    EBIC_TRY(sur_forward_scores(s, d_seq + (size_t)b0 * stride, d_len + b0, stride, m,
                                s->act.ptr, d_out + b0, st, nullptr));
    count_launches(1);
  }
  if (!stream) {
    int e = 0;
    EBIC_CUDA_TRY(cudaMemcpyAsync(&e, s->ferr.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    EBIC_CUDA_TRY(cudaStreamSynchronize(st));
    if (e) return fail(EBIC_ERR_TIMEOUT, "a bounded wait for the surrogate's weights expired");
  }
  return EBIC_OK;
}

}  // extern "C"
