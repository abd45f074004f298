// Step 6 ("prepare biclusters": the indices of the rows that match each
// series of columns), Step 7's expansion by negative trends, and the recovery
// and relevance scores of Eq. (2)-(3).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ebic_internal.cuh"
#include "ebic_support.cuh"

namespace ebic {

// ---------------------------------------------------------------------------
// Rows of a series.  One CTA per series walks the column-major matrix in
// chunks of 1,024 rows, each thread four consecutive rows (one float4 per
// column): a row is kept when its values rise strictly along the series (or,
// mode 1, rise or fall strictly).  With APPROX a row is kept when at most
// `breaks` of its adjacent pairs do not rise strictly (mode 1: or at most
// `breaks` do not fall strictly), counted per row.  The counting launch
// writes the number of kept rows; the writing launch stores their indices,
// ascending, from row_off[series] on (a block-wide scan orders them).
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 256;

template <bool WRITE, bool APPROX>
__global__ void __launch_bounds__(kRowThreads)
k_rows(const float* __restrict__ A_c, int32_t R, int32_t R_pad, const int32_t* __restrict__ off,
       const int32_t* __restrict__ cols, int32_t mode, int32_t breaks,
       int32_t* __restrict__ counts, const long long* __restrict__ row_off,
       int32_t* __restrict__ rows) {
  __shared__ int s_warp[kRowThreads / 32];
  const int sid = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = off[sid], L = off[sid + 1] - b;
  long long written = 0;
  int total = 0;
  for (int r0 = 0; r0 < R_pad; r0 += 4 * kRowThreads) {
    const int r = r0 + 4 * tid;
    uint32_t keep = 0u;
    if (r < R_pad) {
      uint32_t rise = 0xFu, fall = 0xFu;
      int up_breaks[4] = {0, 0, 0, 0}, down_breaks[4] = {0, 0, 0, 0};
      float4 prev = *reinterpret_cast<const float4*>(A_c + (size_t)cols[b] * R_pad + r);
      for (int i = 1; i < L; ++i) {
        const float4 cur = *reinterpret_cast<const float4*>(A_c + (size_t)cols[b + i] * R_pad + r);
        const uint32_t up = lt4(prev, cur), down = gt4(prev, cur);
        if (APPROX) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            up_breaks[j] += ((up >> j) & 1u) ? 0 : 1;
            down_breaks[j] += ((down >> j) & 1u) ? 0 : 1;
          }
        } else {
          rise &= up;
          fall &= down;
        }
        prev = cur;
      }
      if (APPROX) {
        rise = fall = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          rise |= up_breaks[j] <= breaks ? 1u << j : 0u;
          fall |= down_breaks[j] <= breaks ? 1u << j : 0u;
        }
      }
      const uint32_t valid = (r < R ? 1u : 0u) | (r + 1 < R ? 2u : 0u) | (r + 2 < R ? 4u : 0u) |
                             (r + 3 < R ? 8u : 0u);
      keep = (rise | (mode == 1 ? fall : 0u)) & valid;
    }
    const int c = __popc(keep);
    if (!WRITE) {
      total += c;
      continue;
    }
    // exclusive position of this thread's rows within the chunk
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int before = 0, chunk = 0;
    for (int w = 0; w < kRowThreads / 32; ++w) {
      const int v = s_warp[w];
      before += w < warp ? v : 0;
      chunk += v;
    }
    int pos = (int)(written) + before + incl - c;
    int32_t* out = rows + row_off[sid];
    for (int j = 0; j < 4; ++j)
      if ((keep >> j) & 1u) out[pos++] = r + j;
    written += chunk;
    __syncthreads();                       // s_warp is reused by the next chunk
  }
  if (!WRITE) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) s_warp[warp] = total;
    __syncthreads();
    if (tid == 0) {
      int t = 0;
      for (int w = 0; w < kRowThreads / 32; ++w) t += s_warp[w];
      counts[sid] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// Eq. (2)-(3).  One warp per (expected e, found f) pair computes the Jaccard
// index of the two biclusters as sets of cells: |Re & Rf| |Ce & Cf| /
// (|Re| |Ce| + |Rf| |Cf| - |Re & Rf| |Ce & Cf|); intersections of ascending
// index lists by binary search of one list's entries in the other.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long intersect_sorted(const int32_t* a, int na, const int32_t* b,
                                                      int nb, int lane) {
  long long n = 0;
  for (int i = lane; i < na; i += 32) {
    const int32_t v = a[i];
    int lo = 0, hi = nb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (b[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    n += (lo < nb && b[lo] == v) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  return n;
}

__global__ void __launch_bounds__(256)
k_jaccard(int32_t E, int32_t F, const long long* __restrict__ er_off, const int32_t* __restrict__ er,
          const long long* __restrict__ ec_off, const int32_t* __restrict__ ec,
          const long long* __restrict__ fr_off, const int32_t* __restrict__ fr,
          const long long* __restrict__ fc_off, const int32_t* __restrict__ fc,
          double* __restrict__ J) {
  const int lane = threadIdx.x & 31;
  const long long pair = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (pair >= (long long)E * F) return;
  const int e = (int)(pair / F), f = (int)(pair % F);
  const int ner = (int)(er_off[e + 1] - er_off[e]), nec = (int)(ec_off[e + 1] - ec_off[e]);
  const int nfr = (int)(fr_off[f + 1] - fr_off[f]), nfc = (int)(fc_off[f + 1] - fc_off[f]);
  const long long ir = intersect_sorted(er + er_off[e], ner, fr + fr_off[f], nfr, lane);
  const long long ic = intersect_sorted(ec + ec_off[e], nec, fc + fc_off[f], nfc, lane);
  if (lane == 0) {
    const long long inter = ir * ic;
    const long long uni = (long long)ner * nec + (long long)nfr * nfc - inter;
    J[pair] = uni > 0 ? (double)inter / (double)uni : 0.0;
  }
}

// recovery = mean over e of max over f of J, relevance = mean over f of max
// over e (one CTA; fixed summation order)
__global__ void k_recovery_relevance(int32_t E, int32_t F, const double* __restrict__ J,
                                     double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double rec = 0.0, rel = 0.0;
  for (int e = 0; e < E; ++e) {
    double m = 0.0;
    for (int f = 0; f < F; ++f) m = fmax(m, J[(size_t)e * F + f]);
    rec += m;
  }
  for (int f = 0; f < F; ++f) {
    double m = 0.0;
    for (int e = 0; e < E; ++e) m = fmax(m, J[(size_t)e * F + f]);
    rel += m;
  }
  out[0] = rec / (double)E;
  out[1] = rel / (double)F;
}

}  // namespace ebic

using namespace ebic;

namespace {

struct Guard {
  int prev = -1, dev;
  explicit Guard(int d) : dev(d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~Guard() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

// ascending, distinct, within [0, bound)
bool strictly_ascending(const int32_t* v, long long n, int32_t bound) {
  for (long long i = 0; i < n; ++i) {
    if (v[i] < 0 || v[i] >= bound) return false;
    if (i && v[i] <= v[i - 1]) return false;
  }
  return true;
}

}  // namespace

extern "C" {

// Steps 6 / 7 for ebic_extract_rows (breaks < 0: strict trends) and
// ebic_extract_rows_approx (at most `breaks` broken pairs per row).
static ebic_status extract_rows(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                                int32_t P, int32_t mode, int32_t breaks, int64_t* row_offsets,
                                int32_t* rows, int64_t* inout_capacity) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (P < 0 || P > (1 << 24)) return fail(EBIC_ERR_ARG, "P = %d outside [0, 2^24]", P);
  if (!offsets || !row_offsets || !inout_capacity || *inout_capacity < 0)
    return fail(EBIC_ERR_ARG, "null pointer");
  if (mode != EBIC_ROWS_RISING && mode != EBIC_ROWS_RISING_OR_FALLING)
    return fail(EBIC_ERR_ARG, "bad rows mode %d", mode);
  if (P == 0) {
    row_offsets[0] = 0;
    *inout_capacity = 0;
    return EBIC_OK;
  }
  if (!cols) return fail(EBIC_ERR_ARG, "null pointer");
  if (offsets[0] != 0) return fail(EBIC_ERR_ARG, "offsets[0] must be 0");
  for (int32_t i = 0; i < P; ++i) {
    const int32_t L = offsets[i + 1] - offsets[i];
    if (L < 1 || L > EBIC_MAX_EVAL_LEN)
      return fail(EBIC_ERR_ARG, "series %d has length %d outside [1, %d]", i, L, EBIC_MAX_EVAL_LEN);
  }
  const int32_t total = offsets[P];
  for (int32_t k = 0; k < total; ++k)
    if (cols[k] < 0 || cols[k] >= h->C)
      return fail(EBIC_ERR_ARG, "column index %d at position %d outside [0, %d)", cols[k], k, h->C);
  Guard g(h->device);
  const cudaStream_t s = h->stream;
  DevBuf d_off, d_cols, d_cnt, d_roff, d_rows;
  auto release = [&]() {
    d_off.release();
    d_cols.release();
    d_cnt.release();
    d_roff.release();
    d_rows.release();
  };
  ebic_status st = EBIC_OK;
  std::vector<int32_t> cnt((size_t)P);
  do {
    if ((st = d_off.reserve((size_t)(P + 1) * sizeof(int32_t))) != EBIC_OK) break;
    if ((st = d_cols.reserve((size_t)total * sizeof(int32_t))) != EBIC_OK) break;
    if ((st = d_cnt.reserve((size_t)P * sizeof(int32_t))) != EBIC_OK) break;
    if (cudaMemcpyAsync(d_off.ptr, offsets, (size_t)(P + 1) * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_cols.ptr, cols, (size_t)total * sizeof(int32_t), cudaMemcpyHostToDevice,
                        s) != cudaSuccess) {
      st = fail(EBIC_ERR_CUDA, "copy of the series failed");
      break;
    }
    if (breaks < 0)
      k_rows<false, false><<<(unsigned)P, kRowThreads, 0, s>>>(
          h->A_c, h->R, h->R_pad, d_off.as<int32_t>(), d_cols.as<int32_t>(), mode, 0,
          d_cnt.as<int32_t>(), nullptr, nullptr);
    else
      k_rows<false, true><<<(unsigned)P, kRowThreads, 0, s>>>(
          h->A_c, h->R, h->R_pad, d_off.as<int32_t>(), d_cols.as<int32_t>(), mode, breaks,
          d_cnt.as<int32_t>(), nullptr, nullptr);
    count_launches(1);
    if (cudaMemcpyAsync(cnt.data(), d_cnt.ptr, (size_t)P * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = fail(EBIC_ERR_CUDA, "row counting failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
  } while (false);
  if (st != EBIC_OK) {
    release();
    return st;
  }
  std::vector<long long> roff((size_t)P + 1, 0);
  for (int32_t i = 0; i < P; ++i) roff[i + 1] = roff[i] + cnt[i];
  const long long need = roff[P];
  if (need > *inout_capacity || (need > 0 && !rows)) {
    const long long cap = *inout_capacity;
    *inout_capacity = need;
    release();
    return fail(EBIC_ERR_ARG, "the rows need %lld entries, the buffer holds %lld", need, cap);
  }
  do {
    if (need > 0) {
      if ((st = d_roff.reserve(roff.size() * sizeof(long long))) != EBIC_OK) break;
      if ((st = d_rows.reserve((size_t)need * sizeof(int32_t))) != EBIC_OK) break;
      if (cudaMemcpyAsync(d_roff.ptr, roff.data(), roff.size() * sizeof(long long),
                          cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(EBIC_ERR_CUDA, "copy of the row offsets failed");
        break;
      }
      if (breaks < 0)
        k_rows<true, false><<<(unsigned)P, kRowThreads, 0, s>>>(
            h->A_c, h->R, h->R_pad, d_off.as<int32_t>(), d_cols.as<int32_t>(), mode, 0, nullptr,
            d_roff.as<long long>(), d_rows.as<int32_t>());
      else
        k_rows<true, true><<<(unsigned)P, kRowThreads, 0, s>>>(
            h->A_c, h->R, h->R_pad, d_off.as<int32_t>(), d_cols.as<int32_t>(), mode, breaks,
            nullptr, d_roff.as<long long>(), d_rows.as<int32_t>());
      count_launches(1);
      if (cudaMemcpyAsync(rows, d_rows.ptr, (size_t)need * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = fail(EBIC_ERR_CUDA, "row extraction failed: %s",
                  cudaGetErrorString(cudaGetLastError()));
        break;
      }
    }
  } while (false);
  release();
  if (st != EBIC_OK) return st;
  for (int32_t i = 0; i <= P; ++i) row_offsets[i] = roff[i];
  *inout_capacity = need;
  return EBIC_OK;
}

ebic_status ebic_extract_rows(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                              int32_t P, int32_t mode, int64_t* row_offsets, int32_t* rows,
                              int64_t* inout_capacity) {
  return extract_rows(h, offsets, cols, P, mode, -1, row_offsets, rows, inout_capacity);
}

ebic_status ebic_extract_rows_approx(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                                     int32_t P, int32_t max_breaks, int32_t mode,
                                     int64_t* row_offsets, int32_t* rows,
                                     int64_t* inout_capacity) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (max_breaks < 0 || max_breaks > EBIC_MAX_EVAL_LEN)
    return fail(EBIC_ERR_ARG, "max_breaks = %d outside [0, %d]", max_breaks, EBIC_MAX_EVAL_LEN);
  return extract_rows(h, offsets, cols, P, mode, max_breaks, row_offsets, rows, inout_capacity);
}

ebic_status ebic_recovery_relevance(int32_t E, const int64_t* e_row_off, const int32_t* e_rows,
                                    const int64_t* e_col_off, const int32_t* e_cols, int32_t F,
                                    const int64_t* f_row_off, const int32_t* f_rows,
                                    const int64_t* f_col_off, const int32_t* f_cols,
                                    double* out_recovery, double* out_relevance,
                                    double* out_jaccard) {
  if (E < 0 || F < 0 || (int64_t)E * F > (1ll << 26))
    return fail(EBIC_ERR_ARG, "E = %d, F = %d out of range", E, F);
  if (!out_recovery || !out_relevance) return fail(EBIC_ERR_ARG, "null pointer");
  if (E == 0 || F == 0) {
    *out_recovery = 0.0;
    *out_relevance = 0.0;
    return EBIC_OK;
  }
  if (!e_row_off || !e_rows || !e_col_off || !e_cols || !f_row_off || !f_rows || !f_col_off ||
      !f_cols)
    return fail(EBIC_ERR_ARG, "null pointer");
  const struct {
    const int64_t* off;
    const int32_t* v;
    int32_t n;
  } lists[4] = {{e_row_off, e_rows, E}, {e_col_off, e_cols, E}, {f_row_off, f_rows, F},
                {f_col_off, f_cols, F}};
  for (const auto& li : lists) {
    if (li.off[0] != 0) return fail(EBIC_ERR_ARG, "index lists must start at offset 0");
    for (int32_t i = 0; i < li.n; ++i) {
      if (li.off[i + 1] < li.off[i]) return fail(EBIC_ERR_ARG, "offsets must not decrease");
      if (!strictly_ascending(li.v + li.off[i], li.off[i + 1] - li.off[i], 0x7fffffff))
        return fail(EBIC_ERR_ARG, "bicluster %d: indices must be distinct, ascending, >= 0", i);
    }
  }
  DevBuf d[8], dJ, dout;
  auto release = [&]() {
    for (DevBuf& b : d) b.release();
    dJ.release();
    dout.release();
  };
  ebic_status st = EBIC_OK;
  const cudaStream_t s = nullptr;
  for (int i = 0; i < 4 && st == EBIC_OK; ++i) {
    const size_t no = (size_t)lists[i].n + 1, nv = (size_t)std::max<int64_t>(lists[i].off[lists[i].n], 1);
    if ((st = d[2 * i].reserve(no * sizeof(int64_t))) != EBIC_OK) break;
    if ((st = d[2 * i + 1].reserve(nv * sizeof(int32_t))) != EBIC_OK) break;
    if (cudaMemcpy(d[2 * i].ptr, lists[i].off, no * sizeof(int64_t), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(d[2 * i + 1].ptr, lists[i].v, (size_t)lists[i].off[lists[i].n] * sizeof(int32_t),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(EBIC_ERR_CUDA, "copy of the biclusters failed");
  }
  const size_t pairs = (size_t)E * F;
  if (st == EBIC_OK) st = dJ.reserve(pairs * sizeof(double));
  if (st == EBIC_OK) st = dout.reserve(2 * sizeof(double));
  if (st == EBIC_OK) {
    k_jaccard<<<(unsigned)((pairs * 32 + 255) / 256), 256, 0, s>>>(
        E, F, d[0].as<long long>(), d[1].as<int32_t>(), d[2].as<long long>(), d[3].as<int32_t>(),
        d[4].as<long long>(), d[5].as<int32_t>(), d[6].as<long long>(), d[7].as<int32_t>(),
        dJ.as<double>());
    k_recovery_relevance<<<1, 32, 0, s>>>(E, F, dJ.as<double>(), dout.as<double>());
    count_launches(2);
    double out[2];
    if (cudaMemcpy(out, dout.ptr, sizeof(out), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (out_jaccard &&
         cudaMemcpy(out_jaccard, dJ.ptr, pairs * sizeof(double), cudaMemcpyDeviceToHost) !=
             cudaSuccess)) {
      st = fail(EBIC_ERR_CUDA, "scoring failed: %s", cudaGetErrorString(cudaGetLastError()));
    } else {
      *out_recovery = out[0];
      *out_relevance = out[1];
    }
  }
  release();
  return st;
}

}  // extern "C"
