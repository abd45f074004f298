// Per-item device code of the support kernels (K3): the same functions serve
// the single-problem launches (ebic_matrix.cu) and the multi-problem
// persistent launch (ebic_batch.cu).
#pragma once

#include "ebic_internal.cuh"

namespace ebic {

// ---------------------------------------------------------------------------
// K3 shared pieces
// ---------------------------------------------------------------------------
constexpr int kBatch = 4;          // AND steps issued together before an exit test
constexpr unsigned kFull = 0xffffffffu;

// Eq. (1) for one series and the write-out of its results.
__device__ __forceinline__ void finish_series(const EvalArgs& a, const double* __restrict__ LN,
                                              int64_t i, uint32_t inc, uint32_t dec, int32_t L) {
  a.inc[i] = inc;
  if (a.dec) a.dec[i] = dec;
  int64_t n = (a.mode == EBIC_SUPPORT_INC_PLUS_DEC) ? (int64_t)inc + (int64_t)dec : (int64_t)inc;
  double f = 0.0;
  if (n > 1) {
    int64_t e = n - (int64_t)a.sigma;
    if (e > 0) e = 0;
    if (e < -2000) e = -2000;
    f = __dmul_rn(ldexp(LN[n - 1], (int)e), (double)L);
  }
  a.fit[i] = f;
  if (a.lnf) a.lnf[i] = f > 0.0 ? (float)log(f) : -INFINITY;
}

// Adds one part's counts into per-series scratch; the part that arrives last
// writes the results.  Rising counts only: one 64-bit word per series packs
// (parts arrived << 32 | count); a single atomicAdd both adds and takes a
// ticket, and its return value gives the last arriver the exact total -- no
// fence needed -- after which it puts the word back to zero.  With falling
// counts as well, a second word holds them and the arrival is fenced.  The
// scratch is zero when allocated and after every launch.
__device__ __forceinline__ void add_part(const EvalArgs& a, const double* __restrict__ LN,
                                         uint32_t* __restrict__ scratch, int32_t items_per,
                                         int32_t i, int64_t o, uint32_t inc, uint32_t dec,
                                         int32_t L, bool with_dec) {
  if (items_per == 1) {
    finish_series(a, LN, o, inc, dec, L);
    return;
  }
  unsigned long long* word = reinterpret_cast<unsigned long long*>(scratch) + 2 * (size_t)i;
  if (!with_dec) {
    const unsigned long long old = atomicAdd(word, (1ull << 32) | (unsigned long long)inc);
    if ((uint32_t)(old >> 32) == (uint32_t)items_per - 1) {
      *word = 0ull;
      finish_series(a, LN, o, (uint32_t)old + inc, 0u, L);
    }
    return;
  }
  unsigned long long* dword = word + 1;
  atomicAdd(dword, (unsigned long long)dec);
  __threadfence();
  const unsigned long long old = atomicAdd(word, (1ull << 32) | (unsigned long long)inc);
  if ((uint32_t)(old >> 32) == (uint32_t)items_per - 1) {
    __threadfence();
    const uint32_t n_dec = (uint32_t)atomicExch(dword, 0ull);
    *word = 0ull;
    finish_series(a, LN, o, (uint32_t)old + inc, n_dec, L);
  }
}

__device__ __forceinline__ uint32_t popc4(const uint4& v) {
  return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

__device__ __forceinline__ uint4 and4(const uint4& a, const uint4& b) {
  return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ bool nz4(const uint4& v) { return (v.x | v.y | v.z | v.w) != 0u; }

__device__ __forceinline__ uint4 ld_table(const uint4* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// K3 bitmask path, one warp per (series, part).  Lane l holds words
// [4 v, 4 v + 4) of the running AND for the vectors v = vb + l of the part.
// Steps are walked in windows of 32: lane t computes the pair index of step
// w0 + t and the warp broadcasts it with shuffles.  Every loop condition is
// warp-uniform; the warp leaves when its AND is zero in every lane.
// ---------------------------------------------------------------------------
template <bool DEC, bool CHECK, int NV, int KB, class Pop>
__device__ __forceinline__ void bitmask_warp_item(const uint32_t* __restrict__ LT, int32_t C,
                                                  int32_t W, int32_t R, const Pop& pop,
                                                  const EvalArgs& a, int32_t vecs_per_item,
                                                  int32_t items_per, uint32_t* __restrict__ tickets,
                                                  const double* __restrict__ LN,
                                                  int* __restrict__ err, int32_t sid, int32_t part,
                                                  int lane) {
  int64_t begin = 0;
  int32_t L = 0;
  bool ok = pop.range(sid, &begin, &L);
  bool bad = !ok;
  if (CHECK) {
    bool lb = false;
    if (ok)
      for (int t = lane; t < L; t += 32) lb |= (uint32_t)pop.col(begin, t) >= (uint32_t)C;
    if (__any_sync(kFull, lb)) bad = true;
    ok = ok && !bad;
  }
  const int32_t nsteps = ok ? L - 1 : 0;                 // warp-uniform
  const int32_t V = W >> 2;
  const int32_t v_lo = part * vecs_per_item;
  const int32_t v_hi = min(v_lo + vecs_per_item, V);
  const uint4* LT4 = reinterpret_cast<const uint4*>(LT);
  const size_t row4 = (size_t)V;
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  const uint4 zeros = make_uint4(0u, 0u, 0u, 0u);
  uint32_t cnt_inc = 0, cnt_dec = 0;

  for (int32_t vb = v_lo; vb < v_hi; vb += 32 * NV) {
    bool on[NV];
    uint4 mi[NV], md[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      on[k] = nsteps > 0 && vb + lane + 32 * k < v_hi;
      mi[k] = on[k] ? ones : zeros;
      md[k] = (DEC && on[k]) ? ones : zeros;
    }
    bool alive = nsteps > 0;                               // warp-uniform
    for (int32_t w0 = 0; alive && w0 < nsteps; w0 += 32) {
      uint32_t pi = 0, pd = 0;                             // pair indices x * C + y
      if (w0 + lane < nsteps) {
        uint32_t x = (uint32_t)pop.col(begin, w0 + lane);
        uint32_t y = (uint32_t)pop.col(begin, w0 + lane + 1);
        pi = x * (uint32_t)C + y;
        pd = y * (uint32_t)C + x;
      }
      const int32_t wn = min(32, nsteps - w0);             // warp-uniform
      for (int32_t t = 0; alive && t < wn; t += KB) {
        // a lane stops fetching for a block whose running AND is already zero
        bool live[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) live[k] = on[k] && (nz4(mi[k]) || (DEC && nz4(md[k])));
        uint4 xi[KB][NV], xd[KB][NV];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
          const uint32_t qi = __shfl_sync(kFull, pi, (t + u) & 31);
          const uint32_t qd = DEC ? __shfl_sync(kFull, pd, (t + u) & 31) : 0u;
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            const bool use = live[k] && (t + u) < wn;
            const int32_t vec = vb + lane + 32 * k;
            xi[u][k] = use ? ld_table(LT4 + (size_t)qi * row4 + vec) : ones;
            if (DEC) xd[u][k] = use ? ld_table(LT4 + (size_t)qd * row4 + vec) : ones;
          }
        }
        bool any_nz = false;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
#pragma unroll
          for (int u = 0; u < KB; ++u) {
            mi[k] = and4(mi[k], xi[u][k]);
            if (DEC) md[k] = and4(md[k], xd[u][k]);
          }
          any_nz |= on[k] && (nz4(mi[k]) || (DEC && nz4(md[k])));
        }
        alive = __any_sync(kFull, any_nz);
      }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      if (on[k]) {
        cnt_inc += popc4(mi[k]);
        if (DEC) cnt_dec += popc4(md[k]);
      }
    }
  }
  if (ok && L == 1 && part == 0 && lane == 0) cnt_inc = cnt_dec = (uint32_t)R;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt_inc += __shfl_xor_sync(kFull, cnt_inc, o);
    cnt_dec += __shfl_xor_sync(kFull, cnt_dec, o);
  }
  if (lane == 0) {
    if (bad) {
      atomicOr(err, 1);
      cnt_inc = cnt_dec = 0;
    }
    add_part(a, LN, tickets, items_per, sid, pop.out(sid), cnt_inc, DEC ? cnt_dec : 0u,
             bad ? 1 : L, DEC);
  }
}


// ---------------------------------------------------------------------------
// K3 gather path.  A warp owns one (series, part); lane l holds 4 consecutive
// rows (one float4 of each column read) and a 4-bit mask per direction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lt4(const float4& a, const float4& b) {
  return (uint32_t)(a.x < b.x) | ((uint32_t)(a.y < b.y) << 1) | ((uint32_t)(a.z < b.z) << 2) |
         ((uint32_t)(a.w < b.w) << 3);
}
__device__ __forceinline__ uint32_t gt4(const float4& a, const float4& b) {
  return (uint32_t)(a.x > b.x) | ((uint32_t)(a.y > b.y) << 1) | ((uint32_t)(a.z > b.z) << 2) |
         ((uint32_t)(a.w > b.w) << 3);
}

template <bool DEC, bool CHECK, class Pop>
__device__ __forceinline__ void gather_item(const float* __restrict__ A_c, int32_t C,
                                            int32_t R_pad, int32_t R, const Pop& pop,
                                            const EvalArgs& a, int32_t vecs_per_item,
                                            int32_t items_per, uint32_t* __restrict__ tickets,
                                            const double* __restrict__ LN, int* __restrict__ err,
                                            int32_t sid, int32_t part, int lane) {
  int64_t begin = 0;
  int32_t L = 0;
  bool ok = pop.range(sid, &begin, &L);
  bool bad = !ok;
  if (CHECK) {
    bool lb = false;
    if (ok)
      for (int t = lane; t < L; t += 32) lb |= (uint32_t)pop.col(begin, t) >= (uint32_t)C;
    if (__any_sync(kFull, lb)) bad = true;
    ok = ok && !bad;
  }
  const int32_t nsteps = ok ? L - 1 : 0;
  const int32_t V = R_pad >> 2;
  const int32_t v_lo = part * vecs_per_item;
  const int32_t v_hi = min(v_lo + vecs_per_item, V);
  const float4* A4 = reinterpret_cast<const float4*>(A_c);
  const size_t col4 = (size_t)V;
  uint32_t cnt_inc = 0, cnt_dec = 0;
  const size_t first = nsteps > 0 ? (size_t)(uint32_t)pop.col(begin, 0) * col4 : 0;

  for (int32_t vb = v_lo; vb < v_hi; vb += 32) {
    const int32_t vec = vb + lane;
    const bool lane_on = nsteps > 0 && vec < v_hi;
    uint32_t mi = lane_on ? 0xFu : 0u;
    uint32_t md = (DEC && lane_on) ? 0xFu : 0u;
    float4 prev = lane_on ? __ldg(A4 + first + vec) : make_float4(0.f, 0.f, 0.f, 0.f);
    bool alive = nsteps > 0;
    for (int32_t w0 = 0; alive && w0 < nsteps; w0 += 32) {
      uint32_t cl = 0;
      if (w0 + lane < nsteps) cl = (uint32_t)pop.col(begin, w0 + lane + 1);
      const int32_t wn = min(32, nsteps - w0);
      for (int32_t t = 0; alive && t < wn; t += kBatch) {
        float4 cur[kBatch];
        const bool live = lane_on && (mi | md) != 0u;   // own rows still rising/falling
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const uint32_t c = __shfl_sync(kFull, cl, (t + u) & 31);
          cur[u] = (live && t + u < wn) ? __ldg(A4 + (size_t)c * col4 + vec) : prev;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          if (t + u < wn) {
            mi &= lt4(prev, cur[u]);
            if (DEC) md &= gt4(prev, cur[u]);
            prev = cur[u];
          }
        }
        alive = __any_sync(kFull, (mi | md) != 0u);
      }
    }
    cnt_inc += __popc(mi);
    if (DEC) cnt_dec += __popc(md);
  }
  if (ok && L == 1 && part == 0 && lane == 0) cnt_inc = cnt_dec = (uint32_t)R;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt_inc += __shfl_xor_sync(kFull, cnt_inc, o);
    cnt_dec += __shfl_xor_sync(kFull, cnt_dec, o);
  }
  if (lane == 0) {
    if (bad) {
      atomicOr(err, 1);
      cnt_inc = cnt_dec = 0;
    }
    add_part(a, LN, tickets, items_per, sid, pop.out(sid), cnt_inc, DEC ? cnt_dec : 0u,
             bad ? 1 : L, DEC);
  }
}


}  // namespace ebic
