// K3 bitmask path with the table rows staged in shared memory by bulk copies
// (launch shape "kernel 3" of the evaluation).
//
// Why: a series' support is an AND over its L - 1 table rows.  Every 128-row
// block of a series stays alive through its first few AND steps (a block of
// iid rows keeps about 128 / (t + 1)! rising rows after t steps), so those
// rows are needed whole for every series, and their addresses depend on
// nothing but the series' columns.  They are fetched by the copy engine
// (cp.async.bulk into shared memory, completed through an mbarrier), which
// keeps far more bytes in flight per SM than loads into registers can.  The
// sparse tail -- the later steps, taken only by the 128-row blocks still
// alive -- is read with per-thread loads and early exit per block, as in the
// warp kernel.
//
// One CTA holds `groups` groups of one scout warp and gw consumer warps.
//   scout      takes the items (series, part) s, s + S, s + 2S, ... (s its
//              group's index in the grid, S the number of groups) for the
//              first `static_rounds` rounds (by default all of them); any
//              items left it claims one at a time from a counter (each claim
//              issued one item ahead), so that groups whose items were quick
//              take more.  While an item's columns are in flight it reads the
//              next item's offsets; it writes the pair indices of the item's
//              first 64 AND steps to the stage header and issues one bulk
//              copy per staged ("dense") step: the item's vectors of that
//              step's table row.
//   consumers  thread j of the group owns vectors part * vpp + j + m * 32 gw
//              (m < NVT, 1 to 3).  It ANDs the staged rows, then walks the
//              remaining steps with loads of its own vectors, four steps per
//              batch (two with three vectors), until their AND is zero.  Each
//              warp adds its count to the stage's ticket word in shared
//              memory; the warp that
//              arrives last applies Eq. (1) (the log-table value it asks for
//              is brought in by an asynchronous copy and used one item
//              later, so no warp waits for it) and every warp then releases
//              the stage to the scout.
// Each group owns `ns` stages used as a ring: item k of the group is in stage
// k % ns.  Every mbarrier wait is bounded; a wait that gives up sets the
// device error flag (code 2) and that warp stops taking items.
#pragma once

#include "ebic_async.cuh"
#include "ebic_support.cuh"

namespace ebic {

constexpr int kStagedMaxPairs = 64;   // pair indices kept in a stage header
// Tail steps per batch: four, or two when a thread carries three vectors
// (the batch's loads stay within the register budget).
template <int NVT> struct StagedKB { static constexpr int value = NVT >= 3 ? 2 : 4; };
constexpr int kStagedMaxDense = 8;

struct StagedHdr {
  int64_t begin;     // start of the series in the population view
  int32_t sid;       // series, or -1: no more items
  int32_t part;
  int32_t L;
  int32_t flags;     // bit 0: valid series, bit 1: invalid (bad column or range)
  int32_t pad[2];
  uint32_t pair[kStagedMaxPairs];
};

// Launch geometry, computed on the host.
struct StagedGeom {
  int32_t groups;       // groups per CTA
  int32_t gw;           // consumer warps per group
  int32_t nvt;          // vectors per consumer thread (1 to 3)
  int32_t vpp;          // vectors per item (part), at most 32 * gw * nvt
  int32_t items_per;    // parts per series
  int32_t dense;        // AND steps staged by bulk copies (1 .. kStagedMaxDense)
  int32_t ns;           // stages per group
  int32_t data_bytes;   // dense * vpp * 16, rounded up to 128
  int32_t stage_bytes;  // data_bytes + header, rounded up to 128
  int32_t n_scouts;     // groups in the whole grid
  int32_t static_rounds;  // items per scout taken in the fixed stride first
};

// Deferred Eq. (1) write-out of one consumer warp (used by its lane 0): the
// log-table value is brought in by an asynchronous copy and read one item
// later.
struct StagedPend {
  double ln;
  int64_t out;
  uint32_t inc;
  int32_t L;        // 0: nothing pending
};

// Dynamic shared memory of one CTA: the stages, then the full and empty
// barriers and the ticket word of every stage, then one StagedPend per
// consumer warp.
__host__ __device__ inline size_t staged_smem_bytes(const StagedGeom& g) {
  return (size_t)g.groups * g.ns * g.stage_bytes + (size_t)g.groups * g.ns * 3 * 8 +
         (size_t)g.groups * g.gw * sizeof(StagedPend);
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive1(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Eq. (1) of one series from its count and LN[n - 1] (unused for n <= 1), as
// in finish_series, and the write-out of the rising count and fitness.
__device__ __forceinline__ void staged_write(const EvalArgs& a, int64_t out, uint32_t inc,
                                             int32_t L, double ln) {
  const int64_t n = (int64_t)inc;
  double f = 0.0;
  if (n > 1) {
    int64_t e = n - (int64_t)a.sigma;
    if (e > 0) e = 0;
    if (e < -2000) e = -2000;
    f = __dmul_rn(ldexp(ln, (int)e), (double)L);
  }
  a.inc[out] = inc;
  a.fit[out] = f;
  if (a.lnf) a.lnf[out] = f > 0.0 ? (float)log(f) : -INFINITY;
}

// Rising counts only (a.dec == nullptr, mode EBIC_SUPPORT_INC).  One CTA per
// SM (up to 1,024 threads, 64 registers a thread).
template <bool CHECK, class Pop, int NVT>
__global__ void __launch_bounds__(1024, 1)
k_support_staged(const uint32_t* __restrict__ LT, int32_t C, int32_t W, int32_t R, Pop pop,
                 EvalArgs a, StagedGeom g, uint32_t* __restrict__ tickets,
                 const double* __restrict__ LN, int* __restrict__ err,
                 uint32_t* __restrict__ claim) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!pop.active()) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gsize = g.gw + 1;                         // warps per group
  const int grp = warp / gsize;
  const int wg = warp % gsize;                        // 0 = scout
  unsigned char* gbase = smem + (size_t)grp * g.ns * g.stage_bytes;
  const int GS = g.groups * g.ns;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(smem + (size_t)GS * g.stage_bytes);
  unsigned long long* full = bars + (size_t)grp * g.ns;
  unsigned long long* empty = bars + GS + (size_t)grp * g.ns;
  unsigned long long* tick = bars + 2 * GS + (size_t)grp * g.ns;
  for (int i = threadIdx.x; i < GS; i += blockDim.x) {
    mbar_init(bars + i, 1);              // full: the scout
    mbar_init(bars + GS + i, g.gw);      // empty: each consumer warp
    bars[2 * GS + i] = 0ull;             // tickets
  }
  __syncthreads();

  const uint32_t V = (uint32_t)W >> 2;
  const uint4* LT4 = reinterpret_cast<const uint4*>(LT);
  const uint32_t n_items = (uint32_t)a.P * (uint32_t)g.items_per;
  const uint32_t S = (uint32_t)g.n_scouts;
  // Items below n_static go in a fixed stride (scout s: s, s + S, s + 2S,
  // ...); the rest are claimed one at a time from a counter, so that groups
  // that finish early take more of them.
  const uint32_t n_static = min(n_items, S * (uint32_t)g.static_rounds);

  if (wg == 0) {
    // ------------------------------------------------------------ scout
    const uint32_t first = blockIdx.x * g.groups + grp;
    uint32_t ks = 0;                                 // static items taken
    bool dyn = false;
    uint32_t raw = 0;                                // lane 0: the claim in flight
    bool pending = n_static < n_items;               // (warp-uniform)
    if (lane == 0 && pending) raw = atomicAdd(claim, 1u);
    // The next item; a dynamic one reads the claim issued earlier and issues
    // the claim of the one after.  Every claim is read before the scout ends.
    auto next_item = [&]() -> uint32_t {
      if (!dyn) {
        const uint32_t it = first + ks * S;
        if (it < n_static) {
          ++ks;
          return it;
        }
        dyn = true;
        if (!pending) return n_items;
      }
      const uint32_t it = n_static + __shfl_sync(kFull, raw, 0);
      pending = it < n_items;
      if (lane == 0 && pending) raw = atomicAdd(claim, 1u);
      return it;
    };
    uint32_t item = next_item();
    int64_t begin = 0;
    int32_t L = 0;
    bool ok = false;
    if (item < n_items) ok = pop.range((int32_t)(item / g.items_per), &begin, &L);
    int k = 0;
    bool alive = true;
    for (; item < n_items; ++k) {
      const int32_t sid = (int32_t)(item / g.items_per);
      const int32_t part = (int32_t)(item % g.items_per);
      // columns of steps 0 .. 63: lane t holds columns t, t + 32 (and lane 31 column 64)
      uint32_t c0 = 0, c1 = 0, c2 = 0;
      if (ok) {
        if (lane < L) c0 = (uint32_t)pop.col(begin, lane);
        if (lane + 32 < L) c1 = (uint32_t)pop.col(begin, lane + 32);
        if (lane == 31 && 64 < L) c2 = (uint32_t)pop.col(begin, 64);
      }
      // the next item's offsets, while those columns are in flight
      const uint32_t nitem = next_item();
      int64_t nbegin = 0;
      int32_t nL = 0;
      bool nok = false;
      if (nitem < n_items) nok = pop.range((int32_t)(nitem / g.items_per), &nbegin, &nL);
      bool lb = false;
      if (CHECK && ok) {
        lb = (lane < L && c0 >= (uint32_t)C) || (lane + 32 < L && c1 >= (uint32_t)C);
        for (int t = lane + 64; t < L; t += 32) lb |= (uint32_t)pop.col(begin, t) >= (uint32_t)C;
      }
      const bool bad = !ok || __any_sync(kFull, lb);
      const int32_t nsteps = bad ? 0 : L - 1;
      const uint32_t nx0 = __shfl_down_sync(kFull, c0, 1);
      const uint32_t nx1 = __shfl_down_sync(kFull, c1, 1);
      const uint32_t first1 = __shfl_sync(kFull, c1, 0);
      const uint32_t p0 = c0 * (uint32_t)C + (lane < 31 ? nx0 : first1);   // step lane
      const uint32_t p1 = c1 * (uint32_t)C + (lane < 31 ? nx1 : c2);       // step lane + 32
      const int s = k % g.ns;
      unsigned char* st = gbase + (size_t)s * g.stage_bytes;
      StagedHdr* hd = reinterpret_cast<StagedHdr*>(st + g.data_bytes);
      if (k >= g.ns && !mbar_wait(&empty[s], (uint32_t)((k / g.ns) - 1) & 1u)) {
        if (lane == 0) atomicOr(err, 2);
        alive = false;
        break;
      }
      if (lane < nsteps) hd->pair[lane] = p0;
      if (lane + 32 < nsteps) hd->pair[lane + 32] = p1;
      if (lane == 0) {
        hd->begin = begin;
        hd->sid = sid;
        hd->part = part;
        hd->L = L;
        hd->flags = bad ? 2 : 1;
      }
      __syncwarp();
      if (lane == 0) {
        const int32_t rows = min(nsteps, g.dense);
        const int32_t v0 = part * g.vpp;
        const int32_t vlen = min(g.vpp, (int32_t)V - v0);
        const uint32_t row_bytes = (uint32_t)vlen * 16u;
        if (rows > 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_tx(&full[s], row_bytes * (uint32_t)rows);
          for (int t = 0; t < rows; ++t)
            bulk_copy(st + (size_t)t * row_bytes, LT4 + (size_t)hd->pair[t] * V + v0, row_bytes,
                      &full[s]);
        } else {
          mbar_arrive1(&full[s]);
        }
      }
      item = nitem;
      begin = nbegin;
      L = nL;
      ok = nok;
    }
    // a scout that gave up still reads its claim in flight, so that the
    // counter reset below comes after every claim of this launch
    if (pending && __shfl_sync(kFull, raw, 0) == 0xffffffffu && lane == 0) atomicOr(err, 4);
    // No copy may still be landing when the CTA leaves (which could only
    // happen after a consumer gave up): wait until the latest phase of every
    // stage -- one of the last ns items -- is complete.  Only the scout
    // arrives on the full barriers, so these are their current phases.
    for (int t = max(0, k - g.ns); t < k; ++t)
      if (!mbar_wait(&full[t % g.ns], (uint32_t)(t / g.ns) & 1u)) {
        if (lane == 0) atomicOr(err, 2);
      }
    if (alive) {
      // end marker
      const int s = k % g.ns;
      StagedHdr* hd =
          reinterpret_cast<StagedHdr*>(gbase + (size_t)s * g.stage_bytes + g.data_bytes);
      if (k >= g.ns && !mbar_wait(&empty[s], (uint32_t)((k / g.ns) - 1) & 1u)) {
        if (lane == 0) atomicOr(err, 2);
      } else if (lane == 0) {
        hd->sid = -1;
        mbar_arrive1(&full[s]);
      }
    }
    // The last scout to finish puts the claim counter back to zero for the
    // next launch (every scout's claims have returned by now).
    if (lane == 0 && n_static < n_items) {
      __threadfence();
      const uint32_t done = atomicAdd(claim + 1, 1u);
      if (done == S - 1) {
        claim[0] = 0u;
        claim[1] = 0u;
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int j = (wg - 1) * 32 + lane;                 // thread within the group
  const int stride = g.gw * 32;
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  const bool direct = g.items_per == 1;               // else add_part's tickets
  StagedPend* pend = reinterpret_cast<StagedPend*>(bars + 3 * GS) + (size_t)grp * g.gw + (wg - 1);
  if (lane == 0) pend->L = 0;
  for (int k = 0;; ++k) {
    const int s = k % g.ns;
    const unsigned char* st = gbase + (size_t)s * g.stage_bytes;
    const StagedHdr* hd = reinterpret_cast<const StagedHdr*>(st + g.data_bytes);
    if (!mbar_wait(&full[s], (uint32_t)(k / g.ns) & 1u)) {
      if (lane == 0) atomicOr(err, 2);
      break;
    }
    const int32_t sid = hd->sid;
    if (sid < 0) break;
    const int32_t part = hd->part, L = hd->L, flags = hd->flags;
    const bool good = (flags & 1) != 0;
    const int32_t nsteps = good ? L - 1 : 0;
    const int32_t v0 = part * g.vpp;
    const int32_t vlen = min(g.vpp, (int32_t)V - v0);
    const int32_t rows = min(nsteps, g.dense);
    uint4 m[NVT];
    bool on[NVT];
    const uint4* sd = reinterpret_cast<const uint4*>(st);
#pragma unroll
    for (int q = 0; q < NVT; ++q) {
      const int jj = j + q * stride;
      on[q] = nsteps > 0 && jj < vlen;
      m[q] = on[q] ? ones : make_uint4(0u, 0u, 0u, 0u);
      if (on[q])
        for (int t = 0; t < rows; ++t) m[q] = and4(m[q], sd[(size_t)t * vlen + jj]);
    }
    // the remaining steps, all of this thread's live vectors together
    constexpr int KB = StagedKB<NVT>::value;
    for (int32_t t = rows; t < nsteps; t += KB) {
      bool live[NVT], any = false;
#pragma unroll
      for (int q = 0; q < NVT; ++q) {
        live[q] = on[q] && nz4(m[q]);
        any |= live[q];
      }
      if (!any) break;
      uint4 x[KB][NVT];
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const int32_t tt = t + u;
        uint32_t pr = 0;
        if (tt < nsteps)
          pr = tt < kStagedMaxPairs ? hd->pair[tt]
                                    : (uint32_t)pop.col(hd->begin, tt) * (uint32_t)C +
                                          (uint32_t)pop.col(hd->begin, tt + 1);
#pragma unroll
        for (int q = 0; q < NVT; ++q)
          x[u][q] = (live[q] && tt < nsteps)
                        ? ld_table(LT4 + (size_t)pr * V + (uint32_t)(v0 + j + q * stride))
                        : ones;
      }
#pragma unroll
      for (int u = 0; u < KB; ++u)
#pragma unroll
        for (int q = 0; q < NVT; ++q) m[q] = and4(m[q], x[u][q]);
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < NVT; ++q) cnt += on[q] ? popc4(m[q]) : 0u;
    if (good && L == 1 && part == 0 && j == 0) cnt = (uint32_t)R;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane == 0) {
      // the previous item this warp finished: its log value has arrived
      if (pend->L != 0) {
        cp_async_wait_all();
        staged_write(a, pend->out, pend->inc, pend->L, pend->ln);
        pend->L = 0;
      }
      const unsigned long long old = atomicAdd(&tick[s], (1ull << 32) | (unsigned long long)cnt);
      if ((uint32_t)(old >> 32) == (uint32_t)g.gw - 1) {
        tick[s] = 0ull;                               // before the stage is released
        uint32_t tot = (uint32_t)old + cnt;
        const bool bad = (flags & 2) != 0;
        if (bad) {
          atomicOr(err, 1);
          tot = 0;
        }
        const int32_t Lf = bad ? 1 : L;
        if (direct) {
          pend->out = pop.out(sid);
          pend->inc = tot;
          pend->L = Lf;
          if (tot > 1) cp_async8(&pend->ln, LN + (tot - 1));
        } else {
          add_part(a, LN, tickets, g.items_per, sid, pop.out(sid), tot, 0u, Lf, false);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive1(&empty[s]);          // this warp is done with the stage
  }
  if (lane == 0 && pend->L != 0) {
    cp_async_wait_all();
    staged_write(a, pend->out, pend->inc, pend->L, pend->ln);
  }
}

}  // namespace ebic
