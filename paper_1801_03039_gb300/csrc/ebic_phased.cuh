// K3 bitmask path in phases (launch shape "kernel 4" of the evaluation):
// one persistent CTA per SM owns the series blockIdx.x, blockIdx.x + G, ...
// (G CTAs), taken in chunks of at most kPhasedItems series.
//
// Why: in a pipeline where one group of warps follows one series at a time,
// every series pays its own chain of dependent latencies (its offsets, its
// columns, the copy of its rows, each batch of its sparse tail, the count)
// and a group's series queue behind each other.  Here the chunk's set-up is
// paid once and each warp overlaps one series' sparse tail with the next
// series' copies:
//   phase 0  warp 0 reads the chunk's offsets; then warp w < ns (the slot
//            owners) reads the columns of its series w, w + ns, ... into the
//            chunk's column cache in shared memory;
//   phase 1  each slot owner copies the first `dense` table rows of its
//            series -- the rows every 128-row block still needs (a block of
//            iid rows keeps about 128 / (t + 1)! rising rows after t AND
//            steps) -- into its shared-memory slot with bulk copies (one per
//            row, issued by the warp's lanes, completing on the slot's
//            mbarrier), ANDs them, gathers the 16-byte vectors (128 rows)
//            still nonzero, issues the copies of its next series and only
//            then loads the next kPhasedBatch steps of those vectors; what
//            is still alive after that batch goes to the chunk's survivor
//            list;
//   phase 2  the survivors (almost only rows that truly rise) have all their
//            remaining steps spread over several threads of the CTA in one
//            round, combined with atomicAnd in shared memory (live vectors
//            that did not fit a warp's staging area first get their batch
//            here);
//   phase 3  one thread per series applies Eq. (1) (the log table was
//            prefetched into L2 at the start).
// Counts are exact: a series' count is the sum over its vectors of the
// popcount of the AND of all its steps, whichever phase finishes a vector;
// a list that overflows falls back to the walking thread finishing the
// vector itself.  Every mbarrier wait is bounded; a wait that gives up sets
// the device error flag (code 2) and that warp takes no further series.
// Rising counts only (a.dec == nullptr, mode EBIC_SUPPORT_INC).
#pragma once

#include "ebic_staged.cuh"

namespace ebic {

constexpr int kPhasedThreads = 1024;
constexpr int kPhasedItems = 32;        // series per chunk
constexpr int kPhasedCols = 4096;       // columns per chunk (one series: <= EBIC_MAX_EVAL_LEN)
constexpr int kPhasedBatch = 4;         // steps per load batch after the dense ones
constexpr int kPhasedStage = 64;        // live vectors a slot owner keeps per series (2 a lane)
constexpr int kPhasedLive = 512;        // live vectors beyond a warp's staging, per chunk
constexpr int kPhasedSurv = 512;        // vectors alive after the first batch, per chunk
constexpr int kPhasedMaxSlots = kPhasedThreads / 32;   // one slot per warp at most
static_assert(kPhasedCols >= EBIC_MAX_EVAL_LEN, "a chunk holds at least one series");

struct PhasedItem {
  int64_t begin;     // start of the series in the population view
  int32_t sid;       // series index
  int32_t L;         // length (0 when the range is invalid)
  int32_t coff;      // first column in the chunk's column cache
  int32_t flags;     // bit 0: valid, bit 1: invalid (range or column)
  uint32_t cnt;      // rising rows counted so far
  int32_t pad;
};

// Launch geometry, computed on the host.
struct PhasedGeom {
  int32_t dense;       // AND steps copied into the slots (1 .. kStagedMaxDense)
  int32_t ns;          // slots: warps 0 .. ns - 1 own one each
  int32_t slot_bytes;  // dense * V * 16, rounded up to 128
};

// Offsets of the dynamic shared memory regions (bytes from the 128-aligned base).
struct PhasedLayout {
  size_t ring, stage_bits, stage_tag, live_bits, surv_bits, live_tag, surv_tag, items, cols, bars,
      misc, total;
};

__host__ __device__ inline PhasedLayout phased_layout(const PhasedGeom& g) {
  PhasedLayout l;
  l.ring = 0;
  l.stage_bits = l.ring + (size_t)g.ns * g.slot_bytes;
  l.stage_tag = l.stage_bits + (size_t)g.ns * kPhasedStage * 16;
  l.live_bits = l.stage_tag + (size_t)g.ns * kPhasedStage * 4;
  l.surv_bits = l.live_bits + (size_t)kPhasedLive * 16;
  l.live_tag = l.surv_bits + (size_t)kPhasedSurv * 16;
  l.surv_tag = l.live_tag + (size_t)kPhasedLive * 4;
  l.items = l.surv_tag + (size_t)kPhasedSurv * 4;
  l.cols = l.items + (size_t)kPhasedItems * sizeof(PhasedItem);
  l.bars = l.cols + (size_t)kPhasedCols * 2;
  l.misc = l.bars + (size_t)kPhasedMaxSlots * 8;
  l.total = l.misc + 64;
  return l;
}

// Pair-table row of AND step t of a series whose columns start at cs.
__device__ __forceinline__ uint32_t phased_pair(const uint16_t* cs, int32_t t, int32_t C) {
  return (uint32_t)cs[t] * (uint32_t)C + (uint32_t)cs[t + 1];
}

// Finishes one live vector alone: steps t0 .. nsteps - 1 in batches, until
// its AND is zero.  Returns its rising rows.
__device__ __forceinline__ uint32_t phased_walk(const uint4* __restrict__ LT4, uint32_t V,
                                                const uint16_t* cs, int32_t C, uint32_t v,
                                                uint4 m, int32_t t0, int32_t nsteps) {
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  for (int32_t t = t0; t < nsteps && nz4(m); t += kPhasedBatch) {
    uint4 x[kPhasedBatch];
#pragma unroll
    for (int u = 0; u < kPhasedBatch; ++u)
      x[u] = t + u < nsteps ? ld_table(LT4 + (size_t)phased_pair(cs, t + u, C) * V + v) : ones;
#pragma unroll
    for (int u = 0; u < kPhasedBatch; ++u) m = and4(m, x[u]);
  }
  return popc4(m);
}

// Copies the dense rows of one series into a slot: one bulk copy per row
// (lane t issues row t), completing on the slot's mbarrier.  The slot must
// have been read by the warp (and the warp synchronised) before.
__device__ __forceinline__ void phased_issue(unsigned char* slot, unsigned long long* bar,
                                             const uint4* __restrict__ LT4, uint32_t V,
                                             const uint16_t* cs, int32_t C, int32_t rows,
                                             int lane) {
  const uint32_t row_bytes = V * 16u;
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_tx(bar, row_bytes * (uint32_t)rows);
  }
  __syncwarp();
  if (lane < rows)
    bulk_copy(slot + (size_t)lane * row_bytes, LT4 + (size_t)phased_pair(cs, lane, C) * V,
              row_bytes, bar);
}

// Rows one vector adds to the count after the batch that ends before step
// tnext, or 0 when it goes to the survivor list (which phase 2 finishes).
__device__ __forceinline__ uint32_t phased_after_batch(const uint4* __restrict__ LT4, uint32_t V,
                                                       const uint16_t* cs, int32_t C, uint4 m,
                                                       int32_t tnext, int32_t nsteps,
                                                       uint32_t tag, uint32_t* n_surv,
                                                       uint4* surv_bits, uint32_t* surv_tag) {
  if (!nz4(m) || nsteps <= tnext) return popc4(m);
  const uint32_t f = atomicAdd(n_surv, 1u);
  if (f < (uint32_t)kPhasedSurv) {
    surv_bits[f] = m;
    surv_tag[f] = tag;
    return 0u;
  }
  return phased_walk(LT4, V, cs, C, tag & 0xFFFFu, m, tnext, nsteps);
}

template <bool CHECK, class Pop>
__global__ void __launch_bounds__(kPhasedThreads, 1)
k_support_phased(const uint32_t* __restrict__ LT, int32_t C, int32_t W, int32_t R, Pop pop,
                 EvalArgs a, PhasedGeom g, const double* __restrict__ LN,
                 int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!pop.active()) return;
  const PhasedLayout ly = phased_layout(g);
  unsigned char* ring = smem + ly.ring;
  uint4* stage_bits = reinterpret_cast<uint4*>(smem + ly.stage_bits);
  uint32_t* stage_tag = reinterpret_cast<uint32_t*>(smem + ly.stage_tag);
  uint4* live_bits = reinterpret_cast<uint4*>(smem + ly.live_bits);
  uint4* surv_bits = reinterpret_cast<uint4*>(smem + ly.surv_bits);
  uint32_t* live_tag = reinterpret_cast<uint32_t*>(smem + ly.live_tag);
  uint32_t* surv_tag = reinterpret_cast<uint32_t*>(smem + ly.surv_tag);
  PhasedItem* items = reinterpret_cast<PhasedItem*>(smem + ly.items);
  uint16_t* cols = reinterpret_cast<uint16_t*>(smem + ly.cols);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + ly.bars);
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + ly.misc);
  uint32_t& n_live = misc[0];
  uint32_t& n_surv = misc[1];
  uint32_t& n_chunk = misc[2];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t V = (uint32_t)W >> 2;
  const uint4* LT4 = reinterpret_cast<const uint4*>(LT);
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  const uint32_t lt_mask = (1u << lane) - 1u;
  if (tid < g.ns) mbar_init(&full[tid], 1);      // the owning warp's lane 0
  uint32_t phase = 0;         // copies this warp has waited for (its slot's phase)
  bool failed = false;        // a wait of this warp gave up
  // The log table into L2 (this CTA's share of its lines), for phase 3.
  if (warp == kPhasedThreads / 32 - 1 && LN) {
    const size_t lines = ((size_t)R * sizeof(double) + 127) / 128;
    const size_t per = (lines + gridDim.x - 1) / gridDim.x;
    const size_t l0 = (size_t)blockIdx.x * per, l1 = min(lines, l0 + per);
    const char* base = reinterpret_cast<const char*>(LN);
    for (size_t l = l0 + lane; l < l1; l += 32)
      asm volatile("prefetch.L2 [%0];" ::"l"(base + l * 128));
  }

  const int32_t G = (int32_t)gridDim.x;
  const int32_t nq = (a.P - (int32_t)blockIdx.x + G - 1) / G;   // this CTA's series
  for (int32_t q0 = 0; q0 < nq;) {
    // ------------------------------------------------ phase 0: the chunk
    if (warp == 0) {
      const int32_t q = q0 + lane;
      int64_t begin = 0;
      int32_t L = 0;
      bool ok = false;
      if (q < nq) ok = pop.range((int32_t)blockIdx.x + G * q, &begin, &L);
      // (the host launches this kernel only for series of at most
      // kPhasedCols columns; a longer one would be reported as invalid)
      if (ok && L > kPhasedCols) ok = false;
      const int32_t Lc = ok ? L : 0;
      int32_t incl = Lc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const bool fits = q < nq && incl <= kPhasedCols;       // a prefix of the lanes
      const int32_t n = __popc(__ballot_sync(kFull, fits));
      if (lane < n) {
        PhasedItem& it = items[lane];
        it.begin = begin;
        it.sid = (int32_t)blockIdx.x + G * q;
        it.L = Lc;
        it.coff = incl - Lc;
        it.flags = ok ? 1 : 2;
        it.cnt = 0u;
      }
      if (lane == 0) {
        n_chunk = (uint32_t)n;
        n_live = 0u;
        n_surv = 0u;
      }
    }
    __syncthreads();
    const int32_t n = (int32_t)n_chunk;

    // -------------------------------- phases 0-1 of the slot owners
    if (warp < g.ns) {
      for (int32_t i = warp; i < n; i += g.ns) {       // the columns of this warp's series
        PhasedItem& it = items[i];
        bool bad = false;
        for (int32_t t = lane; t < it.L; t += 32) {
          const int32_t c = pop.col(it.begin, t);
          if (CHECK) bad |= (uint32_t)c >= (uint32_t)C;
          cols[it.coff + t] = (uint16_t)c;
        }
        if (CHECK && __any_sync(kFull, bad) && lane == 0) it.flags = 2;
      }
      __syncwarp();
      unsigned char* slot = ring + (size_t)warp * g.slot_bytes;
      const uint4* sd = reinterpret_cast<const uint4*>(slot);
      uint4* sb = stage_bits + (size_t)warp * kPhasedStage;
      uint32_t* stg = stage_tag + (size_t)warp * kPhasedStage;
      auto steps_of = [&](int32_t i) {
        return (items[i].flags & 1) ? items[i].L - 1 : 0;
      };
      unsigned long long* bar = &full[warp];
      bool pend = false;                      // copies of the current series in flight
      if (!failed && warp < n && min(steps_of(warp), g.dense) > 0) {
        phased_issue(slot, bar, LT4, V, cols + items[warp].coff, C, min(steps_of(warp), g.dense),
                     lane);
        pend = true;
      }
      for (int32_t i = warp; i < n && !failed; i += g.ns) {
        const int32_t nsteps = steps_of(i);
        const int32_t rows = min(nsteps, g.dense);
        const uint16_t* cs = cols + items[i].coff;
        if (pend) {
          failed = !__all_sync(kFull, mbar_wait(bar, phase & 1u));
          ++phase;
          if (failed) {
            if (lane == 0) atomicOr(err, 2);
            break;
          }
        }
        uint32_t cnt = 0, staged = 0;
        for (int32_t vb = 0; vb < (int32_t)V; vb += 32) {
          const uint32_t v = (uint32_t)(vb + lane);
          const bool in = v < V && nsteps > 0;
          uint4 m = ones;
          if (in)
            for (int32_t t = 0; t < rows; ++t) m = and4(m, sd[(size_t)t * V + v]);
          bool push = false;
          if (in) {
            if (nsteps <= g.dense) cnt += popc4(m);
            else push = nz4(m);
          }
          const uint32_t bal = __ballot_sync(kFull, push);
          if (push) {
            const uint32_t e = staged + (uint32_t)__popc(bal & lt_mask);
            const uint32_t tag = ((uint32_t)i << 16) | v;
            if (e < (uint32_t)kPhasedStage) {
              sb[e] = m;
              stg[e] = tag;
            } else {
              const uint32_t f = atomicAdd(&n_live, 1u);
              if (f < (uint32_t)kPhasedLive) {
                live_bits[f] = m;
                live_tag[f] = tag;
              } else {
                cnt += phased_walk(LT4, V, cs, C, v, m, g.dense, nsteps);
              }
            }
          }
          staged += (uint32_t)__popc(bal);
        }
        __syncwarp();
        const uint32_t ne = min(staged, (uint32_t)kPhasedStage);
        const bool h0 = (uint32_t)lane < ne, h1 = (uint32_t)lane + 32u < ne;
        uint4 m0 = ones, m1 = ones;
        uint32_t g0 = 0, g1 = 0;
        if (h0) {
          m0 = sb[lane];
          g0 = stg[lane];
        }
        if (h1) {
          m1 = sb[lane + 32];
          g1 = stg[lane + 32];
        }
        __syncwarp();                         // slot and staging read: reuse them
        pend = i + g.ns < n && min(steps_of(i + g.ns), g.dense) > 0;
        if (pend)
          phased_issue(slot, bar, LT4, V, cols + items[i + g.ns].coff, C,
                       min(steps_of(i + g.ns), g.dense), lane);
        // the first batch after the dense steps, both entries' loads in flight
        uint4 x0[kPhasedBatch], x1[kPhasedBatch];
#pragma unroll
        for (int u = 0; u < kPhasedBatch; ++u) {
          const int32_t t = g.dense + u;
          const bool st = t < nsteps;
          const uint32_t p = st ? phased_pair(cs, t, C) : 0u;
          x0[u] = h0 && st ? ld_table(LT4 + (size_t)p * V + (g0 & 0xFFFFu)) : ones;
          x1[u] = h1 && st ? ld_table(LT4 + (size_t)p * V + (g1 & 0xFFFFu)) : ones;
        }
#pragma unroll
        for (int u = 0; u < kPhasedBatch; ++u) {
          m0 = and4(m0, x0[u]);
          m1 = and4(m1, x1[u]);
        }
        const int32_t tn = g.dense + kPhasedBatch;
        if (h0) cnt += phased_after_batch(LT4, V, cs, C, m0, tn, nsteps, g0, &n_surv, surv_bits, surv_tag);
        if (h1) cnt += phased_after_batch(LT4, V, cs, C, m1, tn, nsteps, g1, &n_surv, surv_bits, surv_tag);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        if (lane == 0 && cnt) atomicAdd(&items[i].cnt, cnt);
      }
    }
    __syncthreads();

    // ------------------ phase 2: live vectors beyond the staging, survivors
    const uint32_t nl = min(n_live, (uint32_t)kPhasedLive);
    for (uint32_t e = (uint32_t)tid; e < nl; e += blockDim.x) {
      const uint32_t tag = live_tag[e];
      const int32_t i = (int32_t)(tag >> 16);
      const uint32_t v = tag & 0xFFFFu;
      const int32_t nsteps = items[i].L - 1;
      const uint16_t* cs = cols + items[i].coff;
      uint4 m = live_bits[e];
      uint4 x[kPhasedBatch];
#pragma unroll
      for (int u = 0; u < kPhasedBatch; ++u) {
        const int32_t t = g.dense + u;
        x[u] = t < nsteps ? ld_table(LT4 + (size_t)phased_pair(cs, t, C) * V + v) : ones;
      }
#pragma unroll
      for (int u = 0; u < kPhasedBatch; ++u) m = and4(m, x[u]);
      const uint32_t c = phased_after_batch(LT4, V, cs, C, m, g.dense + kPhasedBatch, nsteps, tag,
                                            &n_surv, surv_bits, surv_tag);
      if (c) atomicAdd(&items[i].cnt, c);
    }
    __syncthreads();
    const uint32_t nsv = min(n_surv, (uint32_t)kPhasedSurv);
    if (nsv > 0) {
      // threads per survivor: a power of two, at most 8
      uint32_t tps = 1;
      while (tps < 8 && nsv * tps * 2 <= blockDim.x) tps <<= 1;
      for (uint32_t u = (uint32_t)tid; u < nsv * tps; u += blockDim.x) {
        const uint32_t e = u / tps, r = u % tps;
        const uint32_t tag = surv_tag[e];
        const int32_t i = (int32_t)(tag >> 16);
        const uint32_t v = tag & 0xFFFFu;
        const int32_t nsteps = items[i].L - 1;
        const uint16_t* cs = cols + items[i].coff;
        uint4 m = surv_bits[e];
        const uint4 m0 = m;
        for (int32_t t = g.dense + kPhasedBatch + (int32_t)r * kPhasedBatch; t < nsteps && nz4(m);
             t += (int32_t)tps * kPhasedBatch) {
          uint4 x[kPhasedBatch];
#pragma unroll
          for (int q = 0; q < kPhasedBatch; ++q)
            x[q] = t + q < nsteps ? ld_table(LT4 + (size_t)phased_pair(cs, t + q, C) * V + v)
                                  : ones;
#pragma unroll
          for (int q = 0; q < kPhasedBatch; ++q) m = and4(m, x[q]);
        }
        unsigned int* w = reinterpret_cast<unsigned int*>(&surv_bits[e]);
        if (m.x != m0.x) atomicAnd(w + 0, m.x);
        if (m.y != m0.y) atomicAnd(w + 1, m.y);
        if (m.z != m0.z) atomicAnd(w + 2, m.z);
        if (m.w != m0.w) atomicAnd(w + 3, m.w);
      }
      __syncthreads();
      for (uint32_t e = (uint32_t)tid; e < nsv; e += blockDim.x) {
        const uint32_t c = popc4(surv_bits[e]);
        if (c) atomicAdd(&items[surv_tag[e] >> 16].cnt, c);
      }
    }
    __syncthreads();

    // ------------------------------------------------ phase 3: Eq. (1)
    if (tid < n) {
      const PhasedItem& it = items[tid];
      const bool bad = (it.flags & 2) != 0;
      uint32_t tot = it.cnt;
      if (!bad && it.L == 1) tot = (uint32_t)R;
      if (bad) {
        atomicOr(err, 1);
        tot = 0u;
      }
      const double ln = tot > 1 ? LN[tot - 1] : 0.0;
      staged_write(a, pop.out(it.sid), tot, bad ? 1 : it.L, ln);
    }
    q0 += n;
    __syncthreads();             // the chunk's tables are rewritten next
  }
  // After a wait that gave up, no copy may land once the CTA has left: the
  // slot's owner waits for that phase once more.
  if (failed && !mbar_wait(&full[warp], (phase - 1u) & 1u) && lane == 0) atomicOr(err, 2);
}

}  // namespace ebic
