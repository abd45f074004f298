// Matrix placement, pair bitmask table and population evaluation.
//
//   K1 k_load_colmajor  -- row-major fp32 -> column-major, NaN-padded to a
//                          multiple of 128 rows (Step 1: data placed on the GPU)
//   K2 k_pair_table     -- LT[p][q][w] = ballot over 32 rows of a[k][p] < a[k][q]
//                          (the pairwise count #{k : a_kp < a_kq}, "Motivation")
//   K3 k_support_bitmask / k_support_gather
//                       -- support of every series (strict chain, "Motivation";
//                          Step 4) reduced to exact counts, with Eq. (1) fused
//                          into the epilogue of the last part of each series.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstring>
#include <vector>

#include "ebic_internal.cuh"
#include "ebic_phased.cuh"
#include "ebic_staged.cuh"
#include "ebic_support.cuh"

namespace ebic {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// errors and buffers
// ---------------------------------------------------------------------------
static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

ebic_status fail(ebic_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

ebic_status DevBuf::reserve(size_t want) {
  if (want <= bytes) return EBIC_OK;
  release();
  if (want == 0) return EBIC_OK;
  EBIC_CUDA_TRY(cudaMalloc(&ptr, want));
  bytes = want;
  return EBIC_OK;
}

ebic_status DevBuf::reserve_zeroed(size_t want, cudaStream_t s) {
  if (want <= bytes) return EBIC_OK;
  EBIC_TRY(reserve(want));
  EBIC_CUDA_TRY(cudaMemsetAsync(ptr, 0, bytes, s));
  return EBIC_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

ebic_status HostBuf::reserve(size_t want) {
  if (want <= bytes) return EBIC_OK;
  release();
  if (want == 0) return EBIC_OK;
  EBIC_CUDA_TRY(cudaMallocHost(&ptr, want));
  bytes = want;
  return EBIC_OK;
}

void HostBuf::release() {
  if (ptr) cudaFreeHost(ptr);
  ptr = nullptr;
  bytes = 0;
}

// Makes the handle's device current for the lifetime of the object.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else if (prev == dev) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------------------
// K1: column-major placement
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_load_colmajor(const float* __restrict__ src, int32_t R, int32_t C, int32_t R_pad,
                float* __restrict__ dst) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  const float qnan = __int_as_float(0x7fc00000);
  for (int j = ty; j < 32; j += 8) {
    int r = r0 + j, c = c0 + tx;
    tile[j][tx] = (r < R && c < C) ? src[(size_t)r * C + c] : qnan;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    int c = c0 + j, r = r0 + tx;
    if (c < C && r < R_pad) dst[(size_t)c * R_pad + r] = tile[tx][j];
  }
}

// ---------------------------------------------------------------------------
// K2: pair bitmask table.  Layout: entry (p, q) is W words = V 16-byte vectors;
// vector b covers rows 128 b .. 128 b + 127, and bit l of its word i is the
// row 128 b + 4 l + i (each lane of a warp reads one float4 = 4 consecutive
// rows, and one ballot per component gives one word).  Counting only ANDs and
// popcounts whole vectors, so the order of bits inside a vector is free.
// One CTA = 8 columns p (one per warp) x 8 vectors (1,024 rows); each warp
// keeps its column's 8 float4 in registers and walks every q; the 8 warps read
// the same q values, which L1 serves after the first.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_pair_table(const float* __restrict__ A_c, int32_t C, int32_t R_pad, int32_t W,
             uint32_t* __restrict__ LT) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = blockIdx.y * 8 + warp;
  const int V = R_pad >> 7;                      // 128-row vectors per column
  const int b0 = blockIdx.x * 8;
  if (p >= C) return;
  const int nb = min(8, V - b0);
  const float qnan = __int_as_float(0x7fc00000);
  const float4 nan4 = make_float4(qnan, qnan, qnan, qnan);
  const float4* A4 = reinterpret_cast<const float4*>(A_c);
  const size_t col4 = (size_t)R_pad >> 2;        // float4 per column
  float4 ap[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) ap[b] = (b < nb) ? A4[(size_t)p * col4 + (size_t)(b0 + b) * 32 + lane] : nan4;
  uint32_t* out = LT + (size_t)p * C * W + (size_t)b0 * 4;
  for (int q = 0; q < C; ++q) {
    const float4* colq = A4 + (size_t)q * col4 + (size_t)b0 * 32;
    uint32_t mine = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float4 aq = (b < nb) ? colq[b * 32 + lane] : nan4;
      const uint32_t w0 = __ballot_sync(0xffffffffu, ap[b].x < aq.x);
      const uint32_t w1 = __ballot_sync(0xffffffffu, ap[b].y < aq.y);
      const uint32_t w2 = __ballot_sync(0xffffffffu, ap[b].z < aq.z);
      const uint32_t w3 = __ballot_sync(0xffffffffu, ap[b].w < aq.w);
      if (lane == 4 * b + 0) mine = w0;
      if (lane == 4 * b + 1) mine = w1;
      if (lane == 4 * b + 2) mine = w2;
      if (lane == 4 * b + 3) mine = w3;
    }
    if (lane < 4 * nb) out[(size_t)q * W + lane] = mine;
  }
}

// ---------------------------------------------------------------------------
// K3 kernels: one warp per (series, part) calls the per-item code of
// ebic_support.cuh; the lane kernel serves short tables.
// ---------------------------------------------------------------------------
template <bool DEC, bool CHECK, int NV, int KB, class Pop>
__global__ void __launch_bounds__(256)
k_support_bitmask_warp(const uint32_t* __restrict__ LT, int32_t C, int32_t W, int32_t R,
                       Pop pop, EvalArgs a, int32_t vecs_per_item, int32_t items_per,
                       uint32_t* __restrict__ tickets, const double* __restrict__ LN,
                       int* __restrict__ err) {
  if (!pop.active()) return;
  const int lane = threadIdx.x & 31;
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_items = (int64_t)a.P * items_per;
  if (item >= n_items) return;                           // warp-uniform
  bitmask_warp_item<DEC, CHECK, NV, KB, Pop>(LT, C, W, R, pop, a, vecs_per_item, items_per,
                                             tickets, LN, err, (int32_t)(item / items_per),
                                             (int32_t)(item % items_per), lane);
}

// ---------------------------------------------------------------------------
// K3 bitmask path for short tables (at most 32 16-byte vectors per entry, i.e.
// up to 4096 rows): one lane per (series, vector).  The VP = 2^k lanes of a
// series are consecutive and aligned, each walks the whole chain for its own
// vector with its own early exit -- no warp-level vote inside the loops -- and
// a butterfly over the VP lanes sums the counts at the end.
// ---------------------------------------------------------------------------
template <bool DEC, bool CHECK, class Pop>
__global__ void __launch_bounds__(256)
k_support_bitmask_lane(const uint32_t* __restrict__ LT, int32_t C, int32_t W, int32_t R,
                       Pop pop, EvalArgs a, int32_t VP, const double* __restrict__ LN,
                       int* __restrict__ err) {
  if (!pop.active()) return;
  const int lane = threadIdx.x & 31;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t sid64 = tid / VP;
  const int32_t v = (int32_t)(tid % VP);
  const bool valid = sid64 < a.P;
  const int32_t sid = valid ? (int32_t)sid64 : 0;
  int64_t begin = 0;
  int32_t L = 0;
  bool ok = valid && pop.range(sid, &begin, &L);
  uint32_t bad = (valid && !ok) ? 1u : 0u;
  if (CHECK && ok)
    for (int t = v; t < L; t += VP) bad |= (uint32_t)pop.col(begin, t) >= (uint32_t)C ? 1u : 0u;
  for (int o = 1; o < VP; o <<= 1) bad |= __shfl_xor_sync(kFull, bad, o);
  ok = ok && !bad;
  const int32_t V = W >> 2;
  const int32_t nsteps = ok ? L - 1 : 0;
  const bool lane_on = nsteps > 0 && v < V;
  const uint4* LT4 = reinterpret_cast<const uint4*>(LT);
  const size_t row4 = (size_t)V;
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  uint4 mi = lane_on ? ones : make_uint4(0u, 0u, 0u, 0u);
  uint4 md = (DEC && lane_on) ? ones : make_uint4(0u, 0u, 0u, 0u);
  if (lane_on) {
    uint32_t x = (uint32_t)pop.col(begin, 0);
    for (int32_t i = 0; i < nsteps; i += kBatch) {
      uint4 xi[kBatch], xd[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (i + u < nsteps) {
          const uint32_t y = (uint32_t)pop.col(begin, i + u + 1);
          xi[u] = ld_table(LT4 + (size_t)(x * (uint32_t)C + y) * row4 + v);
          if (DEC) xd[u] = ld_table(LT4 + (size_t)(y * (uint32_t)C + x) * row4 + v);
          x = y;
        } else {
          xi[u] = ones;
          if (DEC) xd[u] = ones;
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        mi = and4(mi, xi[u]);
        if (DEC) md = and4(md, xd[u]);
      }
      if (!(nz4(mi) || (DEC && nz4(md)))) break;
    }
  }
  uint32_t cnt_inc = lane_on ? popc4(mi) : 0u;
  uint32_t cnt_dec = (DEC && lane_on) ? popc4(md) : 0u;
  if (ok && L == 1 && v == 0) cnt_inc = cnt_dec = (uint32_t)R;
  for (int o = 1; o < VP; o <<= 1) {
    cnt_inc += __shfl_xor_sync(kFull, cnt_inc, o);
    cnt_dec += __shfl_xor_sync(kFull, cnt_dec, o);
  }
  (void)lane;
  if (valid && v == 0) {
    if (bad) {
      atomicOr(err, 1);
      cnt_inc = cnt_dec = 0;
    }
    finish_series(a, LN, pop.out(sid), cnt_inc, DEC ? cnt_dec : 0u, bad ? 1 : L);
  }
}

template <bool DEC, bool CHECK, class Pop>
__global__ void __launch_bounds__(256)
k_support_gather(const float* __restrict__ A_c, int32_t C, int32_t R_pad, int32_t R, Pop pop,
                 EvalArgs a, int32_t vecs_per_item, int32_t items_per,
                 uint32_t* __restrict__ tickets, const double* __restrict__ LN,
                 int* __restrict__ err) {
  if (!pop.active()) return;
  const int lane = threadIdx.x & 31;
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_items = (int64_t)a.P * items_per;
  if (item >= n_items) return;
  gather_item<DEC, CHECK, Pop>(A_c, C, R_pad, R, pop, a, vecs_per_item, items_per, tickets, LN,
                               err, (int32_t)(item / items_per), (int32_t)(item % items_per),
                               lane);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
constexpr int kSMs = 152;          // GB300
constexpr int kTargetWarps = kSMs * 48 * 3;   // about three warps per resident slot
constexpr int kWarpsPerCta = 2;    // small CTAs: the block scheduler balances uneven series

// Split each series' vectors into parts so that the launch has enough warps.
static void choose_split(int32_t P, int32_t V, int32_t forced_vpi, int32_t* vecs_per_item,
                         int32_t* items_per, int32_t lanes_vecs = 32) {
  if (forced_vpi > 0) {
    *vecs_per_item = std::max(forced_vpi / 32, 1) * 32;
    *items_per = (V + *vecs_per_item - 1) / *vecs_per_item;
    return;
  }
  int32_t chunks = (V + lanes_vecs - 1) / lanes_vecs;
  int64_t want = (kTargetWarps + (int64_t)P - 1) / std::max<int64_t>(P, 1);
  int32_t parts = (int32_t)std::min<int64_t>(std::max<int64_t>(want, 1), chunks);
  int32_t per = (chunks + parts - 1) / parts;
  *vecs_per_item = per * lanes_vecs;
  *items_per = (V + *vecs_per_item - 1) / *vecs_per_item;
}

int32_t resolve_path(ebic_ctx* h) {
  if (h->path == EBIC_PATH_GATHER) return EBIC_PATH_GATHER;
  if (h->path == EBIC_PATH_BITMASK) return EBIC_PATH_BITMASK;
  return h->LT ? EBIC_PATH_BITMASK : EBIC_PATH_GATHER;
}

// Geometry of the staged kernel for this handle and tuning; false if it
// cannot run here (a group does not fit one CTA).  Parts hold at most 256
// vectors; a consumer thread carries `vecs_per_lane` of them (1 to 3; 0 =
// 2 for parts over 64 vectors).
constexpr int kStagedMaxSmem = 227 * 1024;   // the per-CTA opt-in limit of sm_100 / sm_103

static bool staged_geometry(const ebic_ctx* h, const ebic_eval_tuning_t& tu, int32_t P,
                            StagedGeom* out) {
  StagedGeom g{};
  const int32_t V = h->W >> 2;
  // an item holds at most 256 vectors (or the tuning's part size), the
  // parts of a series as even as possible
  const int32_t cap = tu.vecs_per_part_bitmask > 0 ? std::min(tu.vecs_per_part_bitmask, 256) : 256;
  const int32_t parts = (V + cap - 1) / cap;
  g.vpp = (V + parts - 1) / parts;
  g.items_per = parts;
  g.nvt = (tu.vecs_per_lane >= 1 && tu.vecs_per_lane <= 3) ? tu.vecs_per_lane
                                                           : (g.vpp > 64 ? 2 : 1);
  g.gw = (g.vpp + 32 * g.nvt - 1) / (32 * g.nvt);
  g.dense = tu.dense_steps > 0 ? tu.dense_steps : 4;
  g.ns = tu.stages > 0 ? tu.stages : 2;
  g.data_bytes = (g.dense * g.vpp * 16 + 127) / 128 * 128;
  g.stage_bytes = (g.data_bytes + (int32_t)sizeof(StagedHdr) + 127) / 128 * 128;
  int32_t groups = 0;
  for (int32_t n = 1; n <= 15; ++n) {
    StagedGeom t = g;
    t.groups = n;
    if (n * (g.gw + 1) * 32 > 1024 || staged_smem_bytes(t) > (size_t)kStagedMaxSmem) break;
    groups = n;
  }
  if (tu.groups > 0) groups = std::min(groups, tu.groups);
  if (groups < 1 || (int64_t)P * parts >= (1ll << 31)) return false;
  g.groups = groups;
  *out = g;
  return true;
}

// Queues the staged kernel (rising counts only): one CTA per SM, capped by
// the items.
template <bool CHECK, class Pop, int NVT>
static ebic_status launch_staged(ebic_ctx* h, const Pop& pop, const EvalArgs& a,
                                 const StagedGeom& g0, cudaStream_t s) {
  StagedGeom g = g0;
  const size_t smem = staged_smem_bytes(g);
  const int threads = g.groups * (g.gw + 1) * 32;
  auto kern = k_support_staged<CHECK, Pop, NVT>;
  // The shared-memory opt-in is set to the device maximum (every handle sets
  // the same value, so handles with different shapes never undercut each
  // other) and the occupancy is queried once per shape and handle.
  StagedMemo& memo = h->staged_memo;
  const void* fn = reinterpret_cast<const void*>(kern);
  if (memo.fn != fn || memo.threads != threads || memo.smem != smem) {
    EBIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStagedMaxSmem));
    EBIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&memo.per_sm, kern, threads, smem));
    memo.fn = fn;
    memo.threads = threads;
    memo.smem = smem;
  }
  const int per_sm = memo.per_sm;
  if (per_sm < 1) return fail(EBIC_ERR_CUDA, "staged kernel: no CTA fits an SM");
  const int64_t n_items = (int64_t)a.P * g.items_per;
  const int64_t grid = std::min<int64_t>((int64_t)h->sm_count * per_sm,
                                         (n_items + g.groups - 1) / g.groups);
  g.n_scouts = (int32_t)(grid * g.groups);
  // fixed-stride rounds: the even share less the last `dynamic_rounds`
  // rounds, whose items and the remainder are claimed dynamically; 0 or -1
  // (the default): every item in the fixed stride (measured as fast as any
  // dynamic share on the 20,000 x 200 pass, whose claims cost what the
  // balance gains)
  const int64_t rounds = n_items / g.n_scouts;
  const int32_t dyn_rounds = h->tuning.dynamic_rounds;
  g.static_rounds = dyn_rounds <= 0 ? (int32_t)(rounds + 1)
                                    : (int32_t)std::max<int64_t>(0, rounds - dyn_rounds);
  if (g.items_per > 1)
    EBIC_TRY(h->tickets.reserve_zeroed((size_t)a.P * 2 * sizeof(unsigned long long), s));
  count_launches(1);
  kern<<<(unsigned)grid, threads, smem, s>>>(h->LT, h->C, h->W, h->R, pop, a, g,
                                             h->tickets.as<uint32_t>(), h->LN, h->d_err,
                                             h->d_claim);
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

// Longest series a population view can hold.
static int32_t pop_max_len(const CbfPop&) { return EBIC_MAX_EVAL_LEN; }
static int32_t pop_max_len(const FixedPop& p) { return p.stride; }
static int32_t pop_max_len(const ArchivePop& p) { return p.stride; }

// Geometry of the phased kernel (kernel 4): the slots take the shared memory
// the fixed regions leave, at most one per warp; false when fewer than two
// slots fit or the view can hold series longer than a chunk.
template <class Pop>
static bool phased_geometry(const ebic_ctx* h, const ebic_eval_tuning_t& tu, const Pop& pop,
                            PhasedGeom* out) {
  const int32_t V = h->W >> 2;
  if (V < 1 || V > 65535 || pop_max_len(pop) > kPhasedCols) return false;
  PhasedGeom g{};
  g.dense = tu.dense_steps > 0 ? tu.dense_steps : 5;
  g.slot_bytes = (int32_t)(((int64_t)g.dense * V * 16 + 127) / 128 * 128);
  g.ns = 0;
  const size_t fixed = phased_layout(g).total;           // with no ring
  if (fixed >= (size_t)kStagedMaxSmem) return false;
  const int64_t per_slot = g.slot_bytes + (int64_t)kPhasedStage * 20;   // slot + staging
  const int64_t fit = ((int64_t)kStagedMaxSmem - (int64_t)fixed) / per_slot;
  g.ns = (int32_t)std::min<int64_t>(fit, kPhasedMaxSlots);
  if (tu.stages > 0) g.ns = std::min(g.ns, tu.stages);
  if (g.ns < 2) return false;
  *out = g;
  return true;
}

// Queues the phased kernel: one CTA per SM, at most one per series.
template <bool CHECK, class Pop>
static ebic_status launch_phased(ebic_ctx* h, const Pop& pop, const EvalArgs& a,
                                 const PhasedGeom& g, cudaStream_t s) {
  const size_t smem = phased_layout(g).total;
  auto kern = k_support_phased<CHECK, Pop>;
  StagedMemo& memo = h->phased_memo;
  const void* fn = reinterpret_cast<const void*>(kern);
  if (memo.fn != fn || memo.smem != smem) {
    EBIC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStagedMaxSmem));
    EBIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&memo.per_sm, kern,
                                                                kPhasedThreads, smem));
    memo.fn = fn;
    memo.threads = kPhasedThreads;
    memo.smem = smem;
  }
  if (memo.per_sm < 1) return fail(EBIC_ERR_CUDA, "phased kernel: no CTA fits an SM");
  const int64_t grid = std::min<int64_t>(h->sm_count, a.P);
  count_launches(1);
  kern<<<(unsigned)grid, kPhasedThreads, smem, s>>>(h->LT, h->C, h->W, h->R, pop, a, g, h->LN,
                                                    h->d_err);
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

template <bool CHECK, class Pop>
static ebic_status eval_any(ebic_ctx* h, const Pop& pop, EvalArgs a, cudaStream_t s) {
  if (a.P <= 0) return EBIC_OK;
  const bool dec = a.want_dec != 0 || a.mode == EBIC_SUPPORT_INC_PLUS_DEC;
  if (dec && !a.dec) return fail(EBIC_ERR_ARG, "internal: dec output required");
  const int32_t path = resolve_path(h);
  if (path == EBIC_PATH_BITMASK && !h->LT) EBIC_TRY(build_pair_table(h, s));
  if (path == EBIC_PATH_BITMASK && h->tuning.kernel == 4 && !dec && !a.dec) {
    PhasedGeom g;
    if (phased_geometry(h, h->tuning, pop, &g)) return launch_phased<CHECK, Pop>(h, pop, a, g, s);
  }
  if (path == EBIC_PATH_BITMASK && h->tuning.kernel >= 3 && !dec && !a.dec) {
    StagedGeom g;
    if (staged_geometry(h, h->tuning, a.P, &g))
      return g.nvt == 3   ? launch_staged<CHECK, Pop, 3>(h, pop, a, g, s)
             : g.nvt == 2 ? launch_staged<CHECK, Pop, 2>(h, pop, a, g, s)
                          : launch_staged<CHECK, Pop, 1>(h, pop, a, g, s);
  }
  int32_t vpi = 0, ipc = 1;
  bool lane_kernel = false;
  int32_t VP = 1;
  int32_t nv = 1, kb = 4;
  const ebic_eval_tuning_t& tu = h->tuning;
  if (path == EBIC_PATH_BITMASK) {
    const int32_t V = h->W >> 2;
    lane_kernel = tu.kernel == 1 ? V <= 32 : (tu.kernel == 0 && V <= 16);
    if (lane_kernel) {
      while (VP < V) VP <<= 1;
    } else {
      nv = dec ? 1 : (tu.vecs_per_lane > 0 ? tu.vecs_per_lane : 1);
      kb = dec ? 4 : (tu.batch_steps > 0 ? tu.batch_steps : 8);
      choose_split(a.P, V, tu.vecs_per_part_bitmask, &vpi, &ipc, 32 * nv);
    }
  } else {
    choose_split(a.P, h->R_pad >> 2, tu.vecs_per_part_gather, &vpi, &ipc);
  }
  if (ipc > 1) EBIC_TRY(h->tickets.reserve_zeroed((size_t)a.P * 2 * sizeof(unsigned long long), s));
  uint32_t* tk = h->tickets.as<uint32_t>();
  count_launches(1);
  if (path == EBIC_PATH_BITMASK && lane_kernel) {
    const int64_t threads = (int64_t)a.P * VP;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (dec)
      k_support_bitmask_lane<true, CHECK, Pop><<<blocks, 256, 0, s>>>(h->LT, h->C, h->W, h->R,
                                                                      pop, a, VP, h->LN, h->d_err);
    else
      k_support_bitmask_lane<false, CHECK, Pop><<<blocks, 256, 0, s>>>(h->LT, h->C, h->W, h->R,
                                                                       pop, a, VP, h->LN, h->d_err);
  } else {
    const unsigned blocks = (unsigned)(((int64_t)a.P * ipc + kWarpsPerCta - 1) / kWarpsPerCta);
    if (path == EBIC_PATH_BITMASK) {
#define EBIC_BM(D, N, K)                                                                   \
  k_support_bitmask_warp<D, CHECK, N, K, Pop><<<blocks, 32 * kWarpsPerCta, 0, s>>>(h->LT, h->C, h->W, h->R, \
                                                                      pop, a, vpi, ipc, tk,  \
                                                                      h->LN, h->d_err)
      if (dec) EBIC_BM(true, 1, 4);
      else if (nv == 1 && kb == 4) EBIC_BM(false, 1, 4);
      else if (nv == 1) EBIC_BM(false, 1, 8);
      else if (nv == 2 && kb == 4) EBIC_BM(false, 2, 4);
      else if (nv == 2) EBIC_BM(false, 2, 8);
      else EBIC_BM(false, 4, 4);
#undef EBIC_BM
    } else {
      if (dec)
        k_support_gather<true, CHECK, Pop><<<blocks, 32 * kWarpsPerCta, 0, s>>>(
            h->A_c, h->C, h->R_pad, h->R, pop, a, vpi, ipc, tk, h->LN, h->d_err);
      else
        k_support_gather<false, CHECK, Pop><<<blocks, 32 * kWarpsPerCta, 0, s>>>(
            h->A_c, h->C, h->R_pad, h->R, pop, a, vpi, ipc, tk, h->LN, h->d_err);
    }
  }
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

// ---------------------------------------------------------------------------
// Read-bandwidth probe: every 16-byte vector of a device buffer is loaded once
// per pass (grid-stride, 4 vectors in flight per thread) and XOR-folded; the
// fold is stored only if it equals a value no buffer produces by chance, so
// the loads cannot be dropped.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512)
k_read_probe(const uint4* __restrict__ buf, size_t n4, uint32_t magic, uint32_t* __restrict__ sink) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                d = __ldcg(buf + i + 3 * stride);
    acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^
           d.z ^ d.w;
  }
  for (; i < n4; i += stride) {
    const uint4 a = __ldcg(buf + i);
    acc ^= a.x ^ a.y ^ a.z ^ a.w;
  }
  if (acc == magic) *sink = acc;
}

// Autotuner: times candidate launch shapes on the caller's population (each
// candidate once to warm up, then 3 launches each between two events, or 5
// after emptying the L2 with `cold`) and keeps the fastest in h->tuning.  The candidates are evaluations, so the outputs
// hold valid results afterwards.
template <bool CHECK, class Pop>
static ebic_status autotune_any(ebic_ctx* h, const Pop& pop, const EvalArgs& a, cudaStream_t s,
                                float* best_us, bool cold = false) {
  std::vector<ebic_eval_tuning_t> cands;
  const int32_t path = resolve_path(h);
  const bool dec = a.want_dec != 0 || a.mode == EBIC_SUPPORT_INC_PLUS_DEC;
  if (path == EBIC_PATH_BITMASK) {
    const int32_t V = h->W >> 2;
    if (V <= 32) cands.push_back({1, 0, 0, 0, 0, 0, 0, 0, 0});
    if (!dec && V > 32) {
      for (int32_t nvt : {1, 2})
        for (int32_t dense : {4, 6}) cands.push_back({3, 0, 0, 0, nvt, dense, 2, 0, 0});
      cands.push_back({3, 0, 0, 0, 0, 4, 3, 0, 0});
      for (int32_t dense : {5, 6}) cands.push_back({4, 0, 0, 0, 0, dense, 0, 0, 0});
    }
    const int32_t parts[] = {32, 64, 128, 256, 0};
    for (int32_t vp : parts) {
      if (vp > 0 && vp / 2 >= V) continue;
      cands.push_back({2, vp, 0, 8, 1, 0, 0, 0, 0});
      if (!dec) {
        cands.push_back({2, vp, 0, 4, 1, 0, 0, 0, 0});
        cands.push_back({2, vp, 0, 4, 2, 0, 0, 0, 0});
      }
    }
  } else {
    const int32_t V = h->R_pad >> 2;
    const int32_t parts[] = {32, 64, 128, 256, 512, 1024, 0};
    for (int32_t vp : parts) {
      if (vp > 0 && vp / 2 >= V) continue;
      cands.push_back({0, 0, vp, 0, 0, 0, 0, 0, 0});
    }
  }
  // With `cold`, every timed launch follows an overwrite of one buffer of
  // twice the L2 size and a read of another: the L2 then holds no line of
  // the workload and no dirty line.
  void* flush = nullptr;
  size_t flush_bytes = 0;
  if (cold) {
    int l2 = 0;
    EBIC_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device));
    flush_bytes = std::max<size_t>((size_t)2 * (size_t)l2, (size_t)64 << 20) / 16 * 16;
    EBIC_CUDA_TRY(cudaMalloc(&flush, 2 * flush_bytes));
  }
  auto clear_l2 = [&]() {
    cudaMemsetAsync(flush, 0x5a, flush_bytes, s);
    k_read_probe<<<(unsigned)h->sm_count * 4, 512, 0, s>>>(
        reinterpret_cast<const uint4*>(static_cast<char*>(flush) + flush_bytes), flush_bytes / 16,
        0x9e3779b9u, static_cast<uint32_t*>(flush));
  };
  const int reps = cold ? 5 : 3;      // timed launches per candidate
  cudaEvent_t ev[10];
  for (cudaEvent_t& e : ev) EBIC_CUDA_TRY(cudaEventCreate(&e));
  float best = 1e30f;
  ebic_eval_tuning_t chosen = cands.empty() ? ebic_eval_tuning_t{} : cands[0];
  ebic_status st = EBIC_OK;
  for (const ebic_eval_tuning_t& c : cands) {
    h->tuning = c;
    if ((st = eval_any<CHECK>(h, pop, a, s)) != EBIC_OK) break;
    for (int r = 0; r < reps && st == EBIC_OK; ++r) {
      if (cold) clear_l2();
      cudaEventRecord(ev[2 * r], s);
      st = eval_any<CHECK>(h, pop, a, s);
      cudaEventRecord(ev[2 * r + 1], s);
    }
    if (st != EBIC_OK) break;
    if (cudaEventSynchronize(ev[2 * reps - 1]) != cudaSuccess) {
      st = fail(EBIC_ERR_CUDA, "autotune: event wait failed");
      break;
    }
    float ms = 0.f;
    for (int r = 0; r < reps; ++r) {
      float x = 0.f;
      cudaEventElapsedTime(&x, ev[2 * r], ev[2 * r + 1]);
      ms += x;
    }
    if (ms < best) {
      best = ms;
      chosen = c;
    }
  }
  for (cudaEvent_t& e : ev) cudaEventDestroy(e);
  if (flush) {
    cudaStreamSynchronize(s);
    cudaFree(flush);
  }
  h->tuning = chosen;
  if (best_us) *best_us = best * 1000.f / (float)reps;
  return st;
}

ebic_status autotune_fixed(ebic_ctx* h, const uint16_t* d_seq, const int32_t* d_len,
                           int32_t stride, const EvalArgs& a, cudaStream_t s, float* best_us) {
  FixedPop pop{d_seq, d_len, stride};
  return autotune_any<false>(h, pop, a, s, best_us);
}

ebic_status eval_archive(ebic_ctx* h, const ArchivePop& pop, const EvalArgs& a, cudaStream_t s) {
  return eval_any<false>(h, pop, a, s);
}

ebic_status autotune_archive(ebic_ctx* h, const ArchivePop& pop, const EvalArgs& a,
                             cudaStream_t s, float* best_us) {
  return autotune_any<false>(h, pop, a, s, best_us);
}

ebic_status eval_cbf(ebic_ctx* h, const int32_t* d_off, const int32_t* d_cols, int32_t total,
                     const EvalArgs& a, cudaStream_t s) {
  CbfPop pop{d_off, d_cols, total};
  return eval_any<true>(h, pop, a, s);
}

ebic_status eval_fixed(ebic_ctx* h, const uint16_t* d_seq, const int32_t* d_len, int32_t stride,
                       const EvalArgs& a, cudaStream_t s) {
  FixedPop pop{d_seq, d_len, stride};
  return eval_any<false>(h, pop, a, s);
}

ebic_status build_pair_table(ebic_ctx* h, cudaStream_t s) {
  if (h->LT) return EBIC_OK;
  const size_t bytes = (size_t)h->C * (size_t)h->C * (size_t)h->W * sizeof(uint32_t);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(EBIC_ERR_OOM, "pair table of %zu bytes does not fit: %s", bytes,
                cudaGetErrorString(e));
  }
  h->LT = static_cast<uint32_t*>(p);
  h->LT_bytes = bytes;
  dim3 grid((unsigned)((h->R_pad / 128 + 7) / 8), (unsigned)((h->C + 7) / 8));
  k_pair_table<<<grid, 256, 0, s>>>(h->A_c, h->C, h->R_pad, h->W, h->LT);
  count_launches(1);
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

static ebic_status create_handle(int32_t rows, int32_t cols, ebic_ctx** out) {
  if (rows < 1 || rows > (1 << 26) || cols < 1 || cols > 65535)
    return fail(EBIC_ERR_ARG, "matrix shape %d x %d outside [1, 2^26] x [1, 65535]", rows, cols);
  ebic_ctx* h = new ebic_ctx();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(EBIC_ERR_CUDA, "no CUDA device");
  }
  h->R = rows;
  h->C = cols;
  h->R_pad = (rows + 127) / 128 * 128;
  h->W = h->R_pad / 32;
  *out = h;
  return EBIC_OK;
}

static void destroy(ebic_ctx* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  ea_release(h);
  if (h->screen_sur) sur_attach(h->screen_sur, -1);
  h->screen_sur = nullptr;
  if (h->A_c) cudaFree(h->A_c);
  if (h->LN) cudaFree(h->LN);
  if (h->LT) cudaFree(h->LT);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_claim) cudaFree(h->d_claim);
  h->tickets.release();
  h->st_off.release();
  h->st_cols.release();
  h->st_inc.release();
  h->st_dec.release();
  h->st_fit.release();
  h->h_stage.release();
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Allocates the per-matrix buffers and places the matrix (rowmajor_dev is a
// device pointer); the caller's stream orders the work.
static ebic_status place(ebic_ctx* h, const float* rowmajor_dev, cudaStream_t s) {
  EBIC_CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
  EBIC_CUDA_TRY(cudaMalloc(&h->A_c, (size_t)h->C * h->R_pad * sizeof(float)));
  EBIC_CUDA_TRY(cudaMalloc(&h->d_err, sizeof(int)));
  EBIC_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  EBIC_CUDA_TRY(cudaMalloc(&h->d_claim, 2 * sizeof(uint32_t)));
  EBIC_CUDA_TRY(cudaMemsetAsync(h->d_claim, 0, 2 * sizeof(uint32_t), s));
  EBIC_CUDA_TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
  // LN[m] = log(m) with the host C library, m = 0 .. 2R + 1.
  const size_t nln = 2 * (size_t)h->R + 2;
  EBIC_CUDA_TRY(cudaMalloc(&h->LN, nln * sizeof(double)));
  EBIC_TRY(h->h_stage.reserve(nln * sizeof(double)));
  double* ln = h->h_stage.as<double>();
  ln[0] = -INFINITY;
  for (size_t m = 1; m < nln; ++m) ln[m] = std::log((double)m);
  EBIC_CUDA_TRY(cudaMemcpyAsync(h->LN, ln, nln * sizeof(double), cudaMemcpyHostToDevice, s));
  dim3 grid((unsigned)(h->R_pad / 32), (unsigned)((h->C + 31) / 32));
  k_load_colmajor<<<grid, 256, 0, s>>>(rowmajor_dev, h->R, h->C, h->R_pad, h->A_c);
  count_launches(1);
  EBIC_CUDA_TRY(cudaGetLastError());
  // The pinned LN staging is reused by later calls: finish the copy first.
  EBIC_CUDA_TRY(cudaStreamSynchronize(s));
  return EBIC_OK;
}

// ---------------------------------------------------------------------------
// Evaluation without any allocation.  Some callers cannot let a library call
// cudaMalloc: a host framework that owns all device memory through its own
// pool, or a latency-critical loop that cannot afford the implicit device
// synchronisation an allocation may cause.  This variant of the split-series
// support launch keeps its per-series scratch (the partial counts and arrival
// tickets of series that several warps share) in the fixed array below
// instead of memory owned by the handle, and it never builds the pair table.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[2 * (size_t)EBIC_NOALLOC_MAX_SERIES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256] = {};   // device address of the array, per device

// Device address of g_noalloc_scratch on the current device.  Host code only
// holds a stand-in for the symbol, so the real address is fetched once per
// device, with that device current.
static ebic_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= 256) return fail(EBIC_ERR_ARG, "device ordinal %d", device);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(EBIC_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s",
                  cudaGetErrorString(e));
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return EBIC_OK;
}

}  // namespace ebic

using namespace ebic;

extern "C" ebic_status ebic_eval_population_dev_noalloc(ebic_handle h, const int32_t* d_offsets,
                                                        const int32_t* d_cols, int32_t P,
                                                        int32_t total_cols, int32_t sigma,
                                                        uint32_t* d_inc, double* d_fitness,
                                                        void* stream) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (P < 0 || P > EBIC_NOALLOC_MAX_SERIES)
    return fail(EBIC_ERR_ARG,
                "P = %d outside [0, %d]: the no-allocation evaluation has fixed scratch for at "
                "most EBIC_NOALLOC_MAX_SERIES series per call",
                P, EBIC_NOALLOC_MAX_SERIES);
  if (P == 0) return EBIC_OK;
  if (!d_offsets || !d_cols || !d_inc || !d_fitness) return fail(EBIC_ERR_ARG, "null pointer");
  if (total_cols < 0) return fail(EBIC_ERR_ARG, "negative total_cols");
  DeviceGuard g(h->device);
  void* scratch = nullptr;
  EBIC_TRY(noalloc_scratch(h->device, &scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the words this call uses start at zero (the kernel also leaves them zero)
  EBIC_CUDA_TRY(cudaMemsetAsync(scratch, 0, (size_t)P * 2 * sizeof(unsigned long long), s));
  EvalArgs a{};
  a.P = P;
  a.sigma = sigma;
  a.mode = EBIC_SUPPORT_INC;
  a.want_dec = 0;
  a.inc = d_inc;
  a.dec = nullptr;
  a.fit = d_fitness;
  a.lnf = nullptr;
  CbfPop pop{d_offsets, d_cols, total_cols};
  uint32_t* sc = static_cast<uint32_t*>(scratch);
  const bool bitmask = h->LT != nullptr && h->path != EBIC_PATH_GATHER;
  int32_t vpi = 0, ipc = 1;
  if (bitmask) {
    choose_split(P, h->W >> 2, 0, &vpi, &ipc, 32);
    const unsigned blocks = (unsigned)(((int64_t)P * ipc + kWarpsPerCta - 1) / kWarpsPerCta);
    k_support_bitmask_warp<false, true, 1, 8, CbfPop><<<blocks, 32 * kWarpsPerCta, 0, s>>>(
        h->LT, h->C, h->W, h->R, pop, a, vpi, ipc, sc, h->LN, h->d_err);
  } else {
    choose_split(P, h->R_pad >> 2, 0, &vpi, &ipc);
    const unsigned blocks = (unsigned)(((int64_t)P * ipc + kWarpsPerCta - 1) / kWarpsPerCta);
    k_support_gather<false, true, CbfPop><<<blocks, 32 * kWarpsPerCta, 0, s>>>(
        h->A_c, h->C, h->R_pad, h->R, pop, a, vpi, ipc, sc, h->LN, h->d_err);
  }
  count_launches(1);
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}


extern "C" ebic_status ebic_probe_read_bandwidth(const void* d_buf, uint64_t bytes, int32_t reps,
                                                 void* stream, float* out_best_us) {
  if (!d_buf || !out_best_us || reps < 1 || bytes < 16 || bytes % 16)
    return fail(EBIC_ERR_ARG, "probe: need a device buffer of a multiple of 16 bytes and reps >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  EBIC_CUDA_TRY(cudaGetDevice(&dev));
  EBIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint32_t* sink = nullptr;
  EBIC_CUDA_TRY(cudaMalloc(&sink, sizeof(uint32_t)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const size_t n4 = bytes / 16;
  const unsigned grid = (unsigned)sms * 4;
  float best = 1e30f;
  ebic_status st = EBIC_OK;
  for (int r = 0; r <= reps && st == EBIC_OK; ++r) {     // pass 0 warms the caches
    cudaEventRecord(e0, s);
    k_read_probe<<<grid, 512, 0, s>>>(static_cast<const uint4*>(d_buf), n4, 0x9e3779b9u, sink);
    cudaEventRecord(e1, s);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = fail(EBIC_ERR_CUDA, "probe launch failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (st == EBIC_OK) *out_best_us = best * 1000.f;
  return st;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* ebic_last_error(void) { return g_last_error; }
uint64_t ebic_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }
int32_t ebic_abi_version(void) { return EBIC_ABI_VERSION; }

ebic_status ebic_load_matrix(const float* host_rowmajor, int32_t rows, int32_t cols,
                             ebic_handle* out) {
  if (!host_rowmajor || !out) return fail(EBIC_ERR_ARG, "null pointer");
  ebic_ctx* h = nullptr;
  EBIC_TRY(create_handle(rows, cols, &h));
  DeviceGuard g(h->device);
  float* tmp = nullptr;
  size_t bytes = (size_t)rows * cols * sizeof(float);
  ebic_status st = EBIC_OK;
  cudaError_t e = cudaMalloc(&tmp, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy(h);
    return fail(EBIC_ERR_OOM, "matrix staging: %s", cudaGetErrorString(e));
  }
  st = [&]() -> ebic_status {
    EBIC_CUDA_TRY(cudaMemcpy(tmp, host_rowmajor, bytes, cudaMemcpyHostToDevice));
    return place(h, tmp, nullptr);
  }();
  cudaFree(tmp);
  if (st != EBIC_OK) {
    destroy(h);
    return st;
  }
  *out = h;
  return EBIC_OK;
}

ebic_status ebic_load_matrix_dev(const float* dev_rowmajor, int32_t rows, int32_t cols,
                                 void* stream, ebic_handle* out) {
  if (!dev_rowmajor || !out) return fail(EBIC_ERR_ARG, "null pointer");
  ebic_ctx* h = nullptr;
  EBIC_TRY(create_handle(rows, cols, &h));
  DeviceGuard g(h->device);
  ebic_status st = place(h, dev_rowmajor, static_cast<cudaStream_t>(stream));
  if (st != EBIC_OK) {
    destroy(h);
    return st;
  }
  *out = h;
  return EBIC_OK;
}

void ebic_free(ebic_handle h) { destroy(h); }

ebic_status ebic_matrix_shape(ebic_handle h, int32_t* rows, int32_t* cols) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (rows) *rows = h->R;
  if (cols) *cols = h->C;
  return EBIC_OK;
}

ebic_status ebic_build_pair_table(ebic_handle h, void* stream) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  DeviceGuard g(h->device);
  return build_pair_table(h, static_cast<cudaStream_t>(stream));
}

ebic_status ebic_pair_table_bytes(ebic_handle h, uint64_t* bytes, int32_t* built) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (bytes) *bytes = (uint64_t)h->C * (uint64_t)h->C * (uint64_t)h->W * 4u;
  if (built) *built = h->LT != nullptr;
  return EBIC_OK;
}

ebic_status ebic_read_pair_words(ebic_handle h, int32_t p, int32_t q, int32_t w0, int32_t n,
                                 uint32_t* host_out) {
  if (!h || !host_out) return fail(EBIC_ERR_ARG, "null pointer");
  if (!h->LT) return fail(EBIC_ERR_STATE, "pair table not built");
  if (p < 0 || p >= h->C || q < 0 || q >= h->C || w0 < 0 || n < 0 || w0 + n > h->W)
    return fail(EBIC_ERR_ARG, "pair words out of range");
  DeviceGuard g(h->device);
  EBIC_CUDA_TRY(cudaDeviceSynchronize());
  EBIC_CUDA_TRY(cudaMemcpy(host_out, h->LT + ((size_t)p * h->C + q) * h->W + w0,
                           (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return EBIC_OK;
}

ebic_status ebic_set_path(ebic_handle h, int32_t path) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (path < EBIC_PATH_AUTO || path > EBIC_PATH_BITMASK) return fail(EBIC_ERR_ARG, "bad path");
  h->path = path;
  if (path == EBIC_PATH_BITMASK && !h->LT) {
    DeviceGuard g(h->device);
    EBIC_TRY(build_pair_table(h, h->stream));
    EBIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  return EBIC_OK;
}

ebic_status ebic_set_eval_tuning(ebic_handle h, const ebic_eval_tuning_t* t) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  ebic_eval_tuning_t z{};
  if (!t) t = &z;
  if (t->kernel < 0 || t->kernel > 4) return fail(EBIC_ERR_ARG, "kernel must be 0 .. 4");
  if (t->dense_steps < 0 || t->dense_steps > kStagedMaxDense)
    return fail(EBIC_ERR_ARG, "dense_steps must be 0 .. %d", kStagedMaxDense);
  if (!(t->stages == 0 || (t->stages >= 2 && t->stages <= 4)))
    return fail(EBIC_ERR_ARG, "stages must be 0 or 2 .. 4");
  if (t->groups < 0 || t->groups > 15) return fail(EBIC_ERR_ARG, "groups must be 0 .. 15");
  if (t->dynamic_rounds < -1 || t->dynamic_rounds > 64)
    return fail(EBIC_ERR_ARG, "dynamic_rounds must be -1 .. 64");
  if (t->vecs_per_part_bitmask < 0 || t->vecs_per_part_gather < 0)
    return fail(EBIC_ERR_ARG, "negative part size");
  if (!(t->batch_steps == 0 || t->batch_steps == 4 || t->batch_steps == 8))
    return fail(EBIC_ERR_ARG, "batch_steps must be 0, 4 or 8");
  if (!(t->vecs_per_lane == 0 || t->vecs_per_lane == 1 || t->vecs_per_lane == 2 ||
        t->vecs_per_lane == 4 || (t->vecs_per_lane == 3 && t->kernel == 3)))
    return fail(EBIC_ERR_ARG, "vecs_per_lane must be 0, 1, 2 or 4 (3: kernel 3 only)");
  if (t->vecs_per_lane == 4 && t->batch_steps == 8)
    return fail(EBIC_ERR_ARG, "vecs_per_lane 4 allows batch_steps 4 only");
  h->tuning = *t;
  return EBIC_OK;
}

ebic_status ebic_eval_population(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                                 int32_t P, int32_t sigma, int32_t support_mode,
                                 uint32_t* out_inc, uint32_t* out_dec, double* out_fitness) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (P < 0 || P > (1 << 24)) return fail(EBIC_ERR_ARG, "P = %d outside [0, 2^24]", P);
  if (P == 0) return EBIC_OK;
  if (!offsets || !cols || !out_inc || !out_fitness) return fail(EBIC_ERR_ARG, "null pointer");
  if (support_mode != EBIC_SUPPORT_INC && support_mode != EBIC_SUPPORT_INC_PLUS_DEC)
    return fail(EBIC_ERR_ARG, "bad support mode %d", support_mode);
  if (offsets[0] != 0) return fail(EBIC_ERR_ARG, "offsets[0] must be 0");
  // the lengths, in one pass without early exit; the offending series only
  // when there is one
  bool bad_len = false;
  for (int32_t i = 0; i < P; ++i) {
    const int32_t L = offsets[i + 1] - offsets[i];
    bad_len |= (L < 1) | (L > EBIC_MAX_EVAL_LEN);
  }
  if (bad_len)
    for (int32_t i = 0; i < P; ++i) {
      const int32_t L = offsets[i + 1] - offsets[i];
      if (L < 1 || L > EBIC_MAX_EVAL_LEN)
        return fail(EBIC_ERR_ARG, "series %d has length %d outside [1, %d]", i, L,
                    EBIC_MAX_EVAL_LEN);
    }
  const int32_t total = offsets[P];
  DeviceGuard g(h->device);
  cudaStream_t s = h->stream;
  // device staging: the CBF, then [fitness | inc | dec] in one buffer so that
  // one copy brings every result back into the pinned host stage
  const size_t nres = (size_t)P * (sizeof(double) + 2 * sizeof(uint32_t));
  EBIC_TRY(h->st_off.reserve((size_t)(P + 1) * sizeof(int32_t)));
  EBIC_TRY(h->st_cols.reserve((size_t)std::max(total, 1) * sizeof(int32_t)));
  EBIC_TRY(h->st_fit.reserve(nres));
  EBIC_TRY(h->h_stage.reserve(nres));
  EBIC_CUDA_TRY(cudaMemcpyAsync(h->st_off.ptr, offsets, (size_t)(P + 1) * sizeof(int32_t),
                                cudaMemcpyHostToDevice, s));
  EBIC_CUDA_TRY(cudaMemcpyAsync(h->st_cols.ptr, cols, (size_t)total * sizeof(int32_t),
                                cudaMemcpyHostToDevice, s));
  double* d_fit = h->st_fit.as<double>();
  uint32_t* d_inc = reinterpret_cast<uint32_t*>(d_fit + P);
  uint32_t* d_dec = d_inc + P;
  const bool with_dec = out_dec != nullptr;
  EvalArgs a{};
  a.P = P;
  a.sigma = sigma;
  a.mode = support_mode;
  a.want_dec = with_dec;
  a.inc = d_inc;
  a.dec = (with_dec || support_mode == EBIC_SUPPORT_INC_PLUS_DEC) ? d_dec : nullptr;
  a.fit = d_fit;
  a.lnf = nullptr;
  EBIC_TRY(eval_cbf(h, h->st_off.as<int32_t>(), h->st_cols.as<int32_t>(), total, a, s));
  const size_t back = (size_t)P * (sizeof(double) + (with_dec ? 2 : 1) * sizeof(uint32_t));
  EBIC_CUDA_TRY(cudaMemcpyAsync(h->h_stage.ptr, d_fit, back, cudaMemcpyDeviceToHost, s));
  // the column indices are checked while the device works (the kernels
  // bound-check every index themselves, so a bad one only raises the device
  // flag, which is cleared again below); nothing reaches the caller's
  // buffers unless every index is valid
  int32_t lo = 0, hi = 0;
  for (int32_t k = 0; k < total; ++k) {
    lo = std::min(lo, cols[k]);
    hi = std::max(hi, cols[k]);
  }
  EBIC_CUDA_TRY(cudaStreamSynchronize(s));
  if (lo < 0 || hi >= h->C) {
    EBIC_CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
    for (int32_t k = 0; k < total; ++k)
      if (cols[k] < 0 || cols[k] >= h->C)
        return fail(EBIC_ERR_ARG, "column index %d at position %d outside [0, %d)", cols[k], k,
                    h->C);
  }
  const unsigned char* hs = h->h_stage.as<unsigned char>();
  std::memcpy(out_fitness, hs, (size_t)P * sizeof(double));
  std::memcpy(out_inc, hs + (size_t)P * sizeof(double), (size_t)P * sizeof(uint32_t));
  if (with_dec)
    std::memcpy(out_dec, hs + (size_t)P * (sizeof(double) + sizeof(uint32_t)),
                (size_t)P * sizeof(uint32_t));
  return EBIC_OK;
}

ebic_status ebic_eval_population_dev(ebic_handle h, const int32_t* d_offsets,
                                     const int32_t* d_cols, int32_t P, int32_t total_cols,
                                     int32_t sigma, int32_t support_mode, uint32_t* d_inc,
                                     uint32_t* d_dec, double* d_fitness, void* stream) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (P < 0 || P > (1 << 24)) return fail(EBIC_ERR_ARG, "P = %d outside [0, 2^24]", P);
  if (P == 0) return EBIC_OK;
  if (!d_offsets || !d_cols || !d_inc || !d_fitness) return fail(EBIC_ERR_ARG, "null pointer");
  if (total_cols < 0) return fail(EBIC_ERR_ARG, "negative total_cols");
  if (support_mode != EBIC_SUPPORT_INC && support_mode != EBIC_SUPPORT_INC_PLUS_DEC)
    return fail(EBIC_ERR_ARG, "bad support mode %d", support_mode);
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EvalArgs a{};
  a.P = P;
  a.sigma = sigma;
  a.mode = support_mode;
  a.want_dec = d_dec != nullptr;
  a.inc = d_inc;
  a.fit = d_fitness;
  a.lnf = nullptr;
  if (d_dec) {
    a.dec = d_dec;
  } else if (support_mode == EBIC_SUPPORT_INC_PLUS_DEC) {
    EBIC_TRY(h->st_dec.reserve((size_t)P * sizeof(uint32_t)));
    a.dec = h->st_dec.as<uint32_t>();
  }
  return eval_cbf(h, d_offsets, d_cols, total_cols, a, s);
}

ebic_status ebic_autotune_eval(ebic_handle h, const int32_t* d_offsets, const int32_t* d_cols,
                               int32_t P, int32_t total_cols, int32_t sigma, int32_t support_mode,
                               uint32_t* d_inc, uint32_t* d_dec, double* d_fitness, void* stream,
                               int32_t flags, ebic_eval_tuning_t* chosen, float* best_us) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (P <= 0 || P > (1 << 24)) return fail(EBIC_ERR_ARG, "P = %d outside [1, 2^24]", P);
  if (!d_offsets || !d_cols || !d_inc || !d_fitness) return fail(EBIC_ERR_ARG, "null pointer");
  if (support_mode != EBIC_SUPPORT_INC && support_mode != EBIC_SUPPORT_INC_PLUS_DEC)
    return fail(EBIC_ERR_ARG, "bad support mode %d", support_mode);
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EvalArgs a{};
  a.P = P;
  a.sigma = sigma;
  a.mode = support_mode;
  a.want_dec = d_dec != nullptr;
  a.inc = d_inc;
  a.fit = d_fitness;
  if (d_dec) {
    a.dec = d_dec;
  } else if (support_mode == EBIC_SUPPORT_INC_PLUS_DEC) {
    EBIC_TRY(h->st_dec.reserve((size_t)P * sizeof(uint32_t)));
    a.dec = h->st_dec.as<uint32_t>();
  }
  if (resolve_path(h) == EBIC_PATH_BITMASK && !h->LT) EBIC_TRY(build_pair_table(h, s));
  CbfPop pop{d_offsets, d_cols, total_cols};
  if (flags & ~EBIC_TUNE_COLD_L2) return fail(EBIC_ERR_ARG, "unknown autotune flags %d", flags);
  EBIC_TRY(autotune_any<true>(h, pop, a, s, best_us, (flags & EBIC_TUNE_COLD_L2) != 0));
  if (chosen) *chosen = h->tuning;
  return EBIC_OK;
}

ebic_status ebic_get_eval_tuning(ebic_handle h, ebic_eval_tuning_t* out) {
  if (!h || !out) return fail(EBIC_ERR_ARG, "null pointer");
  *out = h->tuning;
  return EBIC_OK;
}

ebic_status ebic_check_device_error(ebic_handle h) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  DeviceGuard g(h->device);
  EBIC_CUDA_TRY(cudaDeviceSynchronize());
  int v = 0;
  EBIC_CUDA_TRY(cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    EBIC_CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
    // a staged launch that gave up may have left its item counter unreset
    EBIC_CUDA_TRY(cudaMemset(h->d_claim, 0, 2 * sizeof(uint32_t)));
    return fail(EBIC_ERR_DEVICE, "a kernel flagged invalid input (code %d)", v);
  }
  return EBIC_OK;
}

}  // extern "C"
