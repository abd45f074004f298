// Many independent problems in one launch: each problem is a matrix (its own
// handle) and a population, as produced by many EBIC runs or restarts side by
// side (Step 4 of the "EBIC Algorithm" section, repeated over problems).
//
// A persistent kernel (one grid that fills the GPU) pulls work items --
// (problem, series, part of the series' rows) -- from a list ordered by
// decreasing estimated cost (longest-processing-time first), so that the
// long, heavy series start early and short ones fill the gaps.  Each item is
// evaluated by the same per-item code as the single-problem kernels, on the
// path (pair bitmask or gather) and split chosen for its problem by the
// autotuner.  The launch (counter reset + kernel) can be captured once as a
// CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "ebic_internal.cuh"
#include "ebic_support.cuh"

namespace ebic {

struct BatchProb {
  const float* A_c;
  const uint32_t* LT;
  const double* LN;
  int* err;
  int32_t R, C, R_pad, W;
  CbfPop pop;
  EvalArgs a;
  int32_t path;          // EBIC_PATH_GATHER or EBIC_PATH_BITMASK
  int32_t vpi, ipc;      // vectors per part, parts per series
  uint32_t* scratch;     // split accumulators of this problem (2 x 64-bit per series)
};

constexpr int kBatchThreads = 256;
constexpr int kBatchKB = 8;   // bitmask steps between exit tests in the batch launch

__global__ void __launch_bounds__(kBatchThreads)
k_support_batch(const BatchProb* __restrict__ probs, const int2* __restrict__ work,
                long long n_items, unsigned long long* __restrict__ counter) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(counter, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if ((long long)i >= n_items) break;                  // warp-uniform
    const int2 w = work[i];
    const BatchProb& pb = probs[w.x];
    const int32_t ipc = pb.ipc;
    const int32_t sid = w.y / ipc, part = w.y % ipc;
    if (pb.path == EBIC_PATH_BITMASK)
      bitmask_warp_item<false, true, 1, kBatchKB, CbfPop>(pb.LT, pb.C, pb.W, pb.R, pb.pop, pb.a,
                                                          pb.vpi, ipc, pb.scratch, pb.LN, pb.err,
                                                          sid, part, lane);
    else
      gather_item<false, true, CbfPop>(pb.A_c, pb.C, pb.R_pad, pb.R, pb.pop, pb.a, pb.vpi, ipc,
                                       pb.scratch, pb.LN, pb.err, sid, part, lane);
  }
}

}  // namespace ebic

struct ebic_batch_ctx {
  int device = 0;
  int32_t n = 0;
  int32_t flags = 0;
  std::vector<ebic::BatchProb> probs;
  std::vector<long long> items_per_prob;
  ebic::DevBuf d_probs, d_work, d_scratch, d_counter;
  long long n_items = 0;
  int grid = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaStream_t own = nullptr;   // blocking stream used when the caller passes none
};

namespace ebic {

// Median-free timing of one shape on one problem with the single-problem
// warp kernels (same per-item code as the batch launch).
static ebic_status time_shape(ebic_ctx* h, const ebic_batch_item_t& it, int32_t path,
                              int32_t vpp, cudaStream_t s, float* us) {
  // vpp 0 = whole series in one part, as in the batch launch
  if (vpp <= 0) vpp = ((path == EBIC_PATH_BITMASK ? h->W / 4 : h->R_pad / 4) + 31) / 32 * 32;
  const int32_t saved_path = h->path;
  const ebic_eval_tuning_t saved = h->tuning;
  h->path = path;
  h->tuning = ebic_eval_tuning_t{};
  h->tuning.kernel = 2;
  h->tuning.batch_steps = kBatchKB;
  h->tuning.vecs_per_lane = 1;
  if (path == EBIC_PATH_BITMASK) h->tuning.vecs_per_part_bitmask = vpp;
  else h->tuning.vecs_per_part_gather = vpp;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ebic_status st = ebic_eval_population_dev(h, it.d_offsets, it.d_cols, it.P, it.total_cols,
                                            it.sigma, EBIC_SUPPORT_INC, it.d_inc, nullptr,
                                            it.d_fitness, s);
  cudaEventRecord(e0, s);
  for (int r = 0; r < 3 && st == EBIC_OK; ++r)
    st = ebic_eval_population_dev(h, it.d_offsets, it.d_cols, it.P, it.total_cols, it.sigma,
                                  EBIC_SUPPORT_INC, it.d_inc, nullptr, it.d_fitness, s);
  cudaEventRecord(e1, s);
  float ms = 1e30f;
  if (st == EBIC_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->path = saved_path;
  h->tuning = saved;
  *us = ms * 1000.f / 3.f;
  return st;
}

// Vectors per part (rounded to warps) and parts per series, as the
// single-problem launch computes them for a forced part size.
static void split_for(int32_t V, int32_t vpp, int32_t* vpi, int32_t* ipc) {
  if (vpp <= 0 || vpp >= V) {
    *vpi = ((V + 31) / 32) * 32;
    *ipc = 1;
    return;
  }
  *vpi = std::max(vpp / 32, 1) * 32;
  *ipc = (V + *vpi - 1) / *vpi;
}

}  // namespace ebic

using namespace ebic;

extern "C" {

ebic_status ebic_batch_create(const ebic_handle* handles, const ebic_batch_item_t* items,
                              int32_t n, int32_t flags, void* stream, ebic_batch* out) {
  if (!handles || !items || !out || n < 1) return fail(EBIC_ERR_ARG, "bad batch arguments");
  const int dev = handles[0] ? handles[0]->device : -1;
  for (int32_t i = 0; i < n; ++i) {
    if (!handles[i]) return fail(EBIC_ERR_ARG, "null handle %d", i);
    if (handles[i]->device != dev) return fail(EBIC_ERR_ARG, "handles on different devices");
    const ebic_batch_item_t& it = items[i];
    if (it.P < 1 || it.P > (1 << 24) || !it.d_offsets || !it.d_cols || !it.d_inc ||
        !it.d_fitness || it.total_cols < 0)
      return fail(EBIC_ERR_ARG, "bad batch item %d", i);
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ebic_batch_ctx* b = new ebic_batch_ctx();
  b->device = dev;
  b->n = n;
  b->flags = flags;
  if (cudaStreamCreate(&b->own) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return fail(EBIC_ERR_CUDA, "cannot create the batch stream");
  }
  ebic_status st = EBIC_OK;
  auto fin = [&](ebic_status r) {
    if (r != EBIC_OK) ebic_batch_free(b);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return r;
  };

  // Per problem: path and split.  With EBIC_BATCH_BUILD_TABLES the pair
  // table is built where it fits (half the free memory, cumulative); with
  // EBIC_BATCH_AUTOTUNE both paths and a few part sizes are timed.
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  size_t budget = free_b / 2;
  b->probs.resize((size_t)n);
  size_t scratch_words = 0;
  std::vector<size_t> scratch_off((size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    ebic_ctx* h = handles[i];
    const ebic_batch_item_t& it = items[i];
    if ((flags & EBIC_BATCH_BUILD_TABLES) && !h->LT) {
      const size_t need = (size_t)h->C * h->C * h->W * sizeof(uint32_t);
      if (need <= budget) {
        if ((st = build_pair_table(h, s)) != EBIC_OK) return fin(st);
        budget -= need;
      }
    }
    int32_t best_path = h->LT ? EBIC_PATH_BITMASK : EBIC_PATH_GATHER, best_vpp = 0;
    if (flags & EBIC_BATCH_AUTOTUNE) {
      float best = 1e30f;
      const int32_t paths[2] = {EBIC_PATH_GATHER, EBIC_PATH_BITMASK};
      for (int32_t path : paths) {
        if (path == EBIC_PATH_BITMASK && !h->LT) continue;
        const int32_t V = path == EBIC_PATH_BITMASK ? h->W / 4 : h->R_pad / 4;
        const int32_t vpps[] = {32, 64, 128, 256, 512, 0};
        for (int32_t vpp : vpps) {
          if (vpp > 0 && vpp / 2 >= V) continue;
          float us = 0.f;
          if ((st = time_shape(h, it, path, vpp, s, &us)) != EBIC_OK) return fin(st);
          if (us < best) {
            best = us;
            best_path = path;
            best_vpp = vpp;
          }
        }
      }
    }
    BatchProb& pb = b->probs[(size_t)i];
    pb.A_c = h->A_c;
    pb.LT = h->LT;
    pb.LN = h->LN;
    pb.err = h->d_err;
    pb.R = h->R;
    pb.C = h->C;
    pb.R_pad = h->R_pad;
    pb.W = h->W;
    pb.pop = CbfPop{it.d_offsets, it.d_cols, it.total_cols};
    pb.a = EvalArgs{};
    pb.a.P = it.P;
    pb.a.sigma = it.sigma;
    pb.a.mode = EBIC_SUPPORT_INC;
    pb.a.want_dec = 0;
    pb.a.inc = it.d_inc;
    pb.a.dec = nullptr;
    pb.a.fit = it.d_fitness;
    pb.a.lnf = nullptr;
    pb.path = best_path;
    split_for(best_path == EBIC_PATH_BITMASK ? h->W / 4 : h->R_pad / 4, best_vpp, &pb.vpi,
              &pb.ipc);
    if ((long long)it.P * pb.ipc >= (1ll << 31))
      return fin(fail(EBIC_ERR_ARG, "problem %d: too many work items", i));
    scratch_off[(size_t)i] = scratch_words;
    scratch_words += (pb.ipc > 1 ? (size_t)it.P * 4 : 0);   // 2 x 64-bit words per series
  }
  // scratch for split series
  if ((st = b->d_scratch.reserve_zeroed(std::max<size_t>(scratch_words, 4) * sizeof(uint32_t), s)) !=
      EBIC_OK)
    return fin(st);
  for (int32_t i = 0; i < n; ++i)
    b->probs[(size_t)i].scratch = b->d_scratch.as<uint32_t>() + scratch_off[(size_t)i];

  // work list, longest estimated cost first: cost = (L - 1) x vectors of the part
  struct W {
    float cost;
    int2 w;
  };
  std::vector<W> work;
  for (int32_t i = 0; i < n; ++i) {
    const ebic_batch_item_t& it = items[i];
    const BatchProb& pb = b->probs[(size_t)i];
    std::vector<int32_t> off((size_t)it.P + 1);
    if (cudaMemcpy(off.data(), it.d_offsets, off.size() * sizeof(int32_t),
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return fin(fail(EBIC_ERR_CUDA, "reading offsets of problem %d", i));
    }
    const int32_t V = pb.path == EBIC_PATH_BITMASK ? pb.W / 4 : pb.R_pad / 4;
    const float unit = pb.path == EBIC_PATH_BITMASK ? 1.f : 32.f;   // bytes per row-step / 16
    for (int32_t sid = 0; sid < it.P; ++sid) {
      const int32_t L = std::max(off[(size_t)sid + 1] - off[(size_t)sid], 1);
      for (int32_t q = 0; q < pb.ipc; ++q) {
        const int32_t vecs = std::min(pb.vpi, V - q * pb.vpi);
        work.push_back({unit * (float)(L - 1 > 0 ? L - 1 : 1) * (float)vecs,
                        make_int2(i, sid * pb.ipc + q)});
      }
    }
  }
  std::stable_sort(work.begin(), work.end(), [](const W& x, const W& y) { return x.cost > y.cost; });
  std::vector<int2> wl(work.size());
  for (size_t i = 0; i < work.size(); ++i) wl[i] = work[i].w;
  b->n_items = (long long)wl.size();
  if ((st = b->d_work.reserve(std::max<size_t>(wl.size(), 1) * sizeof(int2))) != EBIC_OK) return fin(st);
  if ((st = b->d_probs.reserve(b->probs.size() * sizeof(BatchProb))) != EBIC_OK) return fin(st);
  if ((st = b->d_counter.reserve(sizeof(unsigned long long))) != EBIC_OK) return fin(st);
  if (cudaMemcpyAsync(b->d_work.ptr, wl.data(), wl.size() * sizeof(int2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_probs.ptr, b->probs.data(), b->probs.size() * sizeof(BatchProb),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return fin(fail(EBIC_ERR_CUDA, "uploading the batch work list"));
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_support_batch, kBatchThreads, 0);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = std::max(1, per_sm) * std::max(1, sms);
  *out = b;
  return fin(EBIC_OK);
}

ebic_status ebic_batch_eval(ebic_batch b, void* stream) {
  if (!b) return fail(EBIC_ERR_ARG, "null batch");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  // The legacy default stream cannot be captured: use the batch's own
  // blocking stream instead (blocking streams stay ordered with it).
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->own;
  auto launch = [&]() -> ebic_status {
    EBIC_CUDA_TRY(cudaMemsetAsync(b->d_counter.ptr, 0, sizeof(unsigned long long), s));
    k_support_batch<<<b->grid, kBatchThreads, 0, s>>>(
        b->d_probs.as<BatchProb>(), b->d_work.as<int2>(), b->n_items,
        b->d_counter.as<unsigned long long>());
    EBIC_CUDA_TRY(cudaGetLastError());
    return EBIC_OK;
  };
  ebic_status st = EBIC_OK;
  if (b->flags & EBIC_BATCH_GRAPH) {
    if (!b->exec) {
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        st = fail(EBIC_ERR_CUDA, "cannot capture on this stream");
      } else {
        st = launch();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st == EBIC_OK && e == cudaSuccess && g) {
          b->graph = g;
          if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            cudaGetLastError();
            st = fail(EBIC_ERR_CUDA, "graph instantiation failed");
          }
        } else if (st == EBIC_OK) {
          cudaGetLastError();
          st = fail(EBIC_ERR_CUDA, "graph capture failed");
        }
      }
    }
    if (st == EBIC_OK && cudaGraphLaunch(b->exec, s) != cudaSuccess) {
      cudaGetLastError();
      st = fail(EBIC_ERR_CUDA, "graph launch failed");
    }
  } else {
    st = launch();
  }
  if (st == EBIC_OK) count_launches(1);
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  return st;
}

ebic_status ebic_batch_describe(ebic_batch b, int32_t problem, int32_t* path,
                                int32_t* vecs_per_part, int32_t* parts, int64_t* work_items,
                                int32_t* grid) {
  if (!b || problem < 0 || problem >= b->n) return fail(EBIC_ERR_ARG, "bad batch / problem");
  const BatchProb& pb = b->probs[(size_t)problem];
  if (path) *path = pb.path;
  if (vecs_per_part) *vecs_per_part = pb.vpi;
  if (parts) *parts = pb.ipc;
  if (work_items) *work_items = b->n_items;
  if (grid) *grid = b->grid;
  return EBIC_OK;
}

void ebic_batch_free(ebic_batch b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->d_probs.release();
  b->d_work.release();
  b->d_scratch.release();
  b->d_counter.release();
  if (b->own) cudaStreamDestroy(b->own);
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
