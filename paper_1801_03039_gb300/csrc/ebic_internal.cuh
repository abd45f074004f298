// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "ebic.h"

namespace ebic {

// Thread-local message of the last failing call.
void set_error(const char* fmt, ...);
ebic_status fail(ebic_status st, const char* fmt, ...);

#define EBIC_CUDA_TRY(expr)                                                           \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                             \
      return ::ebic::fail(e_ == cudaErrorMemoryAllocation ? EBIC_ERR_OOM : EBIC_ERR_CUDA, \
                          "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                          __FILE__, __LINE__);                                        \
    }                                                                                 \
  } while (0)

#define EBIC_TRY(expr)                  \
  do {                                  \
    ebic_status s_ = (expr);            \
    if (s_ != EBIC_OK) return s_;       \
  } while (0)

// A growable device buffer owned by a handle.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  ebic_status reserve(size_t want);
  ebic_status reserve_zeroed(size_t want, cudaStream_t s);  // new bytes are zero
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// A growable pinned host buffer.
struct HostBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  ebic_status reserve(size_t want);
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

struct EaState;     // generation-loop state (ebic_ea.cu)

}  // namespace ebic

// The last launch shape of the staged (or phased) kernel on a handle and its
// occupancy, so that repeated evaluations skip the occupancy query.
struct StagedMemo {
  const void* fn = nullptr;
  int threads = 0;
  size_t smem = 0;
  int per_sm = 0;
};

// The opaque handle.
struct ebic_ctx {
  int device = 0;
  int32_t R = 0;          // rows
  int32_t C = 0;          // columns
  int32_t R_pad = 0;      // rows padded to a multiple of 128 (NaN padding)
  int32_t W = 0;          // 32-row words per column pair = R_pad / 32 (multiple of 4)
  float* A_c = nullptr;   // column-major [C][R_pad]
  double* LN = nullptr;   // LN[m] = log(m), m = 0 .. 2R + 1 (LN[0] unused)
  uint32_t* LT = nullptr; // pair bitmask table [C][C][W] (nullptr until built)
  size_t LT_bytes = 0;
  int32_t path = EBIC_PATH_AUTO;
  ebic_eval_tuning_t tuning{};     // launch shape of evaluations (zeros = automatic)
  cudaStream_t stream = nullptr;  // internal stream for the host-buffer calls
  int* d_err = nullptr;           // device error flag (0 = none)
  uint32_t* d_claim = nullptr;    // item counter of the staged kernel and its
                                  // finished-scout count (zero between launches)
  int32_t sm_count = 0;           // streaming multiprocessors of the device
  StagedMemo staged_memo;         // kernel 3
  StagedMemo phased_memo;         // kernel 4
  ebic::DevBuf tickets;           // per-series partial counts and arrivals of split
                                  // series (2 x 64-bit words each, zero between launches)
  ebic::DevBuf st_off, st_cols, st_inc, st_dec, st_fit;   // staging for host calls
  ebic::HostBuf h_stage;          // pinned staging for host calls
  ebic::EaState* ea = nullptr;
  // offspring screening applied by the next ebic_run_init
  ebic_surrogate_ctx* screen_sur = nullptr;
  int32_t screen_v = 1;
  int32_t screen_mode = 0;
  int32_t ktime_slots = 0;        // in-graph timing of Step 3's builder (0: off)
};

namespace ebic {

// Population views used by the support kernels.
// A view supplies range(i) (start and length of series i; false if invalid),
// col(begin, t), out(i) (index at which series i's results are written) and
// active() (false skips the whole launch).
struct CbfPop {          // caller CBF: offsets[P + 1], cols[total]
  const int32_t* offsets;
  const int32_t* cols;
  int32_t total;
  __device__ __forceinline__ bool active() const { return true; }
  __device__ __forceinline__ int64_t out(int32_t i) const { return i; }
  __device__ __forceinline__ bool range(int32_t i, int64_t* begin, int32_t* len) const {
    int32_t b = offsets[i], e = offsets[i + 1];
    *begin = b;
    *len = e - b;
    return b >= 0 && e <= total && e - b >= 1 && e - b <= EBIC_MAX_EVAL_LEN;
  }
  __device__ __forceinline__ int32_t col(int64_t begin, int32_t t) const { return cols[begin + t]; }
};

struct FixedPop {        // EA layout: seq[P][stride] (uint16), len[P]
  const uint16_t* seq;
  const int32_t* len;
  int32_t stride;
  __device__ __forceinline__ bool active() const { return true; }
  __device__ __forceinline__ int64_t out(int32_t i) const { return i; }
  __device__ __forceinline__ bool range(int32_t i, int64_t* begin, int32_t* L) const {
    *begin = (int64_t)i * stride;
    *L = len[i];
    return *L >= 1 && *L <= stride;
  }
  __device__ __forceinline__ int32_t col(int64_t begin, int32_t t) const { return seq[begin + t]; }
};

// The current generation of the EA archive: series i of generation g is
// archive entry g * P + i.  g and the stop flag are read on the device, so a
// captured launch follows the run from generation to generation.
struct ArchivePop {
  const uint16_t* seq;   // [entries][stride]
  const int32_t* len;    // [entries]
  int32_t stride;
  int32_t P;
  const int32_t* gen;    // current generation
  const int32_t* stop;   // nonzero: the run has stopped
  __device__ __forceinline__ bool active() const { return *(volatile const int32_t*)stop == 0; }
  __device__ __forceinline__ int64_t out(int32_t i) const { return (int64_t)(*gen) * P + i; }
  __device__ __forceinline__ bool range(int32_t i, int64_t* begin, int32_t* L) const {
    const int64_t e = out(i);
    *begin = e * stride;
    *L = len[e];
    return *L >= 1 && *L <= stride;
  }
  __device__ __forceinline__ int32_t col(int64_t begin, int32_t t) const { return seq[begin + t]; }
};

// Arguments of one evaluation launch.
struct EvalArgs {
  int32_t P;
  int32_t sigma;
  int32_t mode;           // ebic_support_mode
  int32_t want_dec;       // compute dec (needed when mode == INC_PLUS_DEC or dec requested)
  uint32_t* inc;
  uint32_t* dec;          // may be nullptr when only inc is returned
  double* fit;
  float* lnf;             // optional: log(fitness) as float (EA tournaments), -inf for 0
};

// Evaluate a population on the handle's matrix (Step 4 + Eq. (1)), queued on s.
ebic_status eval_cbf(ebic_ctx* h, const int32_t* d_off, const int32_t* d_cols, int32_t total,
                     const EvalArgs& a, cudaStream_t s);
ebic_status eval_fixed(ebic_ctx* h, const uint16_t* d_seq, const int32_t* d_len, int32_t stride,
                       const EvalArgs& a, cudaStream_t s);
ebic_status eval_archive(ebic_ctx* h, const ArchivePop& pop, const EvalArgs& a, cudaStream_t s);
ebic_status autotune_archive(ebic_ctx* h, const ArchivePop& pop, const EvalArgs& a,
                             cudaStream_t s, float* best_us);
// Times candidate launch shapes on a device-resident EA population and keeps
// the fastest in h->tuning (synchronises s).
ebic_status autotune_fixed(ebic_ctx* h, const uint16_t* d_seq, const int32_t* d_len,
                           int32_t stride, const EvalArgs& a, cudaStream_t s, float* best_us);
// Which path an evaluation of this handle would take now.
int32_t resolve_path(ebic_ctx* h);
ebic_status build_pair_table(ebic_ctx* h, cudaStream_t s);

void ea_release(ebic_ctx* h);
// The evaluated part of the handle's run archive (device pointers; entry e is
// seq[e * stride ..], len[e], fit[e]; n entries).  Synchronises the stream.
ebic_status ea_archive(ebic_ctx* h, const uint16_t** seq, const int32_t** len, const double** fit,
                       long long* n, int32_t* stride);

// Surrogate forward pass for screening (ebic_surrogate.cu): y[n] receives the
// predictions of n series (act is unused: the fused kernel keeps no
// activations).  Launches only (no allocation, no synchronisation): safe
// under stream capture.
size_t sur_act_bytes(long long rows);
ebic_status sur_forward_scores(ebic_surrogate_ctx* s, const uint16_t* seq, const int32_t* len,
                               int32_t stride, int32_t n, void* act, float* y, cudaStream_t st,
                               int* launches);
int32_t sur_columns(const ebic_surrogate_ctx* s);
void sur_attach(ebic_surrogate_ctx* s, int delta);
// Adds n to the process-wide count of kernels this library launched.
void count_launches(uint64_t n);

}  // namespace ebic
