// The generation loop of EBIC on the device: Steps 1-5 of the "EBIC
// Algorithm" section (elitism, tournament selection with the crowding
// penalty, crossover and the four mutations of Fig. 1, the tabu list, Step 4
// evaluation and the top-rank list), kept entirely on one GPU.
//
// One generation = five launches, captured once into a CUDA graph (two
// branches: tabu insertion beside evaluation, Step 5 beside the next
// generation's k_spec) and replayed; every kernel reads the generation number
// and the stop flag from a device control block, so replays need no host
// involvement:
//   k_spec         parallel over attempts j < 2P + 1: draws the attempt's
//                  random numbers (Philox-4x32-10, keyed by seed, generation,
//                  attempt) and builds the child for EVERY possible outcome of
//                  its tournament(s); probes the tabu list for each.
//   k_build        one CTA: the sequential part of Step 3 -- elites, then the
//                  attempts in order, each tournament decided with the penalty
//                  counts as they stand, the precomputed child picked,
//                  duplicates (tabu or earlier in this generation) counted as
//                  hits; more than P hits stop the run.
//   k_tabu_insert  parallel: the accepted children enter the tabu hash table.
//   K3 evaluation  support + Eq. (1) of the new population (ebic_matrix.cu).
//   k_rank         one CTA: sorts by fitness and runs the Step 5 top-rank
//                  update (k_rank_warp: the visit by one warp from shared
//                  column bitsets, up to 256 columns).
// At most 2P + 1 attempts are ever needed: every attempt either adds one of at
// most P individuals or is one of at most P + 1 hits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ebic_async.cuh"
#include "ebic_internal.cuh"

namespace ebic {

// ---------------------------------------------------------------------------
// device state
// ---------------------------------------------------------------------------
struct Ctl {
  int32_t gen;          // generation being built (0 = Step 1)
  int32_t stop;         // nonzero once the run has stopped
  int32_t stop_reason;  // 1 tabu hits > P, 2 Step 1 could not fill the population, 3 internal
  int32_t n_top;        // records in the top-rank list
  int32_t n_elite;      // elites at the front of the current population
  int32_t last_hits;    // tabu hits in the last Step 3
  int32_t gens_done;    // Steps 2-5 passes completed
  int32_t spec_gen;     // generation whose attempt records come next (set by k_build)
  long long hits_total, attempts_total, evals_total, exact_total;
};

struct EaDev {
  int32_t P, C, S, Lmin, Lmax, k, T, mode, J, ncombo, WC, pad;
  double tau, elite_frac, pc;
  uint64_t seed;
  // archive: entry g * P + i is individual i of generation g
  uint16_t* seq;
  int32_t* len;
  double* fit;
  float* lnf;
  // tabu list: open addressing, key = 64-bit hash (0 = empty), ref = archive entry
  unsigned long long* tkey;
  int32_t* tref;
  unsigned long long tmask;
  // attempts of the current generation: one record of rec_bytes per attempt
  // (layout rec_layout), written by k_spec and streamed into k_build
  char* rec;
  int32_t rec_bytes;
  int32_t pad2;
  // top-rank list (archive entries and their fitness), capacity T + P
  int32_t* list_ref;
  double* list_f;
  // crowding penalty: base^(S/L) for S in [0, L P], from the host C library
  const double* pow_tab;
  const long long* pow_off;     // [Lmax + 1]
  const float* c_over_L;        // [Lmax + 1] log(base) / L as float
  Ctl* ctl;
  // offspring screening (V candidates per attempt and tournament outcome):
  // candidate v of (attempt j, outcome c) is row (j * ncombo + c) * V + v
  int32_t V, screen;
  uint16_t* var_seq;            // [rows][S]
  int32_t* var_len;             // [rows]
  float* var_score;             // [rows]
};

constexpr int kMaxLen = EBIC_MAX_EA_LEN;

// Words of the column bitsets kept in attempt records: 4 for up to 128
// columns, 8 for up to 256, none beyond (the builder's generic path).
__host__ __device__ inline int bit_words(int WC) { return WC <= 4 ? 4 : (WC <= 8 ? 8 : 0); }

// Layout of one attempt record (byte offsets; 8-byte fields first, size a
// multiple of 16 so that records can be bulk-copied).  ne = 2k entrant slots
// (first tournament, then second), nc = k * k candidate children (winner
// positions ta * k + tb), S = series stride, nw = bitset words (ebit / cbit:
// the column sets of the entrants / children as bitsets).
struct RecLayout {
  int chash, ef, ent, cross, elnf, eL, cL, ctabu, ebit, cbit, ecols, ccols, bytes, nw;
};

__host__ __device__ inline RecLayout rec_layout(int k, int S, bool init, int nw) {
  const int ne = init ? 0 : 2 * k, nc = init ? 1 : k * k;
  if (init) nw = 0;
  RecLayout l{};
  int o = 0;
  l.nw = nw;
  l.chash = o; o += nc * 8;
  l.ef = o;    o += ne * 8;
  o = (o + 15) & ~15;                 // bitsets: 16-byte aligned for vector loads
  l.ebit = o;  o += ne * nw * 4;
  l.cbit = o;  o += nc * nw * 4;
  l.ent = o;   o += 8 * 4;
  l.cross = o; o += 4;
  l.elnf = o;  o += ne * 4;
  l.eL = o;    o += ne * 4;
  l.cL = o;    o += nc * 4;
  l.ctabu = o; o += nc * 4;
  l.ecols = o; o += ne * S * 2;
  l.ccols = o; o += nc * S * 2;
  l.bytes = (o + 15) & ~15;
  return l;
}

// The column set of a series as nw bitset words.
// (gathered in registers, eight columns read per round; nw <= 8)
__device__ __forceinline__ void write_bits(uint32_t* out, int nw, const uint16_t* s, int L) {
  uint32_t acc[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) acc[w] = 0u;
  for (int c0 = 0; c0 < L; c0 += 8) {
    uint32_t col[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = c0 + i < L ? (uint32_t)s[c0 + i] : 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t bit = col[i] != 0xffffffffu ? 1u << (col[i] & 31) : 0u;
#pragma unroll
      for (int w = 0; w < 8; ++w) acc[w] |= (col[i] >> 5) == (uint32_t)w ? bit : 0u;
    }
  }
#pragma unroll
  for (int w = 0; w < 8; ++w)
    if (w < nw) out[w] = acc[w];
}

// Copies L columns, eight loads in flight per round.
__device__ __forceinline__ void copy_cols(uint16_t* dst, const uint16_t* src, int L) {
  for (int c0 = 0; c0 < L; c0 += 8) {
    uint16_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = c0 + i < L ? src[c0 + i] : (uint16_t)0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c0 + i < L) dst[c0 + i] = v[i];
  }
}

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11): counter (j, g, block, 0), key = seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_block(uint32_t j, uint32_t g, uint32_t blk, uint64_t seed,
                                             uint32_t out[4]) {
  uint32_t x0 = j, x1 = g, x2 = blk, x3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    const uint32_t y0 = hi1 ^ x1 ^ k0;
    const uint32_t y2 = hi0 ^ x3 ^ k1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

// Draw d of attempt j in generation g (word d % 4 of block d / 4).
struct Draws {
  uint64_t seed;
  uint32_t g, j;
  int blk;
  uint32_t w[4];
  __device__ Draws(uint64_t s, uint32_t gg, uint32_t jj) : seed(s), g(gg), j(jj), blk(-1) {}
  __device__ uint32_t operator()(int d) {
    if (d / 4 != blk) {
      blk = d / 4;
      philox_block(j, g, (uint32_t)blk, seed, w);
    }
    return w[d & 3];
  }
};

__device__ __forceinline__ uint32_t below(uint32_t r, uint32_t n) {
  return (uint32_t)(((unsigned long long)r * n) >> 32);
}

// k-th (0-based) column, in increasing order, that is not among s[0 .. L):
// start from k and step over every used column that is not above the answer.
__device__ int kth_absent(const uint16_t* s, int L, uint32_t k) {
  uint16_t t[kMaxLen];
  for (int i = 0; i < L; ++i) {
    uint16_t v = s[i];
    int m = i;
    while (m > 0 && t[m - 1] > v) {
      t[m] = t[m - 1];
      --m;
    }
    t[m] = v;
  }
  uint32_t c = k;
  for (int i = 0; i < L; ++i) {
    if (t[i] <= c) ++c;
    else break;
  }
  return (int)c;
}

__device__ __forceinline__ bool holds(const uint16_t* s, int L, int c) {
  for (int i = 0; i < L; ++i)
    if (s[i] == c) return true;
  return false;
}

// A set of columns below 256 as eight words in registers (every word index
// resolved by unrolled selects): membership in O(1) and the k-th absent
// column by a popcount walk -- the same answers as holds / kth_absent.
struct ColSet8 {
  uint32_t w[8];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = 0u;
  }
  __device__ __forceinline__ void add(uint32_t c) {
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] |= (c >> 5) == (uint32_t)i ? 1u << (c & 31) : 0u;
  }
  __device__ __forceinline__ bool has(uint32_t c) const {
    uint32_t r = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) r |= (c >> 5) == (uint32_t)i ? w[i] : 0u;
    return (r >> (c & 31)) & 1u;
  }
  __device__ __forceinline__ void fill(const uint16_t* s, int L) {
    clear();
    for (int i = 0; i < L; ++i) add(s[i]);
  }
  // k-th (0-based) column below C, in increasing order, not in the set
  __device__ __forceinline__ int kth_absent(uint32_t k, int C) const {
    int found = -1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int lo = 32 * i;
      uint32_t z = ~w[i];
      if (C - lo < 32) z &= C - lo > 0 ? (1u << (C - lo)) - 1u : 0u;
      const uint32_t cnt = (uint32_t)__popc(z);
      if (found < 0) {
        if (k < cnt) {
          for (uint32_t t = 0; t < k; ++t) z &= z - 1u;     // drop the k lowest
          found = lo + __ffs(z) - 1;
        } else {
          k -= cnt;
        }
      }
    }
    return found;
  }
};

// The four mutations (Fig. 1a-d): one, chosen uniformly among those that keep
// the series in [Lmin, Lmax] with distinct columns (insert, delete, swap,
// substitute in that order).
__device__ __forceinline__ void mutate(uint16_t* x, int& L, int C, int Lmin, int Lmax, uint32_t rt,
                                       uint32_t r1, uint32_t r2, const ColSet8* cs = nullptr) {
  int allowed[4];
  int n = 0;
  if (L < Lmax && L < C) allowed[n++] = 0;
  if (L > Lmin) allowed[n++] = 1;
  if (L >= 2) allowed[n++] = 2;
  if (L < C) allowed[n++] = 3;
  if (n == 0) return;
  const int kind = allowed[below(rt, (uint32_t)n)];
  if (kind == 0) {
    const int pos = (int)below(r1, (uint32_t)(L + 1));
    const uint32_t kk = below(r2, (uint32_t)(C - L));
    const int col = cs ? cs->kth_absent(kk, C) : kth_absent(x, L, kk);
    for (int i = L; i > pos; --i) x[i] = x[i - 1];
    x[pos] = (uint16_t)col;
    ++L;
  } else if (kind == 1) {
    const int pos = (int)below(r1, (uint32_t)L);
    for (int i = pos; i + 1 < L; ++i) x[i] = x[i + 1];
    --L;
  } else if (kind == 2) {
    const int i = (int)below(r1, (uint32_t)L);
    int j = (int)below(r2, (uint32_t)(L - 1));
    if (j >= i) ++j;
    const uint16_t t = x[i];
    x[i] = x[j];
    x[j] = t;
  } else {
    const int pos = (int)below(r1, (uint32_t)L);
    const uint32_t kk = below(r2, (uint32_t)(C - L));
    x[pos] = (uint16_t)(cs ? cs->kth_absent(kk, C) : kth_absent(x, L, kk));
  }
}

// 64-bit hash of an ordered series (never 0: 0 marks an empty slot).
__device__ __forceinline__ unsigned long long seq_hash(const uint16_t* s, int L) {
  unsigned long long h = 0xcbf29ce484222325ull ^ (unsigned long long)L;
  h *= 0x100000001b3ull;
  for (int i = 0; i < L; ++i) {
    h ^= s[i];
    h *= 0x100000001b3ull;
  }
  h ^= h >> 30;
  h *= 0xbf58476d1ce4e5b9ull;
  h ^= h >> 27;
  h *= 0x94d049bb133111ebull;
  h ^= h >> 31;
  return h | 1ull;
}

__device__ __forceinline__ bool same_series(const uint16_t* a, int La, const uint16_t* b, int Lb) {
  if (La != Lb) return false;
  bool eq = true;
  for (int c0 = 0; c0 < La && eq; c0 += 8) {    // eight columns of each side per round
    uint32_t x[8], y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[i] = c0 + i < La ? a[c0 + i] : 0u;
      y[i] = c0 + i < La ? b[c0 + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) eq = eq && x[i] == y[i];
  }
  return eq;
}

__device__ bool tabu_contains(const EaDev& d, unsigned long long key, const uint16_t* s, int L) {
  unsigned long long i = key & d.tmask;
  for (unsigned long long n = 0; n <= d.tmask; ++n) {
    const unsigned long long k = d.tkey[i];
    if (k == 0ull) return false;
    if (k == key) {
      const int32_t r = d.tref[i];
      if (r >= 0 && same_series(d.seq + (size_t)r * d.S, d.len[r], s, L)) return true;
    }
    i = (i + 1) & d.tmask;
  }
  return false;
}

// ---------------------------------------------------------------------------
// k_spec: every child an attempt can produce.  Thread = (attempt, combo);
// combo = ta * k + tb names the winning positions of the two tournaments.
// ---------------------------------------------------------------------------
// SCREEN: thread = (attempt, combo, candidate v); candidate v repeats the
// crossover cuts and the mutation with draws 2k + 1 + 5v .. 2k + 5 + 5v (v = 0
// is the plain child) and goes to the candidate buffers; k_pick completes the
// record once the candidates are scored.
template <bool INIT, bool SCREEN>
__global__ void __launch_bounds__(128) k_spec(EaDev d) {
  if (*(volatile int32_t*)&d.ctl->stop) return;
  // generation g's records are built while Step 5 of generation g - 1 may
  // still be running (it advances ctl->gen), so g comes from spec_gen
  const int g = INIT ? 0 : d.ctl->spec_gen;
  const int nc = INIT ? 1 : d.ncombo;
  const int V = SCREEN ? d.V : 1;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)d.J * nc * V) return;
  const int v = SCREEN ? (int)(tid % V) : 0;
  const long long jc = SCREEN ? tid / V : tid;
  const int j = (int)(jc / nc), c = (int)(jc % nc);
  const RecLayout l = rec_layout(d.k, d.S, INIT, bit_words(d.WC));
  char* rec = d.rec + (size_t)j * d.rec_bytes;
  Draws r(d.seed, (uint32_t)g, (uint32_t)j);
  uint16_t x[kMaxLen];
  int L = 0;
  if (INIT) {
    // Step 1: length uniform in [Lmin, Lmax], then distinct uniform columns.
    L = d.Lmin + (int)below(r(0), (uint32_t)(d.Lmax - d.Lmin + 1));
    if (d.C <= 256) {
      ColSet8 cs;
      cs.clear();
      for (int i = 0; i < L; ++i) {
        x[i] = (uint16_t)cs.kth_absent(below(r(1 + i), (uint32_t)(d.C - i)), d.C);
        cs.add(x[i]);
      }
    } else {
      for (int i = 0; i < L; ++i) x[i] = (uint16_t)kth_absent(x, i, below(r(1 + i), (uint32_t)(d.C - i)));
    }
  } else {
    const int k = d.k;
    const uint32_t P = (uint32_t)d.P;
    const int ta = c / k, tb = c % k;
    const bool cross = (double)r(k) * 0x1p-32 < d.pc;
    const long long prev = (long long)(g - 1) * d.P;
    // entrant slots e = c, c + nc, ... of this attempt's record
    for (int e = c; e < 2 * k && v == 0; e += nc) {
      const int idx = (int)below(r(e < k ? e : k + 1 + (e - k)), P);
      const long long er = prev + idx;
      const int eL = d.len[er];
      reinterpret_cast<double*>(rec + l.ef)[e] = d.fit[er];
      reinterpret_cast<float*>(rec + l.elnf)[e] = d.lnf[er];
      reinterpret_cast<int32_t*>(rec + l.eL)[e] = eL;
      reinterpret_cast<int32_t*>(rec + l.ent)[e < k ? e : 4 + (e - k)] = idx;
      uint16_t* ec = reinterpret_cast<uint16_t*>(rec + l.ecols) + (size_t)e * d.S;
      uint16_t t[kMaxLen];
      copy_cols(t, d.seq + (size_t)er * d.S, eL);
      copy_cols(ec, t, eL);
      if (l.nw) write_bits(reinterpret_cast<uint32_t*>(rec + l.ebit) + (size_t)e * l.nw, l.nw, t, eL);
    }
    if (c == 0 && v == 0) reinterpret_cast<int32_t*>(rec + l.cross)[0] = cross ? 1 : 0;
    const int base = 2 * k + 1 + 5 * v;
    const int ia = (int)below(r(ta), P);
    const int La = d.len[prev + ia];
    copy_cols(x, d.seq + (size_t)(prev + ia) * d.S, La);
    const uint16_t* a = x;
    L = La;
    if (cross) {
      const int ib = (int)below(r(k + 1 + tb), P);
      const int Lb = d.len[prev + ib];
      uint16_t b[kMaxLen];
      copy_cols(b, d.seq + (size_t)(prev + ib) * d.S, Lb);
      const int cut_a = 1 + (int)below(r(base), (uint32_t)La);
      const int cut_b = (int)below(r(base + 1), (uint32_t)Lb);
      uint16_t y[kMaxLen];
      int Ly = 0;
      for (int i = 0; i < cut_a; ++i) y[Ly++] = a[i];
      if (d.C <= 256) {
        ColSet8 ys;
        ys.fill(y, Ly);
        for (int i = cut_b; i < Lb; ++i) {
          if (Ly >= d.Lmax) break;
          if (!ys.has(b[i])) {
            ys.add(b[i]);
            y[Ly++] = b[i];
          }
        }
      } else {
        for (int i = cut_b; i < Lb; ++i) {
          if (Ly >= d.Lmax) break;
          if (!holds(y, Ly, b[i])) y[Ly++] = b[i];
        }
      }
      if (Ly >= d.Lmin) {
        for (int i = 0; i < Ly; ++i) x[i] = y[i];
        L = Ly;
      }
    }
    if (d.C <= 256) {
      ColSet8 xs;
      xs.fill(x, L);
      mutate(x, L, d.C, d.Lmin, d.Lmax, r(base + 2), r(base + 3), r(base + 4), &xs);
    } else {
      mutate(x, L, d.C, d.Lmin, d.Lmax, r(base + 2), r(base + 3), r(base + 4));
    }
  }
  if (SCREEN) {
    const long long row = jc * V + v;
    uint16_t* out = d.var_seq + (size_t)row * d.S;
    for (int i = 0; i < L; ++i) out[i] = x[i];
    d.var_len[row] = L;
    return;
  }
  uint16_t* out = reinterpret_cast<uint16_t*>(rec + l.ccols) + (size_t)c * d.S;
  for (int i = 0; i < L; ++i) out[i] = x[i];
  reinterpret_cast<int32_t*>(rec + l.cL)[c] = L;
  if (l.nw) write_bits(reinterpret_cast<uint32_t*>(rec + l.cbit) + (size_t)c * l.nw, l.nw, x, L);
  const unsigned long long h = seq_hash(x, L);
  reinterpret_cast<unsigned long long*>(rec + l.chash)[c] = h;
  reinterpret_cast<int32_t*>(rec + l.ctabu)[c] = INIT ? 0 : (tabu_contains(d, h, x, L) ? 1 : 0);
}

// Pseudo scores (testing the screening logic without a model): candidate v of
// (attempt j, outcome c) scores word 0 of Philox(j, g, 65536 + c * V + v) >> 8.
__global__ void __launch_bounds__(256) k_pseudo_score(EaDev d) {
  if (*(volatile int32_t*)&d.ctl->stop) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.J * d.ncombo * d.V) return;
  const int v = (int)(t % d.V);
  const long long jc = t / d.V;
  const int j = (int)(jc / d.ncombo), c = (int)(jc % d.ncombo);
  uint32_t w[4];
  philox_block((uint32_t)j, (uint32_t)d.ctl->spec_gen, 65536u + (uint32_t)(c * d.V + v), d.seed, w);
  d.var_score[t] = (float)(w[0] >> 8);
}

// k_pick: the candidates of each (attempt, outcome) are visited by decreasing
// score (ties: lower v; NaN after every number) and the first one that is not
// in the tabu list becomes the record's child; when all are, the
// best-scoring one does (a tabu hit).  The tabu list is the one left by the
// previous generation: this generation's own duplicates are the builder's.
__global__ void __launch_bounds__(128) k_pick(EaDev d) {
  if (*(volatile int32_t*)&d.ctl->stop) return;
  const long long jc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (jc >= (long long)d.J * d.ncombo) return;
  const int j = (int)(jc / d.ncombo), c = (int)(jc % d.ncombo);
  const float* sc = d.var_score + jc * d.V;
  float scv[16];                                    // the scores, read once (V <= 16)
  for (int v = 0; v < d.V; ++v) {
    const float x = sc[v];
    scv[v] = x != x ? -INFINITY : x;
  }
  // each visited candidate is read once into t (eight loads in flight per
  // round); its hash, tabu probe and write-out work on that copy
  uint16_t t[kMaxLen];
  uint32_t seen = 0u;
  int first = -1, chosen = -1, L = 0;
  unsigned long long chosen_h = 0ull, first_h = 0ull;
  for (int r = 0; r < d.V && chosen < 0; ++r) {
    int bv = -1;
    float bs = 0.f;
    for (int v = 0; v < d.V; ++v) {
      if ((seen >> v) & 1u) continue;
      if (bv < 0 || scv[v] > bs) {
        bv = v;
        bs = scv[v];
      }
    }
    seen |= 1u << bv;
    const long long row = jc * d.V + bv;
    L = d.var_len[row];
    copy_cols(t, d.var_seq + (size_t)row * d.S, L);
    const unsigned long long h = seq_hash(t, L);
    if (first < 0) {
      first = bv;
      first_h = h;
    }
    if (!tabu_contains(d, h, t, L)) {
      chosen = bv;
      chosen_h = h;
    }
  }
  const bool hit = chosen < 0;
  if (hit) {                                        // every candidate is in the list
    chosen = first;
    chosen_h = first_h;
    const long long row = jc * d.V + chosen;
    L = d.var_len[row];
    copy_cols(t, d.var_seq + (size_t)row * d.S, L);
  }
  const RecLayout l = rec_layout(d.k, d.S, false, bit_words(d.WC));
  char* rec = d.rec + (size_t)j * d.rec_bytes;
  uint16_t* out = reinterpret_cast<uint16_t*>(rec + l.ccols) + (size_t)c * d.S;
  for (int i = 0; i < L; ++i) out[i] = t[i];
  reinterpret_cast<int32_t*>(rec + l.cL)[c] = L;
  if (l.nw) write_bits(reinterpret_cast<uint32_t*>(rec + l.cbit) + (size_t)c * l.nw, l.nw, t, L);
  reinterpret_cast<unsigned long long*>(rec + l.chash)[c] = chosen_h;
  reinterpret_cast<int32_t*>(rec + l.ctabu)[c] = hit ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Tournament comparison.  Penalised fitness p = f / base^(S/L) in binary64,
// exactly as the reading of the paper defines it.  Fast path: compare the
// log-domain scores ln f - S * ln(base) / L in float; when they differ by more
// than a margin that bounds every rounding error of both the float scores and
// the binary64 values (pow within 1 ulp, S / L rounded once, the quotient
// rounded once), the sign is the binary64 sign.  Otherwise -- and whenever a
// value might be zero, subnormal or infinite -- compute the binary64 values
// with the host-built power table and compare them exactly.
// ---------------------------------------------------------------------------
// One tournament entrant as the builder sees it.  f = 0 exactly when
// lnf = -inf (lnf is log(f) rounded to float, finite for every f > 0), so the
// fast path needs no binary64 arithmetic; f itself is read only on the exact
// path.
struct Entrant {
  float lnf;
  float cl;          // log(base) / L as float
  int32_t S, L, idx;
  const double* f;   // the entrant's binary64 fitness (shared memory)
};

// Bit 0 of the result: x beats y.  Bit 1: the exact path decided.  The float
// decision is formed with selects; only an undecided comparison branches to
// the exact path.
__device__ __forceinline__ int beats(const Entrant& x, const Entrant& y, const EaDev& d) {
  if (x.idx == y.idx) return 0;
  const bool zx = x.lnf == -INFINITY, zy = y.lnf == -INFINITY;
  const float cx = (float)x.S * x.cl;
  const float cy = (float)y.S * y.cl;
  const float gx = x.lnf - cx, gy = y.lnf - cy;
  const bool safe_x = zx || (cx < 700.f && gx > -700.f);
  const bool safe_y = zy || (cy < 700.f && gy > -700.f);
  const float diff = gx - gy;
  const float margin = 0x1p-16f * (fabsf(x.lnf) + fabsf(y.lnf) + cx + cy + 1.f);
  const bool decided = (zx && zy) || (zx && safe_y) || (zy && safe_x) ||
                       (!zx && !zy && safe_x && safe_y && fabsf(diff) > margin);
  if (decided) {
    const bool win = (zx && zy) ? x.idx < y.idx : (zx ? false : (zy ? true : diff > 0.f));
    return win ? 1 : 0;
  }
  const double px = __ddiv_rn(*x.f, d.pow_tab[d.pow_off[x.L] + x.S]);
  const double py = __ddiv_rn(*y.f, d.pow_tab[d.pow_off[y.L] + y.S]);
  return 2 | ((px > py || (px == py && x.idx < y.idx)) ? 1 : 0);
}

// Lane-local tournament decisions for tournament size K (1 or 2): entrant
// slots 0 .. K - 1 form the first tournament, K .. 2K - 1 the second (when the
// attempt crosses over).  Returns the child index ta * K + tb; *nex counts
// exact-path comparisons.
template <int K>
__device__ __forceinline__ int decide_small(const EaDev& d, int cr, const float (&ln)[2 * K],
                                            const float (&cl)[2 * K],
                                            const int32_t (&Sx)[2 * K],
                                            const int32_t (&Lx)[2 * K],
                                            const int32_t (&id)[2 * K], const double* ef,
                                            int* nex) {
  int ta = 0, tb = 0;
  if (K == 2) {
    {
      const Entrant x{ln[1], cl[1], Sx[1], Lx[1], id[1], ef + 1};
      const Entrant y{ln[0], cl[0], Sx[0], Lx[0], id[0], ef + 0};
      const int r = beats(x, y, d);
      *nex += r >> 1;
      if ((r & 1) && id[1] != id[0]) ta = 1;
    }
    if (cr) {
      const Entrant x{ln[K + 1], cl[K + 1], Sx[K + 1], Lx[K + 1], id[K + 1], ef + K + 1};
      const Entrant y{ln[K], cl[K], Sx[K], Lx[K], id[K], ef + K};
      const int r = beats(x, y, d);
      *nex += r >> 1;
      if ((r & 1) && id[K + 1] != id[K]) tb = 1;
    }
  }
  return ta * K + tb;
}

// Within-generation duplicate check: open addressing on the 64-bit hash in
// shared memory; a hash match is confirmed on the columns of the earlier
// child (warp-wide compare).  Returns true for a duplicate; *slot = the first
// empty slot after the probe otherwise.
template <int NCT>   // combos per record when known at compile time (0: runtime nc)
__device__ __forceinline__ bool gen_duplicate(const EaDev& d, const RecLayout& l,
                                              const unsigned long long* hkey,
                                              const int32_t* href, int hmask, int nc_rt, int RB,
                                              unsigned long long key, const uint16_t* child,
                                              int L, int lane, int* slot) {
  const int nc = NCT ? NCT : nc_rt;
  int sl = (int)(key & (unsigned long long)hmask);
  for (int probe = 0; probe <= hmask; ++probe) {
    const unsigned long long kk = hkey[sl];
    if (kk == 0ull) break;
    if (kk == key) {
      const int32_t r = href[sl];
      const char* orec = d.rec + (size_t)(r / nc) * RB;
      const int oc = r % nc;
      const uint16_t* other = reinterpret_cast<const uint16_t*>(orec + l.ccols) + (size_t)oc * d.S;
      const int oL = reinterpret_cast<const int32_t*>(orec + l.cL)[oc];
      const bool same =
          oL == L &&
          __all_sync(0xffffffffu, lane >= L || other[lane] == child[lane]) &&
          __all_sync(0xffffffffu, lane + 32 >= L || other[lane + 32] == child[lane + 32]);
      if (same) return true;
    }
    sl = (sl + 1) & hmask;
  }
  *slot = sl;
  return false;
}

// Float part of one tournament comparison (see beats) with the constants of
// the pair precomputed once per sub-chunk.  During a sub-chunk a penalty sum
// can only grow, by at most 31 * L (31 earlier acceptances, each sharing at
// most L columns with the entrant), so the range checks of beats are settled
// in advance for the whole interval: a pair that passes them for every sum up
// to that bound compares in float; one that does not always takes the exact
// path.  Pairs whose outcome does not depend on the sums (the same individual
// twice, a zero fitness on either side) are decided once.
struct PairConst {
  float lx, ly, clx, cly, base;   // base = 2^-16 (|lx| + |ly| + 1)
  int fixed;                      // -1: depends on the sums; else the outcome
  bool exact_always, xlow;        // xlow: idx_x < idx_y
};

__device__ __forceinline__ PairConst pair_const(float lx, float ly, float clx, float cly,
                                                int32_t ix, int32_t iy, int32_t Sx, int32_t Sy,
                                                int32_t Lx, int32_t Ly) {
  PairConst p;
  p.lx = lx;
  p.ly = ly;
  p.clx = clx;
  p.cly = cly;
  p.xlow = ix < iy;
  const bool zx = lx == -INFINITY, zy = ly == -INFINITY;
  p.base = (zx || zy) ? 0.f : 0x1p-16f * (fabsf(lx) + fabsf(ly) + 1.f);
  // the range checks at the largest sums the sub-chunk can reach (the checks
  // are monotone in the sum)
  const float cxm = (float)(Sx + 31 * Lx) * clx, cym = (float)(Sy + 31 * Ly) * cly;
  const bool safe_x = zx || (cxm < 700.f && lx - cxm > -700.f);
  const bool safe_y = zy || (cym < 700.f && ly - cym > -700.f);
  p.fixed = -1;
  p.exact_always = false;
  if (ix == iy) p.fixed = 0;
  else if (zx && zy) p.fixed = p.xlow ? 1 : 0;
  else if (!(safe_x && safe_y)) p.exact_always = true;
  else if (zx) p.fixed = 0;
  else if (zy) p.fixed = 1;
  return p;
}

// 1 / 0 when decided in float, -1 when the exact path must decide.
__device__ __forceinline__ int pair_fast(const PairConst& p, int32_t Sx, int32_t Sy) {
  const float cx = (float)Sx * p.clx, cy = (float)Sy * p.cly;
  const float diff = (p.lx - cx) - (p.ly - cy);
  const float margin = p.base + 0x1p-16f * (cx + cy);
  int r = fabsf(diff) > margin ? (diff > 0.f ? 1 : 0) : -1;
  r = p.exact_always ? -1 : r;
  return p.fixed >= 0 ? p.fixed : r;
}

// Exact binary64 comparison (the definition; see beats) for an undecided pair.
__device__ __noinline__ int pair_exact(const EaDev& d, const double* fx, const double* fy,
                                       int32_t Lx, int32_t Ly, int32_t Sx, int32_t Sy,
                                       bool xlow) {
  const double px = __ddiv_rn(*fx, d.pow_tab[d.pow_off[Lx] + Sx]);
  const double py = __ddiv_rn(*fy, d.pow_tab[d.pow_off[Ly] + Sy]);
  return (px > py || (px == py && xlow)) ? 1 : 0;
}

// Carry-save adder: a + b + c = 2 h + l, bit by bit.
__device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t u = a ^ b;
  h = (a & b) | (u & c);
  l = u ^ c;
}

// Harley-Seal accumulation of eight words into bit-sliced counters: keeps
// ones + 2 twos + 4 fours + 8 eights (ones, twos, fours counted bit by bit)
// equal to the number of set bits added so far, with one popcount per eight
// words instead of eight.
__device__ __forceinline__ void hs8(const uint32_t (&v)[8], uint32_t& ones, uint32_t& twos,
                                    uint32_t& fours, int& eights) {
  uint32_t c1, s1, c2, s2, c3, s3, c4, d1, e1, d2, f1;
  csa(c1, s1, v[0], v[1], v[2]);
  csa(c2, s2, v[3], v[4], v[5]);
  csa(c3, s3, s1, s2, v[6]);
  csa(c4, ones, ones, s3, v[7]);
  csa(d1, e1, c1, c2, c3);
  csa(d2, twos, twos, e1, c4);
  csa(f1, fours, fours, d1, d2);
  eights += __popc(f1);
}

// Named barrier 1 over the builder's CTA: warp 0 and the helper warps meet
// there four times per batch (job posted, penalty sums done, children
// posted, overlap shares done) and once per chunk (release).
// Eight warps: warp w takes entrant w % 4 of the overlap pass over half
// w / 4 of the earlier lanes.
constexpr int kBuildThreads = 256;
// Step 3 fast path: a bit filter over the keys of the generation's committed
// children (one bit per key, chosen by the key's high 32 bits) in front of a
// dense list of those keys; a clear bit proves a child new.
constexpr int kFilterBits = 1 << 17;
constexpr int kFilterWords = kFilterBits / 32;
__device__ __forceinline__ void bar_team() {
  asm volatile("bar.sync 1, %0;" ::"n"(kBuildThreads) : "memory");
}

// One entrant's share of a batch's overlap pass: for the attempt of lane a
// (record sb + a of the chunk), sum over earlier lanes b < a with b in
// [b_lo, b_hi) of |entrant e & child_b|, the children's bitsets in s_cw
// (Harley-Seal).  b_lo and b_hi are even.
template <int K, int NV>
__device__ __forceinline__ int pass0_share(const RecLayout& l, const char* cur, int sb, int avail,
                                           int e, int lane, int RB, const uint4* s_cw, int b_lo,
                                           int b_hi) {
  constexpr int NW = 4 * NV;
  const bool have = lane < avail;
  const char* ra = cur + (size_t)(have ? sb + lane : sb) * RB;
  const int cr = have ? *reinterpret_cast<const int32_t*>(ra + l.cross) : 0;
  const bool on = have && (e < K || cr);
  uint4 bits[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v)
    bits[v] = on ? reinterpret_cast<const uint4*>(ra + l.ebit)[e * NV + v]
                 : make_uint4(0u, 0u, 0u, 0u);
  uint32_t h1 = 0u, h2 = 0u, h4 = 0u;
  int h8 = 0;
  const int b_end = min(b_hi, avail);
  for (int b = b_lo; b + 1 < b_end; b += 2) {
    uint32_t m[2][NW];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const bool in = lane > b + i;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const uint4 w = s_cw[(b + i) * NV + v];
        m[i][4 * v + 0] = in ? w.x : 0u;
        m[i][4 * v + 1] = in ? w.y : 0u;
        m[i][4 * v + 2] = in ? w.z : 0u;
        m[i][4 * v + 3] = in ? w.w : 0u;
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const uint32_t x[8] = {bits[v].x & m[0][4 * v], bits[v].y & m[0][4 * v + 1],
                             bits[v].z & m[0][4 * v + 2], bits[v].w & m[0][4 * v + 3],
                             bits[v].x & m[1][4 * v], bits[v].y & m[1][4 * v + 1],
                             bits[v].z & m[1][4 * v + 2], bits[v].w & m[1][4 * v + 3]};
      hs8(x, h1, h2, h4, h8);
    }
  }
  return 8 * h8 + 4 * __popc(h4) + 2 * __popc(h2) + __popc(h1);
}

// Shared words of the builder's team protocol.
struct Team {
  int job, sb, avail;
  int sx[2][4][32];     // penalty sum of entrant e of lane a over half h of its columns
  int ov[2][32 * 4];    // entrant e of lane a, half h of the earlier lanes: ov[h][4 a + e]
};

// One entrant's penalty sum over half h of its columns (the first
// ceil(L / 2) or the rest), eight column loads in flight per round.
template <int K>
__device__ __forceinline__ int pen_share(const RecLayout& l, const char* cur, int sb, int avail,
                                         int S, int e, int h, int lane, int RB,
                                         const uint32_t* pen) {
  const bool have = lane < avail;
  const char* ra = cur + (size_t)(have ? sb + lane : sb) * RB;
  const int cr = have ? *reinterpret_cast<const int32_t*>(ra + l.cross) : 0;
  if (!(have && (e < K || cr))) return 0;
  const int L = reinterpret_cast<const int32_t*>(ra + l.eL)[e];
  const int half = (L + 1) >> 1;
  const int c_lo = h ? half : 0, c_hi = h ? L : half;
  const uint16_t* cs = reinterpret_cast<const uint16_t*>(ra + l.ecols) + (size_t)e * S;
  int sum = 0;
  for (int c0 = c_lo; c0 < c_hi; c0 += 8) {
    uint32_t col[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = c0 + i < c_hi ? cs[c0 + i] : 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c0 + i < c_hi) sum += (int)pen[col[i]];
  }
  return sum;
}

// Helper warps (1 .. 7) during one chunk of the fast path: each batch warp w
// computes, for all 32 lanes, the penalty sum of entrant w % 4 over half
// w / 4 of its columns, then (once warp 0 has posted the children) that
// entrant's overlap share over half w / 4 of the earlier lanes; a job of 0
// ends the chunk.  Four meetings at named barrier 1 per batch.
template <int NV>
__device__ __forceinline__ void team_helper(const RecLayout& l, const char* cur, int RB, int S,
                                            int warp, int lane, Team* tm, const uint4* s_cw,
                                            const uint32_t* pen) {
  for (;;) {
    bar_team();
    if (*(volatile int*)&tm->job == 0) break;
    const int sb = tm->sb, avail = tm->avail;
    const int e = warp & 3, h = warp >> 2;
    tm->sx[h][e][lane] = pen_share<2>(l, cur, sb, avail, S, e, h, lane, RB, pen);
    bar_team();
    bar_team();
    tm->ov[h][4 * lane + e] = pass0_share<2, NV>(l, cur, sb, avail, e, lane, RB, s_cw, 16 * h,
                                                 16 * h + 16);
    bar_team();
  }
}

// Equal series test of two children (lane-local).
__device__ __forceinline__ bool same_cols(const uint16_t* a, const uint16_t* b, int L) {
  for (int i = 0; i < L; ++i)
    if (a[i] != b[i]) return false;
  return true;
}

// The same test with sixteen columns of both series loaded before any is
// compared (for a series in global memory, one round trip per sixteen).
__device__ __forceinline__ bool same_cols_wide(const uint16_t* a, const uint16_t* b, int L) {
  bool eq = true;
  for (int c0 = 0; c0 < L && eq; c0 += 16) {
    uint32_t x[16], y[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      x[i] = c0 + i < L ? a[c0 + i] : 0u;
      y[i] = c0 + i < L ? b[c0 + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) eq = eq && x[i] == y[i];
  }
  return eq;
}

constexpr int kTwinSlots = 4096;    // lane-id scratch of the twin pre-check

// The Step 3 consumer for tournaments of K <= 2 entrants and NW-word column
// bitsets, run by one warp on one chunk of records in shared memory, 32
// attempts (one per lane) at a time.
//
// The sequential rule -- each tournament sees the penalty counts left by every
// earlier acceptance -- is solved as a fixpoint.  Assuming every attempt of
// the batch is accepted, lane a's penalty sums are its sums at the batch
// start plus |entrant & child_b| for the chosen child of every earlier lane
// b; its outcome is the tournament result for those sums.  Starting from the
// outcomes at the batch start, all lanes recompute their outcomes from the
// current children of the earlier lanes until none changes (Jacobi
// iteration).  Lane 0 is final after the first pass and lane k after pass k,
// so the iteration stops after at most 32 passes, at the unique fixpoint: the
// outcomes of taking the attempts one by one.  Then duplicates are found in
// parallel (the record's tabu flag; the filter bit of the key and, where it
// is set, a warp-wide scan of the generation's committed keys; equal keys
// among earlier lanes of the batch).  The first duplicate is a hit: its child
// leaves the later lanes' sums, which are re-decided (and, if a child
// changed, re-checked) in the next round.  Once no hit remains (or the
// population is full, or the tabu rule stops the run) the accepted lanes are
// committed together, and the next batch starts from penalty counts that
// include every acceptance so far.
template <int K, int NW>
__device__ __forceinline__ void build_batch(const EaDev& d, const RecLayout& l, const char* cur,
                                            int cnt, int j0, uint32_t* pen, const float* cLf,
                                            unsigned long long* lkey, int32_t* lref,
                                            uint32_t* fbits, int E, uint8_t* s_twin,
                                            int* s_dec, uint4* s_cw, Team* tm, long long base,
                                            int RB,
                                            int lane, int& n, int& hits, int& stopped,
                                            long long& attempts, long long& exact) {
  constexpr int NE = 2 * K, NC = K * K, NV = NW / 4;
  const int S = d.S;
  const unsigned FULL = 0xffffffffu;
  long long ex_lane = 0;                 // exact tournaments of this lane's attempts
  int sb = 0;
  while (sb < cnt && n < d.P && !stopped) {
    const int avail = min(32, cnt - sb);
    const bool have = lane < avail;
    const char* ra = cur + (size_t)(have ? sb + lane : sb) * RB;
    const int cr = have ? *reinterpret_cast<const int32_t*>(ra + l.cross) : 0;
    int32_t Sx[NE], Lx[NE];
    uint4 bits[NE][NV];
    PairConst pc[2];
    const double* efa = reinterpret_cast<const double*>(ra + l.ef);
    if (K == 2) {
      float ln[NE], cl[NE];
      int32_t id[NE];
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        ln[e] = 0.f;
        cl[e] = 0.f;
        Sx[e] = Lx[e] = id[e] = 0;
#pragma unroll
        for (int v = 0; v < NV; ++v) bits[e][v] = make_uint4(0u, 0u, 0u, 0u);
        if (have && (e < K || cr)) {
          ln[e] = reinterpret_cast<const float*>(ra + l.elnf)[e];
          Lx[e] = reinterpret_cast<const int32_t*>(ra + l.eL)[e];
          cl[e] = cLf[Lx[e]];
          id[e] = reinterpret_cast<const int32_t*>(ra + l.ent)[e < K ? e : 4 + (e - K)];
          const uint4* eb = reinterpret_cast<const uint4*>(ra + l.ebit) + e * NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) bits[e][v] = eb[v];
        }
      }
      // penalty sums of the entrants: the team's job, one (entrant, half of
      // its columns) per warp; entrant 0's first half here
      if (lane == 0) {
        tm->sb = sb;
        tm->avail = avail;
        tm->job = 1;
      }
      __syncwarp();
      bar_team();
      const int s00 = pen_share<K>(l, cur, sb, avail, S, 0, 0, lane, RB, pen);
      bar_team();
      Sx[0] = s00 + tm->sx[1][0][lane];
#pragma unroll
      for (int e = 1; e < NE; ++e) Sx[e] = tm->sx[0][e][lane] + tm->sx[1][e][lane];
      pc[0] = pair_const(ln[1], ln[0], cl[1], cl[0], id[1], id[0], Sx[1], Sx[0], Lx[1], Lx[0]);
      pc[1] = pair_const(ln[3], ln[2], cl[3], cl[2], id[3], id[2], Sx[3], Sx[2], Lx[3], Lx[2]);
    }
    auto decide = [&](int* ne) -> int {
      if (K == 1 || !have) return 0;
      int ta = pair_fast(pc[0], Sx[1], Sx[0]);
      if (ta < 0) {
        ta = pair_exact(d, efa + 1, efa + 0, Lx[1], Lx[0], Sx[1], Sx[0], pc[0].xlow);
        ++*ne;
      }
      int tb = 0;
      if (cr) {
        tb = pair_fast(pc[1], Sx[3], Sx[2]);
        if (tb < 0) {
          tb = pair_exact(d, efa + 3, efa + 2, Lx[3], Lx[2], Sx[3], Sx[2], pc[1].xlow);
          ++*ne;
        }
      }
      return ta * K + tb;
    };
    // overlaps of this lane's entrants with another lane's child bitset
    auto add_overlap = [&](const uint4 (&w)[NV], int sign) {
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        int inter = 0;
#pragma unroll
        for (int v = 0; v < NV; ++v)
          inter += __popc(bits[e][v].x & w[v].x) + __popc(bits[e][v].y & w[v].y) +
                   __popc(bits[e][v].z & w[v].z) + __popc(bits[e][v].w & w[v].w);
        Sx[e] += sign * inter;
      }
    };
    int nex = 0;
    int dec = decide(&nex);
    uint4 cw[NV];                       // bitset of this lane's current child
    if (K == 2) {
      const uint4* cb = reinterpret_cast<const uint4*>(ra + l.cbit) + dec * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) cw[v] = cb[v];
      // pass 0: every earlier lane's child, assuming all are accepted (the
      // children's bitsets broadcast from shared memory)
#pragma unroll
      for (int v = 0; v < NV; ++v) s_cw[lane * NV + v] = cw[v];
      __syncwarp();
      // the overlap pass, one (entrant, half of the earlier lanes) per warp
      // of the CTA: release the helpers to it (the job is posted), take
      // entrant 0's first half here, collect the other shares
      bar_team();
      const int ov0 = pass0_share<K, NV>(l, cur, sb, avail, 0, lane, RB, s_cw, 0, 16);
      bar_team();
      Sx[0] += ov0 + tm->ov[1][4 * lane];
#pragma unroll
      for (int e = 1; e < NE; ++e) Sx[e] += tm->ov[0][4 * lane + e] + tm->ov[1][4 * lane + e];
    }
    // Lanes below `first` are settled: accepted (committed together at the
    // end of the batch) or hits.  A round finds the next hit; the hit's child
    // leaves the later lanes' sums and the next round re-decides them.
    int first = 0;
    unsigned hitmask = 0u;              // settled hits
    int acc = 0;                        // settled accepted lanes
    int cut = avail;                    // lanes processed by the batch
    bool done_batch = false;
    // duplicate flags of the lanes' current children; they stay exact for a
    // round that changes no child (after a hit, a child equal to the hit's or
    // to an earlier accepted lane's was already flagged by the twin check,
    // which covers every earlier lane of the batch)
    bool dup = false, dups_valid = false;
    while (!done_batch) {
      bool round_changed = false;
      if (K == 2) {
        // Jacobi passes until no outcome changes (at most 32 passes)
        for (int pass = 0; pass < 33; ++pass) {
          int nx = 0;
          const int nd = decide(&nx);
          unsigned changed = __ballot_sync(FULL, have && lane >= first && nd != dec);
          if (!changed) break;
          round_changed = true;
          uint4 nw[NV];
          const uint4* nb = reinterpret_cast<const uint4*>(ra + l.cbit) + nd * NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) nw[v] = nb[v];
          while (changed) {
            const int b = __ffs(changed) - 1;
            changed &= changed - 1;
            uint4 wo[NV], wn[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              wo[v].x = __shfl_sync(FULL, cw[v].x, b);
              wo[v].y = __shfl_sync(FULL, cw[v].y, b);
              wo[v].z = __shfl_sync(FULL, cw[v].z, b);
              wo[v].w = __shfl_sync(FULL, cw[v].w, b);
              wn[v].x = __shfl_sync(FULL, nw[v].x, b);
              wn[v].y = __shfl_sync(FULL, nw[v].y, b);
              wn[v].z = __shfl_sync(FULL, nw[v].z, b);
              wn[v].w = __shfl_sync(FULL, nw[v].w, b);
            }
            if (lane > b) {
              add_overlap(wo, -1);
              add_overlap(wn, 1);
            }
          }
          if (lane >= first) {
            dec = nd;
            nex = nx;
#pragma unroll
            for (int v = 0; v < NV; ++v) cw[v] = nw[v];
          }
        }
      }
      // duplicates: tabu flag, the generation's children committed by earlier
      // batches (filter, then the key list), equal keys among earlier lanes
      const bool live = have && lane >= first;
      const unsigned long long key =
          have ? reinterpret_cast<const unsigned long long*>(ra + l.chash)[dec] : 0ull;
      const int L = have ? reinterpret_cast<const int32_t*>(ra + l.cL)[dec] : 0;
      const uint16_t* child = reinterpret_cast<const uint16_t*>(ra + l.ccols) + (size_t)dec * S;
      const uint32_t fb = (uint32_t)(key >> 32) & (uint32_t)(kFilterBits - 1);
      if (dups_valid && !round_changed) {
        dup = dup && live;
      } else {
        dups_valid = true;
        dup = live && reinterpret_cast<const int32_t*>(ra + l.ctabu)[dec] != 0;
        const bool maybe = live && !dup && ((fbits[fb >> 5] >> (fb & 31)) & 1u);
        s_dec[lane] = dec;
        __syncwarp();
        unsigned mm = __ballot_sync(FULL, maybe);
        while (mm) {
          // the whole warp scans the committed keys for lane b's child
          const int b = __ffs(mm) - 1;
          mm &= mm - 1;
          const unsigned long long kb = __shfl_sync(FULL, key, b);
          const int Lb = __shfl_sync(FULL, L, b);
          const uint16_t* cb = reinterpret_cast<const uint16_t*>(cur + (size_t)(sb + b) * RB + l.ccols) +
                               (size_t)s_dec[b] * S;
          bool found = false;
#pragma unroll 4
          for (int i = lane; i < n - E; i += 32) {
            if (lkey[i] == kb) {
              const int32_t r = lref[i];
              const char* orec = d.rec + (size_t)(r / NC) * RB;
              const int oc = r % NC;
              if (reinterpret_cast<const int32_t*>(orec + l.cL)[oc] == Lb &&
                  same_cols_wide(reinterpret_cast<const uint16_t*>(orec + l.ccols) + (size_t)oc * S,
                                 cb, Lb))
                found = true;
            }
          }
          if (__any_sync(FULL, found) && lane == b) dup = true;
        }
        // equal keys among earlier lanes of the batch (settled ones too: an
        // accepted lane is not in the key list before the batch commits, and
        // a child equal to a hit's is a duplicate of what the hit duplicated):
        // each lane writes its id into a slot chosen by its key; only when
        // some lane finds another lane's id in its slot does the warp match
        // the keys exactly
        const uint32_t ts = (uint32_t)key & (uint32_t)(kTwinSlots - 1);
        if (have) s_twin[ts] = (uint8_t)lane;
        __syncwarp();
        const bool clash = have && s_twin[ts] != (uint8_t)lane;
        unsigned twins = 0u;
        if (__any_sync(FULL, clash)) {
          twins = __match_any_sync(FULL, key) & ((1u << lane) - 1u);
          if (!live) twins = 0u;
        }
        while (twins && !dup) {
          const int b = __ffs(twins) - 1;
          twins &= twins - 1;
          const char* rbb = cur + (size_t)(sb + b) * RB;
          const int db = s_dec[b];
          if (reinterpret_cast<const int32_t*>(rbb + l.cL)[db] == L &&
              same_cols(reinterpret_cast<const uint16_t*>(rbb + l.ccols) + (size_t)db * S, child, L))
            dup = true;
        }
        __syncwarp();
      }
      // the next hit, unless the population fills before it
      const unsigned dupmask = __ballot_sync(FULL, dup);
      const int first_dup = dupmask ? __ffs(dupmask) - 1 : avail;
      const int need = d.P - n - acc;
      // Several hits at once: when every duplicate of the round is a hit
      // (the population fills after the last one and the tabu rule does not
      // stop the run), take all their children out of the later lanes' sums
      // and re-decide once.  If no lane -- hits included -- changes, these
      // are exactly the sequential outcome's hits and the batch is settled;
      // otherwise the sums go back and the hits are taken one per round.
      const int m = __popc(dupmask);
      bool settled = false;
      if (m >= 2 && (31 - __clz(dupmask) - first) - (m - 1) < need && hits + m <= d.P) {
        int32_t keep_sx[NE];
        if (K == 2) {
#pragma unroll
          for (int e = 0; e < NE; ++e) keep_sx[e] = Sx[e];
          unsigned rest = dupmask;
          while (rest) {
            const int b = __ffs(rest) - 1;
            rest &= rest - 1;
            uint4 wo[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              wo[v].x = __shfl_sync(FULL, cw[v].x, b);
              wo[v].y = __shfl_sync(FULL, cw[v].y, b);
              wo[v].z = __shfl_sync(FULL, cw[v].z, b);
              wo[v].w = __shfl_sync(FULL, cw[v].w, b);
            }
            if (lane > b) add_overlap(wo, -1);
          }
        }
        int nx = 0;
        const int nd = decide(&nx);
        if (!__any_sync(FULL, have && lane >= first && nd != dec)) {
          hitmask |= dupmask;
          hits += m;
          const int free_lanes = (avail - first) - m;
          if (free_lanes >= need) {
            // the need-th accepted lane fills the population and ends the batch
            unsigned am = __ballot_sync(FULL, have && lane >= first && !dup);
            for (int t = 1; t < need; ++t) am &= am - 1;
            cut = __ffs(am);
            acc += need;
          } else {
            acc += free_lanes;
          }
          done_batch = true;
          settled = true;
        } else if (K == 2) {
#pragma unroll
          for (int e = 0; e < NE; ++e) Sx[e] = keep_sx[e];
        }
      }
      if (settled) {
      } else if (first_dup - first >= need) {
        acc += need;
        cut = first + need;
        done_batch = true;
      } else {
        acc += first_dup - first;
        if (first_dup >= avail) {
          done_batch = true;
        } else {
          hitmask |= 1u << first_dup;
          if (++hits > d.P) {
            stopped = 1;
            cut = first_dup + 1;
            done_batch = true;
          } else if (first_dup + 1 >= avail) {
            done_batch = true;
          } else {
            // the hit's child is not accepted: take it out of the later
            // lanes' sums and go on with the rest of the batch
            if (K == 2) {
              uint4 wo[NV];
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                wo[v].x = __shfl_sync(FULL, cw[v].x, first_dup);
                wo[v].y = __shfl_sync(FULL, cw[v].y, first_dup);
                wo[v].z = __shfl_sync(FULL, cw[v].z, first_dup);
                wo[v].w = __shfl_sync(FULL, cw[v].w, first_dup);
              }
              if (lane > first_dup) add_overlap(wo, -1);
            }
            first = first_dup + 1;
          }
        }
      }
      __syncwarp();
    }
    // commit the accepted lanes of [0, cut) in lane order
    {
      const unsigned accm = __ballot_sync(FULL, have && lane < cut && !((hitmask >> lane) & 1u));
      const int k = __popc(accm & ((1u << lane) - 1u));
      if ((accm >> lane) & 1u) {
        const unsigned long long key = reinterpret_cast<const unsigned long long*>(ra + l.chash)[dec];
        const int L = reinterpret_cast<const int32_t*>(ra + l.cL)[dec];
        const uint16_t* child = reinterpret_cast<const uint16_t*>(ra + l.ccols) + (size_t)dec * S;
        const uint32_t fb = (uint32_t)(key >> 32) & (uint32_t)(kFilterBits - 1);
        lkey[n - E + k] = key;
        lref[n - E + k] = (int32_t)((j0 + sb + lane) * NC + dec);
        atomicOr(&fbits[fb >> 5], 1u << (fb & 31));
        uint16_t* dst = d.seq + (size_t)(base + n + k) * S;
        // eight columns per round, loads issued before the stores and the
        // penalty increments that use them
        for (int c0 = 0; c0 < L; c0 += 8) {
          uint32_t v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = c0 + i < L ? child[c0 + i] : 0u;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (c0 + i < L) {
              dst[c0 + i] = (uint16_t)v[i];
              atomicAdd(&pen[v[i]], 1u);
            }
          }
        }
        d.len[base + n + k] = L;
      }
      if (have && lane < cut) ex_lane += nex;
      attempts += cut;
      n += acc;
      sb += cut;
      __syncwarp();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ex_lane += __shfl_xor_sync(FULL, ex_lane, o);
  exact += ex_lane;
}

// ---------------------------------------------------------------------------
// k_build: Steps 2-3 (or the acceptance part of Step 1).  The decisions are
// sequential (each tournament sees the penalty counts left by every earlier
// acceptance), so warp 0 makes them from shared memory only.  The attempt
// records (written by k_spec) are streamed in chunks of kB with TMA bulk
// copies into a double buffer completed through mbarriers, issued by thread 0
// two chunks ahead.  Every wait is bounded: on expiry the kernel records
// stop reason 4, drains its own copies in flight and returns.
// Accepted children go to the archive straight from the shared-memory records
// (at acceptance, or once per 32 attempts in the fast path).
//
// Shared memory: hkey[H] (u64) | href[H] | pen[C] | cLf[Lmax + 1] |
//                fbits[kFilterWords] (16-byte aligned) |
//                2 record buffers of kB records (128-byte aligned).
// hkey / href are the generation's hash set of committed children in the
// general path; the fast path keeps them as a dense list (key, record) in
// commit order behind the bit filter fbits.
// ---------------------------------------------------------------------------
template <bool INIT>
__global__ void __launch_bounds__(kBuildThreads, 1) k_build(EaDev d, int hmask, int kB) {
  extern __shared__ __align__(128) unsigned long long smem_u64[];
  if (*(volatile int32_t*)&d.ctl->stop) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = d.ctl->gen;
  if (tid == 0) d.ctl->spec_gen = g + 1;    // read by the next k_spec only
  const int H = hmask + 1, k = d.k, nc = INIT ? 1 : k * k, S = d.S;
  const RecLayout l = rec_layout(k, S, INIT, bit_words(d.WC));
  const int RB = d.rec_bytes;
  unsigned long long* hkey = smem_u64;
  int32_t* href = reinterpret_cast<int32_t*>(hkey + H);
  uint32_t* pen = reinterpret_cast<uint32_t*>(href + H);
  float* cLf = reinterpret_cast<float*>(pen + d.C);
  // aligned by offsets from the shared base (integer round trips through
  // uintptr_t would lose the shared address space)
  char* const sbase = reinterpret_cast<char*>(smem_u64);
  uint32_t* fbits = reinterpret_cast<uint32_t*>(
      sbase + ((reinterpret_cast<char*>(cLf + d.Lmax + 1) - sbase + 15) & ~(ptrdiff_t)15));
  char* buf0 = sbase + ((reinterpret_cast<char*>(fbits + kFilterWords) - sbase + 127) & ~(ptrdiff_t)127);
  // record buffer i at buf0 + i * kB * RB (computed, not looked up, so that the
  // compiler keeps the shared-memory address space of every record access)
  const size_t buf_bytes = (size_t)kB * RB;
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ int s_n, s_done, s_E, s_fail;
  __shared__ int s_dec[32];              // outcomes of the batch's lanes (fast path)
  __shared__ uint8_t s_twin[kTwinSlots];  // lane ids by key (fast path twin pre-check)
  __shared__ uint4 s_cw[32 * 2];         // their children's bitsets (fast path)
  __shared__ Team s_team;                // the fast path's helper-warp protocol
  // fast path: tournaments of at most 2 entrants, column sets of at most 256 bits
  const bool fast = d.k <= 2 && l.nw > 0;
  // the helper warps share the penalty sums and the overlap pass
  // (tournaments of 2)
  const bool team = !INIT && fast && d.k == 2;

  const int nchunks = (d.J + kB - 1) / kB;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  int issued = 0;                       // chunks whose copy thread 0 has issued
  if (tid == 0) {
    for (; issued < 2 && issued < nchunks; ++issued) {
      const int j0 = issued * kB, cnt = min(kB, d.J - j0);
      bulk_load(buf0 + (issued & 1) * buf_bytes, d.rec + (size_t)j0 * RB, (uint32_t)cnt * RB,
                &bars[issued & 1]);
    }
  }
  for (int i = tid; i < H; i += kBuildThreads) hkey[i] = 0ull;
  if (!INIT && fast)
    for (int i = tid; i < kFilterWords / 4; i += kBuildThreads)
      reinterpret_cast<uint4*>(fbits)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < d.C; i += kBuildThreads) pen[i] = 0u;
  for (int i = tid; i <= d.Lmax; i += kBuildThreads) cLf[i] = d.c_over_L[i];
  const long long base = (long long)g * d.P;
  if (tid == 0) {
    int E = 0;
    if (!INIT) {
      E = (int)ceil(d.elite_frac * (double)d.ctl->n_top);
      if (E > d.P) E = d.P;
    }
    s_E = E;
    s_done = 0;
  }
  __syncthreads();
  const int E = s_E;
  // Step 2: elites copied in order, each column use counted.
  for (int e = warp; e < E; e += kBuildThreads / 32) {
    const int32_t src = d.list_ref[e];
    const int L = d.len[src];
    for (int c = lane; c < L; c += 32) {
      const uint16_t v = d.seq[(size_t)src * S + c];
      d.seq[(size_t)(base + e) * S + c] = v;
      atomicAdd(&pen[v], 1u);
    }
    if (lane == 0) d.len[base + e] = L;
  }
  __syncthreads();

  int n = E, hits = 0, stopped = 0;
  long long attempts = 0, exact = 0;
  int chunk = 0;
  for (; chunk < nchunks; ++chunk) {
    char* cur = buf0 + (chunk & 1) * buf_bytes;
    if (warp == 0) {
      const bool ok = mbar_wait(&bars[chunk & 1], (uint32_t)((chunk >> 1) & 1));
      const int cnt = min(kB, d.J - chunk * kB);
      if (!ok) {
        stopped = 4;
      } else if (!INIT && fast) {
        if (k == 2) {
          if (l.nw == 4)
            build_batch<2, 4>(d, l, cur, cnt, chunk * kB, pen, cLf, hkey, href, fbits, E, s_twin,
                              s_dec, s_cw, &s_team, base, RB,
                             lane, n, hits, stopped, attempts, exact);
          else
            build_batch<2, 8>(d, l, cur, cnt, chunk * kB, pen, cLf, hkey, href, fbits, E, s_twin,
                              s_dec, s_cw, &s_team, base, RB,
                             lane, n, hits, stopped, attempts, exact);
        } else {
          if (l.nw == 4)
            build_batch<1, 4>(d, l, cur, cnt, chunk * kB, pen, cLf, hkey, href, fbits, E, s_twin,
                              s_dec, s_cw, &s_team, base, RB,
                             lane, n, hits, stopped, attempts, exact);
          else
            build_batch<1, 8>(d, l, cur, cnt, chunk * kB, pen, cLf, hkey, href, fbits, E, s_twin,
                              s_dec, s_cw, &s_team, base, RB,
                             lane, n, hits, stopped, attempts, exact);
        }
      } else {
        for (int a = 0; a < kB && n < d.P; ++a) {
          const int j = chunk * kB + a;
          if (j >= d.J) {
            stopped = 3;
            break;
          }
          const char* rc = cur + (size_t)a * RB;
          ++attempts;
          int combo = 0;
          if (!INIT) {
            const int32_t* ent = reinterpret_cast<const int32_t*>(rc + l.ent);
            const int cr = *reinterpret_cast<const int32_t*>(rc + l.cross);
            const double* ef = reinterpret_cast<const double*>(rc + l.ef);
            const float* elnf = reinterpret_cast<const float*>(rc + l.elnf);
            const int32_t* eL = reinterpret_cast<const int32_t*>(rc + l.eL);
            const uint16_t* ecols = reinterpret_cast<const uint16_t*>(rc + l.ecols);
            const int nE = cr ? 2 * k : k;
            // penalty sums: lanes 8q .. 8q + 7 sum entrant 4 * pass + q
            uint32_t part0 = 0u, part1 = 0u;
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
              if (pass * 4 < nE) {
                const int e = pass * 4 + (lane >> 3);
                uint32_t v = 0;
                if (e < nE) {
                  const int L = eL[e];
                  const uint16_t* cs = ecols + (size_t)e * S;
                  for (int c = lane & 7; c < L; c += 8) v += pen[cs[c]];
                }
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                if (pass == 0) part0 = v;
                else part1 = v;
              }
            }
            // tournaments, computed alike on every lane from registers
            int pos0 = 0, pos1 = 0, nex = 0;
            for (int tour = 0; tour < (cr ? 2 : 1); ++tour) {
              Entrant best, x;
              int best_t = 0;
              for (int t = 0; t < k; ++t) {
                const int e = tour * k + t;
                x.lnf = elnf[e];
                x.S = (int32_t)__shfl_sync(0xffffffffu, e < 4 ? part0 : part1, (e & 3) * 8);
                x.L = eL[e];
                x.cl = cLf[x.L];
                x.idx = ent[(tour ? 4 : 0) + t];
                x.f = ef + e;
                if (t == 0) {
                  best = x;
                } else {
                  const int r = beats(x, best, d);
                  nex += r >> 1;
                  if (r & 1) {
                    best = x;
                    best_t = t;
                  }
                }
              }
              for (int t = 0; t < best_t; ++t)
                if (ent[(tour ? 4 : 0) + t] == best.idx) {
                  best_t = t;
                  break;
                }
              if (tour == 0) pos0 = best_t;
              else pos1 = best_t;
            }
            exact += nex;
            combo = pos0 * k + pos1;
          }
          const int L = reinterpret_cast<const int32_t*>(rc + l.cL)[combo];
          const unsigned long long key = reinterpret_cast<const unsigned long long*>(rc + l.chash)[combo];
          const uint16_t* child = reinterpret_cast<const uint16_t*>(rc + l.ccols) + (size_t)combo * S;
          int slot = 0;
          const bool dup = reinterpret_cast<const int32_t*>(rc + l.ctabu)[combo] != 0 ||
                           gen_duplicate<0>(d, l, hkey, href, hmask, nc, RB, key, child, L, lane, &slot);
          if (dup) {
            if (++hits > d.P) {
              stopped = INIT ? 2 : 1;
              break;
            }
            continue;
          }
          const int32_t rec_id = (int32_t)(j * nc + combo);
          uint16_t* dst = d.seq + (size_t)(base + n) * S;
          if (lane < L) {
            pen[child[lane]] += 1u;
            dst[lane] = child[lane];
          }
          if (lane + 32 < L) {
            pen[child[lane + 32]] += 1u;
            dst[lane + 32] = child[lane + 32];
          }
          if (lane == 0) {
            hkey[slot] = key;
            href[slot] = rec_id;
            d.len[base + n] = L;
          }
          __syncwarp();
          ++n;
        }
      }
      if (lane == 0) {
        s_n = n;
        s_done = (n >= d.P || stopped) ? 1 : 0;
        if (stopped == 4) s_fail = 1;
      }
      if (team) {               // release the helpers from this chunk
        if (lane == 0) s_team.job = 0;
        __syncwarp();
        bar_team();
      }
    } else if (team) {
      if (l.nw == 4) team_helper<1>(l, cur, RB, S, warp, lane, &s_team, s_cw, pen);
      else team_helper<2>(l, cur, RB, S, warp, lane, &s_team, s_cw, pen);
    }
    __syncthreads();            // the consumed buffer may now be refilled
    if (s_done) {
      ++chunk;
      break;
    }
    if (tid == 0 && issued < nchunks) {
      const int j0 = issued * kB, cnt = min(kB, d.J - j0);
      bulk_load(buf0 + (issued & 1) * buf_bytes, d.rec + (size_t)j0 * RB, (uint32_t)cnt * RB,
                &bars[issued & 1]);
      ++issued;
    }
  }
  // every attempt consumed without filling the population: cannot happen
  // (2P + 1 attempts always suffice), reported as an internal error
  if (tid == 0 && s_n < d.P && !s_done) s_fail = 2;
  // drain: copies issued but not consumed must land before the CTA exits
  if (tid == 0) {
    for (int c = chunk; c < issued; ++c)
      if (!mbar_wait(&bars[c & 1], (uint32_t)((c >> 1) & 1))) s_fail = 1;
  }
  __syncthreads();
  if (tid == 0) {
    Ctl* ctl = d.ctl;
    ctl->last_hits = hits;
    ctl->hits_total += hits;
    ctl->attempts_total += attempts;
    ctl->exact_total += exact;
    ctl->n_elite = E;
    if (s_fail) stopped = s_fail == 2 ? 3 : 4;
    if (stopped) {
      ctl->stop_reason = stopped;
      __threadfence();
      ctl->stop = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// k_tabu_insert: the generation's new (non-elite) individuals enter the tabu
// list.  Lookups happen in later launches only.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tabu_insert(EaDev d) {
  if (*(volatile int32_t*)&d.ctl->stop) return;
  // the generation k_build just built: Step 5 of that generation may run
  // beside this kernel and advance ctl->gen, so it comes from spec_gen
  const int g = d.ctl->spec_gen - 1;
  const int slot = d.ctl->n_elite + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (slot >= d.P) return;
  const long long e = (long long)g * d.P + slot;
  uint16_t x[kMaxLen];                              // the series, eight loads in flight
  const int L = d.len[e];
  copy_cols(x, d.seq + (size_t)e * d.S, L);
  const unsigned long long key = seq_hash(x, L);
  unsigned long long i = key & d.tmask;
  for (unsigned long long n = 0; n <= d.tmask; ++n) {
    if (atomicCAS(&d.tkey[i], 0ull, key) == 0ull) {
      d.tref[i] = (int32_t)e;
      return;
    }
    i = (i + 1) & d.tmask;
  }
  atomicExch(&d.ctl->stop_reason, 3);   // table full: cannot happen at load <= 1/2
  atomicExch(&d.ctl->stop, 1);
}

// ---------------------------------------------------------------------------
// k_rank: Step 5 (and the list part of Step 1).  One CTA of 1,024 threads.
// The population is sorted by decreasing fitness (ties: lower slot first),
// then visited in that order: an individual joins unless a listed record of
// higher or equal fitness overlaps it (|a & b| / min(|a|, |b|) > tau); when it
// joins it evicts the overlapping records of lower fitness and goes after all
// records of higher or equal fitness.  Finally the list keeps its T best.
//
// The visit stops early once T listed records have a fitness strictly above
// the current individual: records above it can only be evicted by fitter
// individuals (already visited), and everything visited from here on ranks
// below those T records, so it would be cut by the final trim -- and what it
// could still evict also ranks below them.  The result is the same list.
// ---------------------------------------------------------------------------
constexpr int kRankThreads = 1024;

__global__ void __launch_bounds__(kRankThreads) k_rank(EaDev d, int Pp) {
  extern __shared__ unsigned long long smem_u64[];
  if (*(volatile int32_t*)&d.ctl->stop) return;
  const int tid = threadIdx.x;
  const int g = d.ctl->gen;
  const long long base = (long long)g * d.P;
  const int cap = d.T + d.P;
  unsigned long long* skey = smem_u64;                             // [Pp]
  int32_t* sidx = reinterpret_cast<int32_t*>(skey + Pp);           // [Pp]
  double* lf = reinterpret_cast<double*>(sidx + Pp);               // [cap]
  double* lf2 = lf + cap;                                          // [cap]
  int32_t* lr = reinterpret_cast<int32_t*>(lf2 + cap);             // [cap]
  int32_t* lr2 = lr + cap;                                         // [cap]
  uint8_t* ov = reinterpret_cast<uint8_t*>(lr2 + cap);             // [cap]
  uint32_t* xbits = reinterpret_cast<uint32_t*>(ov + ((cap + 15) & ~15));   // [WC]
  __shared__ int s_warp[32];

  // sort keys: ascending (~bits(f), slot) == descending fitness, then slot
  for (int i = tid; i < Pp; i += kRankThreads) {
    if (i < d.P) {
      skey[i] = ~(unsigned long long)__double_as_longlong(d.fit[base + i]);
      sidx[i] = i;
    } else {
      skey[i] = ~0ull;
      sidx[i] = 0x7fffffff;
    }
  }
  __syncthreads();
  for (int size = 2; size <= Pp; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < Pp; i += kRankThreads) {
        const int jx = i ^ stride;
        if (jx > i) {
          const bool up = (i & size) == 0;
          const unsigned long long ka = skey[i], kb = skey[jx];
          const int ia = sidx[i], ib = sidx[jx];
          const bool a_gt_b = ka > kb || (ka == kb && ia > ib);
          if (a_gt_b == up) {
            skey[i] = kb;
            skey[jx] = ka;
            sidx[i] = ib;
            sidx[jx] = ia;
          }
        }
      }
      __syncthreads();
    }
  }

  int n = d.ctl->n_top;
  for (int i = tid; i < n; i += kRankThreads) {
    lr[i] = d.list_ref[i];
    lf[i] = d.list_f[i];
  }
  __syncthreads();

  for (int oi = 0; oi < d.P; ++oi) {
    const int xi = sidx[oi];
    const long long xe = base + xi;
    const double xf = d.fit[xe];
    const int xL = d.len[xe];
    const uint16_t* xs = d.seq + (size_t)xe * d.S;
    int above = 0;
    for (int t0 = 0; t0 < n; t0 += kRankThreads) {
      const int t = t0 + tid;
      above += __syncthreads_count(t < n && lf[t] > xf);
    }
    if (above >= d.T) break;                                   // see the note above
    for (int w = tid; w < d.WC; w += kRankThreads) xbits[w] = 0u;
    __syncthreads();
    if (tid < xL) atomicOr(&xbits[xs[tid] >> 5], 1u << (xs[tid] & 31));
    __syncthreads();
    int blocked = 0;
    for (int t0 = 0; t0 < n; t0 += kRankThreads) {
      const int t = t0 + tid;
      bool hit = false;
      if (t < n) {
        const int32_t r = lr[t];
        const int L = d.len[r];
        const uint16_t* s = d.seq + (size_t)r * d.S;
        int inter = 0;
        for (int c = 0; c < L; ++c) inter += (xbits[s[c] >> 5] >> (s[c] & 31)) & 1u;
        const int mn = L < xL ? L : xL;
        const bool o = (double)inter > d.tau * (double)mn;
        ov[t] = o ? 1 : 0;
        hit = o && lf[t] >= xf;
      }
      blocked += __syncthreads_or(hit);
    }
    if (blocked) continue;
    // evict overlapping records of lower fitness (stable compaction into lr2/lf2)
    int m = 0;
    for (int t0 = 0; t0 < n; t0 += kRankThreads) {
      const int t = t0 + tid;
      const bool keep = t < n && !(ov[t] && lf[t] < xf);
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      const int lane = tid & 31, warp = tid >> 5;
      if (lane == 0) s_warp[warp] = __popc(bal);
      __syncthreads();
      if (warp == 0) {
        int v = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        s_warp[lane] = v;          // inclusive prefix over warps
      }
      __syncthreads();
      const int before = (warp ? s_warp[warp - 1] : 0) + __popc(bal & ((1u << lane) - 1u));
      if (keep) {
        lr2[m + before] = lr[t];
        lf2[m + before] = lf[t];
      }
      const int chunk_total = s_warp[31];
      __syncthreads();
      m += chunk_total;
    }
    // insert after every kept record of higher or equal fitness
    int pos = 0;
    for (int t0 = 0; t0 < m; t0 += kRankThreads) {
      const int t = t0 + tid;
      pos += __syncthreads_count(t < m && lf2[t] >= xf);
    }
    for (int t = tid; t < m; t += kRankThreads) {
      const int dst = t < pos ? t : t + 1;
      lr[dst] = lr2[t];
      lf[dst] = lf2[t];
    }
    if (tid == 0) {
      lr[pos] = (int32_t)xe;
      lf[pos] = xf;
    }
    n = m + 1;
    __syncthreads();
  }
  if (n > d.T) n = d.T;
  for (int i = tid; i < n; i += kRankThreads) {
    d.list_ref[i] = lr[i];
    d.list_f[i] = lf[i];
  }
  if (tid == 0) {
    Ctl* ctl = d.ctl;
    ctl->n_top = n;
    ctl->evals_total += d.P;
    if (g > 0) ctl->gens_done = g;
    ctl->gen = g + 1;
  }
}

// ---------------------------------------------------------------------------
// k_rank_warp: the same Step 5 for column sets of at most NW * 32 columns.
// The whole CTA sorts (as k_rank) and then prefetches, in visiting order, each
// individual's fitness, length and column bitset, and the listed records'
// fitness, reference, length and bitset, into shared memory.  The visit
// itself -- sequential by definition -- is run by warp 0 alone from shared
// memory: overlaps are popcounts of bitset intersections, and
// |a & b| > tau * min(|a|, |b|) is an integer test against floor(tau * m)
// (the binary64 product, as in k_rank).  The list is kept sorted by
// decreasing fitness, so the records of fitness >= f(x) form a prefix of
// length ge; nothing in that prefix can move (evictions need lower fitness,
// and x goes after every record of higher or equal fitness), so an accepted x
// only rewrites the suffix: a stable compaction of the kept records, then a
// shift by one, then x at position ge.
//
// Shared memory: skey[Pp] (u64) | sidx[Pp] | pf[P] (f64) | pL[P] |
//                lm[cap] (RankRec, 16 B) | pbits[P][NW] | lbits[cap][NW] | thr
// ---------------------------------------------------------------------------
struct RankRec {
  double f;
  int32_t r, L;
};

constexpr int kRankWarpThreads = 512;   // register room for the deciding warp

template <int NW>
__device__ __forceinline__ int overlap_bits(const uint32_t* a, const uint32_t (&xb)[NW]) {
  int inter = 0;
#pragma unroll
  for (int v = 0; v < NW / 4; ++v) {
    const uint4 w = reinterpret_cast<const uint4*>(a)[v];
    inter += __popc(w.x & xb[4 * v]) + __popc(w.y & xb[4 * v + 1]) +
             __popc(w.z & xb[4 * v + 2]) + __popc(w.w & xb[4 * v + 3]);
  }
  return inter;
}

// Bitonic sort of N = EPT * kRankWarpThreads (key, index) pairs into
// ascending order (key, then index), thread t holding elements EPT t .. EPT t
// + EPT - 1 in registers: compare-exchanges within a thread, with a partner
// thread of the warp by shuffles, and through shared memory (skey / sidx, N
// entries) only for partners in other warps.
template <int EPT>
__device__ __forceinline__ void sort_pairs(unsigned long long* skey, int32_t* sidx, int tid) {
  constexpr int N = EPT * kRankWarpThreads;
  unsigned long long k[EPT];
  int32_t x[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    k[q] = skey[EPT * tid + q];
    x[q] = sidx[EPT * tid + q];
  }
  // element e of the block-direction `up` keeps the smaller of the pair when
  // it is the lower position of an ascending block (or the upper of a
  // descending one), the larger otherwise
  auto keep = [](unsigned long long& ka, int32_t& xa, unsigned long long kb, int32_t xb,
                 bool want_min) {
    const bool a_gt_b = ka > kb || (ka == kb && xa > xb);
    if (a_gt_b == want_min) {
      ka = kb;
      xa = xb;
    }
  };
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32 * EPT) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          skey[EPT * tid + q] = k[q];
          sidx[EPT * tid + q] = x[q];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int e = EPT * tid + q, p = e ^ stride;
          keep(k[q], x[q], skey[p], sidx[p], (e < p) == ((e & size) == 0));
        }
      } else if (stride >= EPT) {
        const int lane_x = stride / EPT;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int e = EPT * tid + q, p = e ^ stride;
          const unsigned long long kp = __shfl_xor_sync(0xffffffffu, k[q], lane_x);
          const int32_t xp = __shfl_xor_sync(0xffffffffu, x[q], lane_x);
          keep(k[q], x[q], kp, xp, (e < p) == ((e & size) == 0));
        }
      } else {
        // (the in-thread stride as a compile-time constant keeps k and x in
        // registers)
#pragma unroll
        for (int ls = EPT / 2; ls > 0; ls >>= 1) {
          if (ls != stride) continue;
#pragma unroll
          for (int q = 0; q < EPT; ++q) {
            if (q & ls) continue;
            const int e = EPT * tid + q;
            const bool up = (e & size) == 0;
            const unsigned long long ka = k[q], kb = k[q ^ ls];
            const int32_t xa = x[q], xb = x[q ^ ls];
            const bool a_gt_b = ka > kb || (ka == kb && xa > xb);
            if (a_gt_b == up) {
              k[q] = kb;
              x[q] = xb;
              k[q ^ ls] = ka;
              x[q ^ ls] = xa;
            }
          }
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    skey[EPT * tid + q] = k[q];
    sidx[EPT * tid + q] = x[q];
  }
  __syncthreads();
}

template <int NW>
__global__ void __launch_bounds__(kRankWarpThreads) k_rank_warp(EaDev d, int Pp) {
  extern __shared__ __align__(128) unsigned long long smem_u64[];
  if (*(volatile int32_t*)&d.ctl->stop) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = d.ctl->gen;
  const long long base = (long long)g * d.P;
  const int cap = d.T + d.P, P = d.P;
  const int Ns = Pp > kRankWarpThreads ? Pp : kRankWarpThreads;   // sorted entries
  unsigned long long* skey = smem_u64;
  int32_t* sidx = reinterpret_cast<int32_t*>(skey + Ns);
  double* pf = reinterpret_cast<double*>(sidx + Ns);
  int32_t* pL = reinterpret_cast<int32_t*>(pf + P);
  // the records and bitsets are read as 16-byte vectors: align by offset
  char* const sb = reinterpret_cast<char*>(smem_u64);
  RankRec* lm = reinterpret_cast<RankRec*>(
      sb + ((reinterpret_cast<char*>(pL + P) - sb + 15) & ~(ptrdiff_t)15));
  uint32_t* pbits = reinterpret_cast<uint32_t*>(lm + cap);
  uint32_t* lbits = pbits + (size_t)P * NW;
  int32_t* thr = reinterpret_cast<int32_t*>(lbits + (size_t)cap * NW);

  // Every individual's fitness, length and column bitset, by population
  // index, read before the sort (the bitsets' column loads go out eight at
  // a time); the visit reaches them through the sorted index.
  for (int i = tid; i < Ns; i += kRankWarpThreads) {
    if (i < P) {
      const double f = d.fit[base + i];
      skey[i] = ~(unsigned long long)__double_as_longlong(f);
      sidx[i] = i;
      pf[i] = f;
      const int L = d.len[base + i];
      pL[i] = L;
      write_bits(pbits + (size_t)i * NW, NW, d.seq + (size_t)(base + i) * d.S, L);
    } else {
      skey[i] = ~0ull;
      sidx[i] = 0x7fffffff;
    }
  }
  for (int m = tid; m <= d.Lmax; m += kRankWarpThreads) thr[m] = (int32_t)floor(d.tau * (double)m);
  int n = d.ctl->n_top;
  for (int t = tid; t < n; t += kRankWarpThreads) {
    const int32_t r = d.list_ref[t];
    const int L = d.len[r];
    lm[t] = RankRec{d.list_f[t], r, L};
    write_bits(lbits + (size_t)t * NW, NW, d.seq + (size_t)r * d.S, L);
  }
  __syncthreads();
  switch (Ns / kRankWarpThreads) {     // Ns is a power of two >= 512
    case 1: sort_pairs<1>(skey, sidx, tid); break;
    case 2: sort_pairs<2>(skey, sidx, tid); break;
    case 4: sort_pairs<4>(skey, sidx, tid); break;
    default: sort_pairs<8>(skey, sidx, tid); break;
  }


  if (tid < 32) {
    const unsigned FULL = 0xffffffffu;
    for (int oi = 0; oi < P; ++oi) {
      const int xi = sidx[oi];                  // population index of the oi-th visited
      const double xf = pf[xi];
      const int xL = pL[xi];
      uint32_t xb[NW];
#pragma unroll
      for (int v = 0; v < NW / 4; ++v) {
        const uint4 w = reinterpret_cast<const uint4*>(pbits + (size_t)xi * NW)[v];
        xb[4 * v] = w.x;
        xb[4 * v + 1] = w.y;
        xb[4 * v + 2] = w.z;
        xb[4 * v + 3] = w.w;
      }
      // records strictly fitter (above), of higher or equal fitness (ge, a
      // prefix), and whether one of the latter overlaps x (blocks it)
      int above = 0, ge = 0;
      bool block = false;
      for (int t0 = 0; t0 < n; t0 += 32) {
        const int t = t0 + lane;
        bool is_ge = false;
        if (t < n) {
          const RankRec rec = lm[t];
          above += rec.f > xf ? 1 : 0;
          is_ge = rec.f >= xf;
          if (is_ge) block = block || overlap_bits<NW>(lbits + (size_t)t * NW, xb) > thr[min(rec.L, xL)];
        }
        const unsigned gb = __ballot_sync(FULL, is_ge);
        ge += __popc(gb);
        if (gb != FULL) break;                  // the prefix ends in this chunk
      }
      above = __reduce_add_sync(FULL, (unsigned)above);
      if (above >= d.T) break;                  // see k_rank
      if (__any_sync(FULL, block)) continue;
      // suffix [ge, n): stable compaction of the kept records (not:
      // overlapping and less fit) ...
      int m = ge;
      for (int t0 = ge; t0 < n; t0 += 32) {
        const int t = t0 + lane;
        bool keep = false;
        RankRec rec{0.0, 0, 0};
        uint4 b[NW / 4];
        if (t < n) {
          rec = lm[t];
#pragma unroll
          for (int v = 0; v < NW / 4; ++v) b[v] = reinterpret_cast<const uint4*>(lbits + (size_t)t * NW)[v];
          keep = !(overlap_bits<NW>(lbits + (size_t)t * NW, xb) > thr[min(rec.L, xL)]);
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) {
          const int dst = m + __popc(bal & ((1u << lane) - 1u));
          lm[dst] = rec;
#pragma unroll
          for (int v = 0; v < NW / 4; ++v) reinterpret_cast<uint4*>(lbits + (size_t)dst * NW)[v] = b[v];
        }
        __syncwarp();
        m += __popc(bal);
      }
      // ... shifted up by one (from the end), and x at ge
      for (int t0 = ((m - 1) & ~31); t0 >= ge - 31 && t0 >= 0; t0 -= 32) {
        const int t = t0 + lane;
        const bool mv = t >= ge && t < m;
        RankRec rec{0.0, 0, 0};
        uint4 b[NW / 4];
        if (mv) {
          rec = lm[t];
#pragma unroll
          for (int v = 0; v < NW / 4; ++v) b[v] = reinterpret_cast<const uint4*>(lbits + (size_t)t * NW)[v];
        }
        __syncwarp();
        if (mv) {
          lm[t + 1] = rec;
#pragma unroll
          for (int v = 0; v < NW / 4; ++v) reinterpret_cast<uint4*>(lbits + (size_t)(t + 1) * NW)[v] = b[v];
        }
        __syncwarp();
      }
      if (lane == 0) lm[ge] = RankRec{xf, (int32_t)(base + xi), xL};
#pragma unroll
      for (int w = 0; w < NW; ++w)
        if (lane == w) lbits[(size_t)ge * NW + w] = xb[w];
      __syncwarp();
      n = m + 1;
    }
    if (n > d.T) n = d.T;
    for (int i = lane; i < n; i += 32) {
      const RankRec rec = lm[i];
      d.list_ref[i] = rec.r;
      d.list_f[i] = rec.f;
    }
    if (lane == 0) {
      Ctl* ctl = d.ctl;
      ctl->n_top = n;
      ctl->evals_total += d.P;
      if (g > 0) ctl->gens_done = g;
      ctl->gen = g + 1;
    }
  }
}

// Shared bytes of k_rank_warp<NW> for population P (padded Pp), list T.
static size_t rank_warp_smem(int P, int Pp, int T, int Lmax, int NW) {
  const size_t cap = (size_t)T + P;
  const size_t Ns = (size_t)std::max(Pp, kRankWarpThreads);
  return Ns * 12 + (size_t)P * 12 + 16 + cap * sizeof(RankRec) +
         ((size_t)P + cap) * NW * 4 + (size_t)(Lmax + 1) * 4;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct EaState {
  ebic_params_t p{};
  int32_t S = 0, J = 0, ncombo = 0, WC = 0, Pp = 0, hmask = 0, kB = 64;
  long long entries = 0;
  DevBuf seq, len, inc, dec, fit, lnf;
  DevBuf tkey, tref;
  DevBuf rec;
  int32_t rec_bytes = 0;
  DevBuf list_ref, list_f;
  DevBuf pow_tab, pow_off, c_over_L;
  DevBuf ctl, gather;
  HostBuf h_ctl, h_gather;
  size_t smem_build = 0, smem_rank = 0;
  int32_t rank_nw = 0;           // k_rank_warp<rank_nw> (0: k_rank)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  EaDev dev{};
  ArchivePop apop{};
  EvalArgs eargs{};
  ebic_eval_tuning_t tuning{};   // evaluation shape chosen at Step 1
  bool initialised = false;
  // offspring screening
  ebic_surrogate_ctx* sur = nullptr;   // attached surrogate (EBIC_SCREEN_SURROGATE)
  long long var_rows = 0;
  DevBuf var_seq, var_len, var_score, act;
  int32_t launches_per_gen = 5;
  cudaStream_t side = nullptr;         // second branch of the generation graph
  cudaEvent_t fork_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // In-graph timing of k_build: two event-record nodes bracket it in the
  // graph; each replay points them at the next pair of a ring of events.
  int32_t tslots = 0;
  std::vector<cudaEvent_t> tev;        // [2 * tslots]: begin, end per slot
  cudaGraphNode_t tnode[2] = {nullptr, nullptr};
  long long tlaunched = 0, tharvested = 0, tcount = 0;
  double tsum_ms = 0.0;

  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    for (cudaEvent_t& e : fork_ev) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    for (cudaEvent_t& e : tev)
      if (e) cudaEventDestroy(e);
    tev.clear();
    tslots = 0;
    if (side) cudaStreamDestroy(side);
    side = nullptr;
    for (DevBuf* b : {&seq, &len, &inc, &dec, &fit, &lnf, &tkey, &tref, &rec, &list_ref,
                      &list_f, &pow_tab, &pow_off, &c_over_L, &ctl, &gather, &var_seq, &var_len,
                      &var_score, &act})
      b->release();
    sur = nullptr;
    h_ctl.release();
    h_gather.release();
    initialised = false;
  }
};

void ea_release(ebic_ctx* h) {
  if (h->ea) {
    h->ea->release();
    delete h->ea;
    h->ea = nullptr;
  }
}

static ebic_status validate(const ebic_ctx* h, const ebic_params_t* p) {
  if (!p) return fail(EBIC_ERR_ARG, "null params");
  if (h->C > 8192) return fail(EBIC_ERR_ARG, "the EA supports at most 8192 columns");
  if (p->pop_size < 2 || p->pop_size > 4096)
    return fail(EBIC_ERR_ARG, "pop_size %d outside [2, 4096]", p->pop_size);
  if (p->len_min < 1 || p->len_max < p->len_min || p->len_max > h->C ||
      p->len_max > EBIC_MAX_EA_LEN)
    return fail(EBIC_ERR_ARG, "lengths [%d, %d] invalid for %d columns (max %d)", p->len_min,
                p->len_max, h->C, EBIC_MAX_EA_LEN);
  if (p->iterations < 0) return fail(EBIC_ERR_ARG, "negative iterations");
  if (p->toprank_size < 1 || p->toprank_size > 4096)
    return fail(EBIC_ERR_ARG, "toprank_size %d outside [1, 4096]", p->toprank_size);
  if (p->tournament_k < 1 || p->tournament_k > EBIC_MAX_TOURNAMENT)
    return fail(EBIC_ERR_ARG, "tournament_k %d outside [1, %d]", p->tournament_k,
                EBIC_MAX_TOURNAMENT);
  if (p->support_mode != EBIC_SUPPORT_INC && p->support_mode != EBIC_SUPPORT_INC_PLUS_DEC)
    return fail(EBIC_ERR_ARG, "bad support mode");
  if (!(p->overlap_tau >= 0.0 && p->overlap_tau <= 1.0)) return fail(EBIC_ERR_ARG, "tau");
  if (!(p->elite_frac >= 0.0 && p->elite_frac <= 1.0)) return fail(EBIC_ERR_ARG, "elite_frac");
  if (!(p->penalty_base >= 1.0 && p->penalty_base < 1e6)) return fail(EBIC_ERR_ARG, "base");
  if (!(p->p_crossover >= 0.0 && p->p_crossover <= 1.0)) return fail(EBIC_ERR_ARG, "p_crossover");
  return EBIC_OK;
}

// Attempt records of one Steps 2-5 generation: k_spec, or (screening) the
// candidates, their scores and the pick.  Returns the launch count in *n.
// With `mid` (profiling, screening only), events mid[0] and mid[1] are
// recorded after the candidates and after their scores.
static ebic_status launch_records(EaState* st, cudaStream_t s, int* n,
                                  cudaEvent_t* mid = nullptr) {
  const EaDev& d = st->dev;
  const long long jc = (long long)st->J * st->ncombo;
  if (d.V <= 1) {
    k_spec<false, false><<<(unsigned)((jc + 127) / 128), 128, 0, s>>>(d);
    *n = 1;
    return EBIC_OK;
  }
  const long long rows = jc * d.V;
  k_spec<false, true><<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(d);
  if (mid) cudaEventRecord(mid[0], s);
  int ns = 1;
  if (d.screen == EBIC_SCREEN_SURROGATE) {
    EBIC_TRY(sur_forward_scores(st->sur, d.var_seq, d.var_len, d.S, (int32_t)rows, st->act.ptr,
                                d.var_score, s, &ns));
  } else {
    k_pseudo_score<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(d);
  }
  if (mid) cudaEventRecord(mid[1], s);
  k_pick<<<(unsigned)((jc + 127) / 128), 128, 0, s>>>(d);
  *n = 2 + ns;
  EBIC_CUDA_TRY(cudaGetLastError());
  return EBIC_OK;
}

static void launch_rank(const EaState* st, cudaStream_t s) {
  if (st->rank_nw == 4)
    k_rank_warp<4><<<1, kRankWarpThreads, st->smem_rank, s>>>(st->dev, st->Pp);
  else if (st->rank_nw == 8)
    k_rank_warp<8><<<1, kRankWarpThreads, st->smem_rank, s>>>(st->dev, st->Pp);
  else
    k_rank<<<1, kRankThreads, st->smem_rank, s>>>(st->dev, st->Pp);
}

// One generation g as captured for replay.  Step 3 first; then tabu
// insertion beside the evaluation; Step 5 of g as soon as the evaluation is
// done, beside the attempt records of g + 1 (which need g's fitness and tabu
// list, not its top-rank list, which only the next Step 2 reads; tabu
// insertion and the records take the generation from spec_gen, not from
// the counter Step 5 advances):
//
//   k_build(g) -+- eval(g) -+- k_rank(g) ---------------+- (next replay)
//               |           +---------+                 |
//               +- k_tabu_insert(g) --+- records(g + 1) -+
//
// The records of generation 1 are built at the end of ebic_run_init.
static ebic_status launch_generation(ebic_ctx* h, EaState* st, cudaStream_t s) {
  const EaDev& d = st->dev;
  cudaStream_t s2 = st->side;
  if (st->tslots) EBIC_CUDA_TRY(cudaEventRecordWithFlags(st->tev[0], s, cudaEventRecordExternal));
  k_build<false><<<1, kBuildThreads, st->smem_build, s>>>(d, st->hmask, st->kB);
  if (st->tslots) EBIC_CUDA_TRY(cudaEventRecordWithFlags(st->tev[1], s, cudaEventRecordExternal));
  EBIC_CUDA_TRY(cudaEventRecord(st->fork_ev[0], s));
  EBIC_CUDA_TRY(cudaStreamWaitEvent(s2, st->fork_ev[0], 0));
  k_tabu_insert<<<(unsigned)((st->p.pop_size + 255) / 256), 256, 0, s2>>>(d);
  EBIC_CUDA_TRY(cudaGetLastError());
  EBIC_TRY(eval_archive(h, st->apop, st->eargs, s));
  // Step 5 right after the evaluation (it needs the fitness, not the tabu
  // list); the next attempt records after both
  EBIC_CUDA_TRY(cudaEventRecord(st->fork_ev[1], s));
  EBIC_CUDA_TRY(cudaStreamWaitEvent(s2, st->fork_ev[1], 0));
  launch_rank(st, s);
  EBIC_CUDA_TRY(cudaGetLastError());
  int nrec = 0;
  EBIC_TRY(launch_records(st, s2, &nrec));
  st->launches_per_gen = nrec + 4;
  EBIC_CUDA_TRY(cudaEventRecord(st->fork_ev[3], s2));
  EBIC_CUDA_TRY(cudaStreamWaitEvent(s, st->fork_ev[3], 0));
  return EBIC_OK;
}

static ebic_status read_ctl(EaState* st, cudaStream_t s, Ctl* out) {
  EBIC_CUDA_TRY(cudaMemcpyAsync(st->h_ctl.ptr, st->ctl.ptr, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  EBIC_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(out, st->h_ctl.ptr, sizeof(Ctl));
  return EBIC_OK;
}

static void fill_stats(const Ctl& c, ebic_stats_t* stats) {
  if (!stats) return;
  stats->generations_done = c.gens_done;
  stats->stop_reason = c.stop_reason;
  stats->tabu_hits_total = c.hits_total;
  stats->attempts_total = c.attempts_total;
  stats->evaluations_total = c.evals_total;
  stats->last_gen_hits = c.last_hits;
  stats->toprank_n = c.n_top;
  stats->exact_tournaments = c.exact_total;
}

static ebic_status run_init(ebic_ctx* h, const ebic_params_t* p) {
  EBIC_TRY(validate(h, p));
  ea_release(h);
  EaState* st = new EaState();
  h->ea = st;
  st->p = *p;
  const int32_t P = p->pop_size, k = p->tournament_k, T = p->toprank_size;
  st->S = p->len_max;
  st->J = 2 * P + 1;
  st->ncombo = k * k;
  st->WC = (h->C + 31) / 32;
  st->Pp = 1;
  while (st->Pp < P) st->Pp <<= 1;
  int H = 1;
  while (H < 2 * P) H <<= 1;
  st->hmask = H - 1;
  st->entries = (long long)(p->iterations + 1) * P;
  const cudaStream_t s = h->stream;
  const size_t E = (size_t)st->entries;
  EBIC_TRY(st->seq.reserve(E * st->S * sizeof(uint16_t)));
  EBIC_TRY(st->len.reserve(E * sizeof(int32_t)));
  EBIC_TRY(st->inc.reserve(E * sizeof(uint32_t)));
  EBIC_TRY(st->dec.reserve(E * sizeof(uint32_t)));
  EBIC_TRY(st->fit.reserve(E * sizeof(double)));
  EBIC_TRY(st->lnf.reserve(E * sizeof(float)));
  unsigned long long tcap = 1;
  while (tcap < 2ull * E) tcap <<= 1;
  EBIC_TRY(st->tkey.reserve(tcap * sizeof(unsigned long long)));
  EBIC_TRY(st->tref.reserve(tcap * sizeof(int32_t)));
  EBIC_CUDA_TRY(cudaMemsetAsync(st->tkey.ptr, 0, tcap * sizeof(unsigned long long), s));
  EBIC_CUDA_TRY(cudaMemsetAsync(st->dec.ptr, 0, E * sizeof(uint32_t), s));
  // attempt records: sized for the larger (Steps 2-5) layout
  st->rec_bytes = rec_layout(k, st->S, false, bit_words((h->C + 31) / 32)).bytes;
  EBIC_TRY(st->rec.reserve((size_t)st->J * st->rec_bytes));
  EBIC_TRY(st->list_ref.reserve((size_t)(T + P) * sizeof(int32_t)));
  EBIC_TRY(st->list_f.reserve((size_t)(T + P) * sizeof(double)));
  EBIC_TRY(st->ctl.reserve(sizeof(Ctl)));
  EBIC_TRY(st->h_ctl.reserve(sizeof(Ctl)));
  EBIC_CUDA_TRY(cudaMemsetAsync(st->ctl.ptr, 0, sizeof(Ctl), s));

  // Crowding-penalty table base^(S / L) (host C library pow), L in
  // [len_min, len_max], S in [0, L * P]; and log(base) / L as float.
  std::vector<long long> off((size_t)p->len_max + 1, 0);
  long long total = 0;
  for (int L = p->len_min; L <= p->len_max; ++L) {
    off[L] = total;
    total += (long long)L * P + 1;
  }
  std::vector<double> tab((size_t)total);
  for (int L = p->len_min; L <= p->len_max; ++L)
    for (long long S = 0; S <= (long long)L * P; ++S)
      tab[(size_t)(off[L] + S)] = std::pow(p->penalty_base, (double)S / (double)L);
  std::vector<float> cl((size_t)p->len_max + 1, 0.f);
  for (int L = 1; L <= p->len_max; ++L) cl[L] = (float)(std::log(p->penalty_base) / (double)L);
  EBIC_TRY(st->pow_tab.reserve(tab.size() * sizeof(double)));
  EBIC_TRY(st->pow_off.reserve(off.size() * sizeof(long long)));
  EBIC_TRY(st->c_over_L.reserve(cl.size() * sizeof(float)));
  EBIC_CUDA_TRY(cudaMemcpyAsync(st->pow_tab.ptr, tab.data(), tab.size() * sizeof(double),
                                cudaMemcpyHostToDevice, s));
  EBIC_CUDA_TRY(cudaMemcpyAsync(st->pow_off.ptr, off.data(), off.size() * sizeof(long long),
                                cudaMemcpyHostToDevice, s));
  EBIC_CUDA_TRY(cudaMemcpyAsync(st->c_over_L.ptr, cl.data(), cl.size() * sizeof(float),
                                cudaMemcpyHostToDevice, s));

  EaDev& d = st->dev;
  d.P = P;
  d.C = h->C;
  d.S = st->S;
  d.Lmin = p->len_min;
  d.Lmax = p->len_max;
  d.k = k;
  d.T = T;
  d.mode = p->support_mode;
  d.J = st->J;
  d.ncombo = st->ncombo;
  d.WC = st->WC;
  d.tau = p->overlap_tau;
  d.elite_frac = p->elite_frac;
  d.pc = p->p_crossover;
  d.seed = p->seed;
  d.seq = st->seq.as<uint16_t>();
  d.len = st->len.as<int32_t>();
  d.fit = st->fit.as<double>();
  d.lnf = st->lnf.as<float>();
  d.tkey = st->tkey.as<unsigned long long>();
  d.tref = st->tref.as<int32_t>();
  d.tmask = tcap - 1;
  d.rec = st->rec.as<char>();
  d.rec_bytes = st->rec_bytes;
  d.list_ref = st->list_ref.as<int32_t>();
  d.list_f = st->list_f.as<double>();
  d.pow_tab = st->pow_tab.as<double>();
  d.pow_off = st->pow_off.as<long long>();
  d.c_over_L = st->c_over_L.as<float>();
  d.ctl = st->ctl.as<Ctl>();

  // Offspring screening: candidate buffers (zeroed, so that a pass over rows
  // no k_spec has written yet reads empty series), scores, activations.
  d.V = 1;
  d.screen = EBIC_SCREEN_OFF;
  if (h->screen_mode != EBIC_SCREEN_OFF && h->screen_v > 1) {
    const int32_t V = h->screen_v;
    if (h->screen_mode == EBIC_SCREEN_SURROGATE && !h->screen_sur)
      return fail(EBIC_ERR_STATE, "surrogate screening without a surrogate");
    const long long rows = (long long)st->J * st->ncombo * V;
    if (rows > (1ll << 22))
      return fail(EBIC_ERR_ARG, "screening needs %lld candidate rows per generation (max %lld)",
                  rows, 1ll << 22);
    EBIC_TRY(st->var_seq.reserve_zeroed((size_t)rows * st->S * sizeof(uint16_t), s));
    EBIC_TRY(st->var_len.reserve_zeroed((size_t)rows * sizeof(int32_t), s));
    EBIC_TRY(st->var_score.reserve((size_t)rows * sizeof(float)));
    if (h->screen_mode == EBIC_SCREEN_SURROGATE) st->sur = h->screen_sur;
    st->var_rows = rows;
    d.V = V;
    d.screen = h->screen_mode;
    d.var_seq = st->var_seq.as<uint16_t>();
    d.var_len = st->var_len.as<int32_t>();
    d.var_score = st->var_score.as<float>();
  }

  st->apop.seq = d.seq;
  st->apop.len = d.len;
  st->apop.stride = st->S;
  st->apop.P = P;
  st->apop.gen = &d.ctl->gen;
  st->apop.stop = &d.ctl->stop;
  EvalArgs& a = st->eargs;
  a.P = P;
  a.sigma = p->sigma;
  a.mode = p->support_mode;
  a.want_dec = p->support_mode == EBIC_SUPPORT_INC_PLUS_DEC;
  a.inc = st->inc.as<uint32_t>();
  a.dec = a.want_dec ? st->dec.as<uint32_t>() : nullptr;
  a.fit = d.fit;
  a.lnf = d.lnf;

  // build: hash set / key list + pen + cL + filter, then two record buffers of kB attempts
  const size_t fixed = (size_t)H * (sizeof(unsigned long long) + sizeof(int32_t)) +
                       (size_t)h->C * sizeof(uint32_t) +
                       (size_t)(p->len_max + 2) * sizeof(float) + 16 +
                       (size_t)kFilterWords * sizeof(uint32_t) + 128;
  st->kB = 64;
  while (st->kB > 2 && fixed + 2 * (size_t)st->kB * st->rec_bytes > 200 * 1024) st->kB >>= 1;
  st->smem_build = fixed + 2 * (size_t)st->kB * st->rec_bytes;
  const size_t cap = (size_t)T + P;
  st->smem_rank = (size_t)st->Pp * (sizeof(unsigned long long) + sizeof(int32_t)) +
                  cap * (2 * sizeof(double) + 2 * sizeof(int32_t)) + ((cap + 15) & ~(size_t)15) +
                  (size_t)st->WC * sizeof(uint32_t);
  // Step 5 by one warp from shared bitsets when the columns and sizes allow
  st->rank_nw = 0;
  const int rnw = bit_words(st->WC);
  if (rnw && st->Pp <= 8 * kRankWarpThreads) {    // the register sort holds 8 per thread
    const size_t need = rank_warp_smem(P, st->Pp, T, p->len_max, rnw);
    if (need <= 200 * 1024) {
      st->rank_nw = rnw;
      st->smem_rank = need;
    }
  }
  if (st->smem_build > 220 * 1024 || st->smem_rank > 220 * 1024)
    return fail(EBIC_ERR_ARG, "population / top-rank sizes need more shared memory than a CTA has "
                              "(build %zu B, rank %zu B)", st->smem_build, st->smem_rank);
  EBIC_CUDA_TRY(cudaFuncSetAttribute(k_build<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)st->smem_build));
  EBIC_CUDA_TRY(cudaFuncSetAttribute(k_build<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)st->smem_build));
  if (st->rank_nw == 4)
    EBIC_CUDA_TRY(cudaFuncSetAttribute(k_rank_warp<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)st->smem_rank));
  else if (st->rank_nw == 8)
    EBIC_CUDA_TRY(cudaFuncSetAttribute(k_rank_warp<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)st->smem_rank));
  else
    EBIC_CUDA_TRY(cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)st->smem_rank));

  // The pair table pays for itself over a run; build it when it fits.
  if (h->path != EBIC_PATH_GATHER && !h->LT) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t need = (size_t)h->C * h->C * h->W * sizeof(uint32_t);
    if (need < free_b / 2) EBIC_TRY(build_pair_table(h, s));
  }

  // Step 1: initial population, evaluation (autotuned once), top-rank list.
  const EaDev& dd = st->dev;
  const unsigned sblocks = (unsigned)((st->J + 127) / 128);
  k_spec<true, false><<<sblocks, 128, 0, s>>>(dd);
  k_build<true><<<1, kBuildThreads, st->smem_build, s>>>(dd, st->hmask, st->kB);
  k_tabu_insert<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(dd);
  count_launches(3);
  EBIC_CUDA_TRY(cudaGetLastError());
  Ctl c{};
  EBIC_TRY(read_ctl(st, s, &c));
  // The evaluation of the initial population, with the launch shape set by
  // hand (a nonzero kernel), else with the one the autotuner picks on it
  // (its candidates are evaluations of that population).  Either way any
  // scratch the shape needs is allocated here, before the capture below.
  const ebic_eval_tuning_t user_tuning = h->tuning;
  if (!c.stop) {
    if (user_tuning.kernel != 0) {
      EBIC_TRY(eval_archive(h, st->apop, a, s));
    } else {
      float us = 0.f;
      EBIC_TRY(autotune_archive(h, st->apop, a, s, &us));
    }
  }
  launch_rank(st, s);
  count_launches(1);
  EBIC_CUDA_TRY(cudaGetLastError());
  // attempt records of generation 1
  int nrec = 0;
  EBIC_TRY(launch_records(st, s, &nrec));
  count_launches((uint64_t)nrec);

  // One generation (Steps 2-5) captured as a graph for replay.
  st->tuning = h->tuning;
  EBIC_CUDA_TRY(cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking));
  for (cudaEvent_t& e : st->fork_ev) EBIC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (h->ktime_slots > 0) {
    st->tev.assign(2 * (size_t)h->ktime_slots, nullptr);
    st->tslots = h->ktime_slots;
    for (cudaEvent_t& e : st->tev) EBIC_CUDA_TRY(cudaEventCreate(&e));
  }
  EBIC_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  ebic_status cap_st = launch_generation(h, st, s);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  h->tuning = user_tuning;
  if (cap_st != EBIC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return cap_st;
  }
  EBIC_CUDA_TRY(ce);
  st->graph = graph;
  if (st->tslots) {
    size_t n = 0;
    EBIC_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    EBIC_CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      EBIC_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
      if (t != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t e = nullptr;
      EBIC_CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nd, &e));
      for (int j = 0; j < 2; ++j)
        if (e == st->tev[j]) st->tnode[j] = nd;
    }
    if (!st->tnode[0] || !st->tnode[1])
      return fail(EBIC_ERR_DEVICE, "the captured generation has no timing nodes");
  }
  EBIC_CUDA_TRY(cudaGraphInstantiate(&st->exec, graph, 0));
  EBIC_CUDA_TRY(cudaStreamSynchronize(s));
  st->initialised = true;
  return EBIC_OK;
}

// Adds the k_build time of timing slot `slot` to the running sum (waits for
// that replay to finish).
static ebic_status harvest_timing(EaState* st, long long slot) {
  cudaEvent_t a = st->tev[2 * (size_t)(slot % st->tslots)];
  cudaEvent_t b = st->tev[2 * (size_t)(slot % st->tslots) + 1];
  EBIC_CUDA_TRY(cudaEventSynchronize(b));
  float ms = 0.f;
  EBIC_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
  st->tsum_ms += ms;
  st->tcount += 1;
  return EBIC_OK;
}

// One replay of the generation graph; with in-graph timing on, its two event
// nodes first move to the next slot of the ring (harvesting the replay that
// used the slot before).
static ebic_status graph_launch(EaState* st, cudaStream_t s) {
  if (st->tslots) {
    if (st->tlaunched - st->tharvested >= st->tslots) EBIC_TRY(harvest_timing(st, st->tharvested++));
    const size_t k = 2 * (size_t)(st->tlaunched % st->tslots);
    EBIC_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(st->exec, st->tnode[0], st->tev[k]));
    EBIC_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(st->exec, st->tnode[1], st->tev[k + 1]));
  }
  EBIC_CUDA_TRY(cudaGraphLaunch(st->exec, s));
  if (st->tslots) st->tlaunched += 1;    // a slot counts once its replay is queued
  return EBIC_OK;
}

static ebic_status run_step(ebic_ctx* h, int32_t generations, ebic_stats_t* stats) {
  EaState* st = h->ea;
  if (!st || !st->initialised) return fail(EBIC_ERR_STATE, "ebic_run_init has not run");
  if (generations < 0) return fail(EBIC_ERR_ARG, "negative generation count");
  const cudaStream_t s = h->stream;
  Ctl c{};
  EBIC_TRY(read_ctl(st, s, &c));
  if (!c.stop && c.gens_done + generations > st->p.iterations)
    return fail(EBIC_ERR_STATE, "the run was sized for %d generations (%d done, %d asked)",
                st->p.iterations, c.gens_done, generations);
  int32_t left = c.stop ? 0 : generations;
  while (left > 0) {
    const int32_t chunk = std::min<int32_t>(left, 64);
    for (int32_t i = 0; i < chunk; ++i) EBIC_TRY(graph_launch(st, s));
    count_launches((uint64_t)chunk * st->launches_per_gen);
    left -= chunk;
    EBIC_TRY(read_ctl(st, s, &c));
    if (c.stop) break;
  }
  EBIC_TRY(read_ctl(st, s, &c));
  fill_stats(c, stats);
  if (c.stop_reason == 3) return fail(EBIC_ERR_DEVICE, "internal EA error (code 3)");
  if (c.stop_reason == 4)
    return fail(EBIC_ERR_TIMEOUT, "a bounded wait for streamed attempt records expired");
  return EBIC_OK;
}

ebic_status ea_archive(ebic_ctx* h, const uint16_t** seq, const int32_t** len, const double** fit,
                       long long* n, int32_t* stride) {
  EaState* st = h->ea;
  if (!st || !st->initialised) return fail(EBIC_ERR_STATE, "the handle has no run");
  Ctl c{};
  EBIC_TRY(read_ctl(st, h->stream, &c));
  *seq = st->seq.as<uint16_t>();
  *len = st->len.as<int32_t>();
  *fit = st->fit.as<double>();
  *stride = st->S;
  // generations 0 .. c.gen - 1 are evaluated (c.gen counts Step 1 as one)
  *n = std::min<long long>((long long)c.gen * st->p.pop_size, st->entries);
  return EBIC_OK;
}

// Gathers n records (archive entries refs[i], or g * P + i when refs is
// null) into packed rows: seq [n][S], then len, inc, dec (int32) and fitness.
__global__ void __launch_bounds__(256) k_gather(EaDev d, const int32_t* refs, long long first,
                                                int n, const uint32_t* inc, const uint32_t* dec,
                                                uint16_t* o_seq, int32_t* o_len, uint32_t* o_inc,
                                                uint32_t* o_dec, double* o_fit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long r = refs ? (long long)refs[i] : first + i;
  const int L = d.len[r];
  for (int c = 0; c < d.S; ++c) o_seq[(size_t)i * d.S + c] = c < L ? d.seq[(size_t)r * d.S + c] : 0;
  o_len[i] = L;
  o_inc[i] = inc[r];
  o_dec[i] = dec[r];
  o_fit[i] = d.fit[r];
}

// Steps 2-5 replayed on the caller's stream without waiting or reading back.
static ebic_status run_step_async(ebic_ctx* h, int32_t generations, cudaStream_t s) {
  EaState* st = h->ea;
  if (!st || !st->initialised) return fail(EBIC_ERR_STATE, "ebic_run_init has not run");
  if (generations < 0) return fail(EBIC_ERR_ARG, "negative generation count");
  for (int32_t i = 0; i < generations; ++i) EBIC_TRY(graph_launch(st, s));
  count_launches((uint64_t)generations * st->launches_per_gen);
  return EBIC_OK;
}

// One generation as five separate launches with events between them.
// One generation as separate launches with events between them, in the
// order of the graph's dependencies: Step 3, tabu insertion, evaluation,
// Step 5, then the next generation's attempt records (reported first).
static ebic_status run_step_profiled(ebic_ctx* h, float* us, cudaStream_t s) {
  EaState* st = h->ea;
  if (!st || !st->initialised) return fail(EBIC_ERR_STATE, "ebic_run_init has not run");
  cudaEvent_t ev[8];
  for (int i = 0; i < 8; ++i) EBIC_CUDA_TRY(cudaEventCreate(&ev[i]));
  const EaDev& d = st->dev;
  cudaEventRecord(ev[0], s);
  k_build<false><<<1, kBuildThreads, st->smem_build, s>>>(d, st->hmask, st->kB);
  cudaEventRecord(ev[1], s);
  k_tabu_insert<<<(unsigned)((st->p.pop_size + 255) / 256), 256, 0, s>>>(d);
  cudaEventRecord(ev[2], s);
  const ebic_eval_tuning_t user = h->tuning;
  h->tuning = st->tuning;
  ebic_status es = eval_archive(h, st->apop, st->eargs, s);
  h->tuning = user;
  cudaEventRecord(ev[3], s);
  launch_rank(st, s);
  cudaEventRecord(ev[4], s);
  int nrec = 0;
  const bool screened = d.V > 1;
  ebic_status rs = launch_records(st, s, &nrec, screened ? ev + 6 : nullptr);
  cudaEventRecord(ev[5], s);
  count_launches((uint64_t)(3 + nrec));
  cudaError_t e = cudaEventSynchronize(ev[5]);
  // kernel_us order: records, build, tabu insertion, evaluation, rank; then,
  // when screening, the records stage split into candidates, scores, pick
  const int from[5] = {4, 0, 1, 2, 3};
  for (int i = 0; i < 5 && us; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[from[i]], ev[from[i] + 1]);
    us[i] = ms * 1000.f;
  }
  if (us) {
    us[5] = us[6] = us[7] = 0.f;
    if (screened && rs == EBIC_OK) {
      const cudaEvent_t* seg[4] = {&ev[4], &ev[6], &ev[7], &ev[5]};
      for (int i = 0; i < 3; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, *seg[i], *seg[i + 1]);
        us[5 + i] = ms * 1000.f;
      }
    }
  }
  for (int i = 0; i < 8; ++i) cudaEventDestroy(ev[i]);
  EBIC_TRY(rs);
  EBIC_TRY(es);
  EBIC_CUDA_TRY(e);
  return EBIC_OK;
}

static ebic_status get_records(ebic_ctx* h, bool toprank, int32_t* offsets, int32_t* cols,
                               double* fitness, uint32_t* inc, uint32_t* dec, int32_t* inout_n) {
  EaState* st = h->ea;
  if (!st || !st->initialised) return fail(EBIC_ERR_STATE, "ebic_run_init has not run");
  if (!offsets || !cols || !inout_n || *inout_n < 0) return fail(EBIC_ERR_ARG, "null pointer");
  const cudaStream_t s = h->stream;
  Ctl c{};
  EBIC_TRY(read_ctl(st, s, &c));
  const int32_t P = st->p.pop_size, S = st->S;
  // the list, or the last evaluated generation (c.gen - 1)
  const int32_t avail = toprank ? c.n_top : (c.gen > 0 ? P : 0);
  const int32_t n = std::min<int32_t>(*inout_n, avail);
  offsets[0] = 0;
  *inout_n = n;
  if (n == 0) return EBIC_OK;
  const size_t row = (size_t)S * sizeof(uint16_t);
  const size_t bytes = (size_t)n * (row + 3 * sizeof(int32_t) + sizeof(double));
  EBIC_TRY(st->gather.reserve(bytes));
  EBIC_TRY(st->h_gather.reserve(bytes));
  // regions by decreasing element size, so every one is aligned:
  // fitness [n] (8 B) | len, inc, dec [n] (4 B) | seq [n][S] (2 B)
  char* dbase = static_cast<char*>(st->gather.ptr);
  double* o_fit = reinterpret_cast<double*>(dbase);
  int32_t* o_len = reinterpret_cast<int32_t*>(o_fit + n);
  uint32_t* o_inc = reinterpret_cast<uint32_t*>(o_len + n);
  uint32_t* o_dec = o_inc + n;
  uint16_t* o_seq = reinterpret_cast<uint16_t*>(o_dec + n);
  k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      st->dev, toprank ? st->list_ref.as<int32_t>() : nullptr, (long long)(c.gen - 1) * P, n,
      st->inc.as<uint32_t>(), st->dec.as<uint32_t>(), o_seq, o_len, o_inc, o_dec, o_fit);
  count_launches(1);
  EBIC_CUDA_TRY(cudaGetLastError());
  EBIC_CUDA_TRY(cudaMemcpyAsync(st->h_gather.ptr, st->gather.ptr, bytes, cudaMemcpyDeviceToHost, s));
  EBIC_CUDA_TRY(cudaStreamSynchronize(s));
  const double* h_fit = static_cast<const double*>(st->h_gather.ptr);
  const int32_t* h_len = reinterpret_cast<const int32_t*>(h_fit + n);
  const uint32_t* h_inc = reinterpret_cast<const uint32_t*>(h_len + n);
  const uint32_t* h_dec = h_inc + n;
  const uint16_t* h_seq = reinterpret_cast<const uint16_t*>(h_dec + n);
  for (int32_t i = 0; i < n; ++i) {
    const int32_t L = h_len[i];
    for (int32_t t = 0; t < L; ++t) cols[offsets[i] + t] = h_seq[(size_t)i * S + t];
    offsets[i + 1] = offsets[i] + L;
    if (fitness) fitness[i] = h_fit[i];
    if (inc) inc[i] = h_inc[i];
    if (dec) dec[i] = h_dec[i];
  }
  return EBIC_OK;
}

}  // namespace ebic

using namespace ebic;

extern "C" {

void ebic_default_params(ebic_params_t* p) {
  if (!p) return;
  p->pop_size = 100;
  p->len_min = 2;
  p->len_max = 6;
  p->iterations = 10;
  p->sigma = 10;
  p->toprank_size = 100;
  p->tournament_k = 2;
  p->support_mode = EBIC_SUPPORT_INC;
  p->overlap_tau = 0.5;
  p->elite_frac = 0.25;
  p->penalty_base = 1.2;
  p->p_crossover = 0.5;
  p->seed = 0;
}

ebic_status ebic_run_init(ebic_handle h, const ebic_params_t* p) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  ebic_status st = run_init(h, p);
  if (st != EBIC_OK) ea_release(h);
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  return st;
}

ebic_status ebic_run_step(ebic_handle h, int32_t generations, ebic_stats_t* stats) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  return run_step(h, generations, stats);
}

ebic_status ebic_run_step_async(ebic_handle h, int32_t generations, void* stream) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  return run_step_async(h, generations, static_cast<cudaStream_t>(stream));
}

ebic_status ebic_run_step_profiled(ebic_handle h, float* kernel_us) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  return run_step_profiled(h, kernel_us, h->stream);
}

ebic_status ebic_set_kernel_timing(ebic_handle h, int32_t slots) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (slots < 0 || slots > (1 << 20)) return fail(EBIC_ERR_ARG, "timing slots %d outside [0, 2^20]", slots);
  h->ktime_slots = slots;
  return EBIC_OK;
}

ebic_status ebic_read_kernel_timing(ebic_handle h, int32_t reset, double* mean_us, long long* count) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  EaState* st = h->ea;
  if (!st || !st->initialised) return fail(EBIC_ERR_STATE, "ebic_run_init has not run");
  if (!st->tslots) return fail(EBIC_ERR_STATE, "the run was started without kernel timing");
  while (st->tharvested < st->tlaunched) EBIC_TRY(harvest_timing(st, st->tharvested++));
  if (mean_us) *mean_us = st->tcount ? 1e3 * st->tsum_ms / (double)st->tcount : 0.0;
  if (count) *count = st->tcount;
  if (reset) {
    st->tsum_ms = 0.0;
    st->tcount = 0;
  }
  return EBIC_OK;
}

ebic_status ebic_run_screen(ebic_handle h, ebic_surrogate s, int32_t oversample, int32_t mode) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  if (oversample < 1 || oversample > 16)
    return fail(EBIC_ERR_ARG, "oversample %d outside [1, 16]", oversample);
  if (mode != EBIC_SCREEN_OFF && mode != EBIC_SCREEN_SURROGATE && mode != EBIC_SCREEN_PSEUDO)
    return fail(EBIC_ERR_ARG, "bad screening mode %d", mode);
  if (mode == EBIC_SCREEN_SURROGATE && !s) return fail(EBIC_ERR_ARG, "surrogate mode needs a surrogate");
  if (mode == EBIC_SCREEN_SURROGATE && sur_columns(s) != h->C)
    return fail(EBIC_ERR_ARG, "the surrogate has %d columns, the matrix %d", sur_columns(s), h->C);
  // the handle holds one reference to its screening surrogate
  if (h->screen_sur) sur_attach(h->screen_sur, -1);
  h->screen_sur = mode == EBIC_SCREEN_SURROGATE ? s : nullptr;
  if (h->screen_sur) sur_attach(h->screen_sur, +1);
  h->screen_v = oversample;
  h->screen_mode = mode;
  return EBIC_OK;
}

ebic_status ebic_get_toprank(ebic_handle h, int32_t* offsets, int32_t* cols, double* fitness,
                             uint32_t* inc, int32_t* inout_n) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  return get_records(h, true, offsets, cols, fitness, inc, nullptr, inout_n);
}

ebic_status ebic_get_population(ebic_handle h, int32_t* offsets, int32_t* cols, uint32_t* inc,
                                uint32_t* dec, double* fitness, int32_t* inout_n) {
  if (!h) return fail(EBIC_ERR_ARG, "null handle");
  return get_records(h, false, offsets, cols, fitness, inc, dec, inout_n);
}

ebic_status ebic_run_generations(ebic_handle h, const ebic_params_t* p, int32_t* out_offsets,
                                 int32_t* out_cols, double* out_fitness, int32_t* inout_n,
                                 ebic_stats_t* stats) {
  if (!h || !p) return fail(EBIC_ERR_ARG, "null pointer");
  EBIC_TRY(ebic_run_init(h, p));
  EBIC_TRY(ebic_run_step(h, p->iterations, stats));
  return ebic_get_toprank(h, out_offsets, out_cols, out_fitness, nullptr, inout_n);
}

}  // extern "C"
