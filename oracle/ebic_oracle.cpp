// EBIC CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
//
// A plain, slow, deliberately unoptimised restatement of what EBIC
// (Orzechowski, Sipper, Huang, Moore: "EBIC: an evolutionary-based parallel
// biclustering algorithm for pattern discovery", arXiv 1801.03039) computes.
// Only the test suite, the smoke check in __graft_entry__ and the CPU-baseline
// leg of bench.py may load this library.  The CUDA library never links,
// includes or calls anything here, and this file includes nothing from it.
//
// Every function follows one passage of the paper:
//   support          -- section "Motivation": #{k : a_kp < a_kq < a_kr ...}
//   fitness          -- Eq. (1)
//   CBF              -- Fig. 3 (offsets + column indices)
//   rows of a series -- Step 6 (and Step 7's negative-trend expansion)
//   tournament/penalty, mutations, crossover, tabu list, elitism,
//   top-rank list    -- section "EBIC Algorithm", Steps 1-5, and the paragraph
//                       on genetic operations and crowding (Fig. 1)
//   Philox-4x32-10   -- Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
//                       as easy as 1, 2, 3", SC'11 (the counter-based generator
//                       used for every random draw of the EA)
//   Step 7 expansion by approximate trends (or_rows_approx) -- the reading
//                       that at most e adjacent pairs of a row may break the
//                       order (the paper does not define "approximate")
//   offspring screening with pseudo scores (make_child, oversample > 1) --
//                       not in the paper: the test form of the learned
//                       pre-screen's candidate generation and pick; pinned by
//                       properties of its definition on single attempts
//                       (or_screen_attempt: candidate 0 is the plain child,
//                       candidates do not depend on V, scores follow the
//                       Philox counter layout, the pick rule) and by its
//                       oversample = 1 case, the plain algorithm
//
// Where the paper is silent the reading is stated next to the code.  Build
// flags: -O2 -fno-fast-math -ffp-contract=off (IEEE binary32/binary64,
// round-to-nearest-even, no fused multiply-add).
//
// Pins (tests/test_oracle_*.py): brute force and sort-based support on tiny
// matrices, the closed-form sum over all L-tuples, reversal/complement
// invariants, planted rows, hand values of Eq. (1), the CBF example of Fig. 3,
// Philox known-answer vectors, operator properties, hand-built top-rank
// cases, and one generation of Steps 2-3 listed attempt by attempt with the
// crowding counts each tournament sees (elites count, accepted children count
// before the next attempt, tabu hits do not).  The full EA trajectory has no
// external pin beyond these parts ("parity unpinned" for the trajectory as a
// whole).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::vector<int32_t> Seq;

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11).  Ten rounds of the Philox S-box on a
// 128-bit counter with a 64-bit key; the key is bumped by the Weyl constants
// before every round after the first.
// ---------------------------------------------------------------------------
const uint32_t kPhiloxM0 = 0xD2511F53u;
const uint32_t kPhiloxM1 = 0xCD9E8D57u;
const uint32_t kPhiloxW0 = 0x9E3779B9u;
const uint32_t kPhiloxW1 = 0xBB67AE85u;

void philox_round(uint32_t x[4], const uint32_t k[2]) {
  uint64_t prod0 = (uint64_t)kPhiloxM0 * (uint64_t)x[0];
  uint64_t prod1 = (uint64_t)kPhiloxM1 * (uint64_t)x[2];
  uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
  uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
  uint32_t y0 = hi1 ^ x[1] ^ k[0];
  uint32_t y1 = lo1;
  uint32_t y2 = hi0 ^ x[3] ^ k[1];
  uint32_t y3 = lo0;
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k[0] += kPhiloxW0; k[1] += kPhiloxW1; }
    philox_round(x, k);
  }
  for (int i = 0; i < 4; ++i) out[i] = x[i];
}

// Draw number d of attempt j in generation g.  Counter = (j, g, d / 4, 0),
// key = the 64-bit seed split into (low, high) words; the draw is word d % 4.
uint32_t draw(uint64_t seed, int32_t g, int32_t j, int32_t d) {
  uint32_t ctr[4] = {(uint32_t)j, (uint32_t)g, (uint32_t)(d / 4), 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  philox4x32_10(ctr, key, out);
  return out[d % 4];
}

// An integer in [0, n) from a 32-bit draw: floor(r * n / 2^32).
uint32_t below(uint32_t r, uint32_t n) {
  return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

// ---------------------------------------------------------------------------
// Support (section "Motivation"): the number of rows k whose values follow the
// series strictly: a[k][s0] < a[k][s1] < ... (inc), or strictly fall (dec).
// Reading: IEEE `<` on the stored fp32 values, so equal values (+0 and -0
// included) break the chain and a NaN makes every comparison false.  A series
// of length 1 imposes no comparison, so every row counts.
// ---------------------------------------------------------------------------
void support_one(const float* A, int32_t R, int32_t C, const int32_t* s, int32_t L,
                 uint32_t* inc, uint32_t* dec) {
  uint32_t n_inc = 0, n_dec = 0;
  for (int32_t k = 0; k < R; ++k) {
    const float* row = A + (size_t)k * (size_t)C;
    bool rising = true, falling = true;
    for (int32_t i = 0; i + 1 < L; ++i) {
      float a = row[s[i]];
      float b = row[s[i + 1]];
      if (!(a < b)) rising = false;
      if (!(a > b)) falling = false;
    }
    if (rising) ++n_inc;
    if (falling) ++n_dec;
  }
  *inc = n_inc;
  *dec = n_dec;
}

// Eq. (1).  n = |I| rows, J = |J| columns, sigma = the expected minimal number
// of rows.  Readings: natural logarithm; binary64 arithmetic; 2^min(n-sigma,0)
// applied with ldexp (exact unless the result leaves the normal range).
double fitness_eq1(int64_t n, int32_t J, int32_t sigma) {
  if (n <= 1) return 0.0;
  int64_t e = n - (int64_t)sigma;
  if (e > 0) e = 0;
  if (e < -2000) e = -2000;  // 2^-2000 is already zero in binary64
  double t = std::ldexp(std::log((double)(n - 1)), (int)e);
  return t * (double)J;
}

// ---------------------------------------------------------------------------
// EA parameters and state (section "EBIC Algorithm").
// ---------------------------------------------------------------------------
struct Params {
  int32_t pop_size;         // P
  int32_t len_min;          // shortest series the EA builds
  int32_t len_max;          // longest series the EA builds (<= C)
  int32_t iterations;       // Steps 2-5 repetitions after Step 1
  int32_t sigma;            // Eq. (1)
  int32_t toprank_size;     // T
  int32_t tournament_k;     // entrants per tournament
  int32_t fitness_support;  // 0: |I| = inc; 1: |I| = inc + dec
  double overlap_tau;       // top-rank overlap threshold
  double elite_frac;        // Step 2 fraction of the top-rank list (1/4)
  double penalty_base;      // crowding penalty base (1.2)
  double p_crossover;       // probability that an attempt uses crossover
  uint64_t seed;
  int32_t oversample = 1;   // candidates per attempt (offspring screening, not in the paper)
};

struct Entry {
  Seq seq;
  double f;
  uint32_t inc, dec;
};

bool contains(const Seq& s, int32_t c) {
  for (size_t i = 0; i < s.size(); ++i)
    if (s[i] == c) return true;
  return false;
}

// The k-th (0-based) column, in increasing column order, that is not in s.
int32_t kth_absent(const Seq& s, int32_t C, uint32_t k) {
  for (int32_t c = 0; c < C; ++c) {
    if (contains(s, c)) continue;
    if (k == 0) return c;
    --k;
  }
  return -1;  // unreachable when k < C - |s|
}

// Step 1: a random series.  Reading: length uniform in [len_min, len_max],
// then distinct columns, each uniform among the columns not yet used.
Seq random_series(uint64_t seed, int32_t g, int32_t j, int32_t C, int32_t Lmin, int32_t Lmax) {
  int32_t L = Lmin + (int32_t)below(draw(seed, g, j, 0), (uint32_t)(Lmax - Lmin + 1));
  Seq s;
  for (int32_t i = 0; i < L; ++i) {
    uint32_t k = below(draw(seed, g, j, 1 + i), (uint32_t)(C - i));
    s.push_back(kth_absent(s, C, k));
  }
  return s;
}

// Crowding (paragraph on genetic operations, Step 3): the fitness of an
// entrant is divided by base^theta, theta = mean over its columns of the
// per-column usage counts.  Reading: division (the only reading that keeps the
// ranking independent of the logarithm base in Eq. (1)), theta = S / L as a
// binary64 quotient, base^theta by the C library's pow.
double penalized(double f, int64_t S, int32_t L, double base) {
  double theta = (double)S / (double)L;
  return f / std::pow(base, theta);
}

int64_t penalty_sum(const Seq& s, const std::vector<int64_t>& pen) {
  int64_t S = 0;
  for (size_t i = 0; i < s.size(); ++i) S += pen[s[i]];
  return S;
}

// Tournament selection (Step 3): the entrant with the largest penalised
// fitness wins; equal values go to the lowest population index.
int32_t tournament(const int32_t* entrants, int32_t k, const std::vector<Seq>& pop,
                   const std::vector<double>& f, const std::vector<int64_t>& pen, double base) {
  int32_t best = -1;
  double best_p = 0.0;
  for (int32_t t = 0; t < k; ++t) {
    int32_t i = entrants[t];
    double p = penalized(f[i], penalty_sum(pop[i], pen), (int32_t)pop[i].size(), base);
    if (best < 0 || p > best_p || (p == best_p && i < best)) {
      best = i;
      best_p = p;
    }
  }
  return best;
}

// Crossover (Fig. 1e; the figure is not available).  Reading: one-point
// crossover.  The child keeps the first cut_a columns of a and then the columns
// of b from position cut_b on, skipping columns it already holds, truncated to
// len_max columns.
Seq crossover(const Seq& a, const Seq& b, int32_t cut_a, int32_t cut_b, int32_t Lmax) {
  Seq child(a.begin(), a.begin() + cut_a);
  for (size_t i = (size_t)cut_b; i < b.size(); ++i) {
    if ((int32_t)child.size() >= Lmax) break;
    if (!contains(child, b[i])) child.push_back(b[i]);
  }
  return child;
}

enum { MUT_INSERT = 0, MUT_DELETE = 1, MUT_SWAP = 2, MUT_SUBSTITUTE = 3, MUT_NONE = 4 };

// The four mutations of Fig. 1a-d.  Reading: exactly one mutation per child,
// chosen uniformly among those that keep the series inside [len_min, len_max]
// with distinct columns (insert, delete, swap, substitute, in that order).
Seq mutate(const Seq& s, int32_t C, int32_t Lmin, int32_t Lmax, uint32_t r_type, uint32_t r1,
           uint32_t r2, int32_t* kind) {
  int32_t L = (int32_t)s.size();
  int32_t allowed[4];
  int32_t n_allowed = 0;
  if (L < Lmax && L < C) allowed[n_allowed++] = MUT_INSERT;
  if (L > Lmin) allowed[n_allowed++] = MUT_DELETE;
  if (L >= 2) allowed[n_allowed++] = MUT_SWAP;
  if (L < C) allowed[n_allowed++] = MUT_SUBSTITUTE;
  Seq out = s;
  if (n_allowed == 0) {
    *kind = MUT_NONE;
    return out;
  }
  *kind = allowed[below(r_type, (uint32_t)n_allowed)];
  if (*kind == MUT_INSERT) {
    int32_t pos = (int32_t)below(r1, (uint32_t)(L + 1));
    int32_t col = kth_absent(s, C, below(r2, (uint32_t)(C - L)));
    out.insert(out.begin() + pos, col);
  } else if (*kind == MUT_DELETE) {
    int32_t pos = (int32_t)below(r1, (uint32_t)L);
    out.erase(out.begin() + pos);
  } else if (*kind == MUT_SWAP) {
    int32_t i = (int32_t)below(r1, (uint32_t)L);
    int32_t j = (int32_t)below(r2, (uint32_t)(L - 1));
    if (j >= i) ++j;
    std::swap(out[i], out[j]);
  } else {  // MUT_SUBSTITUTE
    int32_t pos = (int32_t)below(r1, (uint32_t)L);
    int32_t col = kth_absent(s, C, below(r2, (uint32_t)(C - L)));
    out[pos] = col;
  }
  return out;
}

// One attempt of Step 3: tournament(s), optional crossover, one mutation.
// Draw layout for attempt j of generation g (k = tournament size):
//   0..k-1 first tournament, k crossover coin, k+1..2k second tournament,
//   2k+1 / 2k+2 crossover cuts, 2k+3 mutation kind, 2k+4 / 2k+5 its operands.
//
// Offspring screening (not in the paper), oversample V > 1: candidate v
// repeats the crossover cuts and the mutation with draws 2k+1+5v .. 2k+5+5v
// (v = 0 is the plain child).  The candidates are taken by decreasing pseudo
// score (ties: lowest v) and the first one that is not in the tabu list as it
// stood when the generation began is the child; when all of them are, the
// best-scoring one is (a tabu hit).  The pseudo score of candidate v is word
// 0 of Philox(counter (j, g, 65536 + c V + v, 0), key = seed) shifted right by
// 8, where c = ta k + tb names the tournament outcome: ta (tb) is the first
// position in the first (second) tournament holding its winner, tb = 0
// without crossover.
// What make_child saw, for the tests: every candidate, its pseudo score
// (V > 1) and the tournament outcome c.
struct ScreenTrace {
  std::vector<Seq> cand;
  std::vector<uint32_t> score;
  int32_t outcome = 0;
};

Seq make_child(const Params& p, int32_t C, int32_t g, int32_t j, const std::vector<Seq>& prev,
               const std::vector<double>& prev_f, const std::vector<int64_t>& pen,
               const std::set<Seq>& tabu_at_start, ScreenTrace* tr = nullptr) {
  const int32_t k = p.tournament_k;
  const uint32_t Pprev = (uint32_t)prev.size();
  int32_t ea[8], eb[8];
  for (int32_t t = 0; t < k; ++t) ea[t] = (int32_t)below(draw(p.seed, g, j, t), Pprev);
  bool cross = (double)draw(p.seed, g, j, k) * 0x1p-32 < p.p_crossover;
  for (int32_t t = 0; t < k; ++t) eb[t] = (int32_t)below(draw(p.seed, g, j, k + 1 + t), Pprev);

  const int32_t wa = tournament(ea, k, prev, prev_f, pen, p.penalty_base);
  const int32_t wb = cross ? tournament(eb, k, prev, prev_f, pen, p.penalty_base) : -1;
  const int32_t V = p.oversample;
  std::vector<Seq> cand;
  std::vector<uint32_t> score;
  for (int32_t v = 0; v < V; ++v) {
    const int32_t base = 2 * k + 1 + 5 * v;
    Seq child = prev[wa];
    if (cross) {
      const Seq& a = prev[wa];
      const Seq& b = prev[wb];
      int32_t cut_a = 1 + (int32_t)below(draw(p.seed, g, j, base), (uint32_t)a.size());
      int32_t cut_b = (int32_t)below(draw(p.seed, g, j, base + 1), (uint32_t)b.size());
      Seq x = crossover(a, b, cut_a, cut_b, p.len_max);
      // Reading: a crossover child shorter than len_min is dropped and the
      // first parent goes on to the mutation instead.
      if ((int32_t)x.size() >= p.len_min) child = x;
    }
    int32_t kind;
    Seq m = mutate(child, C, p.len_min, p.len_max, draw(p.seed, g, j, base + 2),
                   draw(p.seed, g, j, base + 3), draw(p.seed, g, j, base + 4), &kind);
    int32_t ta = 0, tb = 0;
    while (ea[ta] != wa) ++ta;
    if (cross)
      while (eb[tb] != wb) ++tb;
    const int32_t c = ta * k + tb;
    if (tr) tr->outcome = c;
    if (V == 1) {
      if (tr) tr->cand.push_back(m);
      return m;
    }
    cand.push_back(m);
    score.push_back(draw(p.seed, g, j, 4 * (65536 + c * V + v)) >> 8);
  }
  if (tr) {
    tr->cand = cand;
    tr->score = score;
  }
  std::vector<int32_t> order((size_t)V);
  for (int32_t v = 0; v < V; ++v) order[v] = v;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return score[a] > score[b]; });
  for (int32_t i = 0; i < V; ++i)
    if (!tabu_at_start.count(cand[order[i]])) return cand[order[i]];
  return cand[order[0]];
}

// Top-rank overlap (Step 5 and the Discussion: the list compares column sets,
// ignoring order).  Reading: |cols(a) & cols(b)| / min(|a|, |b|) > tau.
bool overlaps(const Seq& a, const Seq& b, double tau) {
  int32_t inter = 0;
  for (size_t i = 0; i < a.size(); ++i)
    if (contains(b, a[i])) ++inter;
  double mn = (double)std::min(a.size(), b.size());
  return (double)inter > tau * mn;
}

// Step 5 (and the top-rank part of Step 1).  The population is visited by
// decreasing fitness (equal fitness: lower population slot first).  An
// individual is added unless it overlaps a listed record whose fitness is
// higher or equal (reading: "equal" included, so that a re-evaluated elite
// never enters twice); once added it evicts every overlapping record of lower
// fitness and is placed after all records of higher or equal fitness.
// Finally the list is cut to its T best records.
void toprank_update(std::vector<Entry>& list, const std::vector<Entry>& pop, int32_t T,
                    double tau) {
  std::vector<int32_t> order(pop.size());
  for (size_t i = 0; i < pop.size(); ++i) order[i] = (int32_t)i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return pop[a].f > pop[b].f; });
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const Entry& x = pop[order[oi]];
    bool blocked = false;
    for (size_t e = 0; e < list.size(); ++e) {
      if (list[e].f >= x.f && overlaps(list[e].seq, x.seq, tau)) {
        blocked = true;
        break;
      }
    }
    if (blocked) continue;
    std::vector<Entry> kept;
    for (size_t e = 0; e < list.size(); ++e)
      if (!(list[e].f < x.f && overlaps(list[e].seq, x.seq, tau))) kept.push_back(list[e]);
    size_t pos = 0;
    while (pos < kept.size() && kept[pos].f >= x.f) ++pos;
    kept.insert(kept.begin() + pos, x);
    list.swap(kept);
  }
  if ((int32_t)list.size() > T) list.resize((size_t)T);
}

void evaluate(const float* A, int32_t R, int32_t C, const Params& p, std::vector<Entry>& pop) {
  for (size_t i = 0; i < pop.size(); ++i) {
    support_one(A, R, C, pop[i].seq.data(), (int32_t)pop[i].seq.size(), &pop[i].inc, &pop[i].dec);
    int64_t n = (p.fitness_support == 1) ? (int64_t)pop[i].inc + (int64_t)pop[i].dec
                                         : (int64_t)pop[i].inc;
    pop[i].f = fitness_eq1(n, (int32_t)pop[i].seq.size(), p.sigma);
  }
}

}  // namespace

// ===========================================================================
// C interface used by the tests (ctypes).
// ===========================================================================
extern "C" {

typedef struct {
  int32_t pop_size, len_min, len_max, iterations, sigma, toprank_size, tournament_k,
      fitness_support;
  double overlap_tau, elite_frac, penalty_base, p_crossover;
  uint64_t seed;
  int32_t oversample;   // offspring screening with pseudo scores (1: plain EBIC)
  int32_t reserved;
} or_params;

typedef struct {
  int32_t generations_done;  // Steps 2-5 passes completed
  int32_t stop_reason;       // 0 iterations reached, 1 tabu hits > P, 2 initial population failed
  int64_t tabu_hits_total;
  int64_t attempts_total;
  int64_t evaluations_total;
  int32_t last_gen_hits;
  int32_t toprank_n;
} or_stats;

void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

uint32_t or_draw(uint64_t seed, int32_t g, int32_t j, int32_t d) { return draw(seed, g, j, d); }

// Support of every series of a CBF population (offsets has P + 1 entries).
// A is row-major R x C.  nthreads > 1 splits the series across OpenMP threads.
// Step 6 ("determine ... the indices of rows that match each of the series"):
// the rows whose values rise strictly along the series (mode 0), or -- Step 7's
// expansion by negative trends -- the rows that rise or fall strictly along it
// (mode 1).  Row indices ascending into out_rows; returns their number.
int32_t or_rows(const float* A, int32_t R, int32_t C, const int32_t* s, int32_t L, int32_t mode,
                int32_t* out_rows) {
  int32_t n = 0;
  for (int32_t k = 0; k < R; ++k) {
    const float* row = A + (size_t)k * (size_t)C;
    bool rising = true, falling = true;
    for (int32_t i = 0; i + 1 < L; ++i) {
      if (!(row[s[i]] < row[s[i + 1]])) rising = false;
      if (!(row[s[i]] > row[s[i + 1]])) falling = false;
    }
    if (rising || (mode == 1 && falling)) out_rows[n++] = k;
  }
  return n;
}

// Step 7's expansion by approximate trends (the paper leaves "approximate"
// undefined; reading: a row follows the series approximately when at most e
// of its L - 1 adjacent pairs break the order).  Mode 0: at most e pairs
// that do not rise strictly; mode 1: that, or at most e pairs that do not
// fall strictly.  e = 0 is or_rows.  Row indices ascending into out_rows;
// returns their number.
int32_t or_rows_approx(const float* A, int32_t R, int32_t C, const int32_t* s, int32_t L,
                       int32_t e, int32_t mode, int32_t* out_rows) {
  int32_t n = 0;
  for (int32_t k = 0; k < R; ++k) {
    const float* row = A + (size_t)k * (size_t)C;
    int32_t not_up = 0, not_down = 0;
    for (int32_t i = 0; i + 1 < L; ++i) {
      if (!(row[s[i]] < row[s[i + 1]])) ++not_up;
      if (!(row[s[i]] > row[s[i + 1]])) ++not_down;
    }
    if (not_up <= e || (mode == 1 && not_down <= e)) out_rows[n++] = k;
  }
  return n;
}

void or_support(const float* A, int32_t R, int32_t C, const int32_t* offsets,
                const int32_t* cols, int32_t P, uint32_t* inc, uint32_t* dec, int32_t nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int32_t i = 0; i < P; ++i) {
    uint32_t a, b;
    support_one(A, R, C, cols + offsets[i], offsets[i + 1] - offsets[i], &a, &b);
    inc[i] = a;
    if (dec) dec[i] = b;
  }
  (void)nthreads;
}

double or_fitness(int64_t n, int32_t J, int32_t sigma) { return fitness_eq1(n, J, sigma); }

int32_t or_omp_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Operator entry points for the property tests.
int32_t or_random_series(uint64_t seed, int32_t g, int32_t j, int32_t C, int32_t Lmin,
                         int32_t Lmax, int32_t* out) {
  Seq s = random_series(seed, g, j, C, Lmin, Lmax);
  for (size_t i = 0; i < s.size(); ++i) out[i] = s[i];
  return (int32_t)s.size();
}

int32_t or_crossover(const int32_t* a, int32_t La, const int32_t* b, int32_t Lb, int32_t cut_a,
                     int32_t cut_b, int32_t Lmax, int32_t* out) {
  Seq sa(a, a + La), sb(b, b + Lb);
  Seq c = crossover(sa, sb, cut_a, cut_b, Lmax);
  for (size_t i = 0; i < c.size(); ++i) out[i] = c[i];
  return (int32_t)c.size();
}

int32_t or_mutate(const int32_t* s, int32_t L, int32_t C, int32_t Lmin, int32_t Lmax,
                  uint32_t r_type, uint32_t r1, uint32_t r2, int32_t* out, int32_t* kind) {
  Seq in(s, s + L);
  Seq m = mutate(in, C, Lmin, Lmax, r_type, r1, r2, kind);
  for (size_t i = 0; i < m.size(); ++i) out[i] = m[i];
  return (int32_t)m.size();
}

double or_penalized(double f, int64_t S, int32_t L, double base) {
  return penalized(f, S, L, base);
}

// Tournament over a CBF population with per-column usage counts pen[C].
int32_t or_tournament(const int32_t* entrants, int32_t k, const int32_t* offsets,
                      const int32_t* cols, int32_t P, const double* f, const int64_t* pen,
                      int32_t C, double base) {
  std::vector<Seq> pop(P);
  for (int32_t i = 0; i < P; ++i) pop[i].assign(cols + offsets[i], cols + offsets[i + 1]);
  std::vector<double> fv(f, f + P);
  std::vector<int64_t> pv(pen, pen + C);
  return tournament(entrants, k, pop, fv, pv, base);
}

// One attempt of Step 3 with offspring screening (test access to
// make_child): attempt j of generation g drawn from the population given as
// CBF (offsets, cols; P series) with fitness f and penalty counts pen[C],
// the tabu list as it stood at the generation's start given as CBF (t_off,
// t_cols; n_tabu series).  Writes the V = pp->oversample candidates
// (cand_len[V], cand_cols[V][len_max], padded with -1), their pseudo scores
// (V > 1), the tournament outcome c and the child.  Returns V, or -1 on
// invalid parameters.
int32_t or_screen_attempt(const or_params* pp, int32_t C, int32_t g, int32_t j,
                          const int32_t* offsets, const int32_t* cols, int32_t P, const double* f,
                          const int64_t* pen, const int32_t* t_off, const int32_t* t_cols,
                          int32_t n_tabu, int32_t* cand_len, int32_t* cand_cols,
                          uint32_t* scores, int32_t* outcome, int32_t* child_len,
                          int32_t* child_cols) {
  Params p;
  p.pop_size = pp->pop_size; p.len_min = pp->len_min; p.len_max = pp->len_max;
  p.iterations = pp->iterations; p.sigma = pp->sigma; p.toprank_size = pp->toprank_size;
  p.tournament_k = pp->tournament_k; p.fitness_support = pp->fitness_support;
  p.overlap_tau = pp->overlap_tau; p.elite_frac = pp->elite_frac;
  p.penalty_base = pp->penalty_base; p.p_crossover = pp->p_crossover; p.seed = pp->seed;
  p.oversample = pp->oversample < 1 ? 1 : pp->oversample;
  if (P < 1 || p.len_min < 1 || p.len_max < p.len_min || p.len_max > C ||
      p.tournament_k < 1 || p.tournament_k > 4)
    return -1;
  std::vector<Seq> prev(P);
  for (int32_t i = 0; i < P; ++i) prev[i].assign(cols + offsets[i], cols + offsets[i + 1]);
  std::vector<double> fv(f, f + P);
  std::vector<int64_t> pv(pen, pen + C);
  std::set<Seq> tabu;
  for (int32_t i = 0; i < n_tabu; ++i) tabu.insert(Seq(t_cols + t_off[i], t_cols + t_off[i + 1]));
  ScreenTrace tr;
  const Seq child = make_child(p, C, g, j, prev, fv, pv, tabu, &tr);
  const int32_t V = p.oversample, L = p.len_max;
  for (int32_t v = 0; v < V; ++v) {
    cand_len[v] = (int32_t)tr.cand[v].size();
    for (int32_t c = 0; c < L; ++c)
      cand_cols[(size_t)v * L + c] = c < (int32_t)tr.cand[v].size() ? tr.cand[v][c] : -1;
    scores[v] = V > 1 ? tr.score[v] : 0u;
  }
  *outcome = tr.outcome;
  *child_len = (int32_t)child.size();
  for (int32_t c = 0; c < L; ++c) child_cols[c] = c < (int32_t)child.size() ? child[c] : -1;
  return V;
}

// Top-rank update on CBF inputs; the resulting list is written as CBF with
// at most T records.  Returns the list size.
int32_t or_toprank_update(const int32_t* l_off, const int32_t* l_cols, const double* l_f,
                          int32_t n_list, const int32_t* p_off, const int32_t* p_cols,
                          const double* p_f, int32_t n_pop, int32_t T, double tau,
                          int32_t* out_off, int32_t* out_cols, double* out_f) {
  std::vector<Entry> list(n_list), pop(n_pop);
  for (int32_t i = 0; i < n_list; ++i) {
    list[i].seq.assign(l_cols + l_off[i], l_cols + l_off[i + 1]);
    list[i].f = l_f[i];
    list[i].inc = list[i].dec = 0;
  }
  for (int32_t i = 0; i < n_pop; ++i) {
    pop[i].seq.assign(p_cols + p_off[i], p_cols + p_off[i + 1]);
    pop[i].f = p_f[i];
    pop[i].inc = pop[i].dec = 0;
  }
  toprank_update(list, pop, T, tau);
  out_off[0] = 0;
  for (size_t i = 0; i < list.size(); ++i) {
    for (size_t c = 0; c < list[i].seq.size(); ++c) out_cols[out_off[i] + c] = list[i].seq[c];
    out_off[i + 1] = out_off[i] + (int32_t)list[i].seq.size();
    out_f[i] = list[i].f;
  }
  return (int32_t)list.size();
}

// The whole EA (Steps 1-5), sequential, exactly in the paper's order.
// A is row-major R x C.  Outputs (all caller-owned, nullable where noted):
//   top_len[T], top_cols[T * len_max], top_f[T], top_inc[T]: final top-rank
//   list (columns padded with -1);
//   trace_* (nullable): per generation g = 0 .. iterations, the population
//   (len, columns, inc, dec, fitness; P records each) and the top-rank list
//   after that generation (len, columns, fitness, size).
// Returns 0, or -1 on invalid parameters.
int32_t or_run(const float* A, int32_t R, int32_t C, const or_params* pp, int32_t* top_len,
               int32_t* top_cols, double* top_f, uint32_t* top_inc, or_stats* st,
               int32_t* tr_pop_len, int32_t* tr_pop_cols, uint32_t* tr_pop_inc,
               uint32_t* tr_pop_dec, double* tr_pop_f, int32_t* tr_top_n, int32_t* tr_top_len,
               int32_t* tr_top_cols, double* tr_top_f) {
  Params p;
  p.pop_size = pp->pop_size; p.len_min = pp->len_min; p.len_max = pp->len_max;
  p.iterations = pp->iterations; p.sigma = pp->sigma; p.toprank_size = pp->toprank_size;
  p.tournament_k = pp->tournament_k; p.fitness_support = pp->fitness_support;
  p.overlap_tau = pp->overlap_tau; p.elite_frac = pp->elite_frac;
  p.penalty_base = pp->penalty_base; p.p_crossover = pp->p_crossover; p.seed = pp->seed;
  p.oversample = pp->oversample < 1 ? 1 : pp->oversample;
  if (p.pop_size < 2 || p.len_min < 1 || p.len_max < p.len_min || p.len_max > C ||
      p.tournament_k < 1 || p.tournament_k > 4 || p.toprank_size < 1 || p.iterations < 0)
    return -1;
  const int32_t P = p.pop_size, T = p.toprank_size, Lmax = p.len_max;

  std::memset(st, 0, sizeof(*st));
  std::set<Seq> tabu;
  std::vector<Entry> pop, list;

  auto record = [&](int32_t g) {
    if (!tr_pop_len) return;
    for (int32_t i = 0; i < P; ++i) {
      size_t r = (size_t)g * P + i;
      tr_pop_len[r] = (int32_t)pop[i].seq.size();
      for (int32_t c = 0; c < Lmax; ++c)
        tr_pop_cols[r * Lmax + c] = c < (int32_t)pop[i].seq.size() ? pop[i].seq[c] : -1;
      tr_pop_inc[r] = pop[i].inc;
      tr_pop_dec[r] = pop[i].dec;
      tr_pop_f[r] = pop[i].f;
    }
    tr_top_n[g] = (int32_t)list.size();
    for (int32_t i = 0; i < T; ++i) {
      size_t r = (size_t)g * T + i;
      bool have = i < (int32_t)list.size();
      tr_top_len[r] = have ? (int32_t)list[i].seq.size() : 0;
      for (int32_t c = 0; c < Lmax; ++c)
        tr_top_cols[r * Lmax + c] = (have && c < (int32_t)list[i].seq.size()) ? list[i].seq[c] : -1;
      tr_top_f[r] = have ? list[i].f : 0.0;
    }
  };

  // Step 1: initial population of distinct random series, evaluated, and the
  // top-rank list built from it.
  {
    int32_t hits = 0;
    for (int32_t j = 0; (int32_t)pop.size() < P; ++j) {
      Seq s = random_series(p.seed, 0, j, C, p.len_min, p.len_max);
      st->attempts_total++;
      if (tabu.count(s)) {
        ++hits;
        st->tabu_hits_total++;
        if (hits > P) {
          st->stop_reason = 2;
          st->last_gen_hits = hits;
          return 0;
        }
        continue;
      }
      tabu.insert(s);
      Entry e;
      e.seq = s;
      pop.push_back(e);
    }
    evaluate(A, R, C, p, pop);
    st->evaluations_total += P;
    toprank_update(list, pop, T, p.overlap_tau);
    record(0);
  }

  for (int32_t g = 1; g <= p.iterations; ++g) {
    // Step 2: elitism -- the best ceil(elite_frac * |list|) records are copied
    // into the new population; every column use raises that column's penalty.
    std::vector<int64_t> pen((size_t)C, 0);
    std::vector<Entry> next;
    int32_t n_elite = (int32_t)std::ceil(p.elite_frac * (double)list.size());
    if (n_elite > P) n_elite = P;
    for (int32_t e = 0; e < n_elite; ++e) {
      Entry x;
      x.seq = list[e].seq;
      next.push_back(x);
      for (size_t c = 0; c < x.seq.size(); ++c) pen[x.seq[c]] += 1;
    }
    // Step 3: attempts until the population is full.  A child already in the
    // tabu list is a hit; more than P hits in one generation ends the run.
    std::vector<Seq> prev_seq(pop.size());
    std::vector<double> prev_f(pop.size());
    for (size_t i = 0; i < pop.size(); ++i) {
      prev_seq[i] = pop[i].seq;
      prev_f[i] = pop[i].f;
    }
    int32_t hits = 0;
    std::set<Seq> tabu_at_start;
    if (p.oversample > 1) tabu_at_start = tabu;
    for (int32_t j = 0; (int32_t)next.size() < P; ++j) {
      Seq child = make_child(p, C, g, j, prev_seq, prev_f, pen, tabu_at_start);
      st->attempts_total++;
      if (tabu.count(child)) {
        ++hits;
        st->tabu_hits_total++;
        if (hits > P) {
          st->stop_reason = 1;
          st->last_gen_hits = hits;
          goto finish;
        }
        continue;
      }
      tabu.insert(child);
      for (size_t c = 0; c < child.size(); ++c) pen[child[c]] += 1;
      Entry x;
      x.seq = child;
      next.push_back(x);
    }
    st->last_gen_hits = hits;
    // Step 4: support and Eq. (1) for the new population.
    evaluate(A, R, C, p, next);
    st->evaluations_total += P;
    // Step 5: top-rank update.
    toprank_update(list, next, T, p.overlap_tau);
    pop.swap(next);
    st->generations_done = g;
    record(g);
  }

finish:
  st->toprank_n = (int32_t)list.size();
  for (int32_t i = 0; i < T; ++i) {
    bool have = i < (int32_t)list.size();
    top_len[i] = have ? (int32_t)list[i].seq.size() : 0;
    for (int32_t c = 0; c < Lmax; ++c)
      top_cols[(size_t)i * Lmax + c] = (have && c < (int32_t)list[i].seq.size()) ? list[i].seq[c] : -1;
    top_f[i] = have ? list[i].f : 0.0;
    top_inc[i] = have ? list[i].inc : 0;
  }
  return 0;
}

}  // extern "C"
