/*
 * Seeded synthesiser of block-tridiagonal (QBD-like) Markov generators.
 *
 * This module produces problem INPUTS only: the generator Q of an irreducible
 * continuous-time Markov chain on levels l = 0..L-1 with m phases per level,
 * given as three arrays of row-major m x m FP64 blocks
 *     dn[l]  = Q_{l,l-1} = A2(l)   (down-rates; dn[0]   is all zero)
 *     loc[l] = Q_{l,l}   = A1(l) - diag(row sums of A0(l)+A1(l)+A2(l))
 *     up[l]  = Q_{l,l+1} = A0(l)   (up-rates;   up[L-1] is all zero)
 * It holds none of the solver's arithmetic; both the CPU oracle and the GPU
 * library consume what it writes.
 *
 * Randomness is counter based: every entry is a pure function of
 * (seed, attempt, level key, block kind, i, j, purpose), hashed with the
 * SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Output is therefore identical for any
 * thread count and for any subrange of levels generated on its own.
 *
 * Must be compiled with -ffp-contract=off so that every block is bit-exact
 * across compilers and machines (x86_64 and aarch64).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#include <math.h>

enum { K_A0 = 0, K_A1 = 1, K_A2 = 2, K_AP1 = 3, K_AP2 = 4, K_AM1 = 5, K_AM2 = 6, K_REQ = 7 };
enum { P_BERN = 0, P_VAL = 1 };

static uint64_t sm64_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* 64 random bits for one (stream, level, kind, i, j, purpose) coordinate. */
uint64_t synth_bits(uint64_t seed, uint64_t attempt, uint64_t level, uint64_t kind,
                    uint64_t i, uint64_t j, uint64_t purpose) {
  uint64_t h = sm64_mix(seed ^ (attempt << 56));
  h = sm64_mix(h ^ level);
  h = sm64_mix(h ^ ((kind << 56) | (purpose << 48) | (i << 24) | j));
  return h;
}

/* Uniform double in [0,1) from the top 53 bits. */
double synth_uniform(uint64_t seed, uint64_t attempt, uint64_t level, uint64_t kind,
                     uint64_t i, uint64_t j, uint64_t purpose) {
  return (double)(synth_bits(seed, attempt, level, kind, i, j, purpose) >> 11) * 0x1.0p-53;
}

/* One rate-block entry: structurally nonzero with probability 1/2 (always on
 * the diagonal when force_diag), value Uniform(0.1, 1). */
static double rate_entry(uint64_t seed, uint64_t attempt, uint64_t lk, uint64_t kind,
                         int i, int j, int force_diag, int zero_diag) {
  if (i == j && zero_diag) return 0.0;
  if (!(i == j && force_diag)) {
    if (synth_uniform(seed, attempt, lk, kind, (uint64_t)i, (uint64_t)j, P_BERN) >= 0.5) return 0.0;
  }
  double u = synth_uniform(seed, attempt, lk, kind, (uint64_t)i, (uint64_t)j, P_VAL);
  double a = 0.9 * u;
  return 0.1 + a;
}

static void fill_rate_block(double* B, int m, uint64_t seed, uint64_t attempt, uint64_t lk,
                            uint64_t kind, int force_diag, int zero_diag) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      B[(size_t)i * m + j] = rate_entry(seed, attempt, lk, kind, i, j, force_diag, zero_diag);
}

static double block_sum(const double* B, int m) {
  double s = 0.0;
  for (size_t k = 0; k < (size_t)m * m; ++k) s += B[k];
  return s;
}

/*
 * QBD generator, levels [l0, l1) of an L-level chain.
 * Per level l (level key = l if level_dependent else 0):
 *   A0, A2: entries nonzero w.p. 1/2, diagonal forced positive;
 *   A1: off-diagonal entries nonzero w.p. 1/2, zero diagonal;
 *   A2 scaled by sum(A0) / (ratio * sum(A2))  (sums over all m*m entries,
 *   row-major order, before boundary truncation) so that total up-rate /
 *   total down-rate = ratio;
 *   level 0 keeps no A2, level L-1 keeps no A0;
 *   diagonal of Q_{l,l} = -(row sum of retained A0 + A1 + retained A2), each
 *   row summed A0 first, then A1, then A2, every block left to right.
 * Arrays hold (l1-l0) blocks each.  Returns 0, or -1 on bad arguments.
 */
int synth_qbd_levels(uint64_t seed, uint64_t attempt, int64_t L, int m, double ratio,
                     int level_dependent, int64_t l0, int64_t l1,
                     double* dn, double* loc, double* up) {
  if (L < 1 || m < 1 || m > (1 << 20) || l0 < 0 || l1 > L || l0 > l1 || !(ratio > 0)) return -1;
  const size_t mm = (size_t)m * m;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t l = l0; l < l1; ++l) {
    const uint64_t lk = level_dependent ? (uint64_t)l : 0u;
    double* D = dn + (size_t)(l - l0) * mm;
    double* C = loc + (size_t)(l - l0) * mm;
    double* U = up + (size_t)(l - l0) * mm;
    fill_rate_block(U, m, seed, attempt, lk, K_A0, 1, 0);
    fill_rate_block(C, m, seed, attempt, lk, K_A1, 0, 1);
    fill_rate_block(D, m, seed, attempt, lk, K_A2, 1, 0);
    const double s0 = block_sum(U, m), s2 = block_sum(D, m);
    const double c = s0 / (ratio * s2);
    for (size_t k = 0; k < mm; ++k) D[k] = D[k] * c;
    if (l == 0) memset(D, 0, mm * sizeof(double));
    if (l == L - 1) memset(U, 0, mm * sizeof(double));
    for (int i = 0; i < m; ++i) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc += U[(size_t)i * m + j];
      for (int j = 0; j < m; ++j) acc += C[(size_t)i * m + j];
      for (int j = 0; j < m; ++j) acc += D[(size_t)i * m + j];
      C[(size_t)i * m + i] = -acc;
    }
  }
  return 0;
}

/*
 * Block-pentadiagonal generator with level jumps +-1 and +-2 on L levels of m
 * phases, delivered PAIRED: super-level J = {2J, 2J+1} (L must be even), so the
 * output is a block-tridiagonal generator of L/2 super-levels with blocks of
 * 2m.  Jump blocks A(+1), A(+2), A(-1), A(-2) (diagonals forced positive) and
 * A1 (zero diagonal) are level-independent; A(+-2) are multiplied by scale2;
 * both down blocks are then multiplied by one common factor so that
 * (sum A(+1) + sum A(+2)) / (sum A(-1) + sum A(-2)) = ratio.  Jumps that
 * would leave [0, L-1] are dropped and the diagonal keeps only retained rates.
 * Super-level blocks (rows/cols: first the m phases of level 2J, then 2J+1):
 *   loc'[J] = [[Q_{2J,2J},   A(+1)], [A(-1), Q_{2J+1,2J+1}]]
 *   up'[J]  = [[A(+2), 0],  [A(+1), A(+2)]]
 *   dn'[J]  = [[A(-2), A(-1)], [0, A(-2)]]
 * Fills super-levels [J0, J1).  Returns 0, or -1 on bad arguments.
 */
int synth_penta_levels(uint64_t seed, uint64_t attempt, int64_t L, int m, double ratio,
                       double scale2, int64_t J0, int64_t J1,
                       double* dn, double* loc, double* up) {
  if (L < 2 || (L & 1) || m < 1 || J0 < 0 || J1 > L / 2 || J0 > J1 || !(ratio > 0)) return -1;
  const size_t mm = (size_t)m * m, M = 2 * (size_t)m, MM = M * M;
  double *ap1, *ap2, *am1, *am2, *a1;
  /* the five level-independent m x m blocks, built once */
  double* blocks = (double*)malloc(5 * mm * sizeof(double));
  if (!blocks) return -1;
  ap1 = blocks; ap2 = blocks + mm; am1 = blocks + 2 * mm; am2 = blocks + 3 * mm; a1 = blocks + 4 * mm;
  fill_rate_block(ap1, m, seed, attempt, 0, K_AP1, 1, 0);
  fill_rate_block(ap2, m, seed, attempt, 0, K_AP2, 1, 0);
  fill_rate_block(am1, m, seed, attempt, 0, K_AM1, 1, 0);
  fill_rate_block(am2, m, seed, attempt, 0, K_AM2, 1, 0);
  fill_rate_block(a1, m, seed, attempt, 0, K_A1, 0, 1);
  for (size_t k = 0; k < mm; ++k) { ap2[k] = ap2[k] * scale2; am2[k] = am2[k] * scale2; }
  const double su = block_sum(ap1, m) + block_sum(ap2, m);
  const double sd = block_sum(am1, m) + block_sum(am2, m);
  const double c = su / (ratio * sd);
  for (size_t k = 0; k < mm; ++k) { am1[k] = am1[k] * c; am2[k] = am2[k] * c; }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t J = J0; J < J1; ++J) {
    double* D = dn + (size_t)(J - J0) * MM;
    double* C = loc + (size_t)(J - J0) * MM;
    double* U = up + (size_t)(J - J0) * MM;
    memset(D, 0, MM * sizeof(double));
    memset(C, 0, MM * sizeof(double));
    memset(U, 0, MM * sizeof(double));
    for (int h = 0; h < 2; ++h) {              /* h = 0: level 2J, h = 1: level 2J+1 */
      const int64_t l = 2 * J + h;
      const size_t r0 = (size_t)h * m;         /* row offset inside the super block */
      for (int i = 0; i < m; ++i) {
        double acc = 0.0;
        /* up jumps: l -> l+1 and l -> l+2 */
        if (l + 1 <= L - 1) {
          /* l+1 lies in this super-level (h=0) or the next (h=1) */
          double* T = (h == 0) ? C : U; size_t c0 = (h == 0) ? (size_t)m : 0;
          for (int j = 0; j < m; ++j) { T[(r0 + i) * M + c0 + j] = ap1[(size_t)i * m + j]; acc += ap1[(size_t)i * m + j]; }
        }
        if (l + 2 <= L - 1) {
          size_t c0 = (size_t)h * m;           /* l+2 = 2(J+1)+h */
          for (int j = 0; j < m; ++j) { U[(r0 + i) * M + c0 + j] = ap2[(size_t)i * m + j]; acc += ap2[(size_t)i * m + j]; }
        }
        /* local */
        for (int j = 0; j < m; ++j) { C[(r0 + i) * M + r0 + j] = a1[(size_t)i * m + j]; acc += a1[(size_t)i * m + j]; }
        /* down jumps: l -> l-1 and l -> l-2 */
        if (l - 1 >= 0) {
          double* T = (h == 1) ? C : D; size_t c0 = (h == 1) ? 0 : (size_t)m;
          for (int j = 0; j < m; ++j) { T[(r0 + i) * M + c0 + j] = am1[(size_t)i * m + j]; acc += am1[(size_t)i * m + j]; }
        }
        if (l - 2 >= 0) {
          size_t c0 = (size_t)h * m;           /* l-2 = 2(J-1)+h */
          for (int j = 0; j < m; ++j) { D[(r0 + i) * M + c0 + j] = am2[(size_t)i * m + j]; acc += am2[(size_t)i * m + j]; }
        }
        C[(r0 + i) * M + r0 + i] = -acc;
      }
    }
  }
  free(blocks);
  return 0;
}

/* OR the structural pattern of level l's retained rate blocks into the m x m
 * phase adjacency adj (adj[i*m+j] = 1 iff some retained block has (i,j) > 0). */
static void qbd_pattern(uint64_t seed, uint64_t attempt, int64_t L, int m, int level_dependent,
                        int64_t l, unsigned char* adj) {
  const uint64_t lk = level_dependent ? (uint64_t)l : 0u;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      if (i == j) continue;
      int e = 0;
      if (l < L - 1) e |= rate_entry(seed, attempt, lk, K_A0, i, j, 1, 0) > 0;
      e |= rate_entry(seed, attempt, lk, K_A1, i, j, 0, 1) > 0;
      if (l > 0) e |= rate_entry(seed, attempt, lk, K_A2, i, j, 1, 0) > 0;
      if (e) adj[(size_t)i * m + j] = 1;
    }
}

static int reach_all(const unsigned char* adj, int m, int transpose, unsigned char* seen, int* stack) {
  memset(seen, 0, (size_t)m);
  int top = 0, count = 1; stack[top++] = 0; seen[0] = 1;
  while (top) {
    int v = stack[--top];
    for (int w = 0; w < m; ++w) {
      unsigned char e = transpose ? adj[(size_t)w * m + v] : adj[(size_t)v * m + w];
      if (e && !seen[w]) { seen[w] = 1; ++count; stack[top++] = w; }
    }
  }
  return count == m;
}

/*
 * Irreducibility: every level reaches every other level in the same phase
 * (diagonals of A0, A2 are positive), so the chain is irreducible iff the
 * phase graph (union over levels of the retained A0, A1, A2 patterns) is
 * strongly connected.  Returns the first attempt index in [0, 64) whose
 * generator is irreducible, or -1.  work must hold m*m + m bytes + m ints
 * (caller-provided: adj, seen, stack).
 */
int synth_qbd_first_irreducible(uint64_t seed, int64_t L, int m, int level_dependent,
                                unsigned char* adj, unsigned char* seen, int* stack) {
  if (m == 1) return 0;
  for (int attempt = 0; attempt < 64; ++attempt) {
    memset(adj, 0, (size_t)m * m);
    for (int64_t l = 0; l < L; ++l) {
      qbd_pattern(seed, (uint64_t)attempt, L, m, level_dependent, l, adj);
      if (reach_all(adj, m, 0, seen, stack) && reach_all(adj, m, 1, seen, stack)) return attempt;
      if (!level_dependent && l >= 2) break;    /* interior pattern repeats */
    }
  }
  return -1;
}

/*
 * Block-banded generator: jumps of e levels for e in [-p, q] \ {0}, m phases.
 * Per level l (key = l if level_dependent else 0) and jump e: block A_e with
 * entries nonzero w.p. 1/2 (diagonal forced positive for e = +-1), values
 * Uniform(0.1, 1) times decay^(|e|-1); A1 local with zero diagonal.  All down
 * blocks (e < 0) are then multiplied by one factor so that the level's total
 * up-rate / total down-rate = ratio (sums over all entries, before dropping
 * the jumps that leave [0, L-1]).  Diagonal of Q_{l,l} = -(row sums of the
 * retained blocks, in the order e = -p..q, local at e = 0).
 * out[(e + p) * (l1-l0) + (l - l0)] = Q_{l, l+e} (row-major m x m), e = 0 the
 * local block with its diagonal.  Returns 0 or -1 on bad arguments.
 */
int synth_banded_levels(uint64_t seed, int64_t L, int m, int p, int q, double ratio, double decay,
                        int level_dependent, int64_t l0, int64_t l1, double* out) {
  if (L < 1 || m < 1 || p < 1 || q < 1 || p > 16 || q > 16 || l0 < 0 || l1 > L || l0 > l1 ||
      !(ratio > 0) || !(decay > 0))
    return -1;
  const size_t mm = (size_t)m * m, nl = (size_t)(l1 - l0);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t l = l0; l < l1; ++l) {
    const uint64_t lk = level_dependent ? (uint64_t)l : 0u;
    double su = 0.0, sd = 0.0;
    for (int e = -p; e <= q; ++e) {
      double* B = out + ((size_t)(e + p) * nl + (size_t)(l - l0)) * mm;
      if (e == 0) {
        fill_rate_block(B, m, seed, 0, lk, K_A1, 0, 1);
        continue;
      }
      const uint64_t kind = 16 + (uint64_t)(e + 16);
      fill_rate_block(B, m, seed, 0, lk, kind, e == 1 || e == -1, 0);
      double w = 1.0;
      for (int k = 1; k < (e > 0 ? e : -e); ++k) w *= decay;
      for (size_t t = 0; t < mm; ++t) B[t] = B[t] * w;
      if (e > 0) su += block_sum(B, m); else sd += block_sum(B, m);
    }
    const double c = su / (ratio * sd);
    for (int e = -p; e < 0; ++e) {
      double* B = out + ((size_t)(e + p) * nl + (size_t)(l - l0)) * mm;
      for (size_t t = 0; t < mm; ++t) B[t] = B[t] * c;
    }
    for (int e = -p; e <= q; ++e) {
      if (e == 0) continue;
      if (l + e < 0 || l + e > L - 1) {
        double* B = out + ((size_t)(e + p) * nl + (size_t)(l - l0)) * mm;
        memset(B, 0, mm * sizeof(double));
      }
    }
    double* C = out + ((size_t)p * nl + (size_t)(l - l0)) * mm;
    for (int i = 0; i < m; ++i) {
      double acc = 0.0;
      for (int e = -p; e <= q; ++e) {
        const double* B = out + ((size_t)(e + p) * nl + (size_t)(l - l0)) * mm;
        for (int j = 0; j < m; ++j)
          if (!(e == 0 && j == i)) acc += B[(size_t)i * m + j];
      }
      C[(size_t)i * m + i] = -acc;
    }
  }
  return 0;
}
