/*
 * smcx_oracle.c -- plain, sequential CPU oracle of the SMC-X EPI swap sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library: geometry, random numbers, acceptance tables, energies
 * and the sweep schedule are all re-derived here from their definitions.
 *
 * What it computes (arXiv 2509.20949, "SMC-X"):
 *   - canonical-ensemble target P(sigma) ~ exp(-beta H)          (Sec. 2.1, Eq. 1)
 *   - Metropolis acceptance min(1, exp(-beta dE))                (Sec. 2.1, Eq. 3)
 *   - one MC step = one trial per lattice site                   (Sec. 2.1)
 *   - link cells updated as a checkerboard of non-interacting
 *     blocks, rebuilt ("dynamically constructed") every step      (Sec. 2.2, Eq. 5)
 *   - trial energy change from the local interaction zone only   (Sec. 2.2)
 *   - EPI model: pairwise shell interactions only                 (Sec. 3, "EPI model")
 *   - Warren-Cowley SRO from directed pair counts                 (Sec. 3.2, Eq. 9)
 * The paper leaves the random-number generator, the fixed-point energy
 * scale, the cell sizing rule and the visiting order open; this file follows
 * the readings fixed for this project (Philox4x32-10 keyed by (seed, sweep,
 * cell, attempt); energies in units q = 2^-32 eV held in int64; an integer
 * threshold-table acceptance test; cells of edge L >= floor((1+h_R)/2)+1
 * conventional cells; ascending colours, ascending cell ids, raster order
 * inside a cell).
 *
 * Everything is deliberately unoptimised: every neighbour index is recomputed
 * from coordinates, every energy change is the literal sum with every
 * occurrence of the two swapped sites left out.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no fast-math), with
 * -fopenmp where the compiler has it (only the *_par functions use it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EOVERFLOW 4

#define ORC_FLAG_NO_SHIFT 1u
#define ORC_FLAG_SINGLE_CELL 2u

#define ORC_MODE_NORMAL 0
#define ORC_MODE_ACCEPT_ALL 1 /* beta = 0 (T = +inf) */
#define ORC_MODE_ZERO_T 2     /* beta = +inf (T = 0) */

/* Boltzmann constant in eV/K (CODATA 2018 exact value); the paper gives none. */
static const double ORC_KB = 8.617333262e-5;

typedef struct {
  int32_t kind; /* 0 = BCC, 1 = FCC */
  int32_t n[3]; /* conventional cells per dimension, periodic */
  int32_t K;    /* number of species */
  int32_t M;    /* number of EPI shells in use (1..4) */
  int32_t min_cell;
  uint32_t flags;
  uint64_t seed;
} orc_desc;

typedef struct {
  uint64_t attempts, unlike, accepted;
  int64_t sum_dE;
} orc_stats;

typedef struct {
  int32_t L_override;    /* > 0: force this link-cell edge (used to show the
                            schedule test can fail) */
  int32_t shuffle_cells; /* != 0: visit the cells of one colour in a random
                            permutation instead of ascending id */
  uint64_t shuffle_seed;
} orc_opts;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC11): ten rounds of two   */
/* 32x32->64 multiplications, the high halves xor-ed with the other counter  */
/* words and the round key, the key advanced by the Weyl constants between   */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t MUL_A = 0xD2511F53u, MUL_B = 0xCD9E8D57u;
  const uint32_t WEYL_A = 0x9E3779B9u, WEYL_B = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += WEYL_A;
      k1 += WEYL_B;
    }
    uint64_t prod_a = (uint64_t)MUL_A * (uint64_t)x0;
    uint64_t prod_b = (uint64_t)MUL_B * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod_b;
    uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod_a;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

static void philox_keyed(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                         uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry.  Positions are in half-lattice units h = a/2; the basis */
/* of a conventional cell is BCC {(0,0,0),(1,1,1)}, FCC {(0,0,0),(0,1,1),    */
/* (1,0,1),(1,1,0)}.  Neighbour shells are found by brute force: every       */
/* lattice vector in a box is classified by its squared length, shells are   */
/* the distinct lengths in ascending order, each shell's vectors are sorted  */
/* lexicographically on (dx, dy, dz).                                        */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_SHELLS 4
#define ORC_MAX_DISP 128

static int basis_count(int kind) { return kind == 0 ? 2 : 4; }

static void basis_vec(int kind, int b, int v[3]) {
  static const int bcc[2][3] = {{0, 0, 0}, {1, 1, 1}};
  static const int fcc[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
  const int *src = kind == 0 ? bcc[b] : fcc[b];
  v[0] = src[0];
  v[1] = src[1];
  v[2] = src[2];
}

static int is_lattice_vector(int kind, int dx, int dy, int dz) {
  /* BCC: all three components share one parity; FCC: even component sum. */
  int px = dx & 1, py = dy & 1, pz = dz & 1;
  if (kind == 0) return px == py && py == pz;
  return ((dx + dy + dz) & 1) == 0;
}

static int lex_less(const int *a, const int *b) {
  if (a[0] != b[0]) return a[0] < b[0];
  if (a[1] != b[1]) return a[1] < b[1];
  return a[2] < b[2];
}

typedef struct {
  int M;
  int total;
  int z[ORC_MAX_SHELLS];
  int d2[ORC_MAX_SHELLS];
  int start[ORC_MAX_SHELLS + 1];
  int disp[ORC_MAX_DISP][3];
} shells_t;

static int build_shells(int kind, int M, shells_t *sh) {
  if (M < 1 || M > ORC_MAX_SHELLS) return ORC_EINVAL;
  const int R = 4; /* every vector of the first four shells has |component| <= 3 */
  int lengths[64];
  int n_len = 0;
  for (int dx = -R; dx <= R; ++dx)
    for (int dy = -R; dy <= R; ++dy)
      for (int dz = -R; dz <= R; ++dz) {
        if (!dx && !dy && !dz) continue;
        if (!is_lattice_vector(kind, dx, dy, dz)) continue;
        int d2 = dx * dx + dy * dy + dz * dz;
        int seen = 0;
        for (int t = 0; t < n_len; ++t) seen |= lengths[t] == d2;
        if (!seen && n_len < 64) lengths[n_len++] = d2;
      }
  /* ascending squared lengths (insertion sort) */
  for (int a = 1; a < n_len; ++a)
    for (int b = a; b > 0 && lengths[b - 1] > lengths[b]; --b) {
      int t = lengths[b];
      lengths[b] = lengths[b - 1];
      lengths[b - 1] = t;
    }
  sh->M = M;
  sh->total = 0;
  for (int m = 0; m < M; ++m) {
    sh->d2[m] = lengths[m];
    sh->start[m] = sh->total;
    for (int dx = -R; dx <= R; ++dx)
      for (int dy = -R; dy <= R; ++dy)
        for (int dz = -R; dz <= R; ++dz) {
          if (!is_lattice_vector(kind, dx, dy, dz)) continue;
          if (dx * dx + dy * dy + dz * dz != lengths[m]) continue;
          if (sh->total >= ORC_MAX_DISP) return ORC_EINVAL;
          sh->disp[sh->total][0] = dx;
          sh->disp[sh->total][1] = dy;
          sh->disp[sh->total][2] = dz;
          sh->total++;
        }
    sh->z[m] = sh->total - sh->start[m];
    /* lexicographic order inside the shell (insertion sort) */
    for (int a = sh->start[m] + 1; a < sh->total; ++a)
      for (int b = a; b > sh->start[m] && lex_less(sh->disp[b], sh->disp[b - 1]); --b) {
        int t[3] = {sh->disp[b][0], sh->disp[b][1], sh->disp[b][2]};
        memcpy(sh->disp[b], sh->disp[b - 1], sizeof t);
        memcpy(sh->disp[b - 1], t, sizeof t);
      }
  }
  sh->start[M] = sh->total;
  return ORC_OK;
}

/* Export of the shell tables for the tests.  disp: [cap][3]; returns total. */
int orc_shells(int kind, int M, int *disp, int *z, int *d2, int cap) {
  shells_t sh;
  if (kind != 0 && kind != 1) return -1;
  if (build_shells(kind, M, &sh) != ORC_OK) return -1;
  if (sh.total > cap) return -1;
  for (int t = 0; t < sh.total; ++t)
    for (int c = 0; c < 3; ++c) disp[3 * t + c] = sh.disp[t][c];
  for (int m = 0; m < M; ++m) {
    z[m] = sh.z[m];
    d2[m] = sh.d2[m];
  }
  return sh.total;
}

static int64_t site_count(const orc_desc *d) {
  return (int64_t)basis_count(d->kind) * d->n[0] * d->n[1] * d->n[2];
}

static int64_t site_index(const orc_desc *d, int x, int y, int z, int b) {
  return (((int64_t)z * d->n[1] + y) * d->n[0] + x) * basis_count(d->kind) + b;
}

static int pos_mod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

/* Site reached from site i by displacement disp (half units), periodic. */
static int64_t neighbour(const orc_desc *d, int64_t i, const int disp[3]) {
  int nb = basis_count(d->kind);
  int b = (int)(i % nb);
  int64_t cell = i / nb;
  int x = (int)(cell % d->n[0]);
  int y = (int)((cell / d->n[0]) % d->n[1]);
  int z = (int)(cell / ((int64_t)d->n[0] * d->n[1]));
  int bv[3];
  basis_vec(d->kind, b, bv);
  int p[3] = {2 * x + bv[0] + disp[0], 2 * y + bv[1] + disp[1], 2 * z + bv[2] + disp[2]};
  for (int c = 0; c < 3; ++c) p[c] = pos_mod(p[c], 2 * d->n[c]);
  int par[3] = {p[0] & 1, p[1] & 1, p[2] & 1};
  int nbi = -1;
  for (int t = 0; t < nb; ++t) {
    int v[3];
    basis_vec(d->kind, t, v);
    if (v[0] == par[0] && v[1] == par[1] && v[2] == par[2]) nbi = t;
  }
  if (nbi < 0) return -1; /* not a lattice vector: cannot happen for shell vectors */
  return site_index(d, p[0] >> 1, p[1] >> 1, p[2] >> 1, nbi);
}

static int valid_desc(const orc_desc *d) {
  if (d->kind != 0 && d->kind != 1) return 0;
  for (int c = 0; c < 3; ++c)
    if (d->n[c] < 1) return 0;
  if (d->K < 1 || d->K > 255) return 0;
  if (d->M < 1 || d->M > ORC_MAX_SHELLS) return 0;
  if (site_count(d) >= ((int64_t)1 << 32)) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* EPI Hamiltonian (pairwise only, Sec. 3): H = sum_m sum_i sum_{d in S_m,  */
/* d >lex 0} V_m(s_i, s_{i+d}); every bond once, periodic multiplicity kept. */
/* V is [M][K][K] int64 in units of q = 2^-32 eV, symmetric.                 */
/* ------------------------------------------------------------------------ */
static int lex_positive(const int *v) {
  if (v[0] != 0) return v[0] > 0;
  if (v[1] != 0) return v[1] > 0;
  return v[2] > 0;
}

int orc_energy(const orc_desc *d, const int64_t *V, const uint8_t *occ, int64_t *E) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  const int K = d->K;
  __int128 acc = 0;
  int64_t N = site_count(d);
  for (int64_t i = 0; i < N; ++i)
    for (int m = 0; m < d->M; ++m)
      for (int t = sh.start[m]; t < sh.start[m + 1]; ++t) {
        if (!lex_positive(sh.disp[t])) continue;
        int64_t k = neighbour(d, i, sh.disp[t]);
        acc += V[((int64_t)m * K + occ[i]) * K + occ[k]];
      }
  if (acc > (__int128)INT64_MAX || acc < (__int128)INT64_MIN) return ORC_EOVERFLOW;
  *E = (int64_t)acc;
  return ORC_OK;
}

/* Directed pair counts N_m[p'][p]: centre species p', neighbour species p in */
/* shell m, counted from every site (each bond seen from both ends).          */
int orc_pair_counts(const orc_desc *d, const uint8_t *occ, uint64_t *counts) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  const int K = d->K;
  memset(counts, 0, sizeof(uint64_t) * (size_t)d->M * K * K);
  int64_t N = site_count(d);
  for (int64_t i = 0; i < N; ++i)
    for (int m = 0; m < d->M; ++m)
      for (int t = sh.start[m]; t < sh.start[m + 1]; ++t) {
        int64_t k = neighbour(d, i, sh.disp[t]);
        counts[((int64_t)m * K + occ[i]) * K + occ[k]] += 1;
      }
  return ORC_OK;
}

/* Warren-Cowley SRO, Eq. 9: alpha_m^{p p'} = 1 - P_m^{p|p'} / c_p with the  */
/* conditional probability P_m^{p|p'} = N_m[p'][p] / (N_{p'} z_m) and the    */
/* concentration c_p = N_p / N.  alpha[m][p'][p]; NaN where N_p or N_p' = 0. */
int orc_sro_alpha(const orc_desc *d, const uint64_t *counts, const uint64_t *species_count,
                  double *alpha) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  const int K = d->K;
  double N = (double)site_count(d);
  for (int m = 0; m < d->M; ++m)
    for (int pc = 0; pc < K; ++pc)
      for (int p = 0; p < K; ++p) {
        double n_centre = (double)species_count[pc];
        double n_p = (double)species_count[p];
        double cond = (double)counts[((int64_t)m * K + pc) * K + p] / (n_centre * (double)sh.z[m]);
        double conc = n_p / N;
        alpha[((int64_t)m * K + pc) * K + p] =
            (n_centre > 0 && n_p > 0) ? 1.0 - cond / conc : NAN;
      }
  return ORC_OK;
}

/* Energy change of swapping the species of sites i and j, written out      */
/* literally: over both neighbour lists, every occurrence of i or of j is    */
/* left out, so the i-j bond (unchanged by a swap) never enters.             */
static int64_t delta_e(const orc_desc *d, const shells_t *sh, const int64_t *V,
                       const uint8_t *occ, int64_t i, int64_t j) {
  const int K = d->K;
  int p = occ[i], q = occ[j];
  int64_t dE = 0;
  for (int m = 0; m < d->M; ++m) {
    const int64_t *Vm = V + (int64_t)m * K * K;
    for (int t = sh->start[m]; t < sh->start[m + 1]; ++t) {
      int64_t k = neighbour(d, i, sh->disp[t]);
      if (k != i && k != j) dE += Vm[q * K + occ[k]] - Vm[p * K + occ[k]];
      k = neighbour(d, j, sh->disp[t]);
      if (k != i && k != j) dE += Vm[p * K + occ[k]] - Vm[q * K + occ[k]];
    }
  }
  return dE;
}

int orc_delta_e(const orc_desc *d, const int64_t *V, const uint8_t *occ, int64_t i, int64_t j,
                int64_t *dE) {
  if (!valid_desc(d)) return ORC_EINVAL;
  int64_t N = site_count(d);
  if (i < 0 || j < 0 || i >= N || j >= N) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  *dE = delta_e(d, &sh, V, occ, i, j);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Metropolis acceptance (Sec. 2.1, Eq. 3) as an exact integer test.          */
/*  beta = 1/(k_B T); s = largest integer >= 0 with beta q 2^s <= 2^-20       */
/*  (s = 0 when even s = 0 misses); bins of width 2^s q, evaluated at their   */
/*  lower edge:                                                               */
/*    T_l[i] = min(2^32-1, rint(2^32 exp(-beta q 2^s (i << 9l)))), l = 0,1,2  */
/*  and for dE > 0, idx = dE >> s: reject when idx >= 2^27, otherwise        */
/*    thr = hi32(hi32(T_0[idx & 511] T_1[(idx >> 9) & 511]) T_2[idx >> 18])  */
/*  and accept iff the trial's second Philox word is below thr.              */
/*  T = +inf: every proposal accepted; T = 0: accept iff dE <= 0.             */
/* ------------------------------------------------------------------------ */
int orc_thresholds(double T, uint32_t *tab, int32_t *s_out, int32_t *mode_out) {
  if (isnan(T) || T < 0) return ORC_EINVAL;
  memset(tab, 0, sizeof(uint32_t) * 3 * 512);
  *s_out = 0;
  if (T == 0) {
    *mode_out = ORC_MODE_ZERO_T;
    return ORC_OK;
  }
  if (isinf(T)) {
    *mode_out = ORC_MODE_ACCEPT_ALL;
    return ORC_OK;
  }
  double beta = 1.0 / (ORC_KB * T);
  if (beta == 0.0) {
    *mode_out = ORC_MODE_ACCEPT_ALL;
    return ORC_OK;
  }
  *mode_out = ORC_MODE_NORMAL;
  /* beta*q*2^s = beta * 2^(s-32); compare against 2^-20 (exact: ldexp only) */
  int s = 0;
  while (s < 62 && ldexp(beta, s + 1 - 32) <= ldexp(1.0, -20)) ++s;
  *s_out = s;
  for (int l = 0; l < 3; ++l) {
    double step = ldexp(beta, s - 32 + 9 * l); /* beta * q * 2^s * 2^(9l) */
    for (int i = 0; i < 512; ++i) {
      double x = (double)i * step;
      double v = rint(ldexp(exp(-x), 32));
      if (v > 4294967295.0) v = 4294967295.0;
      tab[l * 512 + i] = (uint32_t)v;
    }
  }
  return ORC_OK;
}

static int accept_move(int64_t dE, uint32_t wb, int mode, int s, const uint32_t *tab) {
  if (dE <= 0) return 1;
  if (mode == ORC_MODE_ZERO_T) return 0;
  if (mode == ORC_MODE_ACCEPT_ALL) return 1;
  uint64_t idx = (uint64_t)dE >> s;
  if (idx >= ((uint64_t)1 << 27)) return 0;
  uint32_t a = tab[idx & 511];
  uint32_t b = tab[512 + ((idx >> 9) & 511)];
  uint32_t c = tab[1024 + (idx >> 18)];
  uint32_t ab = (uint32_t)(((uint64_t)a * b) >> 32);
  uint32_t thr = (uint32_t)(((uint64_t)ab * c) >> 32);
  return wb < thr;
}

/* ------------------------------------------------------------------------ */
/* Link cells (Sec. 2.2, Eq. 5).  h_R = largest |component| of any shell     */
/* vector in use; a cell of edge L conventional cells keeps two same-colour  */
/* cells from interacting when 2L > 1 + h_R, so L_min = floor((1+h_R)/2)+1.  */
/* Per dimension m_d = largest even number <= n_d / L (1 if that is 0, or     */
/* everywhere under SINGLE_CELL); cell c spans [floor(c n/m), floor((c+1)n/m))*/
/* in coordinates shifted by the sweep's random origin.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int L;
  int m[3];
} layout_t;

static int compute_layout(const orc_desc *d, const shells_t *sh, int L_override, layout_t *lay,
                          int local) {
  int hR = 0;
  for (int t = 0; t < sh->total; ++t)
    for (int c = 0; c < 3; ++c) {
      int a = abs(sh->disp[t][c]);
      if (a > hR) hR = a;
    }
  /* a trial reads 1 + h_R half units beyond its cell (EPI: the partner's    */
  /* neighbours), 1 + 2 h_R under the local model (their neighbours too)     */
  int L = local ? (1 + 2 * hR) / 2 + 1 : (1 + hR) / 2 + 1;
  if (d->min_cell > L) L = d->min_cell;
  if (L_override > 0) L = L_override;
  lay->L = L;
  for (int c = 0; c < 3; ++c) {
    int m = d->n[c] / L;
    m -= m & 1;
    if (m < 2 || (d->flags & ORC_FLAG_SINGLE_CELL)) m = 1;
    lay->m[c] = m;
  }
  return ORC_OK;
}

int orc_layout(const orc_desc *d, int32_t *L, int32_t *m) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  layout_t lay;
  compute_layout(d, &sh, 0, &lay, 0);
  *L = lay.L;
  for (int c = 0; c < 3; ++c) m[c] = lay.m[c];
  return ORC_OK;
}

static int cell_colour(const layout_t *lay, int cx, int cy, int cz) {
  (void)lay;
  return (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
}

/* The sweep's origin shift ("dynamically constructed" cells, Sec. 2.2):     */
/* w = Philox(counter (0, 0, t, 1), key seed), s_d = (w_d * n_d) >> 32.      */
static void sweep_shift(const orc_desc *d, uint32_t t, int s[3]) {
  if (d->flags & ORC_FLAG_NO_SHIFT) {
    s[0] = s[1] = s[2] = 0;
    return;
  }
  uint32_t w[4];
  philox_keyed(0, 0, t, 1, d->seed, w);
  for (int c = 0; c < 3; ++c) s[c] = (int)(((uint64_t)w[c] * (uint64_t)d->n[c]) >> 32);
}

typedef struct {
  const orc_desc *d;
  const shells_t *sh;
  const int64_t *V;
  const int64_t *T; /* local-energy table (non-NULL: local model, V unused) */
  int zt;           /* its count axis length */
  uint8_t *occ;
  uint32_t t;
  int shift[3];
  int mode, s;
  const uint32_t *tab;
  layout_t lay;
} sweep_ctx;

static int64_t local_delta_e(const orc_desc *d, const shells_t *sh, const int64_t *T, int zt,
                             uint8_t *occ, int64_t i, int64_t j);

/* All trials of one link cell (Sec. 2.2), in raster order: basis fastest,  */
/* then shifted x, y, z.  Trial k of cell cid in sweep t draws              */
/* Philox(counter (k >> 1, cid, t, 0), key seed); it uses words 2(k&1) and  */
/* 2(k&1)+1: the first picks the partner among the first-shell neighbours   */
/* (multiply-shift, no rejection), the second is the Metropolis variate.    */
static void run_cell(sweep_ctx *cx, uint32_t cid, orc_stats *st) {
  const orc_desc *d = cx->d;
  const int nb = basis_count(d->kind);
  const int mx = cx->lay.m[0], my = cx->lay.m[1];
  int c[3] = {(int)(cid % (uint32_t)mx), (int)((cid / (uint32_t)mx) % (uint32_t)my),
              (int)(cid / ((uint32_t)mx * (uint32_t)my))};
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)(((int64_t)c[a] * d->n[a]) / cx->lay.m[a]);
    hi[a] = (int)(((int64_t)(c[a] + 1) * d->n[a]) / cx->lay.m[a]);
  }
  const int z1 = cx->sh->z[0];
  uint32_t k = 0;
  for (int zs = lo[2]; zs < hi[2]; ++zs)
    for (int ys = lo[1]; ys < hi[1]; ++ys)
      for (int xs = lo[0]; xs < hi[0]; ++xs)
        for (int b = 0; b < nb; ++b, ++k) {
          int x = (xs + cx->shift[0]) % d->n[0];
          int y = (ys + cx->shift[1]) % d->n[1];
          int z = (zs + cx->shift[2]) % d->n[2];
          int64_t i = site_index(d, x, y, z, b);
          uint32_t w[4];
          philox_keyed(k >> 1, cid, cx->t, 0, d->seed, w);
          uint32_t wa = w[2 * (k & 1)], wb = w[2 * (k & 1) + 1];
          uint32_t dir = (uint32_t)(((uint64_t)wa * (uint64_t)z1) >> 32);
          int64_t j = neighbour(d, i, cx->sh->disp[cx->sh->start[0] + dir]);
          st->attempts++;
          if (cx->occ[i] == cx->occ[j]) continue;
          st->unlike++;
          int64_t dE = cx->T ? local_delta_e(d, cx->sh, cx->T, cx->zt, cx->occ, i, j)
                             : delta_e(d, cx->sh, cx->V, cx->occ, i, j);
          if (accept_move(dE, wb, cx->mode, cx->s, cx->tab)) {
            uint8_t tmp = cx->occ[i];
            cx->occ[i] = cx->occ[j];
            cx->occ[j] = tmp;
            st->accepted++;
            st->sum_dE += dE;
          }
        }
}

/* simple 64-bit mixing generator for the cell-order permutation used only */
/* by the schedule-independence test                                        */
static uint64_t splitmix(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* T of sweep i of n: linear from T_first to T_last; constant when they are */
/* equal (so T = +inf stays +inf).                                          */
static double sweep_temperature(double T_first, double T_last, uint32_t i, uint32_t n) {
  if (n <= 1 || T_first == T_last) return T_first;
  return T_first + (T_last - T_first) * (double)i / (double)(n - 1);
}

static int validate_occ(const orc_desc *d, const uint8_t *occ) {
  int64_t N = site_count(d);
  for (int64_t i = 0; i < N; ++i)
    if (occ[i] >= d->K) return 0;
  return 1;
}

/* n_sweeps full MC steps starting at sweep counter t0; temperature linear    */
/* from T_first to T_last over the call.  per_sweep[s] receives the integer   */
/* statistics of sweep s.                                                      */
static int sweeps_impl(const orc_desc *d, const int64_t *V, const int64_t *T, int zt, uint8_t *occ,
                       uint32_t t0, uint32_t n_sweeps, double T_first, double T_last,
                       orc_stats *per_sweep, const orc_opts *opts) {
  if (!valid_desc(d) || !validate_occ(d, occ)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  sweep_ctx cx;
  cx.d = d;
  cx.sh = &sh;
  cx.V = V;
  cx.T = T;
  cx.zt = zt;
  cx.occ = occ;
  compute_layout(d, &sh, opts ? opts->L_override : 0, &cx.lay, T != NULL);
  uint32_t n_cells = (uint32_t)cx.lay.m[0] * cx.lay.m[1] * cx.lay.m[2];
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * n_cells);
  if (!order) return ORC_EINVAL;
  uint64_t rng = opts ? opts->shuffle_seed : 0;
  uint32_t tab[3 * 512];
  for (uint32_t sw = 0; sw < n_sweeps; ++sw) {
    double T = sweep_temperature(T_first, T_last, sw, n_sweeps);
    int st_code = orc_thresholds(T, tab, &cx.s, &cx.mode);
    if (st_code != ORC_OK) {
      free(order);
      return st_code;
    }
    cx.tab = tab;
    cx.t = t0 + sw;
    sweep_shift(d, cx.t, cx.shift);
    orc_stats st = {0, 0, 0, 0};
    for (int colour = 0; colour < 8; ++colour) {
      uint32_t n_sel = 0;
      for (uint32_t cid = 0; cid < n_cells; ++cid) {
        int cxi = (int)(cid % (uint32_t)cx.lay.m[0]);
        int cyi = (int)((cid / (uint32_t)cx.lay.m[0]) % (uint32_t)cx.lay.m[1]);
        int czi = (int)(cid / ((uint32_t)cx.lay.m[0] * (uint32_t)cx.lay.m[1]));
        if (cell_colour(&cx.lay, cxi, cyi, czi) == colour) order[n_sel++] = cid;
      }
      if (opts && opts->shuffle_cells)
        for (uint32_t a = n_sel; a > 1; --a) {
          uint32_t b = (uint32_t)(splitmix(&rng) % a);
          uint32_t tmp = order[a - 1];
          order[a - 1] = order[b];
          order[b] = tmp;
        }
      for (uint32_t a = 0; a < n_sel; ++a) run_cell(&cx, order[a], &st);
    }
    if (per_sweep) per_sweep[sw] = st;
  }
  free(order);
  return ORC_OK;
}

int orc_sweeps(const orc_desc *d, const int64_t *V, uint8_t *occ, uint32_t t0, uint32_t n_sweeps,
               double T_first, double T_last, orc_stats *per_sweep, const orc_opts *opts) {
  return sweeps_impl(d, V, NULL, 0, occ, t0, n_sweeps, T_first, T_last, per_sweep, opts);
}

/* The trials of a chosen set of cells of one colour phase of sweep t (cells */
/* of one colour never interact, so any subset can be replayed alone).  Used */
/* to check sampled cells of lattices too large for full oracle sweeps.      */
int orc_phase_cells(const orc_desc *d, const int64_t *V, uint8_t *occ, uint32_t t, double T,
                    int colour, const uint32_t *cids, uint32_t n, orc_stats *st_out) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  sweep_ctx cx;
  cx.d = d;
  cx.sh = &sh;
  cx.V = V;
  cx.T = NULL;
  cx.zt = 0;
  cx.occ = occ;
  compute_layout(d, &sh, 0, &cx.lay, 0);
  uint32_t tab[3 * 512];
  int code = orc_thresholds(T, tab, &cx.s, &cx.mode);
  if (code != ORC_OK) return code;
  cx.tab = tab;
  cx.t = t;
  sweep_shift(d, t, cx.shift);
  uint32_t n_cells = (uint32_t)cx.lay.m[0] * cx.lay.m[1] * cx.lay.m[2];
  orc_stats st = {0, 0, 0, 0};
  for (uint32_t a = 0; a < n; ++a) {
    uint32_t cid = cids[a];
    if (cid >= n_cells) return ORC_EINVAL;
    int cxi = (int)(cid % (uint32_t)cx.lay.m[0]);
    int cyi = (int)((cid / (uint32_t)cx.lay.m[0]) % (uint32_t)cx.lay.m[1]);
    int czi = (int)(cid / ((uint32_t)cx.lay.m[0] * (uint32_t)cx.lay.m[1]));
    if (cell_colour(&cx.lay, cxi, cyi, czi) != colour) return ORC_EINVAL;
    run_cell(&cx, cid, &st);
  }
  if (st_out) *st_out = st;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The same trials with the cells of one colour shared out over OpenMP      */
/* threads (the CPU baseline on all host cores, and whole-phase replays of  */
/* lattices too large for one core).  Cells of one colour never touch one   */
/* another's interaction zones (the link-cell edge rule of Sec. 2.2), so    */
/* each cell's trials read and write the same values whatever the order or  */
/* thread: the occupancy is that of the sequential functions above, bit for */
/* bit, and the integer statistics are per-thread sums added at the end     */
/* (order-free).  Built without OpenMP these run on one thread.             */
/* ------------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static void run_cells_par(sweep_ctx *cx, const uint32_t *cids, uint32_t n, int n_threads,
                          orc_stats *st) {
  uint64_t att = 0, unl = 0, acc = 0;
  int64_t sde = 0;
  if (n_threads < 1) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads) \
    reduction(+ : att, unl, acc, sde)
#endif
  for (int64_t a = 0; a < (int64_t)n; ++a) {
    orc_stats one = {0, 0, 0, 0};
    run_cell(cx, cids[a], &one);
    att += one.attempts;
    unl += one.unlike;
    acc += one.accepted;
    sde += one.sum_dE;
  }
  st->attempts += att;
  st->unlike += unl;
  st->accepted += acc;
  st->sum_dE += sde;
}

int orc_phase_cells_par(const orc_desc *d, const int64_t *V, uint8_t *occ, uint32_t t, double T,
                        int colour, const uint32_t *cids, uint32_t n, int n_threads,
                        orc_stats *st_out) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  sweep_ctx cx;
  cx.d = d;
  cx.sh = &sh;
  cx.V = V;
  cx.T = NULL;
  cx.zt = 0;
  cx.occ = occ;
  compute_layout(d, &sh, 0, &cx.lay, 0);
  uint32_t tab[3 * 512];
  int code = orc_thresholds(T, tab, &cx.s, &cx.mode);
  if (code != ORC_OK) return code;
  cx.tab = tab;
  cx.t = t;
  sweep_shift(d, t, cx.shift);
  uint32_t n_cells = (uint32_t)cx.lay.m[0] * cx.lay.m[1] * cx.lay.m[2];
  for (uint32_t a = 0; a < n; ++a) {
    uint32_t cid = cids[a];
    if (cid >= n_cells) return ORC_EINVAL;
    int cxi = (int)(cid % (uint32_t)cx.lay.m[0]);
    int cyi = (int)((cid / (uint32_t)cx.lay.m[0]) % (uint32_t)cx.lay.m[1]);
    int czi = (int)(cid / ((uint32_t)cx.lay.m[0] * (uint32_t)cx.lay.m[1]));
    if (cell_colour(&cx.lay, cxi, cyi, czi) != colour) return ORC_EINVAL;
  }
  orc_stats st = {0, 0, 0, 0};
  run_cells_par(&cx, cids, n, n_threads, &st);
  if (st_out) *st_out = st;
  return ORC_OK;
}

int orc_sweeps_par(const orc_desc *d, const int64_t *V, uint8_t *occ, uint32_t t0,
                   uint32_t n_sweeps, double T_first, double T_last, orc_stats *per_sweep,
                   int n_threads) {
  if (!valid_desc(d) || !validate_occ(d, occ)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  sweep_ctx cx;
  cx.d = d;
  cx.sh = &sh;
  cx.V = V;
  cx.T = NULL;
  cx.zt = 0;
  cx.occ = occ;
  compute_layout(d, &sh, 0, &cx.lay, 0);
  uint32_t n_cells = (uint32_t)cx.lay.m[0] * cx.lay.m[1] * cx.lay.m[2];
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * n_cells);
  if (!order) return ORC_EINVAL;
  uint32_t tab[3 * 512];
  for (uint32_t sw = 0; sw < n_sweeps; ++sw) {
    double T = sweep_temperature(T_first, T_last, sw, n_sweeps);
    int st_code = orc_thresholds(T, tab, &cx.s, &cx.mode);
    if (st_code != ORC_OK) {
      free(order);
      return st_code;
    }
    cx.tab = tab;
    cx.t = t0 + sw;
    sweep_shift(d, cx.t, cx.shift);
    orc_stats st = {0, 0, 0, 0};
    for (int colour = 0; colour < 8; ++colour) {
      uint32_t n_sel = 0;
      for (uint32_t cid = 0; cid < n_cells; ++cid) {
        int cxi = (int)(cid % (uint32_t)cx.lay.m[0]);
        int cyi = (int)((cid / (uint32_t)cx.lay.m[0]) % (uint32_t)cx.lay.m[1]);
        int czi = (int)(cid / ((uint32_t)cx.lay.m[0] * (uint32_t)cx.lay.m[1]));
        if (cell_colour(&cx.lay, cxi, cyi, czi) == colour) order[n_sel++] = cid;
      }
      run_cells_par(&cx, order, n_sel, n_threads, &st);
    }
    if (per_sweep) per_sweep[sw] = st;
  }
  free(order);
  return ORC_OK;
}

/* Sweep origin shift, exported for the tests. */
void orc_sweep_shift(const orc_desc *d, uint32_t t, int32_t *s) {
  int v[3];
  sweep_shift(d, t, v);
  s[0] = v[0];
  s[1] = v[1];
  s[2] = v[2];
}

/* ------------------------------------------------------------------------ */
/* Replica exchange (parallel tempering, Sec. 2.2, Eqs. 6-7).  Replicas of   */
/* one system run at temperatures T[0..n); perm[k] is the replica currently  */
/* at temperature T[k], E[r] its energy (q units).  Round `round` attempts   */
/* the neighbour pairs (k, k+1) with k = round mod 2, round mod 2 + 2, ...:  */
/*   Delta = (1/k_B)(1/T_k - 1/T_{k+1}) (E_{perm[k]} - E_{perm[k+1]}) [eV],   */
/*   accepted with probability min(1, exp(Delta)) (Eq. 6), i.e. iff         */
/*   Delta >= 0 or u < exp(Delta), u uniform in [0, 1) from the 53 high bits */
/*   of words 0, 1 of Philox(counter = (k, round, 0, 3), key = seed);        */
/* an accepted pair exchanges its replicas' temperatures (perm[k] and        */
/* perm[k+1] swap).  acc[k] = 1 for an accepted pair (k, k+1), else 0.       */
/* Reading: beta = 1/(k_B T) as for the acceptance tables, the energy        */
/* difference formed exactly in integers and scaled by 2^-32 to eV.          */
/* ------------------------------------------------------------------------ */
int orc_exchange(uint32_t n, const int64_t *E, const double *T, uint64_t seed, uint32_t round,
                 uint32_t *perm, uint8_t *acc) {
  if (n < 2) return ORC_EINVAL;
  for (uint32_t k = 0; k < n; ++k) {
    if (!(T[k] > 0) || isinf(T[k]) || perm[k] >= n) return ORC_EINVAL;
    acc[k] = 0;
  }
  for (uint32_t k = round % 2; k + 1 < n; k += 2) {
    const double beta_a = 1.0 / (ORC_KB * T[k]);
    const double beta_b = 1.0 / (ORC_KB * T[k + 1]);
    const __int128 diff = (__int128)E[perm[k]] - (__int128)E[perm[k + 1]];
    const double de_ev = ldexp((double)diff, -32);
    const double delta = (beta_a - beta_b) * de_ev;
    uint32_t w[4];
    philox_keyed(k, round, 0u, 3u, seed, w);
    const double u = ldexp((double)((((uint64_t)w[0] << 32) | w[1]) >> 11), -53);
    if (delta >= 0.0 || u < exp(delta)) {
      const uint32_t t = perm[k];
      perm[k] = perm[k + 1];
      perm[k + 1] = t;
      acc[k] = 1;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Composition profile along a cylinder (the atom-probe-like analysis of     */
/* Sec. 3.2).  Site (x, y, z, b) sits at h = 2*(x,y,z) + basis_b (half      */
/* units).  Inside: t = (h_axis - o_axis) mod 2n_axis < length, and the sum  */
/* over the other two axes of d^2, d = (h_d - o_d) mod 2n_d taken in        */
/* (-n_d, n_d], is <= r2max.  counts[bin * K + sigma] += 1 with              */
/* bin = t * n_bins / length.                                                */
/* ------------------------------------------------------------------------ */
static int64_t mod_pos(int64_t v, int64_t n) {
  int64_t r = v % n;
  return r < 0 ? r + n : r;
}

int orc_profile(const orc_desc *d, const uint8_t *occ, int axis, const int32_t *origin,
                uint64_t r2max, uint32_t length, uint32_t n_bins, uint64_t *counts) {
  if (!valid_desc(d) || axis < 0 || axis > 2 || n_bins < 1 || length < 1 ||
      length > 2u * (uint32_t)d->n[axis])
    return ORC_EINVAL;
  memset(counts, 0, sizeof(uint64_t) * n_bins * (size_t)d->K);
  const int nb = basis_count(d->kind);
  for (int z = 0; z < d->n[2]; ++z)
    for (int y = 0; y < d->n[1]; ++y)
      for (int x = 0; x < d->n[0]; ++x)
        for (int b = 0; b < nb; ++b) {
          int bv[3];
          basis_vec(d->kind, b, bv);
          const int64_t h[3] = {2 * x + bv[0], 2 * y + bv[1], 2 * z + bv[2]};
          const int64_t t = mod_pos(h[axis] - origin[axis], 2 * (int64_t)d->n[axis]);
          if (t >= (int64_t)length) continue;
          uint64_t r2 = 0;
          for (int k = 0; k < 3; ++k) {
            if (k == axis) continue;
            int64_t dd = mod_pos(h[k] - origin[k], 2 * (int64_t)d->n[k]);
            if (dd > d->n[k]) dd -= 2 * (int64_t)d->n[k];
            r2 += (uint64_t)(dd * dd);
          }
          if (r2 > r2max) continue;
          const uint64_t bin = (uint64_t)t * n_bins / length;
          const uint8_t s = occ[site_index(d, x, y, z, b)];
          if (s >= d->K) return ORC_EINVAL;
          counts[bin * (uint64_t)d->K + s] += 1;
        }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Clusters (precipitates, Sec. 3.2): connected components of the sites     */
/* whose species has its bit set in `mask`, connected through first-shell   */
/* neighbours (periodic).  Sequential union-find over every first-shell     */
/* vector of every member site; sizes[0..*n) in descending order.            */
/* ------------------------------------------------------------------------ */
static int64_t uf_find(int64_t *par, int64_t x) {
  int64_t r = x;
  while (par[r] != r) r = par[r];
  while (par[x] != r) {
    const int64_t nx = par[x];
    par[x] = r;
    x = nx;
  }
  return r;
}

static int cmp_desc_u64(const void *a, const void *b) {
  const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? 1 : (x > y ? -1 : 0);
}

int orc_clusters(const orc_desc *d, const uint8_t *occ, uint32_t mask, uint64_t *sizes,
                 uint64_t *n_out) {
  if (!valid_desc(d)) return ORC_EINVAL;
  shells_t sh;
  if (build_shells(d->kind, 1, &sh) != ORC_OK) return ORC_EINVAL;
  const int64_t N = site_count(d);
  int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  uint64_t *cnt = (uint64_t *)calloc((size_t)N, sizeof(uint64_t));
  if (!par || !cnt) {
    free(par);
    free(cnt);
    return ORC_EINVAL;
  }
  for (int64_t i = 0; i < N; ++i) par[i] = ((mask >> occ[i]) & 1u) ? i : -1;
  for (int64_t i = 0; i < N; ++i) {
    if (par[i] < 0) continue;
    for (int k = 0; k < sh.z[0]; ++k) {
      const int64_t j = neighbour(d, i, sh.disp[k]);
      if (par[j] < 0) continue;
      const int64_t a = uf_find(par, i), b = uf_find(par, j);
      if (a != b) par[a < b ? b : a] = a < b ? a : b;
    }
  }
  for (int64_t i = 0; i < N; ++i)
    if (par[i] >= 0) cnt[uf_find(par, i)] += 1;
  uint64_t n = 0;
  for (int64_t i = 0; i < N; ++i)
    if (cnt[i]) sizes[n++] = cnt[i];
  qsort(sizes, (size_t)n, sizeof(uint64_t), cmp_desc_u64);
  *n_out = n;
  free(par);
  free(cnt);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Local-energy model.  The paper's second model (qSRO, Sec. 3) is a general */
/* nonlinear short-range model: a trial's energy change comes from the local */
/* energies of all the sites of its interaction zone, each recomputed.  Its  */
/* functional form is not printed; the reading taken here:                    */
/*   E = sum_i eps(i),   eps(i) = sum_m sum_s T_m[s_i][s][c_{i,m,s}],         */
/* c_{i,m,s} = the number of shell-m displacements of i that land on species */
/* s (each displacement counted, so a site reached twice on a tiny periodic  */
/* lattice counts twice).  T: [M][K][K][zt] int64 in q units, zt = 1 + the   */
/* largest z_m in use; any function of each count (EPI is the linear case    */
/* T_m[a][s][c] = c V_m(a, s) / 2).  A swap of i and j changes eps only on   */
/* U = {i, j} u shells(i) u shells(j) (shells are closed under negation), so */
/* dE = sum over the distinct sites k of U of eps_after(k) - eps_before(k).  */
/* The trial reads up to 1 + 2 h_R half units from its cell, hence the link  */
/* cells of edge floor((1 + 2 h_R)/2) + 1.  M <= 3, K <= 8.                   */
/* ------------------------------------------------------------------------ */
#define ORC_LOCAL_MAX_K 8
#define ORC_LOCAL_MAX_M 3

static int local_width(const shells_t *sh) {
  int z = 0;
  for (int m = 0; m < sh->M; ++m)
    if (sh->z[m] > z) z = sh->z[m];
  return z + 1;
}

int orc_local_width(int kind, int M) {
  shells_t sh;
  if ((kind != 0 && kind != 1) || M < 1 || M > ORC_LOCAL_MAX_M) return -1;
  if (build_shells(kind, M, &sh) != ORC_OK) return -1;
  return local_width(&sh);
}

static int valid_local(const orc_desc *d) {
  return valid_desc(d) && d->M <= ORC_LOCAL_MAX_M && d->K <= ORC_LOCAL_MAX_K;
}

/* eps of site k: its species and the species counts of each of its shells */
static int64_t local_eps(const orc_desc *d, const shells_t *sh, const int64_t *T, int zt,
                         const uint8_t *occ, int64_t k) {
  const int K = d->K;
  int64_t e = 0;
  for (int m = 0; m < sh->M; ++m) {
    int cnt[ORC_LOCAL_MAX_K] = {0};
    for (int t = sh->start[m]; t < sh->start[m + 1]; ++t) cnt[occ[neighbour(d, k, sh->disp[t])]]++;
    for (int s = 0; s < K; ++s) e += T[(((int64_t)m * K + occ[k]) * K + s) * zt + cnt[s]];
  }
  return e;
}

/* dE of swapping i and j: the distinct sites of U, each eps evaluated with  */
/* the occupancy before and after the swap (the swap is undone on return).   */
static int64_t local_delta_e(const orc_desc *d, const shells_t *sh, const int64_t *T, int zt,
                             uint8_t *occ, int64_t i, int64_t j) {
  int64_t U[2 + 2 * ORC_MAX_DISP];
  int nu = 0;
  int64_t cand[2 + 2 * ORC_MAX_DISP];
  int nc = 0;
  cand[nc++] = i;
  cand[nc++] = j;
  for (int t = 0; t < sh->total; ++t) cand[nc++] = neighbour(d, i, sh->disp[t]);
  for (int t = 0; t < sh->total; ++t) cand[nc++] = neighbour(d, j, sh->disp[t]);
  for (int a = 0; a < nc; ++a) {
    int seen = 0;
    for (int b = 0; b < nu; ++b) seen |= U[b] == cand[a];
    if (!seen) U[nu++] = cand[a];
  }
  int64_t before = 0, after = 0;
  for (int a = 0; a < nu; ++a) before += local_eps(d, sh, T, zt, occ, U[a]);
  uint8_t tmp = occ[i];
  occ[i] = occ[j];
  occ[j] = tmp;
  for (int a = 0; a < nu; ++a) after += local_eps(d, sh, T, zt, occ, U[a]);
  occ[j] = occ[i];
  occ[i] = tmp;
  return after - before;
}

int orc_local_energy(const orc_desc *d, const int64_t *T, const uint8_t *occ, int64_t *E) {
  if (!valid_local(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  const int zt = local_width(&sh);
  __int128 acc = 0;
  const int64_t N = site_count(d);
  for (int64_t k = 0; k < N; ++k) acc += local_eps(d, &sh, T, zt, occ, k);
  if (acc > (__int128)INT64_MAX || acc < (__int128)INT64_MIN) return ORC_EOVERFLOW;
  *E = (int64_t)acc;
  return ORC_OK;
}

int orc_local_delta_e(const orc_desc *d, const int64_t *T, const uint8_t *occ, int64_t i,
                      int64_t j, int64_t *dE) {
  if (!valid_local(d)) return ORC_EINVAL;
  const int64_t N = site_count(d);
  if (i < 0 || j < 0 || i >= N || j >= N) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  uint8_t *o = (uint8_t *)malloc((size_t)N);
  if (!o) return ORC_EINVAL;
  memcpy(o, occ, (size_t)N);
  *dE = local_delta_e(d, &sh, T, local_width(&sh), o, i, j);
  free(o);
  return ORC_OK;
}

int orc_local_layout(const orc_desc *d, int32_t *L, int32_t *m) {
  if (!valid_local(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  layout_t lay;
  compute_layout(d, &sh, 0, &lay, 1);
  *L = lay.L;
  for (int c = 0; c < 3; ++c) m[c] = lay.m[c];
  return ORC_OK;
}

int orc_local_sweeps(const orc_desc *d, const int64_t *T, uint8_t *occ, uint32_t t0,
                     uint32_t n_sweeps, double T_first, double T_last, orc_stats *per_sweep,
                     const orc_opts *opts) {
  if (!valid_local(d)) return ORC_EINVAL;
  shells_t sh;
  build_shells(d->kind, d->M, &sh);
  return sweeps_impl(d, NULL, T, local_width(&sh), occ, t0, n_sweeps, T_first, T_last, per_sweep,
                     opts);
}
