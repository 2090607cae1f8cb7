/*
 * ed_oracle.c -- THE ORACLE.  Test infrastructure only: tests/, the smoke check
 * and the benchmark's CPU-baseline / reference leg may call it; the product path
 * never does.
 *
 * A plain, slow restatement of the symmetry-adapted spin-1/2 Hamiltonian of
 * Wietek & Laeuchli (arXiv:1804.05028), written from the definitions only:
 *
 *   - int(s): label p is bit N-1-p, up = 1 (Sec. II, Eq. 1; ordering by int);
 *   - group action (g s)[perm[g][p]] = s[p];
 *   - representative = the orbit element of smallest int, found by applying
 *     EVERY group element bit by bit (Eqs. 3-4; the "apply all symmetries"
 *     option of Sec. III);
 *   - symmetry-adapted state |s_rho> = (1/N_s) sum_g chi(g)^* g|s> (Eq. 2), whose
 *     squared norm is proportional to sum_{h in Stab(s)} chi(h); a
 *     representative is kept only when that sum is non-zero;
 *   - matrix element of a non-branching term: <j|H_k|i> = c chi(h)^* N_j/N_i with
 *     s_j = h s' the representative of s' = H_k s_i, N_s = sqrt(|G| |Stab(s)|)
 *     (Eq. 5 with the conjugation that Eq. 2 implies).
 *
 * No sublattice tables, no prefix index, no blocking: every call loops over the
 * whole group.  fp64 throughout.  OpenMP only splits independent states.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
  int32_t N;               /* sites, <= 64 */
  int32_t n_sym;           /* |G| */
  int32_t phase_denom;     /* chi(g) = exp(2 pi i phase_num[g] / phase_denom) */
  int32_t n_bonds;
  int32_t n_classes;
  int32_t pad;
  const int32_t *perm;     /* [n_sym][N] */
  const int32_t *phase_num;/* [n_sym] */
  const int32_t *bonds;    /* [n_bonds][2] */
  const int32_t *bond_class;
  const double *J;         /* [n_classes] exchange (flip amplitude J/2) */
  const double *Jz;        /* [n_classes] anisotropy of the S^z S^z part */
  const uint8_t *flip;     /* [n_sym] or NULL: element g also reverses every spin */
} or_problem;

static inline int spin(uint64_t s, int N, int p) { return (int)((s >> (N - 1 - p)) & 1ULL); }

/* (g s)[perm[p]] = s[p], one site at a time; an element with the spin flip then
 * reverses every spin (up <-> down) */
static uint64_t apply_sym(const or_problem *P, int g, uint64_t s) {
  const int32_t *perm = P->perm + (size_t)g * P->N;
  uint64_t r = 0;
  for (int p = 0; p < P->N; p++)
    r |= (uint64_t)spin(s, P->N, p) << (P->N - 1 - perm[p]);
  if (P->flip && P->flip[g]) {
    const uint64_t all = (P->N == 64) ? ~0ULL : ((1ULL << P->N) - 1ULL);
    r ^= all;
  }
  return r;
}

void or_apply_sym(const or_problem *P, int g, const uint64_t *s, int64_t n, uint64_t *out) {
  for (int64_t i = 0; i < n; i++) out[i] = apply_sym(P, g, s[i]);
}

/* Eq. 4 by brute force: smallest orbit element, the first group element (in
 * group order) reaching it, and how many group elements reach it. */
static void representative(const or_problem *P, uint64_t s, uint64_t *rep, int32_t *g_first,
                           int32_t *n_min) {
  uint64_t best = ~0ULL;
  int32_t gb = -1, cnt = 0;
  for (int g = 0; g < P->n_sym; g++) {
    uint64_t t = apply_sym(P, g, s);
    if (t < best) { best = t; gb = g; cnt = 1; }
    else if (t == best) cnt++;
  }
  *rep = best; *g_first = gb; *n_min = cnt;
}

/* Sum of chi over the stabiliser of s, as (re, im): Eq. 2's norm up to |G|/N^2. */
static void stab_char_sum(const or_problem *P, uint64_t s, double *re, double *im, int32_t *order) {
  double a = 0, b = 0;
  int32_t cnt = 0;
  for (int g = 0; g < P->n_sym; g++) {
    if (apply_sym(P, g, s) == s) {
      double ph = 2.0 * M_PI * (double)P->phase_num[g] / (double)P->phase_denom;
      a += cos(ph); b += sin(ph); cnt++;
    }
  }
  *re = a; *im = b; *order = cnt;
}

static int kept(const or_problem *P, uint64_t rep, int32_t *order) {
  double re, im;
  stab_char_sum(P, rep, &re, &im, order);
  return (re * re + im * im) > 0.25;   /* the sum is either 0 or |Stab| >= 1 */
}

/* For each state: representative, first minimising element, |Stab(rep)|, and
 * whether the representative survives the projection. */
void or_representatives(const or_problem *P, const uint64_t *s, int64_t n, uint64_t *rep,
                        int32_t *g, int32_t *stab, int32_t *is_kept) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; i++) {
    int32_t nm, order;
    representative(P, s[i], &rep[i], &g[i], &nm);
    is_kept[i] = kept(P, rep[i], &order);
    stab[i] = order;
  }
}

static int popcount64(uint64_t x) { int c = 0; while (x) { x &= x - 1; c++; } return c; }

/* Is s its own representative (no group element gives a smaller int)? */
static int is_rep(const or_problem *P, uint64_t s) {
  for (int g = 0; g < P->n_sym; g++)
    if (apply_sym(P, g, s) < s) return 0;
  return 1;
}

/* Basis of the sector: every s with n_up up spins, in increasing int, that is
 * its own representative and survives the projection (Alg. 3's loop over all
 * configurations, single process).  Two passes over 64 equal slices of the
 * integer range so that the output is ordered.  Returns the dimension; writes
 * at most `cap` states (out may be NULL to count only). */
int64_t or_basis(const or_problem *P, int n_up, uint64_t *out, int32_t *stab_out, int64_t cap) {
  const int NS = 64;
  const uint64_t total = (P->N == 64) ? 0 : (1ULL << P->N);
  int64_t counts[64];
  uint64_t lo[65];
  for (int c = 0; c <= NS; c++) lo[c] = (uint64_t)(((__uint128_t)total * c) / NS);
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < NS; c++) {
    int64_t k = 0;
    for (uint64_t s = lo[c]; s < lo[c + 1]; s++) {
      if (popcount64(s) != n_up) continue;
      int32_t order;
      if (is_rep(P, s) && kept(P, s, &order)) k++;
    }
    counts[c] = k;
  }
  int64_t off[65];
  off[0] = 0;
  for (int c = 0; c < NS; c++) off[c + 1] = off[c] + counts[c];
  if (out && off[NS] <= cap) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < NS; c++) {
      int64_t k = off[c];
      for (uint64_t s = lo[c]; s < lo[c + 1]; s++) {
        if (popcount64(s) != n_up) continue;
        int32_t order;
        if (is_rep(P, s) && kept(P, s, &order)) {
          out[k] = s;
          if (stab_out) stab_out[k] = order;
          k++;
        }
      }
    }
  }
  return off[NS];
}

/* Column i of the symmetry-adapted Hamiltonian, from the representative s_i:
 *   diagonal  sum_b J_c Jz_c (+1/4 parallel, -1/4 antiparallel)        (Eq. 21)
 *   for each antiparallel bond (in bond order): s' = s_i with both spins
 *   exchanged, amplitude c = J_c/2; representative s_j = h s'; if s_j survives
 *   the projection, emit (s_j, c chi(h)^* sqrt(|Stab_j| / |Stab_i|)), which is
 *   <j|H_k|i> (Eq. 5, conjugation from Eq. 2, N_s = sqrt(|G||Stab(s)|)).
 * Returns the number of emitted terms (at most n_bonds). */
int32_t or_column(const or_problem *P, uint64_t s_i, double *diag, uint64_t *rep_out,
                  double *re_out, double *im_out) {
  int32_t order_i;
  double sre, sim;
  stab_char_sum(P, s_i, &sre, &sim, &order_i);
  double d = 0.0;
  int32_t nt = 0;
  for (int b = 0; b < P->n_bonds; b++) {
    int a = P->bonds[2 * b], c = P->bonds[2 * b + 1];
    int cls = P->bond_class[b];
    int sa = spin(s_i, P->N, a), sc = spin(s_i, P->N, c);
    if (sa == sc) { d += 0.25 * P->J[cls] * P->Jz[cls]; continue; }
    d -= 0.25 * P->J[cls] * P->Jz[cls];
    uint64_t sp = s_i ^ (1ULL << (P->N - 1 - a)) ^ (1ULL << (P->N - 1 - c));
    uint64_t rep; int32_t h, nm, order_j;
    representative(P, sp, &rep, &h, &nm);
    if (!kept(P, rep, &order_j)) continue;
    double amp = 0.5 * P->J[cls] * sqrt((double)order_j / (double)order_i);
    double ph = 2.0 * M_PI * (double)P->phase_num[h] / (double)P->phase_denom;
    rep_out[nt] = rep;
    re_out[nt] = amp * cos(ph);
    im_out[nt] = -amp * sin(ph);   /* chi(h)^* */
    nt++;
  }
  *diag = d;
  return nt;
}

/* or_column for many representatives: terms of column r start at
 * r * n_bonds; nterm[r] says how many are valid. */
void or_columns(const or_problem *P, const uint64_t *s, int64_t n, double *diag, int32_t *nterm,
                uint64_t *rep_out, double *re_out, double *im_out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < n; r++) {
    size_t o = (size_t)r * P->n_bonds;
    nterm[r] = or_column(P, s[r], &diag[r], rep_out + o, re_out + o, im_out + o);
  }
}

/* Position of s in the sorted basis by binary search over the whole array (Sec. IV's
 * Basis without a prefix map), or -1 when s is not in it. */
static int64_t basis_index(const uint64_t *basis, int64_t D, uint64_t s) {
  int64_t lo = 0, hi = D;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (basis[mid] < s) lo = mid + 1; else hi = mid;
  }
  return (lo < D && basis[lo] == s) ? lo : -1;
}

/* Rows [r0, r1) of the symmetry-adapted Hamiltonian as a stored sparse matrix (the
 * stored-matrix alternative to the matrix-free product, Sec. IV).  Row i of the
 * Hermitian H is the complex conjugate of column i:
 *   H[i][j] = conj(<j|H_k|i>) = c chi(h) N_j / N_i,   s_j = h s',  s' = H_k s_i,
 * with the representative s_j found by applying every group element (Eq. 4), and the
 * target's position j its index in the sorted basis `basis` (found by binary search).
 * A representative that is not in the basis is one the projection removes (its
 * stabiliser carries a non-trivial character, Eq. 2): the term contributes nothing.
 * |Stab(s_j)| is read from `stab`, the stabiliser orders that or_basis found for the
 * same states.  Each row gets n_bonds slots starting at (i - r0) * n_bonds; nterm[i - r0]
 * says how many are used, in bond order.  diag[i - r0] is the S^z S^z part (Eq. 21). */
void or_rows_slots(const or_problem *P, const uint64_t *basis, const int32_t *stab, int64_t D,
                   int64_t r0, int64_t r1, double *diag, int32_t *nterm, uint32_t *col,
                   double *re, double *im) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = r0; i < r1; i++) {
    const uint64_t s_i = basis[i];
    const size_t o = (size_t)(i - r0) * (size_t)P->n_bonds;
    double d = 0.0;
    int32_t nt = 0;
    for (int b = 0; b < P->n_bonds; b++) {
      const int a = P->bonds[2 * b], c = P->bonds[2 * b + 1];
      const int cls = P->bond_class[b];
      if (spin(s_i, P->N, a) == spin(s_i, P->N, c)) { d += 0.25 * P->J[cls] * P->Jz[cls]; continue; }
      d -= 0.25 * P->J[cls] * P->Jz[cls];
      if (P->J[cls] == 0.0) continue;   /* no exchange in this class: no off-diagonal entry */
      const uint64_t sp = s_i ^ (1ULL << (P->N - 1 - a)) ^ (1ULL << (P->N - 1 - c));
      uint64_t rep;
      int32_t h, nm;
      representative(P, sp, &rep, &h, &nm);
      const int64_t j = basis_index(basis, D, rep);
      if (j < 0) continue;
      const double amp = 0.5 * P->J[cls] * sqrt((double)stab[j] / (double)stab[i]);
      const double ph = 2.0 * M_PI * (double)P->phase_num[h] / (double)P->phase_denom;
      col[o + nt] = (uint32_t)j;
      re[o + nt] = amp * cos(ph);
      if (im) im[o + nt] = amp * sin(ph);
      nt++;
    }
    diag[i - r0] = d;
    nterm[i - r0] = nt;
  }
}

/* y = H x for n consecutive rows r0 .. r0+n-1 of H stored row by row (CSR: row r0+i
 * holds entries rowptr[i] .. rowptr[i+1]), real entries, fp64; diag and y point at
 * the block's first row, x is the whole vector.  Rows are independent. */
void or_csr_spmv(int64_t n, const int64_t *rowptr, const uint32_t *col, const double *val,
                 const double *diag, const double *x, double *y, int64_t r0) {
#pragma omp parallel for schedule(static, 4096)
  for (int64_t i = 0; i < n; i++) {
    double acc = diag[i] * x[r0 + i];
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) acc += val[k] * x[col[k]];
    y[i] = acc;
  }
}

/* The same for complex entries and vectors, interleaved (re, im). */
void or_csr_spmv_complex(int64_t n, const int64_t *rowptr, const uint32_t *col,
                         const double *vre, const double *vim, const double *diag,
                         const double *x, double *y, int64_t r0) {
#pragma omp parallel for schedule(static, 4096)
  for (int64_t i = 0; i < n; i++) {
    double ar = diag[i] * x[2 * (r0 + i)], ai = diag[i] * x[2 * (r0 + i) + 1];
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      const double xr = x[2 * col[k]], xi = x[2 * col[k] + 1];
      ar += vre[k] * xr - vim[k] * xi;
      ai += vre[k] * xi + vim[k] * xr;
    }
    y[2 * i] = ar;
    y[2 * i + 1] = ai;
  }
}

int or_max_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
