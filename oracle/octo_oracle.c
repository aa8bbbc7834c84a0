/*
 * Oracle for the octree FMM gravity solve (Marcello et al. 2021, Sec. 2.2) -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load this code.
 * It is a plain, slow, obviously correct FP64 restatement of what the solve computes, written
 * from the paper's description and from the mathematics of Cartesian expansions; it shares no
 * code with the CUDA library.
 *
 * Model (Sec. 2.1, Eq. 4 Poisson equation with G = 1, g = -grad phi; Sec. 2.2):
 *   - the domain [-1/2, 1/2]^3 is covered by an octree of 8^3-cell subgrids (Sec. 2.4);
 *     a subgrid is a leaf or has 8 children; proper nesting allows at most one level jump
 *     across subgrid boundaries (Sec. 2.4, Sec. 2.7);
 *   - every leaf cell i is a point mass m_i = rho_i dx^3 at its centre;
 *   - the exact answer being approximated is phi_i = -sum_j m_j/|x_i-x_j|,
 *     g_i = -sum_j m_j (x_i-x_j)/|x_i-x_j|^3 (oracle_direct below).
 *
 * The FMM restated (each step follows its definition; no shifts, blocking or reordering):
 *   1. Multipoles (Sec. 2.2: a cell's multipoles are built from its children's).  Since that
 *      composition is exact, the oracle uses the definition: for a cell A with leaf
 *      descendants i, m_A = sum m_i, X_A = sum m_i x_i / m_A (the expansion centre),
 *      M2_A = sum m_i r r, M3_A = sum m_i r r r with r = x_i - X_A.
 *   2. Opening criterion (Sec. 2.2): cells A, B at one level with geometric centres x_A, x_B
 *      are well separated iff theta' = dx / |x_A - x_B| < theta.  A interacts with B through
 *      the multipole interaction iff they are well separated and their parents are not (at the
 *      coarsest level, where cells have no parent, iff they are well separated).
 *   3. Interaction of A with B (reading of "relative to cell centres" with Dehnen's symmetric
 *      truncation): with R = X_A - X_B and D^(n) = grad^n (1/|R|), the local expansion of A is
 *      the cubic polynomial phi_A(X_A + s) = sum_k (1/k!) L^(k) s^k with
 *        L0  = -(m_B D0 + 1/2 D2:M2_B - 1/6 D3:M3_B)
 *        L1  = -(m_B D1 + 1/2 D3:M2_B)
 *        L2  = -m_B D2,  L3 = -m_B D3           (total order k + n <= 3 in both expansions).
 *      The angular-momentum correction (Sec. 2.2, "additional higher order multipoles"): the
 *      truncated pair force leaves the torque defect -R x C_AB with
 *        C_AB = 1/6 D4 : (m_B M3_A - m_A M3_B),
 *      which a force +C_AB spread over A in proportion to mass (acceleration C_AB / m_A) and
 *      -C_AB over B cancels exactly while keeping the force sum zero.
 *   4. The expansion of a child is derived from its parent's (Sec. 2.2).  Because that shift of
 *      a cubic polynomial is exact, the oracle evaluates every ancestor's polynomial directly at
 *      the leaf: phi_i = sum_{A contains i} phi_A(x_i), g_i = sum_A (-grad phi_A(x_i) + a_A).
 *   5. Leaf pairs whose cells are not well separated at the level of the coarser of the two
 *      leaves interact directly (point-mass sum).  Every leaf pair is then covered exactly once.
 *
 * The time derivative of the potential (Sec. 2.1: the FMM with the numerically computed
 * d(rho)/dt as the source, so that the two parts of the energy source term cancel when summed
 * over the grid): the same operator -- same lists, the same expansion centres X_A (rho's
 * centres of mass), the same truncation -- applied to a source s_i = (d rho/dt)_i dx^3.  About
 * those centres s has a dipole, so a cell carries S0 = sum s, S1 = sum s r, S2 = sum s r r,
 * S3 = sum s r r r (r = x_i - X_A), and expanding -s/|R + t - u| to total order 3 gives
 *        L_k = -sum_(n <= 3 - k) (-1)^n / n! D^(k+n) : S_n,
 * which is step 3 with the dipole terms added (S1 = 0 for rho itself).  Only the potential is
 * evaluated; there is no correction term.  With these centres the operator is symmetric, so
 * sum_i s_i phi_i = sum_i m_i (dphi/dt)_i up to rounding -- the cancellation the paper relies on.
 *
 * Readings where the paper is silent are listed in the design notes; this file implements them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NSUB 8
#define O_MAXLEV 10 /* levels 0..9 (the paper's merger models use 9 refinement levels) */
#define NMOM 40    /* m, X[3], M2[9], M3[27] */
#define NLOC 40    /* L0, L1[3], L2[9], L3[27] */

typedef struct otree {
  int depth;                     /* deepest level that has subgrids */
  int64_t count[O_MAXLEV];       /* subgrids per level */
  int32_t *ijk[O_MAXLEV];        /* [count][3], ordered by Morton key */
  uint8_t *leaf[O_MAXLEV];       /* [count] */
  int32_t *lookup[O_MAXLEV];     /* dense position -> subgrid index at that level, or -1 */
  int64_t *leaf_slot[O_MAXLEV];  /* subgrid -> ordinal among leaf subgrids, or -1 */
  int64_t *inner_slot[O_MAXLEV]; /* subgrid -> ordinal among refined subgrids, or -1 */
  int64_t n_sub, n_leaf_sub, n_inner_sub;
} otree;

/* ------------------------------------------------------------------------------------------ */
/* Tree                                                                                        */
/* ------------------------------------------------------------------------------------------ */
static int64_t pos_index(int lev, int64_t i, int64_t j, int64_t k) {
  int64_t n = (int64_t)1 << lev;
  return (i * n + j) * n + k;
}

static uint64_t morton_key(int lev, int64_t i, int64_t j, int64_t k) {
  uint64_t key = 0;
  for (int b = 0; b < lev; ++b) {
    key |= (uint64_t)((i >> b) & 1) << (3 * b + 2);
    key |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
    key |= (uint64_t)((k >> b) & 1) << (3 * b);
  }
  return key;
}

typedef struct { uint64_t key; int32_t i, j, k; } keyed;

static int cmp_keyed(const void *a, const void *b) {
  uint64_t x = ((const keyed *)a)->key, y = ((const keyed *)b)->key;
  return (x > y) - (x < y);
}

void oracle_tree_free(otree *t) {
  if (!t) return;
  for (int l = 0; l < O_MAXLEV; ++l) {
    free(t->ijk[l]); free(t->leaf[l]); free(t->lookup[l]);
    free(t->leaf_slot[l]); free(t->inner_slot[l]);
  }
  free(t);
}

/* Dense flags: level l (< max_level) holds 8^l entries indexed (i*2^l + j)*2^l + k.  A subgrid
 * that exists is refined when it is flagged or when proper nesting requires it; nesting (no more
 * than one level jump across subgrid boundaries, Sec. 2.4) holds when every refined subgrid
 * has all 26 same-level neighbours inside the domain.  The sets only grow, so iterating the two
 * rules to a fixed point terminates. */
otree *oracle_tree_build(int max_level, const uint8_t *flags, int64_t n_flags) {
  if (max_level < 0 || max_level >= O_MAXLEV) return NULL;
  int64_t need_flags = 0;
  for (int l = 0; l < max_level; ++l) need_flags += (int64_t)1 << (3 * l);
  if (n_flags != need_flags) return NULL;
  uint8_t *ex[O_MAXLEV] = {0}, *ref[O_MAXLEV] = {0}, *need[O_MAXLEV] = {0};
  int64_t off[O_MAXLEV];
  int64_t acc = 0;
  for (int l = 0; l <= max_level; ++l) {
    int64_t np = (int64_t)1 << (3 * l);
    ex[l] = (uint8_t *)calloc(np, 1);
    ref[l] = (uint8_t *)calloc(np, 1);
    need[l] = (uint8_t *)calloc(np, 1);
    off[l] = acc;
    if (l < max_level) acc += np;
  }
  ex[0][0] = 1;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int l = 0; l < max_level; ++l) {
      int64_t n = (int64_t)1 << l;
      for (int64_t p = 0; p < n * n * n; ++p) {
        uint8_t r = ex[l][p] && (flags[off[l] + p] || need[l][p]);
        if (r != ref[l][p]) { ref[l][p] = r; changed = 1; }
      }
      int64_t n2 = 2 * n;
      for (int64_t i = 0; i < n2; ++i)
        for (int64_t j = 0; j < n2; ++j)
          for (int64_t k = 0; k < n2; ++k) {
            uint8_t e = ref[l][pos_index(l, i / 2, j / 2, k / 2)];
            int64_t c = pos_index(l + 1, i, j, k);
            if (e != ex[l + 1][c]) { ex[l + 1][c] = e; changed = 1; }
          }
    }
    for (int l = 1; l < max_level; ++l) {
      int64_t n = (int64_t)1 << l;
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
          for (int64_t k = 0; k < n; ++k) {
            if (!ref[l][pos_index(l, i, j, k)]) continue;
            for (int di = -1; di <= 1; ++di)
              for (int dj = -1; dj <= 1; ++dj)
                for (int dk = -1; dk <= 1; ++dk) {
                  int64_t a = i + di, b = j + dj, c = k + dk;
                  if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) continue;
                  int64_t pp = pos_index(l - 1, a / 2, b / 2, c / 2);
                  if (!need[l - 1][pp]) { need[l - 1][pp] = 1; changed = 1; }
                }
          }
    }
  }
  otree *t = (otree *)calloc(1, sizeof(otree));
  t->depth = 0;
  for (int l = 0; l <= max_level; ++l) {
    int64_t n = (int64_t)1 << l, cnt = 0;
    for (int64_t p = 0; p < n * n * n; ++p) cnt += ex[l][p];
    if (cnt == 0) break;
    t->depth = l;
    keyed *ks = (keyed *)malloc(sizeof(keyed) * cnt);
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j)
        for (int64_t k = 0; k < n; ++k)
          if (ex[l][pos_index(l, i, j, k)]) {
            ks[q].key = morton_key(l, i, j, k);
            ks[q].i = (int32_t)i; ks[q].j = (int32_t)j; ks[q].k = (int32_t)k;
            ++q;
          }
    qsort(ks, cnt, sizeof(keyed), cmp_keyed);
    t->count[l] = cnt;
    t->ijk[l] = (int32_t *)malloc(sizeof(int32_t) * 3 * cnt);
    t->leaf[l] = (uint8_t *)malloc(cnt);
    t->lookup[l] = (int32_t *)malloc(sizeof(int32_t) * n * n * n);
    for (int64_t p = 0; p < n * n * n; ++p) t->lookup[l][p] = -1;
    for (int64_t s = 0; s < cnt; ++s) {
      t->ijk[l][3 * s] = ks[s].i; t->ijk[l][3 * s + 1] = ks[s].j; t->ijk[l][3 * s + 2] = ks[s].k;
      int64_t p = pos_index(l, ks[s].i, ks[s].j, ks[s].k);
      t->leaf[l][s] = (uint8_t)!ref[l][p];
      t->lookup[l][p] = (int32_t)s;
    }
    free(ks);
  }
  for (int l = 0; l <= t->depth; ++l) {
    t->leaf_slot[l] = (int64_t *)malloc(sizeof(int64_t) * (t->count[l] ? t->count[l] : 1));
    t->inner_slot[l] = (int64_t *)malloc(sizeof(int64_t) * (t->count[l] ? t->count[l] : 1));
    for (int64_t s = 0; s < t->count[l]; ++s) {
      t->n_sub++;
      if (t->leaf[l][s]) { t->leaf_slot[l][s] = t->n_leaf_sub++; t->inner_slot[l][s] = -1; }
      else { t->inner_slot[l][s] = t->n_inner_sub++; t->leaf_slot[l][s] = -1; }
    }
  }
  for (int l = 0; l <= max_level; ++l) { free(ex[l]); free(ref[l]); free(need[l]); }
  return t;
}

int oracle_tree_depth(const otree *t) { return t->depth; }
int64_t oracle_tree_n_subgrids(const otree *t) { return t->n_sub; }
int64_t oracle_tree_n_leaf_subgrids(const otree *t) { return t->n_leaf_sub; }

/* Rows (level, i, j, k, is_leaf) of every subgrid, by level then Morton key. */
void oracle_tree_subgrids(const otree *t, int32_t *out) {
  int64_t q = 0;
  for (int l = 0; l <= t->depth; ++l)
    for (int64_t s = 0; s < t->count[l]; ++s, ++q) {
      out[5 * q] = l;
      out[5 * q + 1] = t->ijk[l][3 * s];
      out[5 * q + 2] = t->ijk[l][3 * s + 1];
      out[5 * q + 3] = t->ijk[l][3 * s + 2];
      out[5 * q + 4] = t->leaf[l][s];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Opening criterion and stencil                                                               */
/* ------------------------------------------------------------------------------------------ */
/* theta' = dx / |x_A - x_B| < theta, with the same-level offset d in units of dx. */
static int well_separated(int64_t dx, int64_t dy, int64_t dz, double theta) {
  int64_t d2 = dx * dx + dy * dy + dz * dz;
  if (d2 == 0) return 0;
  return 1.0 / sqrt((double)d2) < theta;
}

static int64_t floordiv2(int64_t a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

/* Same-level interaction offsets for a cell whose position within its parent is `parity`
 * (bits x<<2 | y<<1 | z): offsets d, in lexicographic order, that are well separated while the
 * parents are not.  Returns the number of offsets (written when it fits in cap). */
int oracle_stencil(double theta, int parity, int32_t *out, int cap) {
  int64_t a[3] = {(parity >> 2) & 1, (parity >> 1) & 1, parity & 1};
  int W = 2 * (int)floor(1.0 / theta) + 1;
  int n = 0;
  for (int dx = -W; dx <= W; ++dx)
    for (int dy = -W; dy <= W; ++dy)
      for (int dz = -W; dz <= W; ++dz) {
        if (!well_separated(dx, dy, dz, theta)) continue;
        int64_t px = floordiv2(a[0] + dx), py = floordiv2(a[1] + dy), pz = floordiv2(a[2] + dz);
        if (well_separated(px, py, pz, theta)) continue;
        if (n < cap) { out[3 * n] = dx; out[3 * n + 1] = dy; out[3 * n + 2] = dz; }
        ++n;
      }
  return n;
}

/* ------------------------------------------------------------------------------------------ */
/* Cells                                                                                       */
/* ------------------------------------------------------------------------------------------ */
typedef struct { int lev; int64_t g[3]; } cellref; /* level and global cell coordinates */

static double cell_dx(int lev) { return 1.0 / (double)(NSUB * ((int64_t)1 << lev)); }

static void cell_centre(int lev, const int64_t g[3], double x[3]) {
  double dx = cell_dx(lev);
  for (int a = 0; a < 3; ++a) x[a] = -0.5 + ((double)g[a] + 0.5) * dx;
}

/* Subgrid index at `lev` holding global cell g, or -1 when that subgrid does not exist. */
static int64_t cell_subgrid(const otree *t, int lev, const int64_t g[3]) {
  if (lev > t->depth) return -1;
  int64_t n = (int64_t)NSUB << lev;
  for (int a = 0; a < 3; ++a)
    if (g[a] < 0 || g[a] >= n) return -1;
  return t->lookup[lev][pos_index(lev, g[0] / NSUB, g[1] / NSUB, g[2] / NSUB)];
}

static int64_t local_index(const int64_t g[3]) {
  return ((g[0] % NSUB) * NSUB + (g[1] % NSUB)) * NSUB + (g[2] % NSUB);
}

/* Moments of a cell: leaf cells are point masses at their centres; refined cells use the
 * stored definition-based moments. */
typedef struct {
  const otree *t;
  const double *rho;  /* leaf-cell density, canonical leaf order */
  double *inner_mom;  /* [n_inner_sub * 512][NMOM] */
} ctx_t;

static void cell_moments(const ctx_t *C, int lev, const int64_t g[3], double mom[NMOM]) {
  int64_t s = cell_subgrid(C->t, lev, g);
  if (C->t->leaf[lev][s]) {
    double dx = cell_dx(lev);
    memset(mom, 0, sizeof(double) * NMOM);
    mom[0] = C->rho[C->t->leaf_slot[lev][s] * 512 + local_index(g)] * dx * dx * dx;
    cell_centre(lev, g, mom + 1);
  } else {
    memcpy(mom, C->inner_mom + (C->t->inner_slot[lev][s] * 512 + local_index(g)) * NMOM,
           sizeof(double) * NMOM);
  }
}

/* Visit every leaf cell below (lev, g): callback receives the leaf's level and coordinates. */
typedef void (*leaf_visit_fn)(void *user, int lev, const int64_t g[3]);

static void visit_leaves(const otree *t, int lev, const int64_t g[3], leaf_visit_fn fn, void *user) {
  int64_t s = cell_subgrid(t, lev, g);
  if (s < 0) return;
  if (t->leaf[lev][s]) { fn(user, lev, g); return; }
  for (int o = 0; o < 8; ++o) {
    int64_t c[3] = {2 * g[0] + ((o >> 2) & 1), 2 * g[1] + ((o >> 1) & 1), 2 * g[2] + (o & 1)};
    visit_leaves(t, lev + 1, c, fn, user);
  }
}

/* Compensated (Neumaier 1974) running sum: the moment sums of a coarse cell run over up to
 * 10^6 leaves, and a plain running sum would lose up to ~N eps of their magnitude. */
typedef struct { double s, c; } csum;

static void csum_add(csum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

static double csum_val(const csum *a) { return a->s + a->c; }

typedef struct { const ctx_t *C; csum m, mx[3]; const double *X; csum M2[9], M3[27]; } mom_acc;

static void leaf_mass_of(const ctx_t *C, int lev, const int64_t g[3], double *m, double x[3]) {
  int64_t s = cell_subgrid(C->t, lev, g);
  double dx = cell_dx(lev);
  *m = C->rho[C->t->leaf_slot[lev][s] * 512 + local_index(g)] * dx * dx * dx;
  cell_centre(lev, g, x);
}

static void acc_first(void *u, int lev, const int64_t g[3]) {
  mom_acc *A = (mom_acc *)u;
  double m, x[3];
  leaf_mass_of(A->C, lev, g, &m, x);
  csum_add(&A->m, m);
  for (int a = 0; a < 3; ++a) csum_add(&A->mx[a], m * x[a]);
}

static void acc_second(void *u, int lev, const int64_t g[3]) {
  mom_acc *A = (mom_acc *)u;
  double m, x[3], r[3];
  leaf_mass_of(A->C, lev, g, &m, x);
  for (int a = 0; a < 3; ++a) r[a] = x[a] - A->X[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      csum_add(&A->M2[3 * a + b], m * r[a] * r[b]);
      for (int c = 0; c < 3; ++c) csum_add(&A->M3[9 * a + 3 * b + c], m * r[a] * r[b] * r[c]);
    }
}

/* Definition of the multipoles of one refined cell from all of its leaf descendants. */
static void inner_cell_moments(const ctx_t *C, int lev, const int64_t g[3], double mom[NMOM]) {
  mom_acc A;
  memset(&A, 0, sizeof(A));
  A.C = C;
  visit_leaves(C->t, lev, g, acc_first, &A);
  memset(mom, 0, sizeof(double) * NMOM);
  double m = csum_val(&A.m);
  mom[0] = m;
  if (m > 0) {
    for (int a = 0; a < 3; ++a) mom[1 + a] = csum_val(&A.mx[a]) / m;
  } else {
    cell_centre(lev, g, mom + 1);
  }
  A.X = mom + 1;
  visit_leaves(C->t, lev, g, acc_second, &A);
  for (int k = 0; k < 9; ++k) mom[4 + k] = csum_val(&A.M2[k]);
  for (int k = 0; k < 27; ++k) mom[13 + k] = csum_val(&A.M3[k]);
}

static void compute_inner_moments(ctx_t *C, int nthreads) {
  const otree *t = C->t;
  C->inner_mom = (double *)calloc((size_t)(t->n_inner_sub ? t->n_inner_sub : 1) * 512 * NMOM,
                                  sizeof(double));
  for (int l = 0; l <= t->depth; ++l) {
    int64_t cnt = t->count[l];
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t s = 0; s < cnt; ++s) {
      if (t->leaf[l][s]) continue;
      for (int64_t c = 0; c < 512; ++c) {
        int64_t g[3] = {(int64_t)t->ijk[l][3 * s] * NSUB + c / 64,
                        (int64_t)t->ijk[l][3 * s + 1] * NSUB + (c / 8) % 8,
                        (int64_t)t->ijk[l][3 * s + 2] * NSUB + c % 8};
        inner_cell_moments(C, l, g, C->inner_mom + (t->inner_slot[l][s] * 512 + c) * NMOM);
      }
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Expansions                                                                                  */
/* ------------------------------------------------------------------------------------------ */
static int kd(int a, int b) { return a == b; }

/* D^(n)_{a..} = d^n (1/|R|) / dR_a ..., written out from the derivatives of 1/r:
 *   D0 = 1/r, D1 = -R/r^3, D2 = 3RR/r^5 - I/r^3,
 *   D3 = -15RRR/r^7 + 3(R I)_sym3/r^5,
 *   D4 = 105RRRR/r^9 - 15(RR I)_sym6/r^7 + 3(I I)_sym3/r^5.
 * out: D0 | D1[3] | D2[9] | D3[27] | D4[81] (row-major full tensors). */
void oracle_dtensors(const double R[3], double *out) {
  double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  double r = sqrt(r2);
  double g0 = 1.0 / r;
  double g1 = -g0 / r2;
  double g2 = -3.0 * g1 / r2;
  double g3 = -5.0 * g2 / r2;
  double g4 = -7.0 * g3 / r2;
  double *D0 = out, *D1 = out + 1, *D2 = out + 4, *D3 = out + 13, *D4 = out + 40;
  D0[0] = g0;
  for (int a = 0; a < 3; ++a) {
    D1[a] = g1 * R[a];
    for (int b = 0; b < 3; ++b) {
      D2[3 * a + b] = g2 * R[a] * R[b] + g1 * kd(a, b);
      for (int c = 0; c < 3; ++c) {
        D3[9 * a + 3 * b + c] = g3 * R[a] * R[b] * R[c] +
                                g2 * (R[a] * kd(b, c) + R[b] * kd(a, c) + R[c] * kd(a, b));
        for (int d = 0; d < 3; ++d)
          D4[27 * a + 9 * b + 3 * c + d] =
              g4 * R[a] * R[b] * R[c] * R[d] +
              g3 * (R[a] * R[b] * kd(c, d) + R[a] * R[c] * kd(b, d) + R[a] * R[d] * kd(b, c) +
                    R[b] * R[c] * kd(a, d) + R[b] * R[d] * kd(a, c) + R[c] * R[d] * kd(a, b)) +
              g2 * (kd(a, b) * kd(c, d) + kd(a, c) * kd(b, d) + kd(a, d) * kd(b, c));
      }
    }
  }
}

/* Multipoles of a set of point masses about their centre of mass (the definition). */
void oracle_point_moments(int64_t n, const double *x, const double *m, double *mom) {
  memset(mom, 0, sizeof(double) * NMOM);
  double M = 0, mx[3] = {0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    M += m[i];
    for (int a = 0; a < 3; ++a) mx[a] += m[i] * x[3 * i + a];
  }
  mom[0] = M;
  for (int a = 0; a < 3; ++a) mom[1 + a] = M > 0 ? mx[a] / M : 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = x[3 * i + a] - mom[1 + a];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        mom[4 + 3 * a + b] += m[i] * r[a] * r[b];
        for (int c = 0; c < 3; ++c) mom[13 + 9 * a + 3 * b + c] += m[i] * r[a] * r[b] * r[c];
      }
  }
}

/* Adds the expansion of A due to B (step 3 of the header) into L and, with amc, the
 * angular-momentum-correction acceleration of A into ac. */
void oracle_m2l(const double *momA, const double *momB, int amc, double *L, double *ac) {
  double D[121];
  double R[3] = {momA[1] - momB[1], momA[2] - momB[2], momA[3] - momB[3]};
  oracle_dtensors(R, D);
  const double *D0 = D, *D1 = D + 1, *D2 = D + 4, *D3 = D + 13, *D4 = D + 40;
  double mB = momB[0];
  const double *M2B = momB + 4, *M3B = momB + 13;
  double t2 = 0, t3 = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      t2 += D2[3 * a + b] * M2B[3 * a + b];
      for (int c = 0; c < 3; ++c) t3 += D3[9 * a + 3 * b + c] * M3B[9 * a + 3 * b + c];
    }
  L[0] += -(mB * D0[0] + 0.5 * t2 - t3 / 6.0);
  for (int a = 0; a < 3; ++a) {
    double s = 0;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) s += D3[9 * a + 3 * b + c] * M2B[3 * b + c];
    L[1 + a] += -(mB * D1[a] + 0.5 * s);
    for (int b = 0; b < 3; ++b) {
      L[4 + 3 * a + b] += -mB * D2[3 * a + b];
      for (int c = 0; c < 3; ++c) L[13 + 9 * a + 3 * b + c] += -mB * D3[9 * a + 3 * b + c];
    }
  }
  if (amc && ac) {
    double mA = momA[0];
    const double *M3A = momA + 13;
    if (mA > 0) {
      for (int a = 0; a < 3; ++a) {
        double C = 0;
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d)
              C += D4[27 * a + 9 * b + 3 * c + d] *
                   (mB * M3A[9 * b + 3 * c + d] - mA * M3B[9 * b + 3 * c + d]);
        ac[a] += C / 6.0 / mA;
      }
    }
  }
}

/* Value and minus gradient of the cubic local expansion about X at point y. out: phi, g[3]. */
void oracle_local_eval(const double *L, const double *X, const double *y, double *out) {
  double s[3] = {y[0] - X[0], y[1] - X[1], y[2] - X[2]};
  double phi = L[0];
  for (int a = 0; a < 3; ++a) {
    phi += L[1 + a] * s[a];
    for (int b = 0; b < 3; ++b) {
      phi += 0.5 * L[4 + 3 * a + b] * s[a] * s[b];
      for (int c = 0; c < 3; ++c) phi += L[13 + 9 * a + 3 * b + c] * s[a] * s[b] * s[c] / 6.0;
    }
  }
  out[0] = phi;
  for (int a = 0; a < 3; ++a) {
    double d = L[1 + a];
    for (int b = 0; b < 3; ++b) {
      d += L[4 + 3 * a + b] * s[b];
      for (int c = 0; c < 3; ++c) d += 0.5 * L[13 + 9 * a + 3 * b + c] * s[b] * s[c];
    }
    out[1 + a] = -d;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Interaction lists                                                                           */
/* ------------------------------------------------------------------------------------------ */
/* Calls fn for every existing cell B in the multipole-interaction list of cell (lev, g). */
typedef void (*pair_fn)(void *user, int lev, const int64_t gB[3]);

static void for_each_m2l_partner(const otree *t, int lev, const int64_t g[3], double theta,
                                 pair_fn fn, void *user) {
  int64_t n = (int64_t)NSUB << lev;
  int64_t W = 2 * (int64_t)floor(1.0 / theta) + 1;
  if (lev == 0 || W > n) W = n;
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = g[a] - W < 0 ? 0 : g[a] - W;
    hi[a] = g[a] + W > n - 1 ? n - 1 : g[a] + W;
  }
  int64_t gB[3];
  for (gB[0] = lo[0]; gB[0] <= hi[0]; ++gB[0])
    for (gB[1] = lo[1]; gB[1] <= hi[1]; ++gB[1])
      for (gB[2] = lo[2]; gB[2] <= hi[2]; ++gB[2]) {
        if (!well_separated(gB[0] - g[0], gB[1] - g[1], gB[2] - g[2], theta)) continue;
        if (lev > 0 && well_separated(gB[0] / 2 - g[0] / 2, gB[1] / 2 - g[1] / 2,
                                      gB[2] / 2 - g[2] / 2, theta))
          continue;
        if (cell_subgrid(t, lev, gB) < 0) continue;
        fn(user, lev, gB);
      }
}

/* Calls fn for every cell B at level lev, B != A, that exists and is not well separated from A. */
static void for_each_near_cell(const otree *t, int lev, const int64_t g[3], double theta,
                               pair_fn fn, void *user) {
  int64_t n = (int64_t)NSUB << lev;
  int64_t W = (int64_t)floor(1.0 / theta);
  if (W > n) W = n;
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = g[a] - W < 0 ? 0 : g[a] - W;
    hi[a] = g[a] + W > n - 1 ? n - 1 : g[a] + W;
  }
  int64_t gB[3];
  for (gB[0] = lo[0]; gB[0] <= hi[0]; ++gB[0])
    for (gB[1] = lo[1]; gB[1] <= hi[1]; ++gB[1])
      for (gB[2] = lo[2]; gB[2] <= hi[2]; ++gB[2]) {
        if (gB[0] == g[0] && gB[1] == g[1] && gB[2] == g[2]) continue;
        if (well_separated(gB[0] - g[0], gB[1] - g[1], gB[2] - g[2], theta)) continue;
        if (cell_subgrid(t, lev, gB) < 0) continue;
        fn(user, lev, gB);
      }
}

/* ------------------------------------------------------------------------------------------ */
/* Per-cell work                                                                               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const ctx_t *C;
  double momA[NMOM];
  double L[NLOC], ac[3];
  int amc;
  int64_t n_m2l;
} m2l_acc;

static void m2l_cb(void *u, int lev, const int64_t gB[3]) {
  m2l_acc *A = (m2l_acc *)u;
  double momB[NMOM];
  cell_moments(A->C, lev, gB, momB);
  oracle_m2l(A->momA, momB, A->amc, A->L, A->ac);
  A->n_m2l++;
}

static void cell_expansion(const ctx_t *C, int lev, const int64_t g[3], double theta, int amc,
                           double L[NLOC], double ac[3], int64_t *n_m2l) {
  m2l_acc A;
  memset(&A, 0, sizeof(A));
  A.C = C;
  A.amc = amc;
  cell_moments(C, lev, g, A.momA);
  for_each_m2l_partner(C->t, lev, g, theta, m2l_cb, &A);
  memcpy(L, A.L, sizeof(A.L));
  memcpy(ac, A.ac, sizeof(A.ac));
  if (n_m2l) *n_m2l += A.n_m2l;
}

typedef struct {
  const ctx_t *C;
  double x[3];
  double phi, g[3];
  int target_lev;
  int64_t n_same, n_mixed;
} p2p_acc;

static void p2p_leaf_cb(void *u, int lev, const int64_t gB[3]) {
  p2p_acc *P = (p2p_acc *)u;
  double m, y[3];
  leaf_mass_of(P->C, lev, gB, &m, y);
  double d[3] = {P->x[0] - y[0], P->x[1] - y[1], P->x[2] - y[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  P->phi += -m / r;
  for (int a = 0; a < 3; ++a) P->g[a] += -m * d[a] / (r * r * r);
  if (lev == P->target_lev) P->n_same++; else P->n_mixed++;
}

/* A near cell at the target's own level: a leaf interacts directly; a refined cell passes on
 * every leaf below it. */
static void p2p_same_level_cb(void *u, int lev, const int64_t gB[3]) {
  p2p_acc *P = (p2p_acc *)u;
  visit_leaves(P->C->t, lev, gB, p2p_leaf_cb, P);
}

/* A near cell at a level coarser than the target leaf: only a leaf there is a direct partner
 * (a refined one holds leaves finer than this level, handled at a finer level). */
static void p2p_coarser_cb(void *u, int lev, const int64_t gB[3]) {
  p2p_acc *P = (p2p_acc *)u;
  int64_t s = cell_subgrid(P->C->t, lev, gB);
  if (P->C->t->leaf[lev][s]) p2p_leaf_cb(u, lev, gB);
}

/* phi, g of one leaf cell; counts its directed interactions when counters are given. */
static void leaf_solve(const ctx_t *C, int lev, const int64_t g[3], double theta, int amc,
                       const double *inner_L, double *phi, double *gout, int64_t *cnt) {
  const otree *t = C->t;
  double x[3];
  cell_centre(lev, g, x);
  double ph = 0, gg[3] = {0, 0, 0};
  /* the leaf's own expansion, evaluated at its own centre */
  double L[NLOC], ac[3], ev[4];
  int64_t nm = 0;
  cell_expansion(C, lev, g, theta, amc, L, ac, &nm);
  oracle_local_eval(L, x, x, ev);
  ph += ev[0];
  for (int a = 0; a < 3; ++a) gg[a] += ev[1 + a] + ac[a];
  /* every ancestor's expansion, evaluated at the leaf */
  for (int m = 0; m < lev; ++m) {
    int sh = lev - m;
    int64_t gA[3] = {g[0] >> sh, g[1] >> sh, g[2] >> sh};
    double momA[NMOM], LA[NLOC], acA[3];
    cell_moments(C, m, gA, momA);
    if (inner_L) {
      int64_t s = cell_subgrid(t, m, gA);
      const double *src = inner_L + (t->inner_slot[m][s] * 512 + local_index(gA)) * (NLOC + 3);
      memcpy(LA, src, sizeof(LA));
      memcpy(acA, src + NLOC, sizeof(acA));
    } else {
      cell_expansion(C, m, gA, theta, amc, LA, acA, &nm);
    }
    oracle_local_eval(LA, momA + 1, x, ev);
    ph += ev[0];
    for (int a = 0; a < 3; ++a) gg[a] += ev[1 + a] + acA[a];
  }
  /* direct interactions */
  p2p_acc P;
  memset(&P, 0, sizeof(P));
  P.C = C;
  memcpy(P.x, x, sizeof(x));
  P.target_lev = lev;
  for (int m = 0; m < lev; ++m) {
    int sh = lev - m;
    int64_t gA[3] = {g[0] >> sh, g[1] >> sh, g[2] >> sh};
    for_each_near_cell(t, m, gA, theta, p2p_coarser_cb, &P);
  }
  for_each_near_cell(t, lev, g, theta, p2p_same_level_cb, &P);
  ph += P.phi;
  for (int a = 0; a < 3; ++a) gg[a] += P.g[a];
  *phi = ph;
  for (int a = 0; a < 3; ++a) gout[a] = gg[a];
  if (cnt) { cnt[0] += nm; cnt[1] += P.n_same; cnt[2] += P.n_mixed; }
}

static void leaf_cell_coords(const otree *t, int64_t leaf_cell, int *lev, int64_t g[3]) {
  int64_t ls = leaf_cell / 512, c = leaf_cell % 512;
  for (int l = 0; l <= t->depth; ++l)
    for (int64_t s = 0; s < t->count[l]; ++s)
      if (t->leaf_slot[l][s] == ls) {
        *lev = l;
        g[0] = (int64_t)t->ijk[l][3 * s] * NSUB + c / 64;
        g[1] = (int64_t)t->ijk[l][3 * s + 1] * NSUB + (c / 8) % 8;
        g[2] = (int64_t)t->ijk[l][3 * s + 2] * NSUB + c % 8;
        return;
      }
}

static int resolve_threads(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Public entry points                                                                         */
/* ------------------------------------------------------------------------------------------ */
/* Full solve.  rho: leaf-cell density in canonical leaf order (leaf subgrids by level then
 * Morton key; cells (a*8+b)*8+c).  Outputs phi[n], g[n][3].  counts (optional, 3 entries):
 * directed multipole interactions over all cells and levels, directed same-level direct pairs,
 * directed direct pairs between leaves of different levels. */
void oracle_fmm_solve(const otree *t, const double *rho, double theta, int amc, int nthreads,
                      double *phi, double *g, int64_t *counts) {
  nthreads = resolve_threads(nthreads);
  ctx_t C = {t, rho, NULL};
  compute_inner_moments(&C, nthreads);
  double *inner_L = (double *)calloc((size_t)(t->n_inner_sub ? t->n_inner_sub : 1) * 512 * (NLOC + 3),
                                     sizeof(double));
  int64_t n_m2l = 0, n_same = 0, n_mixed = 0;
  for (int l = 0; l <= t->depth; ++l) {
    int64_t cnt = t->count[l];
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : n_m2l)
    for (int64_t s = 0; s < cnt; ++s) {
      if (t->leaf[l][s]) continue;
      for (int64_t c = 0; c < 512; ++c) {
        int64_t gc[3] = {(int64_t)t->ijk[l][3 * s] * NSUB + c / 64,
                         (int64_t)t->ijk[l][3 * s + 1] * NSUB + (c / 8) % 8,
                         (int64_t)t->ijk[l][3 * s + 2] * NSUB + c % 8};
        double *dst = inner_L + (t->inner_slot[l][s] * 512 + c) * (NLOC + 3);
        int64_t nm = 0;
        cell_expansion(&C, l, gc, theta, amc, dst, dst + NLOC, &nm);
        n_m2l += nm;
      }
    }
  }
  for (int l = 0; l <= t->depth; ++l) {
    int64_t cnt = t->count[l];
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : n_m2l, n_same, n_mixed)
    for (int64_t s = 0; s < cnt; ++s) {
      if (!t->leaf[l][s]) continue;
      for (int64_t c = 0; c < 512; ++c) {
        int64_t gc[3] = {(int64_t)t->ijk[l][3 * s] * NSUB + c / 64,
                         (int64_t)t->ijk[l][3 * s + 1] * NSUB + (c / 8) % 8,
                         (int64_t)t->ijk[l][3 * s + 2] * NSUB + c % 8};
        int64_t i = t->leaf_slot[l][s] * 512 + c;
        int64_t cc[3] = {0, 0, 0};
        leaf_solve(&C, l, gc, theta, amc, inner_L, phi + i, g + 3 * i, cc);
        n_m2l += cc[0];
        n_same += cc[1];
        n_mixed += cc[2];
      }
    }
  }
  if (counts) { counts[0] = n_m2l; counts[1] = n_same; counts[2] = n_mixed; }
  free(inner_L);
  free(C.inner_mom);
}

/* The same solve evaluated only at the leaf cells listed in idx (canonical leaf indices).
 * Multipoles of all refined cells are formed; expansions are formed only along the sampled
 * leaves' ancestor chains. */
void oracle_fmm_sample(const otree *t, const double *rho, double theta, int amc, int nthreads,
                       int64_t ns, const int64_t *idx, double *phi, double *g, int64_t *counts) {
  nthreads = resolve_threads(nthreads);
  ctx_t C = {t, rho, NULL};
  compute_inner_moments(&C, nthreads);
  int64_t n_m2l = 0, n_same = 0, n_mixed = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : n_m2l, n_same, n_mixed)
  for (int64_t q = 0; q < ns; ++q) {
    int lev = 0;
    int64_t gc[3] = {0, 0, 0};
    int64_t cc[3] = {0, 0, 0};
    leaf_cell_coords(t, idx[q], &lev, gc);
    leaf_solve(&C, lev, gc, theta, amc, NULL, phi + q, g + 3 * q, cc);
    n_m2l += cc[0];
    n_same += cc[1];
    n_mixed += cc[2];
  }
  /* counts: multipole interactions evaluated (the sampled leaves' own and their ancestors'),
   * direct pairs at the same level and across a level jump */
  if (counts) { counts[0] = n_m2l; counts[1] = n_same; counts[2] = n_mixed; }
  free(C.inner_mom);
}

/* The same evaluation with the multipoles of the refined cells given by the caller (inner_mom,
 * in the layout of oracle_inner_moments) instead of formed from rho: a rank of a decomposed solve
 * evaluates its cells from its own moments, the summed moments of the shared coarse cells and
 * the moments and densities it received from other ranks.  Entries the evaluation should never
 * read may hold NaN. */
void oracle_fmm_sample_given(const otree *t, const double *rho, const double *inner_mom, double theta,
                             int amc, int nthreads, int64_t ns, const int64_t *idx, double *phi,
                             double *g) {
  nthreads = resolve_threads(nthreads);
  ctx_t C = {t, rho, (double *)inner_mom};
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t q = 0; q < ns; ++q) {
    int lev = 0;
    int64_t gc[3] = {0, 0, 0};
    leaf_cell_coords(t, idx[q], &lev, gc);
    leaf_solve(&C, lev, gc, theta, amc, NULL, phi + q, g + 3 * q, NULL);
  }
}

/* Multipoles (m, X[3], M2[9], M3[27]) of every cell of every refined subgrid, in canonical
 * refined-subgrid order, from the definition. */
void oracle_inner_moments(const otree *t, const double *rho, int nthreads, double *out) {
  nthreads = resolve_threads(nthreads);
  ctx_t C = {t, rho, NULL};
  compute_inner_moments(&C, nthreads);
  memcpy(out, C.inner_mom, sizeof(double) * (size_t)t->n_inner_sub * 512 * NMOM);
  free(C.inner_mom);
}

/* Exact point-mass sums over all pairs: phi_i = -sum_j m_j/r_ij, g_i = -sum_j m_j d_ij/r_ij^3. */
void oracle_direct(int64_t n, const double *x, const double *m, int nthreads, double *phi,
                   double *g) {
  nthreads = resolve_threads(nthreads);
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int64_t i = 0; i < n; ++i) {
    double ph = 0, gg[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      ph += -m[j] / r;
      for (int a = 0; a < 3; ++a) gg[a] += -m[j] * d[a] / (r * r * r);
    }
    phi[i] = ph;
    for (int a = 0; a < 3; ++a) g[3 * i + a] = gg[a];
  }
}

int oracle_max_threads(void) { return resolve_threads(0); }

/* ------------------------------------------------------------------------------------------ */
/* Time derivative of the potential (Sec. 2.1)                                                */
/* ------------------------------------------------------------------------------------------ */
#define NSRC 40 /* S0, S1[3], S2[9], S3[27] about the cell's rho centre of mass */

typedef struct {
  ctx_t C;             /* the rho field: lists, centres of mass */
  const double *src;   /* source density (d rho / dt), canonical leaf order */
  double *inner_src;   /* [n_inner_sub * 512][NSRC] */
} dt_ctx;

static void leaf_source_of(const dt_ctx *D, int lev, const int64_t g[3], double *s, double x[3]) {
  int64_t sg = cell_subgrid(D->C.t, lev, g);
  double dx = cell_dx(lev);
  *s = D->src[D->C.t->leaf_slot[lev][sg] * 512 + local_index(g)] * dx * dx * dx;
  cell_centre(lev, g, x);
}

typedef struct { const dt_ctx *D; const double *X; csum S0, S1[3], S2[9], S3[27]; } src_acc;

static void src_acc_leaf(void *u, int lev, const int64_t g[3]) {
  src_acc *A = (src_acc *)u;
  double sv, x[3], r[3];
  leaf_source_of(A->D, lev, g, &sv, x);
  for (int a = 0; a < 3; ++a) r[a] = x[a] - A->X[a];
  csum_add(&A->S0, sv);
  for (int a = 0; a < 3; ++a) {
    csum_add(&A->S1[a], sv * r[a]);
    for (int b = 0; b < 3; ++b) {
      csum_add(&A->S2[3 * a + b], sv * r[a] * r[b]);
      for (int c = 0; c < 3; ++c) csum_add(&A->S3[9 * a + 3 * b + c], sv * r[a] * r[b] * r[c]);
    }
  }
}

/* Source moments of a cell about its rho centre of mass X (written to X as well). */
static void cell_source_moments(const dt_ctx *D, int lev, const int64_t g[3], double sm[NSRC],
                                double X[3]) {
  double mom[NMOM];
  cell_moments(&D->C, lev, g, mom);
  memcpy(X, mom + 1, sizeof(double) * 3);
  int64_t sg = cell_subgrid(D->C.t, lev, g);
  if (D->C.t->leaf[lev][sg]) {
    double x[3];
    memset(sm, 0, sizeof(double) * NSRC);
    leaf_source_of(D, lev, g, &sm[0], x);
    return;
  }
  memcpy(sm, D->inner_src + (D->C.t->inner_slot[lev][sg] * 512 + local_index(g)) * NSRC,
         sizeof(double) * NSRC);
}

static void compute_inner_sources(dt_ctx *D, int nthreads) {
  const otree *t = D->C.t;
  D->inner_src = (double *)calloc((size_t)(t->n_inner_sub ? t->n_inner_sub : 1) * 512 * NSRC,
                                  sizeof(double));
  for (int l = 0; l <= t->depth; ++l) {
    int64_t cnt = t->count[l];
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t sg = 0; sg < cnt; ++sg) {
      if (t->leaf[l][sg]) continue;
      for (int64_t c = 0; c < 512; ++c) {
        int64_t g[3] = {(int64_t)t->ijk[l][3 * sg] * NSUB + c / 64,
                        (int64_t)t->ijk[l][3 * sg + 1] * NSUB + (c / 8) % 8,
                        (int64_t)t->ijk[l][3 * sg + 2] * NSUB + c % 8};
        double mom[NMOM];
        cell_moments(&D->C, l, g, mom);
        src_acc A;
        memset(&A, 0, sizeof(A));
        A.D = D;
        A.X = mom + 1;
        visit_leaves(t, l, g, src_acc_leaf, &A);
        double *out = D->inner_src + (t->inner_slot[l][sg] * 512 + c) * NSRC;
        out[0] = csum_val(&A.S0);
        for (int k = 0; k < 3; ++k) out[1 + k] = csum_val(&A.S1[k]);
        for (int k = 0; k < 9; ++k) out[4 + k] = csum_val(&A.S2[k]);
        for (int k = 0; k < 27; ++k) out[13 + k] = csum_val(&A.S3[k]);
      }
    }
  }
}

/* Adds the expansion at centre XA due to the source moments smB about XB:
 *   L_k -= sum_(n <= 3 - k) (-1)^n / n! D^(k+n) : S_n. */
void oracle_m2l_source(const double *XA, const double *XB, const double *smB, double *L) {
  double Dt[121];
  double R[3] = {XA[0] - XB[0], XA[1] - XB[1], XA[2] - XB[2]};
  oracle_dtensors(R, Dt);
  const double *D0 = Dt, *D1 = Dt + 1, *D2 = Dt + 4, *D3 = Dt + 13;
  const double S0 = smB[0], *S1 = smB + 1, *S2 = smB + 4, *S3 = smB + 13;
  double l0 = S0 * D0[0];
  for (int a = 0; a < 3; ++a) {
    l0 -= D1[a] * S1[a];
    for (int b = 0; b < 3; ++b) {
      l0 += 0.5 * D2[3 * a + b] * S2[3 * a + b];
      for (int c = 0; c < 3; ++c) l0 -= D3[9 * a + 3 * b + c] * S3[9 * a + 3 * b + c] / 6.0;
    }
  }
  L[0] -= l0;
  for (int a = 0; a < 3; ++a) {
    double l1 = S0 * D1[a];
    for (int b = 0; b < 3; ++b) {
      l1 -= D2[3 * a + b] * S1[b];
      for (int c = 0; c < 3; ++c) l1 += 0.5 * D3[9 * a + 3 * b + c] * S2[3 * b + c];
    }
    L[1 + a] -= l1;
    for (int b = 0; b < 3; ++b) {
      double l2 = S0 * D2[3 * a + b];
      for (int c = 0; c < 3; ++c) l2 -= D3[9 * a + 3 * b + c] * S1[c];
      L[4 + 3 * a + b] -= l2;
      for (int c = 0; c < 3; ++c) L[13 + 9 * a + 3 * b + c] -= S0 * D3[9 * a + 3 * b + c];
    }
  }
}

typedef struct {
  const dt_ctx *D;
  double XA[3];
  double L[NLOC];
} src_m2l_acc;

static void src_m2l_cb(void *u, int lev, const int64_t gB[3]) {
  src_m2l_acc *A = (src_m2l_acc *)u;
  double sm[NSRC], XB[3];
  cell_source_moments(A->D, lev, gB, sm, XB);
  oracle_m2l_source(A->XA, XB, sm, A->L);
}

/* The source expansion of cell (lev, g) about its rho centre of mass. */
static void cell_source_expansion(const dt_ctx *D, int lev, const int64_t g[3], double theta,
                                  double L[NLOC], double XA[3]) {
  src_m2l_acc A;
  memset(&A, 0, sizeof(A));
  A.D = D;
  double mom[NMOM];
  cell_moments(&D->C, lev, g, mom);
  memcpy(A.XA, mom + 1, sizeof(A.XA));
  for_each_m2l_partner(D->C.t, lev, g, theta, src_m2l_cb, &A);
  memcpy(L, A.L, sizeof(A.L));
  memcpy(XA, A.XA, sizeof(A.XA));
}

typedef struct { const dt_ctx *D; double x[3]; double phi; } src_p2p_acc;

static void src_p2p_leaf_cb(void *u, int lev, const int64_t gB[3]) {
  src_p2p_acc *P = (src_p2p_acc *)u;
  double sv, y[3];
  leaf_source_of(P->D, lev, gB, &sv, y);
  double d[3] = {P->x[0] - y[0], P->x[1] - y[1], P->x[2] - y[2]};
  P->phi += -sv / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

static void src_p2p_same_level_cb(void *u, int lev, const int64_t gB[3]) {
  src_p2p_acc *P = (src_p2p_acc *)u;
  visit_leaves(P->D->C.t, lev, gB, src_p2p_leaf_cb, P);
}

static void src_p2p_coarser_cb(void *u, int lev, const int64_t gB[3]) {
  src_p2p_acc *P = (src_p2p_acc *)u;
  int64_t sg = cell_subgrid(P->D->C.t, lev, gB);
  if (P->D->C.t->leaf[lev][sg]) src_p2p_leaf_cb(u, lev, gB);
}

/* dphi/dt of one leaf cell: its own and every ancestor's source expansion evaluated at the
 * leaf's centre, plus the direct sums over the same partners as the rho solve. */
static double leaf_solve_dt(const dt_ctx *D, int lev, const int64_t g[3], double theta) {
  const otree *t = D->C.t;
  double x[3], ev[4], L[NLOC], X[3];
  cell_centre(lev, g, x);
  double ph = 0;
  for (int m = 0; m <= lev; ++m) {
    int sh = lev - m;
    int64_t gA[3] = {g[0] >> sh, g[1] >> sh, g[2] >> sh};
    cell_source_expansion(D, m, gA, theta, L, X);
    oracle_local_eval(L, X, x, ev);
    ph += ev[0];
  }
  src_p2p_acc P;
  memset(&P, 0, sizeof(P));
  P.D = D;
  memcpy(P.x, x, sizeof(x));
  for (int m = 0; m < lev; ++m) {
    int sh = lev - m;
    int64_t gA[3] = {g[0] >> sh, g[1] >> sh, g[2] >> sh};
    for_each_near_cell(t, m, gA, theta, src_p2p_coarser_cb, &P);
  }
  for_each_near_cell(t, lev, g, theta, src_p2p_same_level_cb, &P);
  return ph + P.phi;
}

/* dphi/dt at the leaf cells listed in idx (all leaf cells when idx is NULL and ns is their
 * number): rho fixes the tree's expansion centres, src is the source density. */
void oracle_fmm_sample_dt(const otree *t, const double *rho, const double *src, double theta,
                          int nthreads, int64_t ns, const int64_t *idx, double *phidot) {
  nthreads = resolve_threads(nthreads);
  dt_ctx D;
  memset(&D, 0, sizeof(D));
  D.C.t = t;
  D.C.rho = rho;
  D.src = src;
  compute_inner_moments(&D.C, nthreads);
  compute_inner_sources(&D, nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t q = 0; q < ns; ++q) {
    int lev = 0;
    int64_t gc[3] = {0, 0, 0};
    leaf_cell_coords(t, idx ? idx[q] : q, &lev, gc);
    phidot[q] = leaf_solve_dt(&D, lev, gc, theta);
  }
  free(D.inner_src);
  free(D.C.inner_mom);
}

