/*
 * Seeded synthetic inputs: pressure-Poisson matrices in CSR form and
 * right-hand sides.  This file holds none of the smoother's arithmetic; it
 * only builds the matrices A and vectors b that both the CUDA library and the
 * CPU oracle consume.
 *
 * The paper's matrices (PeleLM nodal projection, Nalu-Wind pressure
 * continuity) are not available, so these generators stand in for them with
 * the properties the paper names: symmetric pressure-Poisson operators
 * (Sec. 2, Eq. nodalP), cut cells with arbitrarily small
 * volume and area fractions and coefficients spanning many orders of
 * magnitude (Sec. 1), and 26 neighbours per row for the unstructured-mesh
 * case (Sec. 6.3, performance model).
 *
 * Kinds (natural lexicographic ordering, x fastest, Dirichlet boundaries
 * eliminated):
 *   SYNTH_POISSON7   7-point constant coefficients: diagonal 6, neighbours -1.
 *   SYNTH_CUTCELL7   7-point variable coefficients.  Cell density
 *                    rho = exp(sigma * N(0,1)); face coefficient
 *                    beta = alpha * 2 / (rho_a + rho_b) (harmonic mean of 1/rho)
 *                    with area fraction alpha = min(vf_a, vf_b); a fraction
 *                    `frac_cut` of the boundary-adjacent cells get volume
 *                    fraction vf = 10^U(-8, 0), all others vf = 1.  A
 *                    Dirichlet face contributes beta = vf * 2 / rho to the
 *                    diagonal only.  Diagonal = sum of face coefficients.
 *   SYNTH_HEX27      27-point graph Laplacian on a hex lattice whose nodes
 *                    are jittered by U[-0.25, 0.25] per axis; weight
 *                    w_ij = sqrt(c_i c_j) / |x_i - x_j|^2 with
 *                    c = exp(sigma * N(0,1)); ghost nodes outside the grid
 *                    contribute to the diagonal only.
 *
 * Random numbers: a counter-based generator.  Every draw is
 * splitmix64(splitmix64(seed ^ stream * K) + index), so any value can be
 * produced independently of the others and generation is embarrassingly
 * parallel and reproducible on any host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_POISSON7 0
#define SYNTH_CUTCELL7 1
#define SYNTH_HEX27 2

/* streams of the counter-based generator */
#define ST_DENSITY 1u
#define ST_CUTPICK 2u
#define ST_CUTVF 3u
#define ST_JX 4u
#define ST_JY 5u
#define ST_JZ 6u
#define ST_COEF 7u

static uint64_t sm64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t draw(uint64_t seed, uint64_t stream, uint64_t idx) {
  return sm64(sm64(seed ^ (stream * 0xd1b54a32d192ed03ULL)) + idx);
}

/* uniform on the open interval (0, 1) */
static double unif(uint64_t seed, uint64_t stream, uint64_t idx) {
  return ((double)(draw(seed, stream, idx) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* standard normal by Box-Muller from two independent uniforms */
static double gauss(uint64_t seed, uint64_t stream, uint64_t idx) {
  double u1 = unif(seed, stream, 2 * idx);
  double u2 = unif(seed, stream, 2 * idx + 1);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

int64_t synth_rows(int nx, int ny, int nz) { return (int64_t)nx * ny * nz; }

/* number of stored entries of the matrix of `kind` on an nx*ny*nz grid */
int64_t synth_nnz(int kind, int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  if (kind == SYNTH_POISSON7 || kind == SYNTH_CUTCELL7) {
    return 7LL * nx * ny * nz - 2LL * ny * nz - 2LL * nx * nz - 2LL * nx * ny;
  }
  if (kind == SYNTH_HEX27) {
    return (3LL * nx - 2) * (3LL * ny - 2) * (3LL * nz - 2);
  }
  return -1;
}

typedef struct {
  int nx, ny, nz;
  uint64_t seed;
  double sigma, frac_cut;
} gen7;

static double cc_rho(const gen7* g, int64_t cell) {
  return exp(g->sigma * gauss(g->seed, ST_DENSITY, (uint64_t)cell));
}

static int boundary_adjacent(const gen7* g, int i, int j, int k) {
  return i == 0 || j == 0 || k == 0 || i == g->nx - 1 || j == g->ny - 1 || k == g->nz - 1;
}

static double cc_vf(const gen7* g, int i, int j, int k) {
  if (!boundary_adjacent(g, i, j, k)) return 1.0;
  int64_t cell = ((int64_t)k * g->ny + j) * g->nx + i;
  if (unif(g->seed, ST_CUTPICK, (uint64_t)cell) >= g->frac_cut) return 1.0;
  return pow(10.0, -8.0 * unif(g->seed, ST_CUTVF, (uint64_t)cell));
}

static int64_t count7(int nx, int ny, int nz, int i, int j, int k) {
  return 1 + (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1);
}

/* row pointer of the 7-point matrix (n+1 entries) */
int synth_rowptr7(int nx, int ny, int nz, int64_t* rp) {
  if (nx < 1 || ny < 1 || nz < 1 || !rp) return 1;
  rp[0] = 0;
  int64_t row = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i, ++row) rp[row + 1] = rp[row] + count7(nx, ny, nz, i, j, k);
  return 0;
}

/*
 * Rows [r0, r1) of a 7-point matrix whose row pointer is complete.  Columns
 * come out in ascending order.  Disjoint row ranges may be filled
 * concurrently.
 */
static void fill7_rows(int kind, const gen7* g, int64_t r0, int64_t r1, const int64_t* rp, int32_t* ci, double* va) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  for (int64_t row = r0; row < r1; ++row) {
    const int i = (int)(row % nx), j = (int)((row / nx) % ny), k = (int)(row / ((int64_t)nx * ny));
    int64_t p = rp[row];
    /* neighbour offsets in ascending column order */
    const int di[6] = {0, 0, -1, 1, 0, 0};
    const int dj[6] = {0, -1, 0, 0, 1, 0};
    const int dk[6] = {-1, 0, 0, 0, 0, 1};
    double coef[6];
    int inside[6];
    double diag = 0.0;
    double rho_a = 0.0, vf_a = 1.0;
    if (kind == SYNTH_CUTCELL7) {
      rho_a = cc_rho(g, row);
      vf_a = cc_vf(g, i, j, k);
    }
    for (int f = 0; f < 6; ++f) {
      const int a = i + di[f], b = j + dj[f], c = k + dk[f];
      inside[f] = (a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz);
      if (kind == SYNTH_POISSON7) {
        coef[f] = 1.0;
        diag += 1.0; /* a Dirichlet ghost contributes to the diagonal */
      } else if (inside[f]) {
        const int64_t nb = ((int64_t)c * ny + b) * nx + a;
        const double rho_b = cc_rho(g, nb);
        const double vf_b = cc_vf(g, a, b, c);
        const double alpha = vf_a < vf_b ? vf_a : vf_b;
        coef[f] = alpha * 2.0 / (rho_a + rho_b);
        diag += coef[f];
      } else {
        coef[f] = vf_a * 2.0 / rho_a;
        diag += coef[f];
      }
    }
    /* lower neighbours (faces 0..2), diagonal, upper neighbours (3..5) */
    for (int f = 0; f < 3; ++f)
      if (inside[f]) {
        ci[p] = (int32_t)(row + (int64_t)dk[f] * nx * ny + (int64_t)dj[f] * nx + di[f]);
        va[p] = -coef[f];
        ++p;
      }
    ci[p] = (int32_t)row;
    va[p] = diag;
    ++p;
    for (int f = 3; f < 6; ++f)
      if (inside[f]) {
        ci[p] = (int32_t)(row + (int64_t)dk[f] * nx * ny + (int64_t)dj[f] * nx + di[f]);
        va[p] = -coef[f];
        ++p;
      }
  }
}

int synth_fill7_range(int kind, int nx, int ny, int nz, uint64_t seed, double sigma, double frac_cut, int64_t r0,
                      int64_t r1, const int64_t* rp, int32_t* ci, double* va) {
  if (nx < 1 || ny < 1 || nz < 1 || !rp || !ci || !va) return 1;
  if (kind != SYNTH_POISSON7 && kind != SYNTH_CUTCELL7) return 1;
  gen7 g = {nx, ny, nz, seed, sigma, frac_cut};
  fill7_rows(kind, &g, r0, r1, rp, ci, va);
  return 0;
}

static void fill7(int kind, const gen7* g, int64_t* rp, int32_t* ci, double* va) {
  synth_rowptr7(g->nx, g->ny, g->nz, rp);
  fill7_rows(kind, g, 0, (int64_t)g->nx * g->ny * g->nz, rp, ci, va);
}

/* node index in the lattice extended by one ghost layer on every side */
static int64_t ext_index(int nx, int ny, int i, int j, int k) {
  return ((int64_t)(k + 1) * (ny + 2) + (j + 1)) * (int64_t)(nx + 2) + (i + 1);
}

/*
 * Jittered node positions (3 per node) and node coefficients of the 27-point
 * lattice, ghost layer included: (nx+2)*(ny+2)*(nz+2) nodes.
 */
int synth_hex27_nodes(int nx, int ny, int nz, uint64_t seed, double sigma, double* xyz, double* coef) {
  if (nx < 1 || ny < 1 || nz < 1 || !xyz || !coef) return 1;
  for (int k = -1; k <= nz; ++k)
    for (int j = -1; j <= ny; ++j)
      for (int i = -1; i <= nx; ++i) {
        const int64_t e = ext_index(nx, ny, i, j, k);
        xyz[3 * e + 0] = i + 0.5 * (unif(seed, ST_JX, (uint64_t)e) - 0.5);
        xyz[3 * e + 1] = j + 0.5 * (unif(seed, ST_JY, (uint64_t)e) - 0.5);
        xyz[3 * e + 2] = k + 0.5 * (unif(seed, ST_JZ, (uint64_t)e) - 0.5);
        coef[e] = exp(sigma * gauss(seed, ST_COEF, (uint64_t)e));
      }
  return 0;
}

static int64_t count27(int nx, int ny, int nz, int i, int j, int k) {
  int ca = 1 + (i > 0) + (i < nx - 1);
  int cb = 1 + (j > 0) + (j < ny - 1);
  int cc = 1 + (k > 0) + (k < nz - 1);
  return (int64_t)ca * cb * cc;
}

/* row pointer of the 27-point matrix (n+1 entries) */
int synth_rowptr27(int nx, int ny, int nz, int64_t* rp) {
  if (nx < 1 || ny < 1 || nz < 1 || !rp) return 1;
  rp[0] = 0;
  int64_t row = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i, ++row) rp[row + 1] = rp[row] + count27(nx, ny, nz, i, j, k);
  return 0;
}

/*
 * Rows [r0, r1) of the 27-point matrix, given the complete row pointer and
 * the node tables of synth_hex27_nodes.  Disjoint row ranges may be filled
 * concurrently.
 */
int synth_fill27_range(int nx, int ny, int nz, const double* xyz, const double* coef, int64_t r0, int64_t r1,
                       const int64_t* rp, int32_t* ci, double* va) {
  if (nx < 1 || ny < 1 || nz < 1 || !xyz || !coef || !rp || !ci || !va) return 1;
  for (int64_t row = r0; row < r1; ++row) {
    const int i = (int)(row % nx), j = (int)((row / nx) % ny), k = (int)(row / ((int64_t)nx * ny));
    const int64_t es = ext_index(nx, ny, i, j, k);
    int64_t p = rp[row];
    int64_t pdiag = -1;
    double diag = 0.0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (di == 0 && dj == 0 && dk == 0) {
            pdiag = p++;
            continue;
          }
          const int a = i + di, b = j + dj, c = k + dk;
          const int64_t en = ext_index(nx, ny, a, b, c);
          const double dx = xyz[3 * es] - xyz[3 * en];
          const double dy = xyz[3 * es + 1] - xyz[3 * en + 1];
          const double dz = xyz[3 * es + 2] - xyz[3 * en + 2];
          const double w = sqrt(coef[es] * coef[en]) / (dx * dx + dy * dy + dz * dz);
          diag += w;
          if (a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz) {
            ci[p] = (int32_t)(row + ((int64_t)dk * ny + dj) * nx + di);
            va[p] = -w;
            ++p;
          }
        }
    ci[pdiag] = (int32_t)row;
    va[pdiag] = diag;
  }
  return 0;
}

/*
 * Fill the whole matrix of `kind`.  row_ptr has n+1 entries, col and val
 * synth_nnz() entries; columns come out in ascending order within a row.
 * Returns 0 on success, 1 on bad arguments, 2 if memory ran out.
 */
int synth_fill(int kind, int nx, int ny, int nz, uint64_t seed, double sigma, double frac_cut, int64_t* rp,
               int32_t* ci, double* va) {
  if (nx < 1 || ny < 1 || nz < 1 || !rp || !ci || !va) return 1;
  if ((int64_t)nx * ny * nz >= 2147483647LL) return 1;
  if (kind == SYNTH_POISSON7 || kind == SYNTH_CUTCELL7) {
    gen7 g = {nx, ny, nz, seed, sigma, frac_cut};
    fill7(kind, &g, rp, ci, va);
    return 0;
  }
  if (kind == SYNTH_HEX27) {
    const int64_t ne = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
    double* xyz = (double*)malloc(sizeof(double) * 3 * (size_t)ne);
    double* coef = (double*)malloc(sizeof(double) * (size_t)ne);
    if (!xyz || !coef) {
      free(xyz);
      free(coef);
      return 2;
    }
    synth_hex27_nodes(nx, ny, nz, seed, sigma, xyz, coef);
    synth_rowptr27(nx, ny, nz, rp);
    synth_fill27_range(nx, ny, nz, xyz, coef, 0, (int64_t)nx * ny * nz, rp, ci, va);
    free(xyz);
    free(coef);
    return 0;
  }
  return 1;
}

/* count values uniform on [lo, hi) drawn from (seed, stream) */
void synth_uniform(uint64_t seed, uint64_t stream, int64_t count, double lo, double hi, double* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = lo + (hi - lo) * unif(seed, 1000u + stream, (uint64_t)i);
}

/* integers uniform on [lo, hi] drawn from (seed, stream) */
void synth_randint(uint64_t seed, uint64_t stream, int64_t count, int lo, int hi, int32_t* out) {
  const uint64_t span = (uint64_t)(hi - lo + 1);
  for (int64_t i = 0; i < count; ++i) out[i] = lo + (int32_t)(draw(seed, 2000u + stream, (uint64_t)i) % span);
}
