/*
 * CPU FP64 oracle for the Co-Sim. SPFD Poisson solve -- TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow, obviously-correct definition of what the GPU
 * path computes.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product library never does, and the two
 * share no code.
 *
 * Method (Haussmann et al., "Towards Real-Time Magnetic Dosimetry Simulations
 * for Inductive Charging Systems"):
 *   Eq. 3 (Sec. II):  G^T M_k G Psi = -G^T M_k a   (discrete Poisson system)
 *   Eq. 1 (Sec. II):  e = -j omega (a + G Psi)       (edge voltages)
 *   Sec. III-A:       only conducting voxels carry unknowns
 *   Sec. II-A:        double precision, relative residual below 1e-12
 *   Sec. III-E:       voxel-averaged |E|
 *
 * Readings of what the paper leaves open (each used below):
 *   R1  M_k holds one conductance per edge, g_e = h * (sum of the sigma of the
 *       four voxels sharing the edge) / 4; voxels outside the grid are air.
 *   R3  a node is an unknown iff one of its incident edges has g_e > 0.
 *   R4  Psi is fixed up to one constant per connected conducting component;
 *       the oracle reports the zero-mean representative of each component.
 *   R5  "relative residual" = ||b - A Psi||_2 / ||b||_2 from Psi_0 = 0, with
 *       the residual recomputed from its definition.
 *   R6  |E| of a voxel = (omega / h) * || (mean of u over the voxel's four
 *       x-edges, ... y-edges, ... z-edges) ||_2 with u = a + G Psi.
 *
 * Layout (shared with the input generators): voxels [k][j][i] (nz,ny,nx),
 * nodes [k][j][i] (nz+1,ny+1,nx+1), edges [d][k][j][i] with d = 0,1,2 for
 * the x,y,z edge leaving node (i,j,k) in the +d direction.
 *
 * Parity status: every function below is pinned by the CPU test suite
 * (closed forms, brute force, invariants); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

static inline i64 node_id(i64 i, i64 j, i64 k, i64 nx, i64 ny) {
  return (k * (ny + 1) + j) * (nx + 1) + i;
}

static inline double vox(const double *s, i64 i, i64 j, i64 k, i64 nx, i64 ny,
                         i64 nz) {
  if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0.0;
  return s[(k * ny + j) * nx + i];
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel loops (timing only; no result depends
 * on it beyond the order of reduction sums). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Edge conductances g (the diagonal of M_k, Eq. 3; averaging rule R1).
 * g has 3*(nx+1)*(ny+1)*(nz+1) entries; slots without an edge are 0. */
void orc_conductances(const double *sigma, int nx_, int ny_, int nz_, double h,
                      double *g) {
  i64 nx = nx_, ny = ny_, nz = nz_;
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k <= nz; k++)
    for (i64 j = 0; j <= ny; j++)
      for (i64 i = 0; i <= nx; i++) {
        i64 n = node_id(i, j, k, nx, ny);
        double gx = 0, gy = 0, gz = 0;
        if (i < nx) /* x edge (i,j,k)->(i+1,j,k): voxels i, j-1..j, k-1..k */
          gx = vox(sigma, i, j - 1, k - 1, nx, ny, nz) + vox(sigma, i, j, k - 1, nx, ny, nz) +
               vox(sigma, i, j - 1, k, nx, ny, nz) + vox(sigma, i, j, k, nx, ny, nz);
        if (j < ny) /* y edge: voxels i-1..i, j, k-1..k */
          gy = vox(sigma, i - 1, j, k - 1, nx, ny, nz) + vox(sigma, i, j, k - 1, nx, ny, nz) +
               vox(sigma, i - 1, j, k, nx, ny, nz) + vox(sigma, i, j, k, nx, ny, nz);
        if (k < nz) /* z edge: voxels i-1..i, j-1..j, k */
          gz = vox(sigma, i - 1, j - 1, k, nx, ny, nz) + vox(sigma, i, j - 1, k, nx, ny, nz) +
               vox(sigma, i - 1, j, k, nx, ny, nz) + vox(sigma, i, j, k, nx, ny, nz);
        g[0 * nn + n] = h * gx / 4.0;
        g[1 * nn + n] = h * gy / 4.0;
        g[2 * nn + n] = h * gz / 4.0;
      }
}

/* The up to six edges at node (i,j,k): neighbour node and conductance. */
static int node_edges(const double *g, i64 i, i64 j, i64 k, i64 nx, i64 ny,
                      i64 nz, i64 nb[6], double ge[6]) {
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
  i64 n = node_id(i, j, k, nx, ny);
  int c = 0;
  if (i > 0) {
    i64 m = node_id(i - 1, j, k, nx, ny);
    nb[c] = m; ge[c] = g[0 * nn + m]; c++;
  }
  if (i < nx) {
    nb[c] = node_id(i + 1, j, k, nx, ny); ge[c] = g[0 * nn + n]; c++;
  }
  if (j > 0) {
    i64 m = node_id(i, j - 1, k, nx, ny);
    nb[c] = m; ge[c] = g[1 * nn + m]; c++;
  }
  if (j < ny) {
    nb[c] = node_id(i, j + 1, k, nx, ny); ge[c] = g[1 * nn + n]; c++;
  }
  if (k > 0) {
    i64 m = node_id(i, j, k - 1, nx, ny);
    nb[c] = m; ge[c] = g[2 * nn + m]; c++;
  }
  if (k < nz) {
    nb[c] = node_id(i, j, k + 1, nx, ny); ge[c] = g[2 * nn + n]; c++;
  }
  return c;
}

/* Unknowns (R3): dof[n] = compact index of node n, or -1.  Returns the count. */
i64 orc_index_nodes(const double *g, int nx_, int ny_, int nz_, i64 *dof) {
  i64 nx = nx_, ny = ny_, nz = nz_, cnt = 0;
  for (i64 k = 0; k <= nz; k++)
    for (i64 j = 0; j <= ny; j++)
      for (i64 i = 0; i <= nx; i++) {
        i64 nb[6];
        double ge[6];
        int c = node_edges(g, i, j, k, nx, ny, nz, nb, ge);
        int act = 0;
        for (int q = 0; q < c; q++) act |= ge[q] > 0.0;
        dof[node_id(i, j, k, nx, ny)] = act ? cnt++ : -1;
      }
  return cnt;
}

/* CSR of A = G^T diag(g) G restricted to the unknowns (Eq. 3):
 * (A x)_n = sum over edges e at n of g_e (x_n - x_other).  Diagonal first in
 * each row, then the off-diagonals -g_e in edge order (-x,+x,-y,+y,-z,+z).
 * rowptr has n_dof+1 entries; col/val need at most 7*n_dof. */
i64 orc_assemble(const double *g, int nx_, int ny_, int nz_, const i64 *dof,
                 i64 *rowptr, i64 *col, double *val) {
  i64 nx = nx_, ny = ny_, nz = nz_, nnz = 0;
  for (i64 k = 0; k <= nz; k++)
    for (i64 j = 0; j <= ny; j++)
      for (i64 i = 0; i <= nx; i++) {
        i64 n = node_id(i, j, k, nx, ny);
        i64 r = dof[n];
        if (r < 0) continue;
        i64 nb[6];
        double ge[6];
        int c = node_edges(g, i, j, k, nx, ny, nz, nb, ge);
        rowptr[r] = nnz;
        i64 dpos = nnz++;
        double diag = 0.0;
        for (int q = 0; q < c; q++) {
          if (ge[q] > 0.0) {
            col[nnz] = dof[nb[q]];
            val[nnz] = -ge[q];
            nnz++;
            diag += ge[q];
          }
        }
        col[dpos] = r;
        val[dpos] = diag;
        rowptr[r + 1] = nnz;
      }
  return nnz;
}

/* Right-hand side of Eq. 3 on the node grid: b = -G^T diag(g) a, i.e.
 * b_n = sum_{e leaving n} g_e a_e - sum_{e entering n} g_e a_e. */
void orc_rhs(const double *g, const double *a, int nx_, int ny_, int nz_,
             double *b) {
  i64 nx = nx_, ny = ny_, nz = nz_;
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k <= nz; k++)
    for (i64 j = 0; j <= ny; j++)
      for (i64 i = 0; i <= nx; i++) {
        i64 n = node_id(i, j, k, nx, ny);
        double s = 0.0;
        if (i < nx) s += g[0 * nn + n] * a[0 * nn + n];
        if (j < ny) s += g[1 * nn + n] * a[1 * nn + n];
        if (k < nz) s += g[2 * nn + n] * a[2 * nn + n];
        if (i > 0) { i64 m = node_id(i - 1, j, k, nx, ny); s -= g[0 * nn + m] * a[0 * nn + m]; }
        if (j > 0) { i64 m = node_id(i, j - 1, k, nx, ny); s -= g[1 * nn + m] * a[1 * nn + m]; }
        if (k > 0) { i64 m = node_id(i, j, k - 1, nx, ny); s -= g[2 * nn + m] * a[2 * nn + m]; }
        b[n] = s;
      }
}

/* y = A x (CSR). */
void orc_matvec(i64 n, const i64 *rowptr, const i64 *col, const double *val,
                const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (i64 r = 0; r < n; r++) {
    double s = 0.0;
    for (i64 p = rowptr[r]; p < rowptr[r + 1]; p++) s += val[p] * x[col[p]];
    y[r] = s;
  }
}

/* Connected components of the graph whose edges are the off-diagonal
 * entries of A (R4), by breadth-first search.  Returns the count. */
i64 orc_components(i64 n, const i64 *rowptr, const i64 *col, i64 *comp) {
  i64 *queue = (i64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
  if (!queue) return -1;
  for (i64 r = 0; r < n; r++) comp[r] = -1;
  i64 nc = 0;
  for (i64 s = 0; s < n; s++) {
    if (comp[s] >= 0) continue;
    i64 head = 0, tail = 0;
    queue[tail++] = s;
    comp[s] = nc;
    while (head < tail) {
      i64 r = queue[head++];
      for (i64 p = rowptr[r]; p < rowptr[r + 1]; p++) {
        i64 c = col[p];
        if (comp[c] < 0) { comp[c] = nc; queue[tail++] = c; }
      }
    }
    nc++;
  }
  free(queue);
  return nc;
}

/* x <- x - (unweighted mean of x over its component), per component (R4). */
int orc_project(i64 n, const i64 *comp, i64 nc, double *x) {
  double *sum = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
  i64 *cnt = (i64 *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(i64));
  if (!sum || !cnt) { free(sum); free(cnt); return -1; }
  for (i64 r = 0; r < n; r++) { sum[comp[r]] += x[r]; cnt[comp[r]]++; }
  for (i64 c = 0; c < nc; c++) sum[c] /= (double)cnt[c];
  for (i64 r = 0; r < n; r++) x[r] -= sum[comp[r]];
  free(sum);
  free(cnt);
  return 0;
}

static double dot(i64 n, const double *x, const double *y) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (i64 r = 0; r < n; r++) s += x[r] * y[r];
  return s;
}

static double true_residual(i64 n, const i64 *rowptr, const i64 *col,
                            const double *val, const double *b,
                            const double *x, double *rt) {
  orc_matvec(n, rowptr, col, val, x, rt);
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (i64 i = 0; i < n; i++) {
    rt[i] = b[i] - rt[i];
    s += rt[i] * rt[i];
  }
  return sqrt(s);
}

/* Jacobi-preconditioned conjugate gradients for A x = b from x = 0 (R5).
 * Stops when the recomputed relative residual ||b - A x|| / ||b|| <= tol.
 * The true residual is recomputed every 50 iterations and whenever the
 * recursive one reaches tol (then it also replaces the recursive one).  If
 * 20 consecutive checks fail to lower the best true residual by 10 %, the
 * solve has hit its rounding floor and stops there.
 * info[0] = iterations, info[1] = final true relative residual,
 * info[2] = 1 if converged, 0 if stopped at the floor or at maxit.
 * Returns 0, or -1 on allocation failure. */
int orc_pcg(i64 n, const i64 *rowptr, const i64 *col, const double *val,
            const double *b, double tol, i64 maxit, double *x, double *info) {
  size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(double);
  double *r = malloc(bytes), *z = malloc(bytes), *p = malloc(bytes);
  double *q = malloc(bytes), *dinv = malloc(bytes), *rt = malloc(bytes);
  if (!r || !z || !p || !q || !dinv || !rt) {
    free(r); free(z); free(p); free(q); free(dinv); free(rt);
    return -1;
  }
  for (i64 i = 0; i < n; i++) {
    double d = 0.0;
    for (i64 t = rowptr[i]; t < rowptr[i + 1]; t++)
      if (col[t] == i) d += val[t];
    dinv[i] = d > 0.0 ? 1.0 / d : 0.0;
    x[i] = 0.0;
    r[i] = b[i];
    z[i] = dinv[i] * r[i];
    p[i] = z[i];
  }
  double bnorm = sqrt(dot(n, b, b));
  i64 it = 0;
  double rel = 0.0;
  if (n > 0 && bnorm > 0.0) {
    double rz = dot(n, r, z);
    double best = INFINITY;
    int stall = 0;
    rel = 1.0;
    for (it = 1; it <= maxit; it++) {
      orc_matvec(n, rowptr, col, val, p, q);
      double pq = dot(n, p, q);
      if (!(pq > 0.0)) break;
      double alpha = rz / pq;
#pragma omp parallel for schedule(static)
      for (i64 i = 0; i < n; i++) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      double rrel = sqrt(dot(n, r, r)) / bnorm;
      if (rrel <= tol || it % 50 == 0) {
        rel = true_residual(n, rowptr, col, val, b, x, rt) / bnorm;
        if (rel <= tol) break;
        if (rel < 0.9 * best) { best = rel; stall = 0; }
        else if (++stall >= 20) break;
        if (rrel <= tol) memcpy(r, rt, bytes);
      }
#pragma omp parallel for schedule(static)
      for (i64 i = 0; i < n; i++) z[i] = dinv[i] * r[i];
      double rz_new = dot(n, r, z);
      double beta = rz_new / rz;
      rz = rz_new;
#pragma omp parallel for schedule(static)
      for (i64 i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    }
    if (it > maxit) it = maxit;
    rel = true_residual(n, rowptr, col, val, b, x, rt) / bnorm;
  }
  info[0] = (double)it;
  info[1] = rel;
  info[2] = rel <= tol ? 1.0 : 0.0;
  free(r); free(z); free(p); free(q); free(dinv); free(rt);
  return 0;
}

/* Voxel-averaged |E| (Eq. 1 with reading R6): for a conducting voxel,
 * E_d = omega / (4 h) * sum over its four d-edges of (a_e + Psi_head - Psi_tail),
 * |E| = sqrt(E_x^2 + E_y^2 + E_z^2); air voxels get 0. psi is on the node grid. */
void orc_efield(const double *sigma, const double *a, const double *psi,
                int nx_, int ny_, int nz_, double h, double omega, double *E) {
  i64 nx = nx_, ny = ny_, nz = nz_;
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k < nz; k++)
    for (i64 j = 0; j < ny; j++)
      for (i64 i = 0; i < nx; i++) {
        i64 v = (k * ny + j) * nx + i;
        if (!(sigma[v] > 0.0)) { E[v] = 0.0; continue; }
        double ex = 0, ey = 0, ez = 0;
        for (int s = 0; s < 2; s++)
          for (int t = 0; t < 2; t++) {
            i64 nxe = node_id(i, j + s, k + t, nx, ny);   /* x edge tail */
            ex += a[0 * nn + nxe] + psi[node_id(i + 1, j + s, k + t, nx, ny)] - psi[nxe];
            i64 nye = node_id(i + s, j, k + t, nx, ny);   /* y edge tail */
            ey += a[1 * nn + nye] + psi[node_id(i + s, j + 1, k + t, nx, ny)] - psi[nye];
            i64 nze = node_id(i + s, j + t, k, nx, ny);   /* z edge tail */
            ez += a[2 * nn + nze] + psi[node_id(i + s, j + t, k + 1, nx, ny)] - psi[nze];
          }
        double c = omega / (4.0 * h);
        ex *= c; ey *= c; ez *= c;
        E[v] = sqrt(ex * ex + ey * ey + ez * ez);
      }
}

/* ---------------------------------------------------------------------------
 * Adjoint gradient of the field energy.
 *
 * Objective (a smooth exposure measure built on Eq. 1 and reading R6):
 *   J = (1 / Nc) * sum over conducting voxels v of |E_v|^2,
 *   E_v,d = c * sum over the four d-edges e of v of u_e,  c = omega / (4 h),
 *   u = a + G Psi,  Psi solving Eq. 3:  A Psi = -G^T M a,  A = G^T M G.
 * Gradients (one extra solve with the same operator, A lambda = G^T gJ):
 *   gJ_e     = dJ/du_e = (1 / Nc) * sum over conducting v at e of 2 c E_v,d(e)
 *   dJ/da_e  = gJ_e - g_e (G lambda)_e
 *   dJ/dg_e  = -(G lambda)_e u_e
 *   dJ/dsigma_v = (h / 4) * sum over the 12 edges e of v of dJ/dg_e
 *                 (g_e = h/4 * sum of the sigma of the 4 voxels at e, R1),
 * for conducting v (the set of conducting voxels is held fixed).  Edges are
 * laid out like a, nodes like Psi, voxels like sigma.  Serial loops keep the
 * summation order fixed.
 * ------------------------------------------------------------------------- */

/* J and gJ.  Returns J; gJ (3 * node count) is overwritten. */
double orc_energy(const double *sigma, const double *a, const double *psi,
                  int nx_, int ny_, int nz_, double h, double omega, double *gJ) {
  i64 nx = nx_, ny = ny_, nz = nz_;
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
  double c = omega / (4.0 * h);
  i64 nc = 0;
  for (i64 v = 0; v < nx * ny * nz; v++) nc += sigma[v] > 0.0;
  for (i64 e = 0; e < 3 * nn; e++) gJ[e] = 0.0;
  if (nc == 0) return 0.0;
  double J = 0.0;
  for (i64 k = 0; k < nz; k++)
    for (i64 j = 0; j < ny; j++)
      for (i64 i = 0; i < nx; i++) {
        i64 v = (k * ny + j) * nx + i;
        if (!(sigma[v] > 0.0)) continue;
        i64 tail[3][4];   /* tail node of the four d-edges of v */
        double E[3] = {0.0, 0.0, 0.0};
        int q = 0;
        for (int s = 0; s < 2; s++)
          for (int t = 0; t < 2; t++, q++) {
            tail[0][q] = node_id(i, j + s, k + t, nx, ny);
            tail[1][q] = node_id(i + s, j, k + t, nx, ny);
            tail[2][q] = node_id(i + s, j + t, k, nx, ny);
            i64 hx = node_id(i + 1, j + s, k + t, nx, ny);
            i64 hy = node_id(i + s, j + 1, k + t, nx, ny);
            i64 hz = node_id(i + s, j + t, k + 1, nx, ny);
            E[0] += a[0 * nn + tail[0][q]] + psi[hx] - psi[tail[0][q]];
            E[1] += a[1 * nn + tail[1][q]] + psi[hy] - psi[tail[1][q]];
            E[2] += a[2 * nn + tail[2][q]] + psi[hz] - psi[tail[2][q]];
          }
        for (int d = 0; d < 3; d++) {
          E[d] *= c;
          J += E[d] * E[d];
          for (q = 0; q < 4; q++) gJ[d * nn + tail[d][q]] += 2.0 * c * E[d] / (double)nc;
        }
      }
  return J / (double)nc;
}

/* out = G^T v on the node grid: (G^T v)_n = sum_{e entering n} v_e -
 * sum_{e leaving n} v_e (G maps node values to head minus tail). */
void orc_div(const double *v, int nx_, int ny_, int nz_, double *out) {
  i64 nx = nx_, ny = ny_, nz = nz_;
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
  for (i64 k = 0; k <= nz; k++)
    for (i64 j = 0; j <= ny; j++)
      for (i64 i = 0; i <= nx; i++) {
        i64 n = node_id(i, j, k, nx, ny);
        double s = 0.0;
        if (i > 0) s += v[0 * nn + node_id(i - 1, j, k, nx, ny)];
        if (j > 0) s += v[1 * nn + node_id(i, j - 1, k, nx, ny)];
        if (k > 0) s += v[2 * nn + node_id(i, j, k - 1, nx, ny)];
        if (i < nx) s -= v[0 * nn + n];
        if (j < ny) s -= v[1 * nn + n];
        if (k < nz) s -= v[2 * nn + n];
        out[n] = s;
      }
}

/* dJ/da (3 * node count) and dJ/dsigma (voxel count) from lambda (node
 * grid, zero off the unknowns), gJ, g, a and Psi. */
void orc_energy_grads(const double *sigma, const double *a, const double *psi,
                      const double *lambda, const double *gJ, const double *g,
                      int nx_, int ny_, int nz_, double h, double *dJda,
                      double *dJdsigma) {
  i64 nx = nx_, ny = ny_, nz = nz_;
  i64 nn = (nx + 1) * (ny + 1) * (nz + 1);
  for (i64 k = 0; k <= nz; k++)
    for (i64 j = 0; j <= ny; j++)
      for (i64 i = 0; i <= nx; i++) {
        i64 n = node_id(i, j, k, nx, ny);
        i64 head[3] = {i < nx ? node_id(i + 1, j, k, nx, ny) : -1,
                       j < ny ? node_id(i, j + 1, k, nx, ny) : -1,
                       k < nz ? node_id(i, j, k + 1, nx, ny) : -1};
        for (int d = 0; d < 3; d++) {
          double gl = head[d] >= 0 ? lambda[head[d]] - lambda[n] : 0.0;
          dJda[d * nn + n] = gJ[d * nn + n] - g[d * nn + n] * gl;
        }
      }
  for (i64 k = 0; k < nz; k++)
    for (i64 j = 0; j < ny; j++)
      for (i64 i = 0; i < nx; i++) {
        i64 v = (k * ny + j) * nx + i;
        if (!(sigma[v] > 0.0)) { dJdsigma[v] = 0.0; continue; }
        double s = 0.0;
        for (int p = 0; p < 2; p++)
          for (int q = 0; q < 2; q++) {
            i64 t[3] = {node_id(i, j + p, k + q, nx, ny), node_id(i + p, j, k + q, nx, ny),
                        node_id(i + p, j + q, k, nx, ny)};
            i64 hd[3] = {node_id(i + 1, j + p, k + q, nx, ny), node_id(i + p, j + 1, k + q, nx, ny),
                         node_id(i + p, j + q, k + 1, nx, ny)};
            for (int d = 0; d < 3; d++) {
              double u = a[d * nn + t[d]] + psi[hd[d]] - psi[t[d]];
              double gl = lambda[hd[d]] - lambda[t[d]];
              s += -gl * u;   /* dJ/dg_e */
            }
          }
        dJdsigma[v] = 0.25 * h * s;
      }
}

/* ---------------------------------------------------------------------------
 * Step 6 of the pipeline (Sec. II-A, step 6; Sec. III-E): the 99th
 * percentile of the voxel-averaged |E|, taken to discard unphysical field
 * peaks.  Reading R14: the p-quantile of a set of n values is the nearest-
 * rank value, the k-th smallest with k the least integer >= p * n (exact
 * arithmetic, k >= 1), taken per tissue label over the conducting voxels
 * (sigma > 0) that carry the label, plus once over every conducting voxel
 * (the whole body).  A library sort gives the order statistics.
 * ------------------------------------------------------------------------- */

/* Least integer k >= p * n for p in (0, 1], computed exactly: p is the
 * binary fraction m / 2^s with m a 53-bit integer. */
i64 orc_nearest_rank(double p, i64 n) {
  if (n <= 0) return 0;
  int e;
  double f = frexp(p, &e);                 /* p = f 2^e, f in [0.5, 1) */
  uint64_t m = (uint64_t)ldexp(f, 53);     /* exact */
  int s = 53 - e;                          /* p = m / 2^s */
  unsigned __int128 x = (unsigned __int128)m * (uint64_t)n;
  i64 k;
  if (s >= 127) k = 1;
  else k = (i64)((x + (((unsigned __int128)1 << s) - 1)) >> s);
  return k < 1 ? 1 : k;
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* out[t] / count[t] for labels t = 0..nlab-1, out[nlab] / count[nlab] for
 * the whole body; groups without a voxel get NaN and 0.  Returns 0, or -1 if
 * memory ran out. */
int orc_percentile(const double *sigma, const double *E, const int *labels, i64 nvox,
                   int nlab, double p, double *out, i64 *count) {
  double *buf = (double *)malloc((size_t)(nvox > 0 ? nvox : 1) * sizeof(double));
  if (!buf) return -1;
  for (int t = 0; t <= nlab; t++) {
    i64 n = 0;
    for (i64 v = 0; v < nvox; v++) {
      if (!(sigma[v] > 0.0)) continue;
      if (t == nlab || labels[v] == t) buf[n++] = E[v];
    }
    count[t] = n;
    if (n == 0) { out[t] = NAN; continue; }
    qsort(buf, (size_t)n, sizeof(double), cmp_double);
    out[t] = buf[orc_nearest_rank(p, n) - 1];
  }
  free(buf);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Eq. 2 (Sec. II): b = C a, the magnetic fluxes through the grid facets as
 * the discrete curl of the edge vector potentials.
 *
 * Facet d at node (i,j,k) is the square spanned by the two edges that leave
 * that node along d1 = (d+1) mod 3 and d2 = (d+2) mod 3; its normal is +d
 * and its boundary is run right-handed about +d (along d1 first):
 *   b_d(n) = a_d1(n) + a_d2(n + e_d1) - a_d1(n + e_d2) - a_d2(n).
 * b has the edge layout [3][nz+1][ny+1][nx+1]; slots of facets that would
 * leave the grid are 0.  Each facet sums its four terms in the order above.
 * ------------------------------------------------------------------------- */
void orc_curl(const double *a, int nx_, int ny_, int nz_, double *b) {
  i64 n[3] = {(i64)nx_ + 1, (i64)ny_ + 1, (i64)nz_ + 1};
  i64 nn = n[0] * n[1] * n[2];
  i64 stride[3] = {1, n[0], n[0] * n[1]};
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k < n[2]; k++)
    for (i64 j = 0; j < n[1]; j++)
      for (i64 i = 0; i < n[0]; i++) {
        i64 idx[3] = {i, j, k};
        i64 v = (k * n[1] + j) * n[0] + i;
        for (int d = 0; d < 3; d++) {
          int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
          if (idx[d1] + 1 >= n[d1] || idx[d2] + 1 >= n[d2]) {
            b[d * nn + v] = 0.0;
            continue;
          }
          const double *a1 = a + d1 * nn, *a2 = a + d2 * nn;
          b[d * nn + v] = a1[v] + a2[v + stride[d1]] - a1[v + stride[d2]] - a2[v];
        }
      }
}
