// C ABI of libspfd: context, build (operator + multigrid hierarchy), solve
// (multigrid-preconditioned CG on the device), |E|.
//
// Paper: Eq. 3 (Sec. II) is the system solved; Sec. II-A fixes double
// precision and a relative-residual target (1e-12 in the paper); Sec. III
// solves it with AMG-preconditioned FGMRES from AmgX, which this library
// replaces by CG (the operator is symmetric positive semidefinite and the
// right-hand side consistent) preconditioned by an operator-dependent
// geometric multigrid V-cycle with Galerkin coarse operators.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "spfd.h"
#include "spfd_internal.cuh"

using namespace spfd;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static spfd_status fail(spfd_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

extern "C" const char *spfd_last_error(void) { return g_err.c_str(); }

#define CU(call)                                                          \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess)                                                \
      return fail(SPFD_ECUDA, "%s failed: %s (%s:%d)", #call,             \
                  cudaGetErrorString(e_), __FILE__, __LINE__);            \
  } while (0)

#define TRY(expr)                    \
  do {                               \
    spfd_status s_ = (expr);         \
    if (s_ != SPFD_OK) return s_;    \
  } while (0)

// ------------------------------------------------------------------ context
struct Level {
  Grid g{};                       // device view
  std::vector<int> hbmap;         // host brick map
  std::vector<int4> hbco;         // host brick coordinates
  size_t S = 0;                   // slots = nb * 512
  int64_t n_active = 0;
  // FP64 operator
  double *gx = nullptr;           // level 0: [3][S] +edge conductances
  double *st = nullptr;           // level >= 1: [27][S] Galerkin stencil
  double *P = nullptr;            // level >= 1: [27][S] interpolation to level-1
  double *diag = nullptr, *dinv = nullptr, *wdinv = nullptr;
  double omega = 0.0, lmax = 0.0;
  // FP64 V-cycle vectors
  double *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
};

struct spfd_ctx {
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0;
  double h = 0.0;
  spfd_opts opts{};
  std::vector<Level> L;
  std::vector<void *> allocs;
  int64_t bytes = 0;
  // fine-level bookkeeping
  unsigned char *mask = nullptr;  // [nz][ny][nx] conducting voxel flags
  int *comp = nullptr;            // [S0] component id or -1
  int ncomp = 0;
  int64_t ndof = 0;
  int *csize = nullptr;           // [ncomp]
  double *csum = nullptr;         // [ncomp] (only when ncomp > 1)
  // Krylov vectors
  double *xk = nullptr, *rk = nullptr, *pk = nullptr, *qk = nullptr, *bk = nullptr;
  Scalars *sc = nullptr;          // device scalars
  Scalars *hsc = nullptr;         // pinned host mirror
  double *partials = nullptr;
  // coarsest level
  int m = 0;
  int *cidx = nullptr;
  double *Binv = nullptr;
  // host-array staging
  double *a_stage = nullptr, *psi_stage = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  spfd_info info{};
  int alloc_count = 0;
};

// Allocation with optional injected failure: SPFD_FAIL_ALLOC_AT=N makes the
// N-th device allocation of a context fail (counted from 1), to test that
// every failure path releases what was already allocated.
template <typename T>
static spfd_status dalloc(spfd_ctx *c, T **p, size_t count) {
  *p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  ++c->alloc_count;
  const char *inj = getenv("SPFD_FAIL_ALLOC_AT");
  if (inj && atoi(inj) == c->alloc_count)
    return fail(SPFD_ENOMEM, "injected allocation failure #%d", c->alloc_count);
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SPFD_ENOMEM : SPFD_ECUDA,
                "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  c->bytes += (int64_t)bytes;
  *p = (T *)q;
  return SPFD_OK;
}

template <typename T>
static void dfree(spfd_ctx *c, T *&p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), (void *)p);
  if (it != c->allocs.end()) c->allocs.erase(it);
  cudaFree(p);
  p = nullptr;
}

static void destroy_ctx(spfd_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

extern "C" void spfd_destroy(spfd_ctx *ctx) { destroy_ctx(ctx); }

extern "C" void spfd_opts_default(spfd_opts *o) {
  if (!o) return;
  o->tol = 1e-8;
  o->maxit = 200;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->smoother = SPFD_SMOOTHER_JACOBI;
  o->cheb_degree = 2;
  o->precision = SPFD_FP64;
  o->coarse_max = 512;
  o->max_levels = 12;
  o->verbose = 0;
}

// ------------------------------------------------------------------ helpers
static spfd_status sync_check(spfd_ctx *c, const char *what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess)
    return fail(SPFD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(SPFD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return SPFD_OK;
}

static spfd_status launch_check(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(SPFD_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return SPFD_OK;
}

// Read the device scalars into the pinned mirror (synchronises the stream).
static spfd_status read_scalars(spfd_ctx *c) {
  CU(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                     c->stream));
  return sync_check(c, "reading solver scalars");
}

// Geometry of a level from its brick activity flags.
static spfd_status make_level(spfd_ctx *c, Level &lv, int NX, int NY, int NZ,
                              const std::vector<unsigned char> &flags) {
  Grid &g = lv.g;
  g.NX = NX; g.NY = NY; g.NZ = NZ;
  g.MX = (NX + 7) / 8; g.MY = (NY + 7) / 8; g.MZ = (NZ + 7) / 8;
  size_t nbm = (size_t)g.MX * g.MY * g.MZ;
  lv.hbmap.assign(nbm, -1);
  lv.hbco.clear();
  for (int bz = 0; bz < g.MZ; ++bz)
    for (int by = 0; by < g.MY; ++by)
      for (int bx = 0; bx < g.MX; ++bx) {
        size_t q = ((size_t)bz * g.MY + by) * g.MX + bx;
        if (flags[q]) {
          lv.hbmap[q] = (int)lv.hbco.size();
          lv.hbco.push_back(make_int4(bx, by, bz, 0));
        }
      }
  if (lv.hbco.size() > (size_t)(INT32_MAX / BV))
    return fail(SPFD_EINVAL, "grid too large: %zu active bricks", lv.hbco.size());
  g.nb = (int)lv.hbco.size();
  lv.S = (size_t)g.nb * BV;
  int *bmap = nullptr;
  int4 *bco = nullptr;
  TRY(dalloc(c, &bmap, nbm));
  TRY(dalloc(c, &bco, lv.hbco.size()));
  CU(cudaMemcpyAsync(bmap, lv.hbmap.data(), nbm * sizeof(int),
                     cudaMemcpyHostToDevice, c->stream));
  if (g.nb)
    CU(cudaMemcpyAsync(bco, lv.hbco.data(), lv.hbco.size() * sizeof(int4),
                       cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));  // host vectors may be reused
  g.bmap = bmap;
  g.bco = bco;
  return SPFD_OK;
}

// Largest eigenvalue of D^-1 A by power iteration (smoother weight).
static spfd_status estimate_lmax(spfd_ctx *c, int l, double *lmax) {
  Level &lv = c->L[l];
  const int nb = lv.g.nb;
  *lmax = 0.0;
  if (nb == 0) return SPFD_OK;
  if (nb > c->L[0].g.nb || !c->partials)
    return fail(SPFD_EINTERNAL, "reduction scratch too small for level %d", l);
  double *v = lv.x, *w = lv.t, *r = lv.r, *zero = lv.b;
  CU(cudaMemsetAsync(zero, 0, lv.S * sizeof(double), c->stream));
  launch_power_init(nb, lv.diag, v, c->stream);
  // v <- D^-1 A v / |D^-1 A v|; after the first step |v| = 1, so |D^-1 A v|
  // is the estimate.
  double est = 0.0;
  for (int it = 0; it < 20; ++it) {
    if (l == 0)
      launch_residual7<double, double>(lv.g, lv.gx, lv.diag, v, zero, r, c->stream);
    else
      launch_residual27<double>(lv.g, lv.st, v, zero, r, c->stream);
    launch_power_step(nb, r, lv.dinv, w, c->sc, c->partials, c->stream);
    TRY(launch_check("power iteration"));
    TRY(read_scalars(c));
    double wn = std::sqrt(c->hsc->aux[4]);
    if (!(wn > 0.0)) break;
    if (it > 0) est = wn;
    launch_scaled_copy(nb, w, 1.0 / wn, v, c->stream);
  }
  *lmax = est;
  return SPFD_OK;
}

// Gauss-Jordan inverse of a dense SPD matrix (row-major, n x n), in place.
static bool invert_spd(std::vector<double> &A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = std::fabs(A[(size_t)col * n + col]);
    for (int r = col + 1; r < n; ++r) {
      double v = std::fabs(A[(size_t)r * n + col]);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0)) return false;
    if (piv != col) {
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)piv * n + k], A[(size_t)col * n + k]);
        std::swap(I[(size_t)piv * n + k], I[(size_t)col * n + k]);
      }
    }
    double d = 1.0 / A[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      A[(size_t)col * n + k] *= d;
      I[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= f * A[(size_t)col * n + k];
        I[(size_t)r * n + k] -= f * I[(size_t)col * n + k];
      }
    }
  }
  A.swap(I);
  return true;
}

// Coarsest level: dense B = A + sum_c mu_c v_c v_c^T (v_c = normalised
// indicator of a connected component of A) is SPD, and B^-1 r = A^+ r for r
// orthogonal to the constants of each component.
static spfd_status setup_coarsest(spfd_ctx *c) {
  Level &lv = c->L.back();
  const size_t S = lv.S;
  c->m = 0;
  if (S == 0) return SPFD_OK;
  std::vector<double> hst(27 * S), hdiag(S);
  CU(cudaMemcpyAsync(hdiag.data(), lv.diag, S * sizeof(double),
                     cudaMemcpyDeviceToHost, c->stream));
  if (c->L.size() > 1) {
    CU(cudaMemcpyAsync(hst.data(), lv.st, 27 * S * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream));
  }
  std::vector<double> hgx;
  if (c->L.size() == 1) {
    hgx.resize(3 * S);
    CU(cudaMemcpyAsync(hgx.data(), lv.gx, 3 * S * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream));
  }
  TRY(sync_check(c, "coarsest copy"));
  std::vector<int> row(S, -1), idx;
  for (size_t s = 0; s < S; ++s)
    if (hdiag[s] > 0.0) { row[s] = (int)idx.size(); idx.push_back((int)s); }
  const int m = (int)idx.size();
  c->m = m;
  if (m == 0) return SPFD_OK;
  if ((int64_t)m * m > (int64_t)1 << 26)
    return fail(SPFD_EINVAL, "coarsest level too large (%d unknowns); raise max_levels", m);
  const Grid &g = lv.g;
  auto slot_of = [&](int i, int j, int k) -> int {
    if (i < 0 || j < 0 || k < 0 || i >= g.NX || j >= g.NY || k >= g.NZ) return -1;
    int b = lv.hbmap[((size_t)(k >> 3) * g.MY + (j >> 3)) * g.MX + (i >> 3)];
    if (b < 0) return -1;
    return b * BV + ((k & 7) * 8 + (j & 7)) * 8 + (i & 7);
  };
  std::vector<double> A((size_t)m * m, 0.0);
  for (int a = 0; a < m; ++a) {
    int s = idx[a];
    int b = s / BV, t = s % BV;
    int4 bc = lv.hbco[b];
    int i = bc.x * 8 + (t & 7), j = bc.y * 8 + ((t >> 3) & 7), k = bc.z * 8 + (t >> 6);
    if (c->L.size() == 1) {
      // 7-point level-0 operator (tiny problems)
      A[(size_t)a * m + a] = hdiag[s];
      const int dd[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
      for (int q = 0; q < 6; ++q) {
        int u = slot_of(i + dd[q][0], j + dd[q][1], k + dd[q][2]);
        if (u < 0 || row[u] < 0) continue;
        int ax = q / 2;
        double ge = (q % 2 == 0) ? hgx[(size_t)ax * S + s] : hgx[(size_t)ax * S + u];
        A[(size_t)a * m + row[u]] -= ge;
      }
    } else {
      for (int e = 0; e < 27; ++e) {
        int u = slot_of(i + e % 3 - 1, j + (e / 3) % 3 - 1, k + e / 9 - 1);
        if (u < 0 || row[u] < 0) continue;
        A[(size_t)a * m + row[u]] += hst[(size_t)e * S + s];
      }
    }
  }
  // components of the coarsest graph
  std::vector<int> cc(m, -1), queue;
  int nc = 0;
  for (int a = 0; a < m; ++a) {
    if (cc[a] >= 0) continue;
    queue.assign(1, a);
    cc[a] = nc;
    for (size_t h = 0; h < queue.size(); ++h) {
      int u = queue[h];
      for (int v = 0; v < m; ++v)
        if (v != u && cc[v] < 0 && A[(size_t)u * m + v] != 0.0) {
          cc[v] = nc;
          queue.push_back(v);
        }
    }
    ++nc;
  }
  std::vector<double> dsum(nc, 0.0);
  std::vector<int> cnt(nc, 0);
  for (int a = 0; a < m; ++a) { dsum[cc[a]] += A[(size_t)a * m + a]; cnt[cc[a]]++; }
  for (int a = 0; a < m; ++a)
    for (int b2 = 0; b2 < m; ++b2)
      if (cc[a] == cc[b2]) {
        int q = cc[a];
        double mu = dsum[q] / cnt[q];  // mean diagonal keeps B well scaled
        A[(size_t)a * m + b2] += mu / cnt[q];
      }
  if (!invert_spd(A, m))
    return fail(SPFD_EINTERNAL, "coarsest-level matrix is singular after regularisation");
  TRY(dalloc(c, &c->cidx, m));
  TRY(dalloc(c, &c->Binv, (size_t)m * m));
  CU(cudaMemcpyAsync(c->cidx, idx.data(), m * sizeof(int), cudaMemcpyHostToDevice,
                     c->stream));
  CU(cudaMemcpyAsync(c->Binv, A.data(), (size_t)m * m * sizeof(double),
                     cudaMemcpyHostToDevice, c->stream));
  return sync_check(c, "coarsest upload");
}

static spfd_status count_active(spfd_ctx *c, const Level &lv, const double *d_dev,
                                int64_t *n, double *maxdiag) {
  std::vector<double> d(lv.S);
  if (lv.S)
    CU(cudaMemcpyAsync(d.data(), d_dev, lv.S * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c, "count"));
  int64_t k = 0;
  double mx = 0.0;
  for (double v : d) { if (v > 0.0) ++k; mx = std::max(mx, v); }
  *n = k;
  if (maxdiag) *maxdiag = mx;
  return SPFD_OK;
}

static spfd_status build_impl(spfd_ctx *c, const double *sigma) {
  cudaStream_t st = c->stream;
  TRY(dalloc(c, &c->sc, 1));
  CU(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), st));
  CU(cudaMallocHost(&c->hsc, sizeof(Scalars)));
  memset(c->hsc, 0, sizeof(Scalars));
  CU(cudaEventCreate(&c->ev0));
  CU(cudaEventCreate(&c->ev1));
  CU(cudaEventRecord(c->ev0, st));

  const int NX = c->nx + 1, NY = c->ny + 1, NZ = c->nz + 1;
  const int MX = (NX + 7) / 8, MY = (NY + 7) / 8, MZ = (NZ + 7) / 8;
  const size_t nbm = (size_t)MX * MY * MZ;
  const size_t nvox = (size_t)c->nx * c->ny * c->nz;
  unsigned char *flags = nullptr;
  TRY(dalloc(c, &flags, nbm));
  TRY(dalloc(c, &c->mask, nvox));
  CU(cudaMemsetAsync(flags, 0, nbm, st));
  launch_sigma_flags(sigma, c->nx, c->ny, c->nz, MX, MY, flags, c->mask,
                     &c->sc->status, st);
  TRY(launch_check("sigma flags"));
  std::vector<unsigned char> hflags(nbm);
  CU(cudaMemcpyAsync(hflags.data(), flags, nbm, cudaMemcpyDeviceToHost, st));
  TRY(read_scalars(c));
  dfree(c, flags);
  if (c->hsc->status & DEV_BAD_SIGMA)
    return fail(SPFD_EINVAL, "sigma holds a negative, NaN or infinite value");

  c->L.clear();
  c->L.emplace_back();
  TRY(make_level(c, c->L[0], NX, NY, NZ, hflags));
  Level &l0 = c->L[0];
  const size_t S0 = l0.S;
  // reduction scratch: level 0 has the most bricks of all levels, and every
  // grid reduction writes at most 2 values per block
  TRY(dalloc(c, &c->partials, 4 * (size_t)std::max(l0.g.nb, 1)));
  TRY(dalloc(c, &l0.gx, 3 * S0));
  TRY(dalloc(c, &l0.diag, S0));
  TRY(dalloc(c, &l0.dinv, S0));
  TRY(dalloc(c, &l0.wdinv, S0));
  launch_build_fine(l0.g, sigma, c->nx, c->ny, c->nz, c->h, l0.gx, l0.diag,
                    l0.dinv, st);
  TRY(launch_check("build fine"));

  // connected components of the conducting nodes
  int *parent = nullptr, *counts = nullptr, *offsets = nullptr;
  TRY(dalloc(c, &parent, S0));
  TRY(dalloc(c, &c->comp, S0));
  launch_components(l0.g, l0.gx, parent, &c->sc->status, st);
  TRY(launch_check("components"));
  const int nb0 = l0.g.nb;
  TRY(dalloc(c, &counts, nb0));
  TRY(dalloc(c, &offsets, nb0));
  launch_root_counts(l0.g, parent, counts, st);
  std::vector<int> hcnt(nb0), hoff(nb0);
  if (nb0)
    CU(cudaMemcpyAsync(hcnt.data(), counts, nb0 * sizeof(int),
                       cudaMemcpyDeviceToHost, st));
  TRY(read_scalars(c));
  if (c->hsc->status & DEV_UF_CAP)
    return fail(SPFD_EINTERNAL, "component labelling hit its iteration cap");
  int64_t tot = 0;
  for (int b = 0; b < nb0; ++b) { hoff[b] = (int)tot; tot += hcnt[b]; }
  c->ncomp = (int)tot;
  if (nb0)
    CU(cudaMemcpyAsync(offsets, hoff.data(), nb0 * sizeof(int),
                       cudaMemcpyHostToDevice, st));
  launch_assign_comp(l0.g, parent, offsets, c->comp, st);
  TRY(dalloc(c, &c->csize, std::max(c->ncomp, 1)));
  CU(cudaMemsetAsync(c->csize, 0, std::max(c->ncomp, 1) * sizeof(int), st));
  launch_comp_sizes(l0.g, c->comp, c->csize, st);
  TRY(launch_check("component sizes"));
  std::vector<int> hsize(std::max(c->ncomp, 1));
  CU(cudaMemcpyAsync(hsize.data(), c->csize, hsize.size() * sizeof(int),
                     cudaMemcpyDeviceToHost, st));
  TRY(sync_check(c, "components"));
  dfree(c, parent);
  dfree(c, counts);
  dfree(c, offsets);
  c->ndof = 0;
  for (int q = 0; q < c->ncomp; ++q) c->ndof += hsize[q];
  l0.n_active = c->ndof;
  if (c->ncomp > 1) TRY(dalloc(c, &c->csum, c->ncomp));

  // multigrid hierarchy
  for (int l = 0;; ++l) {
    Level &f = c->L[l];
    TRY(dalloc(c, &f.x, f.S));
    TRY(dalloc(c, &f.b, f.S));
    TRY(dalloc(c, &f.r, f.S));
    TRY(dalloc(c, &f.t, f.S));
    CU(cudaMemsetAsync(f.x, 0, f.S * sizeof(double), st));
    CU(cudaMemsetAsync(f.t, 0, f.S * sizeof(double), st));
    bool last = f.n_active <= c->opts.coarse_max || l + 1 >= c->opts.max_levels ||
                (f.g.NX <= 3 && f.g.NY <= 3 && f.g.NZ <= 3);
    if (last) break;
    // coarse geometry: coarse node I <-> fine node 2I; coarse brick B covers
    // fine bricks 2B-1 .. 2B+1 on each axis
    const int CX = f.g.NX / 2 + 1, CY = f.g.NY / 2 + 1, CZ = f.g.NZ / 2 + 1;
    const int cMX = (CX + 7) / 8, cMY = (CY + 7) / 8, cMZ = (CZ + 7) / 8;
    std::vector<unsigned char> cfl((size_t)cMX * cMY * cMZ, 0);
    for (int bz = 0; bz < cMZ; ++bz)
      for (int by = 0; by < cMY; ++by)
        for (int bx = 0; bx < cMX; ++bx) {
          bool any = false;
          for (int fz = std::max(0, 2 * bz - 1); fz <= std::min(f.g.MZ - 1, 2 * bz + 1) && !any; ++fz)
            for (int fy = std::max(0, 2 * by - 1); fy <= std::min(f.g.MY - 1, 2 * by + 1) && !any; ++fy)
              for (int fx = std::max(0, 2 * bx - 1); fx <= std::min(f.g.MX - 1, 2 * bx + 1) && !any; ++fx)
                any = f.hbmap[((size_t)fz * f.g.MY + fy) * f.g.MX + fx] >= 0;
          cfl[((size_t)bz * cMY + by) * cMX + bx] = any;
        }
    c->L.emplace_back();
    Level &fl = c->L[l];
    Level &cl = c->L[l + 1];
    TRY(make_level(c, cl, CX, CY, CZ, cfl));
    const size_t Sc = cl.S;
    TRY(dalloc(c, &cl.st, 27 * Sc));
    TRY(dalloc(c, &cl.P, 27 * Sc));
    TRY(dalloc(c, &cl.diag, Sc));
    TRY(dalloc(c, &cl.dinv, Sc));
    TRY(dalloc(c, &cl.wdinv, Sc));
    double *W = nullptr;
    TRY(dalloc(c, &W, 8 * fl.S));
    launch_interp_weights(fl.g, fl.gx, fl.st, fl.diag, W, st);
    TRY(launch_check("interpolation weights"));
    launch_galerkin(fl.g, cl.g, fl.gx, fl.st, fl.diag, W, cl.st, st);
    TRY(launch_check("galerkin"));
    launch_symmetrize(cl.g, cl.st, st);
    launch_pack_P(fl.g, cl.g, W, cl.P, st);
    TRY(launch_check("pack P"));
    TRY(sync_check(c, "coarse level"));
    dfree(c, W);
    int64_t nact = 0;
    double maxdiag = 0.0;
    TRY(count_active(c, cl, cl.st + 13 * Sc, &nact, &maxdiag));
    launch_coarse_diag(cl.g, cl.st, 1e-13 * maxdiag, cl.diag, cl.dinv, st);
    TRY(launch_check("coarse diag"));
    TRY(count_active(c, cl, cl.diag, &cl.n_active, nullptr));
  }

  // smoother weights (weighted Jacobi, omega = 4 / (3 lambda_max(D^-1 A)))
  for (size_t l = 0; l + 1 < c->L.size(); ++l) {
    Level &lv = c->L[l];
    double lm = 0.0;
    TRY(estimate_lmax(c, (int)l, &lm));
    if (!(lm > 0.0)) lm = 2.0;
    lv.lmax = lm;
    lv.omega = 4.0 / (3.0 * 1.05 * lm);
    launch_scaled_copy(lv.g.nb, lv.dinv, lv.omega, lv.wdinv, st);
    CU(cudaMemsetAsync(lv.x, 0, lv.S * sizeof(double), st));
    CU(cudaMemsetAsync(lv.t, 0, lv.S * sizeof(double), st));
  }
  TRY(setup_coarsest(c));

  // Krylov vectors and reduction scratch
  TRY(dalloc(c, &c->xk, S0));
  TRY(dalloc(c, &c->rk, S0));
  TRY(dalloc(c, &c->pk, S0));
  TRY(dalloc(c, &c->qk, S0));
  TRY(dalloc(c, &c->bk, S0));
  for (auto &lv : c->L)
    if (lv.g.nb > c->L[0].g.nb)
      return fail(SPFD_EINTERNAL, "a coarse level has more bricks than level 0");
  CU(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), st));
  CU(cudaEventRecord(c->ev1, st));
  TRY(sync_check(c, "build"));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->info.ms_build = ms;
  c->info.n_dof = c->ndof;
  c->info.n_comp = c->ncomp;
  c->info.n_levels = (int)c->L.size();
  c->info.n_bricks = c->L[0].g.nb;
  c->info.bytes_device = c->bytes;
  if (c->opts.verbose) {
    fprintf(stderr, "[spfd] build: %lld dof, %d comp, %d levels, %.2f ms, %.1f MB\n",
            (long long)c->ndof, c->ncomp, (int)c->L.size(), ms, c->bytes / 1e6);
    for (size_t l = 0; l < c->L.size(); ++l)
      fprintf(stderr, "[spfd]   level %zu: nodes %dx%dx%d, bricks %d, active %lld, lmax %.3f\n",
              l, c->L[l].g.NX, c->L[l].g.NY, c->L[l].g.NZ, c->L[l].g.nb,
              (long long)c->L[l].n_active, c->L[l].lmax);
  }
  return SPFD_OK;
}

extern "C" spfd_status spfd_build(const double *sigma_dev, int nx, int ny,
                                  int nz, double h, const spfd_opts *opts,
                                  void *stream, spfd_ctx **out) {
  if (!out) return fail(SPFD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!sigma_dev) return fail(SPFD_EINVAL, "sigma_dev is NULL");
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(SPFD_EINVAL, "voxel counts must be >= 1 (got %d %d %d)", nx, ny, nz);
  if ((int64_t)(nx + 1) * (ny + 1) * (nz + 1) >= ((int64_t)1 << 31))
    return fail(SPFD_EINVAL, "grid too large");
  if (!(h > 0.0) || !std::isfinite(h)) return fail(SPFD_EINVAL, "h must be > 0");
  spfd_opts o;
  spfd_opts_default(&o);
  if (opts) o = *opts;
  if (o.maxit < 1 || o.nu_pre < 1 || o.nu_post < 1 || o.coarse_max < 1 ||
      o.max_levels < 1 || !(o.tol > 0.0) ||
      (o.precision != SPFD_FP64 && o.precision != SPFD_MIXED) ||
      (o.smoother != SPFD_SMOOTHER_JACOBI && o.smoother != SPFD_SMOOTHER_CHEBYSHEV))
    return fail(SPFD_EINVAL, "invalid options");
  spfd_ctx *c = new (std::nothrow) spfd_ctx();
  if (!c) return fail(SPFD_ENOMEM, "host allocation of the context failed");
  c->nx = nx; c->ny = ny; c->nz = nz; c->h = h; c->opts = o;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return fail(SPFD_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  }
  spfd_status s = build_impl(c, sigma_dev);
  if (s != SPFD_OK) {
    std::string msg = g_err;
    destroy_ctx(c);
    g_err = msg;
    return s;
  }
  *out = c;
  return SPFD_OK;
}

// ------------------------------------------------------------------ solve
static spfd_status project(spfd_ctx *c, double *v);

// V-cycle on level l for right-hand side bl; returns the buffer holding the
// correction (one of L[l].x / L[l].t).  With proj (level 0 only) bl is first
// projected onto the range of A (its per-component mean removed, in place),
// so the preconditioner acts as Pi M Pi and r.z never sees the rounding
// drift of r along the constant nullspace; the single-component case fuses
// this into the first smoothing sweep, using sum(r) from the x/r update.
static double *vcycle(spfd_ctx *c, int l, double *bl, bool proj) {
  Level &lv = c->L[l];
  cudaStream_t st = c->stream;
  const int nl = (int)c->L.size();
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  if (proj && (c->ncomp > 1 || l == nl - 1)) {
    project(c, bl);
    proj = false;
  }
  if (l == nl - 1) {
    cudaMemsetAsync(lv.x, 0, lv.S * sizeof(double), st);
    launch_coarse_solve<double>(c->m, c->cidx, c->Binv, bl, lv.x, st);
    return lv.x;
  }
  double *cur = lv.x, *oth = lv.t;
  if (proj)
    launch_jacobi_first_proj<double>(lv.g, lv.wdinv, bl, cur, c->sc, inv, st);
  else
    launch_jacobi_first<double>(lv.g, lv.wdinv, bl, cur, st);
  for (int s = 1; s < c->opts.nu_pre; ++s) {
    if (l == 0)
      launch_jacobi7<double, double>(lv.g, lv.gx, lv.diag, lv.wdinv, cur, bl, oth, st);
    else
      launch_jacobi27<double>(lv.g, lv.st, lv.wdinv, cur, bl, oth, st);
    std::swap(cur, oth);
  }
  if (l == 0)
    launch_residual7<double, double>(lv.g, lv.gx, lv.diag, cur, bl, lv.r, st);
  else
    launch_residual27<double>(lv.g, lv.st, cur, bl, lv.r, st);
  Level &cl = c->L[l + 1];
  launch_restrict<double>(lv.g, cl.g, cl.P, lv.r, cl.b, st);
  double *ec = vcycle(c, l + 1, cl.b, false);
  launch_prolong<double>(lv.g, cl.g, cl.P, ec, cur, st);
  for (int s = 0; s < c->opts.nu_post; ++s) {
    if (l == 0)
      launch_jacobi7<double, double>(lv.g, lv.gx, lv.diag, lv.wdinv, cur, bl, oth, st);
    else
      launch_jacobi27<double>(lv.g, lv.st, lv.wdinv, cur, bl, oth, st);
    std::swap(cur, oth);
  }
  return cur;
}

// v -= per-component mean of v (aux slot 0 is scratch).
static spfd_status project(spfd_ctx *c, double *v) {
  Level &l0 = c->L[0];
  cudaStream_t st = c->stream;
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  if (c->ncomp > 1) {
    CU(cudaMemsetAsync(c->csum, 0, c->ncomp * sizeof(double), st));
    launch_comp_sum<double>(l0.g.nb, v, c->comp, c->csum, st);
    launch_sub_mean<double>(l0.g.nb, v, c->comp, c->sc, 0, c->csum, c->csize, inv, st);
  } else {
    launch_dot<double>(l0.g.nb, v, nullptr, c->comp, c->sc, c->partials, 0, st);
    launch_sub_mean<double>(l0.g.nb, v, c->comp, c->sc, 0, nullptr, c->csize, inv, st);
  }
  return launch_check("projection");
}

static spfd_status true_residual(spfd_ctx *c, double *rel) {
  Level &l0 = c->L[0];
  launch_residual7<double, double>(l0.g, l0.gx, l0.diag, c->xk, c->bk, l0.r, c->stream);
  launch_dot<double>(l0.g.nb, l0.r, l0.r, c->comp, c->sc, c->partials, 2, c->stream);
  TRY(launch_check("true residual"));
  TRY(read_scalars(c));
  double bb = c->hsc->bb;
  *rel = bb > 0.0 ? std::sqrt(c->hsc->aux[2] / bb) : 0.0;
  return SPFD_OK;
}

static spfd_status solve_fp64(spfd_ctx *c, double tol, spfd_info *out) {
  Level &l0 = c->L[0];
  cudaStream_t st = c->stream;
  const int nb = l0.g.nb;
  const size_t S0 = l0.S;
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  int it = 0;
  double rel = 0.0;
  bool conv = false;

  TRY(project(c, c->bk));
  launch_dot<double>(nb, c->bk, c->bk, c->comp, c->sc, c->partials, 1, st);
  TRY(read_scalars(c));
  if (c->hsc->status & DEV_BAD_A)
    return fail(SPFD_EINVAL, "a holds a non-finite value on a conducting edge");
  const double bb = c->hsc->aux[1];
  CU(cudaMemcpyAsync(&c->sc->bb, &c->sc->aux[1], sizeof(double),
                     cudaMemcpyDeviceToDevice, st));
  CU(cudaMemsetAsync(c->xk, 0, S0 * sizeof(double), st));
  if (!(bb > 0.0)) {
    conv = true;
  } else {
    CU(cudaMemcpyAsync(c->rk, c->bk, S0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemsetAsync(c->pk, 0, S0 * sizeof(double), st));
    CU(cudaMemsetAsync(&c->sc->rsum, 0, sizeof(double), st));  // b is projected
    double *z = vcycle(c, 0, c->rk, true);
    launch_dot_rz<double>(nb, c->rk, z, c->comp, c->sc, c->partials, 1, st);
    if (c->ncomp > 1) {
      CU(cudaMemsetAsync(c->csum, 0, c->ncomp * sizeof(double), st));
      launch_comp_sum<double>(nb, z, c->comp, c->csum, st);
    }
    launch_pupdate<double>(nb, c->pk, z, c->comp, c->sc,
                           c->ncomp > 1 ? c->csum : nullptr, c->csize, inv, st);
    TRY(launch_check("first V-cycle"));
    // Stopping: the recursive residual triggers a recomputation of the true
    // one; if that is still above tol, CG restarts from the true residual
    // (beta = 0).  Three restarts that fail to halve the best true residual
    // mean the rounding floor is reached: stop there (not converged).
    double best_true = INFINITY, min_rrel = INFINITY;
    int stall = 0;
    bool restart = false;
    for (it = 1; it <= c->opts.maxit; ++it) {
      launch_apply_dot<double>(l0.g, l0.gx, l0.diag, c->pk, c->qk, c->sc, c->partials, st);
      launch_update_xr<double>(nb, c->xk, c->rk, c->pk, c->qk, c->sc, c->partials, st);
      TRY(launch_check("CG update"));
      TRY(read_scalars(c));
      double rrel = std::sqrt(c->hsc->rr / bb);
      if (!std::isfinite(rrel) || rrel > 1e8 * std::max(min_rrel, tol)) {
        TRY(true_residual(c, &rel));
        break;  // breakdown: report the current iterate, not converged
      }
      min_rrel = std::min(min_rrel, rrel);
      if (rrel <= tol) {
        TRY(true_residual(c, &rel));
        if (rel <= tol) { conv = true; break; }
        if (rel < 0.5 * best_true) { best_true = rel; stall = 0; }
        else if (++stall >= 3) break;
        CU(cudaMemcpyAsync(c->rk, l0.r, S0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        TRY(project(c, c->rk));
        CU(cudaMemsetAsync(&c->sc->rsum, 0, sizeof(double), st));
        restart = true;
      }
      z = vcycle(c, 0, c->rk, true);
      launch_dot_rz<double>(nb, c->rk, z, c->comp, c->sc, c->partials, restart ? 1 : 0, st);
      restart = false;
      if (c->ncomp > 1) {
        CU(cudaMemsetAsync(c->csum, 0, c->ncomp * sizeof(double), st));
        launch_comp_sum<double>(nb, z, c->comp, c->csum, st);
      }
      launch_pupdate<double>(nb, c->pk, z, c->comp, c->sc,
                             c->ncomp > 1 ? c->csum : nullptr, c->csize, inv, st);
      TRY(launch_check("V-cycle"));
    }
    if (it > c->opts.maxit) it = c->opts.maxit;
    TRY(project(c, c->xk));
    if (!conv) TRY(true_residual(c, &rel));
  }
  out->iters = it;
  out->outer_iters = 0;
  out->converged = conv ? 1 : 0;
  out->rel_res_true = rel;
  return SPFD_OK;
}

static spfd_status solve_device(spfd_ctx *c, const double *a_dev, double tol,
                                double *psi_dev, spfd_info *info) {
  if (!(tol > 0.0)) tol = c->opts.tol;
  cudaStream_t st = c->stream;
  Level &l0 = c->L[0];
  spfd_info res = c->info;
  CU(cudaEventRecord(c->ev0, st));
  CU(cudaMemsetAsync(&c->sc->status, 0, sizeof(int), st));
  if (c->ndof == 0) {
    size_t NN = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    CU(cudaMemsetAsync(psi_dev, 0, NN * sizeof(double), st));
    res.iters = 0;
    res.converged = 1;
    res.rel_res_true = 0.0;
  } else {
    launch_rhs(l0.g, l0.gx, a_dev, c->bk, &c->sc->status, st);
    TRY(launch_check("rhs"));
    TRY(solve_fp64(c, tol, &res));
    launch_scatter<double>(l0.g, c->xk, c->comp, psi_dev, st);
    TRY(launch_check("scatter"));
  }
  CU(cudaEventRecord(c->ev1, st));
  TRY(sync_check(c, "solve"));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  res.ms_solve = ms;
  res.bytes_device = c->bytes;
  c->info = res;
  if (info) *info = res;
  if (c->opts.verbose)
    fprintf(stderr, "[spfd] solve: %d it, rel %.3e, %.3f ms\n", res.iters,
            res.rel_res_true, ms);
  if (!res.converged)
    return fail(SPFD_ENOTCONVERGED, "not converged: rel residual %.3e after %d iterations",
                res.rel_res_true, res.iters);
  return SPFD_OK;
}

extern "C" spfd_status spfd_solve(spfd_ctx *ctx, const double *a_dev,
                                  double tol, double *psi_dev,
                                  spfd_info *info) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!a_dev || !psi_dev) return fail(SPFD_EINVAL, "a_dev / psi_dev is NULL");
  if (std::isnan(tol)) return fail(SPFD_EINVAL, "tol is NaN");
  return solve_device(ctx, a_dev, tol, psi_dev, info);
}

extern "C" spfd_status spfd_solve_host(spfd_ctx *ctx, const double *a_host,
                                       double tol, double *psi_host,
                                       spfd_info *info) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!a_host || !psi_host) return fail(SPFD_EINVAL, "a_host / psi_host is NULL");
  if (std::isnan(tol)) return fail(SPFD_EINVAL, "tol is NaN");
  const size_t NN = (size_t)(ctx->nx + 1) * (ctx->ny + 1) * (ctx->nz + 1);
  if (!ctx->a_stage) TRY(dalloc(ctx, &ctx->a_stage, 3 * NN));
  if (!ctx->psi_stage) TRY(dalloc(ctx, &ctx->psi_stage, NN));
  ctx->info.bytes_device = ctx->bytes;
  CU(cudaMemcpyAsync(ctx->a_stage, a_host, 3 * NN * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  spfd_status s = solve_device(ctx, ctx->a_stage, tol, ctx->psi_stage, info);
  if (s != SPFD_OK && s != SPFD_ENOTCONVERGED) return s;
  std::string msg = g_err;
  CU(cudaMemcpyAsync(psi_host, ctx->psi_stage, NN * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream));
  TRY(sync_check(ctx, "copy psi"));
  g_err = msg;
  return s;
}

extern "C" spfd_status spfd_efield(spfd_ctx *ctx, const double *a_dev,
                                   const double *psi_dev, double omega,
                                   double *E_dev) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!a_dev || !psi_dev || !E_dev) return fail(SPFD_EINVAL, "null array");
  if (!std::isfinite(omega)) return fail(SPFD_EINVAL, "omega must be finite");
  launch_efield(ctx->mask, a_dev, psi_dev, ctx->nx, ctx->ny, ctx->nz, ctx->h,
                omega, E_dev, ctx->stream);
  return launch_check("efield");
}

extern "C" spfd_status spfd_get_info(const spfd_ctx *ctx, spfd_info *info) {
  if (!ctx || !info) return fail(SPFD_EINVAL, "null argument");
  *info = ctx->info;
  info->bytes_device = ctx->bytes;
  return SPFD_OK;
}
