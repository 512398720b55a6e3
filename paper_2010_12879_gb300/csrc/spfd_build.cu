// spfd_build: the operator of Eq. 3 and its multigrid hierarchy.
//
// Paper: Eq. 3 (Sec. II) defines G^T M_k G; Sec. III-A keeps only the
// conducting nodes; Sec. III solves with AMG-preconditioned FGMRES (AmgX).
// Here the hierarchy is geometric and operator-dependent: 2:1 vertex
// coarsening of the brick grid, BoxMG-style interpolation collapsed from the
// operator, Galerkin 27-point coarse operators, weighted-Jacobi smoothing
// with omega from a power-iteration estimate of lambda_max(D^-1 A), and a
// dense regularised inverse on the coarsest level.
#include <chrono>
#include <cstdio>
#include <cstring>

#include "spfd_ctx.cuh"

namespace spfd {

// Geometry of a level from its brick activity flags (host only): brick map,
// brick coordinates and the 27-neighbour brick table.
static spfd_status host_level(Level &lv, int NX, int NY, int NZ,
                              const std::vector<unsigned char> &flags) {
  Grid &g = lv.g;
  g = Grid{};
  g.NX = NX; g.NY = NY; g.NZ = NZ;
  g.MX = (NX + 7) / 8; g.MY = (NY + 7) / 8; g.MZ = (NZ + 7) / 8;
  const size_t nbm = (size_t)g.MX * g.MY * g.MZ;
  lv.hbmap.assign(nbm, -1);
  lv.hbco.clear();
  for (int bz = 0; bz < g.MZ; ++bz)
    for (int by = 0; by < g.MY; ++by)
      for (int bx = 0; bx < g.MX; ++bx) {
        const size_t q = ((size_t)bz * g.MY + by) * g.MX + bx;
        if (flags[q]) {
          lv.hbmap[q] = (int)lv.hbco.size();
          lv.hbco.push_back(make_int4(bx, by, bz, 0));
        }
      }
  if (lv.hbco.size() > (size_t)(INT32_MAX / BV))
    return fail(SPFD_EINVAL, "grid too large: %zu active bricks", lv.hbco.size());
  g.nb = (int)lv.hbco.size();
  lv.S = (size_t)g.nb * BV;
  return SPFD_OK;
}

// Brick activity of the level below fine level f: coarse node I sits on fine
// node 2I, and coarse brick B covers fine bricks 2B-1 .. 2B+1 on each axis.
static void coarse_flags(const Level &f, int *CX, int *CY, int *CZ,
                         std::vector<unsigned char> *cfl) {
  const Grid &fg = f.g;
  *CX = fg.NX / 2 + 1; *CY = fg.NY / 2 + 1; *CZ = fg.NZ / 2 + 1;
  const int cMX = (*CX + 7) / 8, cMY = (*CY + 7) / 8, cMZ = (*CZ + 7) / 8;
  cfl->assign((size_t)cMX * cMY * cMZ, 0);
  for (int bz = 0; bz < cMZ; ++bz)
    for (int by = 0; by < cMY; ++by)
      for (int bx = 0; bx < cMX; ++bx) {
        bool any = false;
        for (int fz = std::max(0, 2 * bz - 1); fz <= std::min(fg.MZ - 1, 2 * bz + 1) && !any; ++fz)
          for (int fy = std::max(0, 2 * by - 1); fy <= std::min(fg.MY - 1, 2 * by + 1) && !any; ++fy)
            for (int fx = std::max(0, 2 * bx - 1); fx <= std::min(fg.MX - 1, 2 * bx + 1) && !any; ++fx)
              any = f.hbmap[((size_t)fz * fg.MY + fy) * fg.MX + fx] >= 0;
        (*cfl)[((size_t)bz * cMY + by) * cMX + bx] = any;
      }
}

// Host-to-device copy for the build.  A pinned block is read by the SMs over
// the chip-to-chip link, which on GB300 reaches the copy engine's bandwidth,
// so the build's uploads do not queue behind a large copy the caller may have
// on the copy engine meanwhile (e.g. the next source field); any other host
// memory goes through cudaMemcpyAsync.
static spfd_status h2d(spfd_ctx *c, void *dst, const void *src, size_t bytes) {
  if (bytes == 0) return SPFD_OK;
  cudaPointerAttributes at{};
  const bool mapped = cudaPointerGetAttributes(&at, src) == cudaSuccess &&
                      at.type == cudaMemoryTypeHost && at.devicePointer != nullptr;
  cudaGetLastError();  // an unregistered pointer is not an error here
  if (mapped && (uintptr_t)dst % 16 == 0 && (uintptr_t)at.devicePointer % 16 == 0) {
    launch_pull(dst, at.devicePointer, bytes, c->stream);
    ++c->launch_count;
    return launch_check("upload");
  }
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
  return SPFD_OK;
}

// One asynchronous upload of host tables: each (host vector, device slot)
// pair is packed into a pinned block, copied into one device block, and the
// slot pointed at its part.  The pinned block stays with the context.
struct TableUpload {
  struct Item {
    const void *src;
    size_t bytes;
    const void **dst;
  };
  std::vector<Item> items;
  template <typename T>
  void add(const std::vector<T> &v, const T **dst) {
    items.push_back({v.data(), v.size() * sizeof(T), (const void **)dst});
  }
  spfd_status run(spfd_ctx *c) {
    size_t total = 0;
    for (auto &it : items) total += (it.bytes + 255) / 256 * 256;
    if (total == 0) return SPFD_OK;
    unsigned char *h = nullptr, *d = nullptr;
    TRY(halloc(c, &h, total));
    TRY(dalloc(c, &d, total));
    size_t off = 0;
    for (auto &it : items) {
      memcpy(h + off, it.src, it.bytes);
      *it.dst = d + off;
      off += (it.bytes + 255) / 256 * 256;
    }
    TRY(h2d(c, d, h, total));
    return SPFD_OK;
  }
};

// Jacobi weights of a 27-point level, omega = 4 / (3 * 1.05 * lambda_max),
// with lambda_max of D^-1 A from a power iteration v <- D^-1 A v from a fixed
// positive start vector: the generalized Rayleigh quotient v.(A v) / v.(D v)
// of the last iterate.  The quotient of the symmetric pencil (A, D) converges
// twice as fast as the ratio of norms, so 8 steps match 16 of the latter.
// The iterates are not normalised (they grow by at most 4^8), and nothing is
// read back: the weights are formed on the device, lambda goes to *lam_dev.
// The iteration runs in FP32 on FP32 copies of the coefficients and of the
// inverse diagonal (an estimate taken with a margin needs no more), with v
// and w in the level's FP64 vectors x and t, cleared afterwards.  The mixed
// form keeps the coefficient copy as its level's FP32 operator; other copies
// go to *tmp, released by the caller once the build's work has ended.
static spfd_status smoother_weights(spfd_ctx *c, int l, double *lam_dev, Scalars *sc,
                                   double *partials, std::vector<float *> *tmp) {
  Level &lv = c->L[l];
  const int nb = lv.g.nb;
  cudaStream_t st = c->stream;
  if (nb == 0) return SPFD_OK;
  if (!partials || !lv.st)
    return fail(SPFD_EINTERNAL, "power iteration needs a 27-point level (%d)", l);
  const size_t S = lv.S;
  float *st32 = nullptr, *dinv32 = nullptr;
  TRY(dalloc(c, &st32, 27 * S));
  if (c->opts.precision == SPFD_MIXED) lv.st32 = st32;
  else tmp->push_back(st32);
  TRY(dalloc(c, &dinv32, S));
  tmp->push_back(dinv32);
  SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0, launch_convert<float>(27 * S, lv.st, 1.0, st32, st));
  SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0, launch_convert<float>(S, lv.dinv, 1.0, dinv32, st));
  float *v = reinterpret_cast<float *>(lv.x), *w = reinterpret_cast<float *>(lv.t);
  SPFD_LAUNCH(c, "setup_power", true, 1, 0, 0, launch_power_init_f32(nb, dinv32, v, st));
  const int iters = 8;
  for (int it = 0; it < iters; ++it) {
    SPFD_LAUNCH(c, "setup_power", true, 1, 0, 0,
                launch_power27_f32(lv.g, st32, dinv32, v, w, sc, partials, st));
    std::swap(v, w);
  }
  SPFD_LAUNCH(c, "setup_power", false, 1, 0, 0,
              launch_jacobi_weights(nb, lv.dinv, sc, 1.05, lv.wdinv, lam_dev, st));
  return launch_check("power iteration");
}

// Inverse of a dense SPD n x n matrix (row-major), in place: Cholesky
// A = L L^T, then L^-1 by forward substitution, then A^-1 = L^-T L^-1.
// Returns false if a pivot is not positive.
static bool invert_spd(std::vector<double> &A, int n) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    const double *lj = &L[(size_t)j * n];
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= lj[k] * lj[k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      const double *li = &L[(size_t)i * n];
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= li[k] * lj[k];
      L[(size_t)i * n + j] = s / ljj;
    }
  }
  // Linv (lower triangular), row-major
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    Li[(size_t)i * n + i] = 1.0 / L[(size_t)i * n + i];
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += L[(size_t)i * n + k] * Li[(size_t)k * n + j];
      Li[(size_t)i * n + j] = -s / L[(size_t)i * n + i];
    }
  }
  // A^-1 = Linv^T Linv: (i,j) = sum_{k >= max(i,j)} Li[k][i] Li[k][j]
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = i; k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
    }
  return true;
}

// Wall-clock phase marks of the build (printed with opts.verbose >= 2).
struct PhaseClock {
  spfd_ctx *c;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double alloc0 = 0.0;
  void mark(const char *what) {
    if (c->opts.verbose < 2) return;
    cudaStreamSynchronize(c->stream);
    auto t1 = std::chrono::steady_clock::now();
    fprintf(stderr, "[spfd]   build phase %-18s %8.3f ms (cudaMalloc %.3f ms)\n", what,
            std::chrono::duration<double, std::milli>(t1 - t0).count(), c->alloc_ms - alloc0);
    t0 = t1;
    alloc0 = c->alloc_ms;
  }
};

// Coarsest level: B = A + sum_c mu_c v_c v_c^T (v_c the normalised indicator
// of a connected component of the coarsest graph, mu_c its mean diagonal) is
// SPD, and B^-1 r = A^+ r for r with zero mean on every component.  The
// symmetrised inverse is applied as a dense FP64 matrix-vector product.
// The host reads the level back to number its unknowns and label the
// components (a breadth-first search over the operator's couplings); the
// dense matrix is assembled, regularised and inverted on the device.
// *spare: a device block the inverse still uses when this returns (the
// caller frees it once the build's streams are synchronised: kernels on the
// side streams allocate after this, and must not be handed it meanwhile).
static spfd_status setup_coarsest(spfd_ctx *c, PhaseClock &clk, double **spare) {
  Level &lv = c->L.back();
  const size_t S = lv.S;
  const bool single = c->L.size() == 1;
  c->m = 0;
  if (S == 0) return SPFD_OK;
  // read-backs live in the context's pinned host blocks (reused across
  // builds): fresh pageable buffers cost more in first-touch page faults
  // than the work on them
  double *hdiag = nullptr, *hop = nullptr;
  const size_t nop = (single ? 3 : 27) * S;
  TRY(halloc(c, &hdiag, S));
  TRY(halloc(c, &hop, nop));
  CU(cudaMemcpyAsync(hdiag, lv.diag, S * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(hop, single ? lv.gx : lv.st, nop * sizeof(double),
                     cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_check(c, "coarsest copy"));
  clk.mark("coarsest read-back");
  std::vector<int> row(S, -1), idx;
  for (size_t s = 0; s < S; ++s)
    if (hdiag[s] > 0.0) { row[s] = (int)idx.size(); idx.push_back((int)s); }
  const int m = (int)idx.size();
  c->m = m;
  if (m == 0) return SPFD_OK;
  if ((int64_t)m * m > ((int64_t)1 << 26))
    return fail(SPFD_EINVAL, "coarsest level too large (%d unknowns); raise max_levels", m);
  const Grid &g = lv.g;
  auto slot_of = [&](int i, int j, int k) -> int {
    if (i < 0 || j < 0 || k < 0 || i >= g.NX || j >= g.NY || k >= g.NZ) return -1;
    int b = lv.hbmap[((size_t)(k >> 3) * g.MY + (j >> 3)) * g.MX + (i >> 3)];
    if (b < 0) return -1;
    return b * BV + ((k & 7) * 8 + (j & 7)) * 8 + (i & 7);
  };
  // the rows v != a that row a couples to (nonzero operator entry), in the
  // order the dense matrix holds them
  std::vector<int> nb;
  auto couplings = [&](int a) {
    nb.clear();
    const int s = idx[a];
    const int4 bc = lv.hbco[s / BV];
    const int t = s % BV;
    const int i = bc.x * 8 + (t & 7), j = bc.y * 8 + ((t >> 3) & 7), k = bc.z * 8 + (t >> 6);
    for (int e = 0; e < 27; ++e) {
      if (e == 13) continue;
      const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
      if (single && (dx != 0) + (dy != 0) + (dz != 0) != 1) continue;
      const int u = slot_of(i + dx, j + dy, k + dz);
      if (u < 0 || row[u] < 0) continue;
      double v;
      if (single) {
        const int ax = dx ? 0 : (dy ? 1 : 2);
        v = hop[(size_t)ax * S + (dx + dy + dz > 0 ? s : u)];
      } else {
        v = hop[(size_t)e * S + s];
      }
      if (v != 0.0) nb.push_back(row[u]);
    }
  };
  // connected components of the coarsest graph
  std::vector<int> cc(m, -1), queue;
  int nc = 0;
  for (int a = 0; a < m; ++a) {
    if (cc[a] >= 0) continue;
    queue.assign(1, a);
    cc[a] = nc;
    for (size_t hd = 0; hd < queue.size(); ++hd) {
      couplings(queue[hd]);
      for (int v : nb)
        if (cc[v] < 0) {
          cc[v] = nc;
          queue.push_back(v);
        }
    }
    ++nc;
  }
  // mu_c / n_c per component from the dense diagonal (as the device
  // assembles it), and the diagonal shift
  std::vector<double> dsum(nc, 0.0), mu(nc);
  std::vector<int> cnt(nc, 0);
  double dmean = 0.0;
  for (int a = 0; a < m; ++a) {
    const int s = idx[a];
    dsum[cc[a]] += single ? hdiag[s] : 0.0 + hop[(size_t)13 * S + s];
    cnt[cc[a]]++;
    dmean += hdiag[s];
  }
  for (int q = 0; q < nc; ++q) mu[q] = (dsum[q] / cnt[q]) / cnt[q];
  dmean /= m;
  // The coarsest Galerkin operator is numerically singular beyond the
  // component constants: coarse basis functions at the conducting boundary
  // can be nearly dependent (on the 2 mm body, 46 of 481 eigenvalues lie
  // below 1e-10 of the largest), and a few such "ghost" rows have diagonals
  // near 1e-13 of the largest.  Any inverse is rounding noise along those
  // directions, and different elimination orders give different noise.  A
  // shift of the whole diagonal by 1e-8 of the mean diagonal bounds the
  // condition number near 1e9, so the unpivoted elimination below stays
  // positive, while it changes the coarse solve of modes above 1e-5 of the
  // spectrum by under 1e-3.  (A shift proportional to each row's own
  // diagonal leaves the tiny ghost rows unregularised: on a 96x96x256 body
  // the condition number stayed at 2e11 and elimination met a negative
  // pivot.)
  const double shift = 1e-8 * dmean;
  TableUpload up;
  const int *d_rowof = nullptr, *d_cc = nullptr, *d_idx = nullptr;
  const double *d_mu = nullptr;
  up.add(idx, &d_idx);
  up.add(row, &d_rowof);
  up.add(cc, &d_cc);
  up.add(mu, &d_mu);
  TRY(up.run(c));
  c->cidx = const_cast<int *>(d_idx);
  double *b0 = nullptr;
  TRY(dalloc(c, &b0, (size_t)m * m));
  CU(cudaMemsetAsync(b0, 0, (size_t)m * m * sizeof(double), c->stream));
  // diagnostics: SPFD_DUMP_COARSEST=<path> writes m (int32) and the
  // assembled coarsest matrix (m x m FP64, row-major) before regularisation
  if (const char *dump = getenv("SPFD_DUMP_COARSEST")) {
    launch_coarse_dense(g, single ? lv.gx : lv.st, !single, S,
                        lv.diag, d_idx, d_rowof, m, nullptr, nullptr, 0.0, b0, c->stream);
    std::vector<double> Ad((size_t)m * m);
    CU(cudaMemcpyAsync(Ad.data(), b0, Ad.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    TRY(sync_check(c, "coarsest dump"));
    if (FILE *f = fopen(dump, "wb")) {
      fwrite(&m, sizeof(int), 1, f);
      fwrite(Ad.data(), sizeof(double), Ad.size(), f);
      fclose(f);
    }
  }
  launch_coarse_dense(g, single ? lv.gx : lv.st, !single, S, lv.diag, d_idx, d_rowof, m, d_cc,
                      d_mu, shift, b0, c->stream);
  c->launch_count += 2;
  TRY(launch_check("coarsest assembly"));
  clk.mark("coarsest assembly");
  if (m <= 64) {  // small: invert on the host
    double *A = nullptr;
    TRY(halloc(c, &A, (size_t)m * m));
    CU(cudaMemcpyAsync(A, b0, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    TRY(sync_check(c, "coarsest matrix"));
    std::vector<double> As(A, A + (size_t)m * m);
    if (!invert_spd(As, m))
      return fail(SPFD_EINTERNAL, "coarsest-level matrix is not positive definite after regularisation");
    memcpy(A, As.data(), (size_t)m * m * sizeof(double));
    TRY(h2d(c, b0, A, (size_t)m * m * sizeof(double)));
    c->Binv = b0;
    return sync_check(c, "coarsest upload");
  }
  // larger: Gauss-Jordan sweeps on the device (ping-pong between two buffers)
  double *b1 = nullptr;
  TRY(dalloc(c, &b1, (size_t)m * m));
  double *inv = nullptr;
  unsigned *bar = nullptr;
  TRY(dalloc(c, &bar, 2));
  CU(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), c->stream));
  SPFD_LAUNCH(c, "setup_coarsest", false, dense_inverse_launches(m), 0, 2.0 * m * m * m,
              inv = launch_dense_inverse(b0, b1, m, &c->sc->status, bar, c->stream));
  TRY(launch_check("coarsest inverse"));
  // a non-positive pivot raises DEV_BAD_PIVOT, read at the end of the build
  c->Binv = inv;
  *spare = inv == b0 ? b1 : b0;
  return SPFD_OK;
}

// FP32 / BF16 copies of the hierarchy for the mixed-precision solve.
// FP32 / BF16 copies of level l for the mixed-precision solve, on
// c->stream (levels are independent; level l needs its smoother weights).
static spfd_status setup_mixed_level(spfd_ctx *c, int l) {
  cudaStream_t st = c->stream;
  Level &lv = c->L[l];
  const size_t S = lv.S;
  TRY(dalloc(c, &lv.x32, S));
  TRY(dalloc(c, &lv.b32, S));
  TRY(dalloc(c, &lv.r32, S));
  TRY(dalloc(c, &lv.t32, S));
  CU(cudaMemsetAsync(lv.x32, 0, S * sizeof(float), st));
  CU(cudaMemsetAsync(lv.t32, 0, S * sizeof(float), st));
  TRY(dalloc(c, &lv.wdinv32, S));
  SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0, launch_convert<float>(S, lv.wdinv, 1.0, lv.wdinv32, st));
  if (lv.Pc) {
    TRY(dalloc(c, &lv.Pc32, 27 * (S / 8)));
    SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0,
                launch_convert<float>(27 * (S / 8), lv.Pc, 1.0, lv.Pc32, st));
  }
  if (l == 0) {
    TRY(dalloc(c, &lv.gx32, 3 * S));
    TRY(dalloc(c, &lv.gxbf, 3 * S));
    TRY(dalloc(c, &lv.diag32, S));
    SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0, launch_convert<float>(3 * S, lv.gx, 1.0, lv.gx32, st));
    SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0,
                launch_convert<__nv_bfloat16>(3 * S, lv.gx, 1.0, lv.gxbf, st));
    SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0, launch_convert<float>(S, lv.diag, 1.0, lv.diag32, st));
  } else {
    if (!lv.st32) {  // the coarsest level (no power iteration)
      TRY(dalloc(c, &lv.st32, 27 * S));
      SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0,
                  launch_convert<float>(27 * S, lv.st, 1.0, lv.st32, st));
    }
    TRY(dalloc(c, &lv.P32, 27 * S));
    SPFD_LAUNCH(c, "setup_convert", false, 1, 0, 0, launch_convert<float>(27 * S, lv.P, 1.0, lv.P32, st));
  }
  return launch_check("mixed-precision copies");
}

// The FP32 inner-solve vectors of the mixed-precision solve.
static spfd_status setup_mixed_krylov(spfd_ctx *c) {
  const size_t S0 = c->L[0].S;
  TRY(dalloc(c, &c->dk32, S0));
  TRY(dalloc(c, &c->rk32, S0));
  TRY(dalloc(c, &c->pk32, S0));
  TRY(dalloc(c, &c->qk32, S0));
  return SPFD_OK;
}

spfd_status build_impl(spfd_ctx *c, const double *sigma) {
  cudaStream_t st = c->stream;
  PhaseClock clk{c};
  TRY(dalloc(c, &c->sc, 1));
  CU(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), st));
  TRY(halloc(c, &c->hsc, 1));
  memset(c->hsc, 0, sizeof(Scalars));
  CU(cudaEventCreate(&c->ev0));
  CU(cudaEventCreate(&c->ev1));
  CU(cudaEventCreateWithFlags(&c->evsc, cudaEventDisableTiming));
  CU(cudaEventRecord(c->ev0, st));
  const int64_t launches0 = c->launch_count;

  const int NX = c->nx + 1, NY = c->ny + 1, NZ = c->nz + 1;
  const int MX = (NX + 7) / 8, MY = (NY + 7) / 8, MZ = (NZ + 7) / 8;
  const size_t nbm = (size_t)MX * MY * MZ;
  const size_t nvox = (size_t)c->nx * c->ny * c->nz;
  unsigned char *flags = nullptr, *hflags_p = nullptr;
  TRY(dalloc(c, &flags, nbm));
  TRY(dalloc(c, &c->mask, nvox));
  TRY(halloc(c, &hflags_p, nbm));
  CU(cudaMemsetAsync(flags, 0, nbm, st));
  SPFD_LAUNCH(c, "setup_flags", false, 1, 9.0 * nvox, 0,
              launch_sigma_flags(sigma, c->nx, c->ny, c->nz, MX, MY, flags, c->mask,
                                 &c->sc->status, st));
  TRY(launch_check("sigma flags"));
  CU(cudaMemcpyAsync(hflags_p, flags, nbm, cudaMemcpyDeviceToHost, st));
  TRY(read_scalars(c));
  dfree(c, flags);
  if (c->hsc->status & DEV_BAD_SIGMA)
    return fail(SPFD_EINVAL, "sigma holds a negative, NaN or infinite value");

  clk.mark("flags");
  c->L.clear();
  c->L.emplace_back();
  {
    const std::vector<unsigned char> hflags(hflags_p, hflags_p + nbm);
    TRY(host_level(c->L[0], NX, NY, NZ, hflags));
    TableUpload up;
    Level &l0 = c->L[0];
    up.add(l0.hbmap, &l0.g.bmap);
    up.add(l0.hbco, &l0.g.bco);
    TRY(up.run(c));
    int *nbr = nullptr;
    TRY(dalloc(c, &nbr, (size_t)std::max(l0.g.nb, 1) * 27));
    launch_brick_nbr(l0.g, nbr, st);
    c->launch_count += l0.g.nb ? 1 : 0;
    l0.g.nbr = nbr;
  }
  clk.mark("level-0 tables");
  const size_t S0 = c->L[0].S;
  const int nb0 = c->L[0].g.nb;
  // reduction scratch: the level-0 CG operator and the last smoothing sweep
  // write at most 8 partials per brick (16 reserved), followed by the finishing reduction's block sums (152); the
  // grid-stride reductions of every level write 2 values per block, on at
  // most 608 blocks
  c->pstride = 16 * (size_t)std::max(nb0, 1) + 2048;
  TRY(dalloc(c, &c->partials, c->pstride));
  int *parent = nullptr, *counts = nullptr, *offsets = nullptr;
  int *comp_hcnt = nullptr, *comp_hstat = nullptr;
  struct CompStream {  // released on every exit (the context is then destroyed)
    spfd_ctx *c;
    cudaStream_t main, s = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    ~CompStream() {
      c->stream = main;
      if (s) cudaStreamDestroy(s);
      if (fork) cudaEventDestroy(fork);
      if (done) cudaEventDestroy(done);
    }
  } comp_side{c, st};
  {
    Level &l0 = c->L[0];
    TRY(dalloc(c, &l0.gx, 3 * S0));
    TRY(dalloc(c, &l0.diag, S0));
    TRY(dalloc(c, &l0.dinv, S0));
    TRY(dalloc(c, &l0.wdinv, S0));
    SPFD_LAUNCH(c, "setup_fine", false, 1, 40.0 * S0, 0,
                launch_build_fine(l0.g, sigma, c->nx, c->ny, c->nz, c->h, l0.gx,
                                  l0.diag, l0.dinv, st));
    TRY(launch_check("build fine"));
    // connected components of the conducting nodes: the union-find and the
    // root counts run on a stream of their own, overlapping the coarse
    // tables and the hierarchy (which do not need them); the numbering that
    // follows runs on the main stream after it
    TRY(dalloc(c, &parent, S0));
    TRY(dalloc(c, &c->comp, S0));
    TRY(dalloc(c, &counts, nb0));
    TRY(dalloc(c, &offsets, nb0));
    TRY(halloc(c, &comp_hcnt, std::max(nb0, 1)));
    TRY(halloc(c, &comp_hstat, 1));
    CU(cudaStreamCreateWithFlags(&comp_side.s, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&comp_side.fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&comp_side.done, cudaEventDisableTiming));
    CU(cudaEventRecord(comp_side.fork, st));
    CU(cudaStreamWaitEvent(comp_side.s, comp_side.fork, 0));
    c->stream = comp_side.s;
    SPFD_LAUNCH(c, "setup_components", false, 3, 0, 0,
                launch_components(l0.g, l0.gx, parent, &c->sc->status, comp_side.s));
    SPFD_LAUNCH(c, "setup_components", false, 1, 0, 0,
                launch_root_counts(l0.g, parent, counts, comp_side.s));
    c->stream = st;
    TRY(launch_check("components"));
    if (nb0)
      CU(cudaMemcpyAsync(comp_hcnt, counts, nb0 * sizeof(int), cudaMemcpyDeviceToHost,
                         comp_side.s));
    CU(cudaMemcpyAsync(comp_hstat, &c->sc->status, sizeof(int), cudaMemcpyDeviceToHost,
                       comp_side.s));
    CU(cudaEventRecord(comp_side.done, comp_side.s));
  }

  // The brick structure of every coarser level follows from the brick maps
  // alone, so it is built on the host while the device labels components.
  // Levels are added until one could hold no more than coarse_max unknowns
  // (its slot and node counts bound them) or the grid is exhausted; the levels past
  // the first one whose actual unknowns fit coarse_max are dropped below.
  for (int l = 0;; ++l) {
    const Level &f = c->L[l];
    const int64_t bound = std::min<int64_t>((int64_t)f.S, (int64_t)f.g.NX * f.g.NY * f.g.NZ);
    if (bound <= c->opts.coarse_max || l + 1 >= c->opts.max_levels ||
        (f.g.NX <= 3 && f.g.NY <= 3 && f.g.NZ <= 3))
      break;
    int CX, CY, CZ;
    std::vector<unsigned char> cfl;
    coarse_flags(f, &CX, &CY, &CZ, &cfl);
    c->L.emplace_back();  // (invalidates references into c->L)
    TRY(host_level(c->L[l + 1], CX, CY, CZ, cfl));
  }
  const int LB = (int)c->L.size();
  clk.mark("coarse tables (host)");
  {
    // brick maps and coordinates from the host; the neighbour, child and
    // parent tables are formed on the device from them
    TableUpload up;
    for (int l = 1; l < LB; ++l) {
      up.add(c->L[l].hbmap, &c->L[l].g.bmap);
      up.add(c->L[l].hbco, &c->L[l].g.bco);
    }
    TRY(up.run(c));
    for (int l = 0; l < LB; ++l) {
      Grid &g = c->L[l].g;
      if (l > 0) {
        int *nbr = nullptr, *kid = nullptr;
        TRY(dalloc(c, &nbr, (size_t)std::max(g.nb, 1) * 27));
        TRY(dalloc(c, &kid, (size_t)std::max(g.nb, 1) * 27));
        launch_brick_nbr(g, nbr, st);
        launch_brick_kid(c->L[l - 1].g, g, kid, st);
        c->launch_count += g.nb ? 2 : 0;
        g.nbr = nbr;
        g.kid = kid;
      }
      if (l + 1 < LB) {
        int *par = nullptr;
        TRY(dalloc(c, &par, (size_t)std::max(g.nb, 1) * 8));
        launch_brick_par(g, c->L[l + 1].g, par, st);
        c->launch_count += g.nb ? 1 : 0;
        g.par = par;
      }
    }
    TRY(launch_check("brick tables"));
  }

  clk.mark("brick tables");

  // Multigrid hierarchy, enqueued without host round trips.  lstat[4l..4l+3]:
  // level l's count and largest entry of the Galerkin diagonal, then the
  // same after the activity threshold (count = unknowns of the level).
  // Ttmp: the product A P of one level, scratch grown to the largest fine
  // level (a coarse level can hold more bricks than the level above it, up
  // to 8 per odd-indexed fine brick).
  unsigned long long *lstat = nullptr;
  double *lam = nullptr;
  TRY(dalloc(c, &lstat, 4 * (size_t)LB));
  TRY(dalloc(c, &lam, LB));
  CU(cudaMemsetAsync(lstat, 0, 4 * LB * sizeof(unsigned long long), st));
  CU(cudaMemsetAsync(lam, 0, LB * sizeof(double), st));
  double *Ttmp = nullptr;
  size_t Tcap = 0;
  for (int l = 0; l < LB; ++l) {
    Level &f = c->L[l];
    TRY(dalloc(c, &f.x, f.S));
    TRY(dalloc(c, &f.b, f.S));
    TRY(dalloc(c, &f.r, f.S));
    TRY(dalloc(c, &f.t, f.S));
    CU(cudaMemsetAsync(f.x, 0, f.S * sizeof(double), st));
    CU(cudaMemsetAsync(f.t, 0, f.S * sizeof(double), st));
    if (l + 1 == LB) break;
    Level &cl = c->L[l + 1];
    const size_t Sc = cl.S;
    TRY(dalloc(c, &cl.st, 27 * Sc));
    TRY(dalloc(c, &cl.P, 27 * Sc));
    TRY(dalloc(c, &cl.diag, Sc));
    TRY(dalloc(c, &cl.dinv, Sc));
    TRY(dalloc(c, &cl.wdinv, Sc));
    TRY(dalloc(c, &f.Pc, 27 * (f.S / 8)));
    if (f.S > Tcap) {
      dfree(c, Ttmp);
      TRY(dalloc(c, &Ttmp, (size_t)ap_rows_per_cell() * (f.S / 8)));
      Tcap = f.S;
    }
    SPFD_LAUNCH(c, "setup_interp", false, 3, 0, 0,
                launch_interp_weights(f.g, f.gx, f.st, f.diag, f.Pc, st));
    unsigned *bits = nullptr;  // the coarse level's activity bits, written with P
    TRY(dalloc(c, &bits, (size_t)std::max(cl.g.nb, 1) * 16));
    SPFD_LAUNCH(c, "setup_galerkin", false, 3, 0, 0,
                launch_galerkin(f.g, cl.g, f.gx, f.st, f.diag, f.Pc, Ttmp, cl.st, cl.P, bits,
                                st));
    cl.g.act = bits;
    // Rows below 1e-13 of the level's largest diagonal are not unknowns:
    // they come only from basis functions constant on a tiny component.
    unsigned long long *ls = lstat + 4 * (l + 1);
    SPFD_LAUNCH(c, "setup_pack", false, 1, 8.0 * Sc, 0,
                launch_diag_stats(cl.st + 13 * Sc, Sc, ls, st));
    SPFD_LAUNCH(c, "setup_pack", false, 1, 0, 0,
                launch_coarse_diag(cl.g, cl.st, ls + 1, 1e-13, cl.diag, cl.dinv, st));
    SPFD_LAUNCH(c, "setup_pack", false, 1, 8.0 * Sc, 0,
                launch_diag_stats(cl.diag, Sc, ls + 2, st));
    TRY(launch_check("coarse level"));
  }
  dfree(c, Ttmp);
  // component numbering, once the side stream's root counts are in (the
  // host waits for that stream alone; the main stream waits for it before
  // the numbering kernels)
  {
    Level &l0 = c->L[0];
    CU(cudaEventSynchronize(comp_side.done));
    if (*comp_hstat & DEV_UF_CAP)
      return fail(SPFD_EINTERNAL, "component labelling hit its iteration cap");
    CU(cudaStreamWaitEvent(st, comp_side.done, 0));
    const int *hcnt = comp_hcnt;
    int *hoff = nullptr;
    TRY(halloc(c, &hoff, nb0));
    int64_t tot = 0;
    for (int b = 0; b < nb0; ++b) { hoff[b] = (int)tot; tot += hcnt[b]; }
    c->ncomp = (int)tot;
    if (nb0)
      TRY(h2d(c, offsets, hoff, nb0 * sizeof(int)));
    SPFD_LAUNCH(c, "setup_components", false, 2, 0, 0, launch_assign_comp(l0.g, parent, offsets, c->comp, st));
    TRY(dalloc(c, &c->csize, std::max(c->ncomp, 1)));
    CU(cudaMemsetAsync(c->csize, 0, std::max(c->ncomp, 1) * sizeof(int), st));
    SPFD_LAUNCH(c, "setup_components", false, 1, 0, 0, launch_comp_sizes(l0.g, c->comp, c->csize, st));
    TRY(launch_check("component sizes"));
    dfree(c, parent);
    dfree(c, counts);
    dfree(c, offsets);
    c->cstride = 3 * c->ncomp + 1;
    if (c->ncomp > 1) TRY(dalloc(c, &c->csum, c->cstride));
  }
  clk.mark("components");
  {
    // the one read-back of the hierarchy: component sizes and the unknowns
    // of every level
    unsigned long long *hl = nullptr;
    int *hsize = nullptr;
    TRY(halloc(c, &hl, 4 * (size_t)LB));
    TRY(halloc(c, &hsize, std::max(c->ncomp, 1)));
    CU(cudaMemcpyAsync(hl, lstat, 4 * LB * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(hsize, c->csize, std::max(c->ncomp, 1) * sizeof(int),
                       cudaMemcpyDeviceToHost, st));
    TRY(sync_check(c, "hierarchy"));
    c->ndof = 0;
    for (int q = 0; q < c->ncomp; ++q) c->ndof += hsize[q];
    c->L[0].n_active = c->ndof;
    for (int l = 1; l < LB; ++l) c->L[l].n_active = (int64_t)hl[4 * l + 2];
  }
  // the coarsest level: the first whose unknowns fit coarse_max
  int LU = LB;
  for (int l = 0; l < LB; ++l)
    if (c->L[l].n_active <= c->opts.coarse_max) { LU = l + 1; break; }
  while ((int)c->L.size() > LU) {
    Level &lv = c->L.back();
    for (double **p : {&lv.st, &lv.P, &lv.diag, &lv.dinv, &lv.wdinv, &lv.x, &lv.b, &lv.r,
                       &lv.t, &lv.Pc})
      dfree(c, *p);
    c->L.pop_back();
  }
  dfree(c, c->L.back().Pc);
  clk.mark("coarse levels");


  // smoother weights (weighted Jacobi): level 0 has D^-1 A the random-walk
  // Laplacian of a bipartite node graph, so lambda_max = 2 exactly and
  // omega = 2/3; coarser levels estimate it on the device by power
  // iterations.  Those are independent of one another and of the coarsest
  // inverse, so each runs on a stream of its own (with its own reduction
  // scratch) while the main stream inverts the coarsest level.  The side
  // streams fork from the main stream before the coarsest level, but their
  // kernels are enqueued after the inverse's cooperative launch: launched
  // first, the inverse takes its SM slots (a quarter of each SM's threads),
  // and the power iterations fill the rest beside it instead of holding
  // every SM until they end.
  {
    Level &l0 = c->L[0];
    l0.lmax = 2.0;
    l0.omega = 2.0 / 3.0;
    SPFD_LAUNCH(c, "setup_power", false, 1, 0, 0,
                launch_scaled_copy(l0.g.nb, l0.dinv, l0.omega, l0.wdinv, st));
    if (c->L.size() > 1) {
      CU(cudaMemsetAsync(l0.x, 0, l0.S * sizeof(double), st));
      CU(cudaMemsetAsync(l0.t, 0, l0.S * sizeof(double), st));
    }
  }
  const int np = std::max(0, (int)c->L.size() - 2);  // levels 1 .. coarsest - 1
  struct SideStreams {  // streams and events are released on every exit
    spfd_ctx *c;
    cudaStream_t main;
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> e;
    ~SideStreams() {
      c->stream = main;
      for (cudaStream_t x : s) if (x) cudaStreamDestroy(x);
      for (cudaEvent_t x : e) if (x) cudaEventDestroy(x);
    }
  };
  // one stream per power iteration, plus one for level 0's mixed-precision
  // copies; the last event is the fork point
  const bool mixed = c->opts.precision == SPFD_MIXED;
  const int ns = np + (mixed ? 1 : 0);
  SideStreams side{c, st, std::vector<cudaStream_t>(ns, nullptr),
                   std::vector<cudaEvent_t>(ns + 1, nullptr)};
  Scalars *psc = nullptr;
  double *ppart = nullptr;
  const size_t part_per_level = 2 * 1024;  // grid_sum<2> over <= 1024 blocks
  if (ns > 0) {
    if (np > 0) {
      TRY(dalloc(c, &psc, np));
      TRY(dalloc(c, &ppart, part_per_level * np));
      CU(cudaMemsetAsync(psc, 0, np * sizeof(Scalars), st));
    }
    CU(cudaEventCreateWithFlags(&side.e[ns], cudaEventDisableTiming));
    CU(cudaEventRecord(side.e[ns], st));
  }
  clk.mark("smoother weights");
  double *gj_spare = nullptr;
  std::vector<float *> tmp32;  // FP32 copies of the power iterations
  TRY(setup_coarsest(c, clk, &gj_spare));
  clk.mark("coarsest inverse");
  if (ns > 0) {
    for (int i = 0; i < ns; ++i) {
      CU(cudaStreamCreateWithFlags(&side.s[i], cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&side.e[i], cudaEventDisableTiming));
      CU(cudaStreamWaitEvent(side.s[i], side.e[ns], 0));
      c->stream = side.s[i];
      if (i < np) {
        const int l = i + 1;
        Level &lv = c->L[l];
        TRY(smoother_weights(c, l, lam + l, psc + i, ppart + part_per_level * i, &tmp32));
        CU(cudaMemsetAsync(lv.x, 0, lv.S * sizeof(double), side.s[i]));
        CU(cudaMemsetAsync(lv.t, 0, lv.S * sizeof(double), side.s[i]));
        if (mixed) TRY(setup_mixed_level(c, l));
      } else {
        TRY(setup_mixed_level(c, 0));
      }
      CU(cudaEventRecord(side.e[i], side.s[i]));
      c->stream = st;
    }
  } else if (mixed) {
    TRY(setup_mixed_level(c, 0));
  }
  if (mixed && c->L.size() > 1) TRY(setup_mixed_level(c, (int)c->L.size() - 1));
  for (int i = 0; i < ns; ++i) CU(cudaStreamWaitEvent(st, side.e[i], 0));
  dfree(c, psc);
  dfree(c, ppart);

  // Krylov vectors
  TRY(dalloc(c, &c->xk, S0));
  TRY(dalloc(c, &c->rk, S0));
  TRY(dalloc(c, &c->pk, S0));
  TRY(dalloc(c, &c->qk, S0));
  TRY(dalloc(c, &c->bk, S0));
  if (mixed) TRY(setup_mixed_krylov(c));
  clk.mark("vectors+mixed");
  // read back the device status and the smoother estimates, then clear the
  // scalars for the solves
  double *hlam = nullptr;
  TRY(halloc(c, &hlam, LB));
  CU(cudaMemcpyAsync(hlam, lam, LB * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  CU(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), st));
  const double inv_ndof = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  launch_set_f64(&c->sc->inv_ndof, inv_ndof, st);
  ++c->launch_count;
  CU(cudaEventRecord(c->ev1, st));
  TRY(sync_check(c, "build"));
  dfree(c, gj_spare);
  for (float *&p : tmp32) dfree(c, p);
  if (c->hsc->status & DEV_BAD_PIVOT)
    return fail(SPFD_EINTERNAL, "coarsest-level matrix is not positive definite after regularisation");
  if (c->hsc->status & DEV_GRID_WAIT)
    return fail(SPFD_EINTERNAL, "coarsest inverse: a grid-wide barrier hit its wait cap");
  for (size_t l = 1; l + 1 < c->L.size(); ++l) {
    c->L[l].lmax = hlam[l];
    c->L[l].omega = 4.0 / (3.0 * 1.05 * hlam[l]);
  }
  dfree(c, lstat);
  dfree(c, lam);
  TRY(prof_flush(c));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->info.ms_build = ms;
  c->info.n_dof = c->ndof;
  c->info.n_comp = c->ncomp;
  c->info.n_levels = (int)c->L.size();
  c->info.n_bricks = nb0;
  c->info.bytes_device = c->bytes;
  c->info.launches = c->launch_count - launches0;
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

}  // namespace spfd
