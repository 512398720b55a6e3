// C ABI of libspfd: context lifetime, solve paths and |E|.
//
// Paper: Eq. 3 (Sec. II) is the system solved; Sec. II-A fixes double
// precision and a relative-residual target (1e-12 in the paper); Sec. III
// solves it with AMG-preconditioned FGMRES from AmgX, which this library
// replaces by CG (the operator is symmetric positive semidefinite and the
// right-hand side consistent) preconditioned by a multigrid V-cycle.  Eq. 1
// with the voxel averaging of Sec. III-E gives |E|.
//
// Two arithmetics (opts.precision):
//   SPFD_FP64   CG, V-cycle and operator all in FP64;
//   SPFD_MIXED  FP64 iterative refinement: r = b - A x in FP64, then an FP32
//               CG (operator with FP32 conductances, V-cycle with BF16
//               finest-level conductances and FP32 accumulation) solves
//               A d = r to a modest relative accuracy, x += d in FP64.
//               Dot products accumulate in FP64; the coarsest solve is FP64.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "spfd_ctx.cuh"

using namespace spfd;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

namespace spfd {
thread_local bool pdl_allowed = true;
spfd_status fail(spfd_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}
void set_error(const std::string &msg) { g_err = msg; }
std::string last_error_copy() { return g_err; }

spfd_status sync_check(spfd_ctx *c, const char *what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SPFD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return SPFD_OK;
}

spfd_status launch_check(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(SPFD_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return SPFD_OK;
}

// Device scalars of the first nk right-hand sides into the pinned mirror
// (synchronises the stream).
spfd_status read_scalars(spfd_ctx *c, int nk) {
  CU(cudaMemcpyAsync(c->hsc, c->sc, (size_t)nk * sizeof(Scalars), cudaMemcpyDeviceToHost,
                     c->stream));
  return sync_check(c, "reading solver scalars");
}

void destroy_ctx(spfd_ctx *c) {
  if (!c) return;
  // idle after the synchronisation: every block goes to the process cache
  cudaStreamSynchronize(c->stream);
  for (size_t k = 0; k < c->allocs.size(); ++k)
    spfd::mem_put(c->device, c->allocs[k], c->alloc_bytes[k]);
  for (auto &b : c->spare) spfd::mem_put(c->device, b.first, b.second);
  c->allocs.clear();
  c->alloc_bytes.clear();
  c->spare.clear();
  for (auto &b : c->hblocks) spfd::host_put(b.first, b.second);
  c->hblocks.clear();
  for (auto &r : c->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evsc) cudaEventDestroy(c->evsc);
  delete c;
}

// ------------------------------------------------------------------ profiling
int stat_index(spfd_ctx *c, const char *name, bool f32) {
  std::string key = std::string(name) + (f32 ? "_f32" : "_f64");
  for (size_t i = 0; i < c->stats.size(); ++i)
    if (c->stats[i].name == key) return (int)i;
  c->stats.push_back(KernelStat{key});
  return (int)c->stats.size() - 1;
}

cudaEvent_t take_event(spfd_ctx *c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_push(spfd_ctx *c, int stat, cudaEvent_t a, cudaEvent_t b,
               double bytes, double flops) {
  c->pending.push_back(ProfRec{stat, a, b, bytes, flops});
}

spfd_status prof_flush(spfd_ctx *c) {
  if (c->pending.empty()) return SPFD_OK;
  TRY(sync_check(c, "profile flush"));
  for (auto &r : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    KernelStat &s = c->stats[r.stat];
    s.launches++;
    s.ms += ms;
    s.bytes += r.bytes;
    s.flops += r.flops;
    c->evpool.push_back(r.a);
    c->evpool.push_back(r.b);
  }
  c->pending.clear();
  return SPFD_OK;
}
}  // namespace spfd

extern "C" const char *spfd_last_error(void) { return g_err.c_str(); }

extern "C" spfd_status spfd_release_cached_memory(size_t *released) {
  const size_t n = spfd::mem_release_all();
  if (released) *released = n;
  return SPFD_OK;
}

extern "C" void spfd_destroy(spfd_ctx *ctx) { destroy_ctx(ctx); }

// Chebyshev smoother: ratio of the eigenvalue bounds of D^-1 A it damps
// (the upper part of the spectrum, which the coarse levels do not correct),
// the margin on coarse levels' lambda_max estimates, and the largest degree
// accepted.  Measured on the 2 mm body with degree 2: ratio 30 took 69
// iterations (too little damping per step on the upper half), ratio 4 or 8
// took 9; margin 1.3 costs no iteration against 1.05 there.
constexpr double CHEB_RATIO = 8.0;
constexpr double CHEB_MARGIN = 1.3;  // on the power-iteration estimate of coarse levels
constexpr int CHEB_MAX_DEGREE = 8;

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
  o->profile = 0;
  o->autotune = 1;
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
  if (o.smoother == SPFD_SMOOTHER_CHEBYSHEV &&
      (o.cheb_degree < 1 || o.cheb_degree > CHEB_MAX_DEGREE))
    return fail(SPFD_EINVAL, "cheb_degree must be in 1..%d (got %d)", CHEB_MAX_DEGREE,
                o.cheb_degree);
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

// ------------------------------------------------------------------ V-cycle
template <typename T> struct Prec;
template <> struct Prec<double> {
  using C7 = double;  // level-0 conductance storage in the V-cycle
  static const double *gx(const Level &l) { return l.gx; }
};
template <> struct Prec<float> {
  using C7 = __nv_bfloat16;
  static const __nv_bfloat16 *gx(const Level &l) { return l.gxbf; }
};

// v -= per-component mean of v for nk right-hand sides (aux slot 0 of each
// one's Scalars is scratch).  j0 selects the first right-hand side.
template <typename T>
spfd_status project(spfd_ctx *c, T *v, int nk, int j0) {
  Level &l0 = c->L[0];
  cudaStream_t st = c->stream;
  const bool f32 = sizeof(T) == 4;
  const double S = (double)l0.S * nk, w = sizeof(T);
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  Scalars *sc = c->sc + j0;
  double *partials = c->partials + (size_t)j0 * c->pstride;
  if (c->ncomp > 1) {
    double *csum = c->csum + (size_t)j0 * c->cstride;
    SPFD_LAUNCH(c, "project", f32, 3, 2 * (w + 4) * S, 12 * S,
                launch_comp_sum<T>(l0.g.nb, v, c->comp, csum, c->ncomp, c->cstride, st, nk));
    SPFD_LAUNCH(c, "project", f32, 1, (2 * w + 4) * S, S,
                launch_sub_mean<T>(l0.g.nb, v, c->comp, sc, 0, csum, c->csize, inv, st, nk,
                                   c->cstride));
  } else {
    SPFD_LAUNCH(c, "project", f32, 1, (w + 4) * S, S,
                launch_dot<T>(l0.g.nb, v, nullptr, c->comp, sc, partials, 0, st, nk,
                              c->pstride));
    SPFD_LAUNCH(c, "project", f32, 1, (2 * w + 4) * S, S,
                launch_sub_mean<T>(l0.g.nb, v, c->comp, sc, 0, nullptr, c->csize, inv, st, nk));
  }
  return launch_check("projection");
}

// Kernel-family name of a V-cycle kernel on level l: levels 0-4 by number
// (level 0 is HBM-sized, levels >= 2 of the 2 mm body are L2-resident and
// latency-bound), deeper levels together.
static const char *lvl_name(const char *const (&names)[6], int l) {
  return names[l < 5 ? l : 5];
}
#define LVL_NAMES(base)                                                          \
  {base "_l0", base "_l1", base "_l2", base "_l3", base "_l4", base "_deep"}

// Chebyshev smoothing of degree k on D^-1 A: eigenvalue bounds
// [hi / CHEB_RATIO, hi] with hi the level's lambda_max (2 on level 0, the
// power-iteration estimate times CHEB_MARGIN above: the polynomial grows
// fast past hi, so an underestimate costs more than with Jacobi's 1.05
// margin), theta and delta their centre
// and half-width; the recurrence of the shifted and scaled Chebyshev
// polynomials gives d_0 = D^-1 r_0 / theta and, for j >= 1,
// rho_j = 1 / (2 theta / delta - rho_{j-1}) (rho_0 = delta / theta),
// d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) D^-1 r_j, with
// x_{j+1} = x_j + d_j.  c1[j], c2[j] are the two factors of step j.
struct ChebCoef {
  double c1[CHEB_MAX_DEGREE], c2[CHEB_MAX_DEGREE];
};
static ChebCoef cheb_coefficients(double hi, int k) {
  ChebCoef cf{};
  const double lo = hi / CHEB_RATIO;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  cf.c1[0] = 0.0;
  cf.c2[0] = 1.0 / theta;
  for (int j = 1; j < k && j < CHEB_MAX_DEGREE; ++j) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    cf.c1[j] = rn * rho;
    cf.c2[j] = 2.0 * rn / delta;
    rho = rn;
  }
  return cf;
}

// V-cycle on level l for the right-hand sides bl (nk of them, S_l apart);
// returns the buffer holding the corrections.  With proj (level 0) bl is
// first projected onto the range of A in place (its per-component mean
// removed), so the preconditioner acts as Pi M Pi and r.z never sees the
// rounding drift of r along the constant nullspace; with one component this
// is fused into the first sweep, using sum(r) left in each right-hand side's
// Scalars by the preceding x/r update.
template <typename T>
T *vcycle(spfd_ctx *c, int l, T *bl, bool proj, int nk, bool rz, bool head) {
  Level &lv = c->L[l];
  cudaStream_t st = c->stream;
  const int nl = (int)c->L.size();
  const bool f32 = sizeof(T) == 4;
  const double w = sizeof(T), S = (double)lv.S * nk;
  const double wc = sizeof(typename Prec<T>::C7);
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  const bool cheb = c->opts.smoother == SPFD_SMOOTHER_CHEBYSHEV;
  if (proj && (cheb || c->ncomp > 1 || l == nl - 1)) {
    project<T>(c, bl, nk);
    proj = false;
  }
  if (l == nl - 1) {
    const double m = c->m;
    cudaMemsetAsync(lv.X<T>(), 0, lv.S * nk * sizeof(T), st);
    SPFD_LAUNCH(c, "coarsest_solve", f32, 1, (8 * m * m + 2 * w * m) * nk, 2 * m * m * nk,
                launch_coarse_solve<T>(c->m, lv.S, c->cidx, c->Binv, bl, lv.X<T>(), st, nk));
    return lv.X<T>();
  }
  const T *wd = lv.WDINV<T>();
  auto residual = [&](const T *xin, T *rout) {
    if (l == 0)
      SPFD_LAUNCH(c, "residual7_l0", f32, 1, (4 * w + 3 * wc) * S, 14 * S,
                  (launch_residual7<T, typename Prec<T>::C7>(lv.g, Prec<T>::gx(lv),
                                                             lv.DIAG<T>(), xin, bl, rout, st,
                                                             nk, block_order(c, TF_RESID, l))));
    else
      SPFD_LAUNCH(c, lvl_name(LVL_NAMES("residual27"), l), f32, 1,
                  30 * w * S, 55 * S,
                  launch_residual27<T>(lv.g, lv.ST<T>(), xin, bl, rout, st, nk,
                                       block_order(c, TF_RESID, l)));
  };
  if (cheb) {
    // Chebyshev: x ping-pongs between the level's two vectors, d lives in
    // its residual vector (free while smoothing; the residual for the
    // restriction overwrites it once pre-smoothing is done)
    const int k = c->opts.cheb_degree;
    const ChebCoef cf = cheb_coefficients(l == 0 ? 2.0 : CHEB_MARGIN * lv.lmax, k);
    const double iw = 1.0 / lv.omega;  // wdinv = omega D^-1
    T *cur = lv.X<T>(), *oth = lv.Tt<T>(), *d = lv.R<T>();
    auto step = [&](int j) {
      if (l == 0)
        SPFD_LAUNCH(c, "cheb7_l0", f32, 1, (7 * w + 3 * wc) * S, 18 * S,
                    (launch_cheb7<T, typename Prec<T>::C7>(lv.g, Prec<T>::gx(lv), lv.DIAG<T>(),
                                                           wd, cur, bl, oth, d, cf.c1[j],
                                                           cf.c2[j] * iw, st, nk)));
      else
        SPFD_LAUNCH(c, lvl_name(LVL_NAMES("cheb27"), l), f32, 1, 34 * w * S, 59 * S,
                    launch_cheb27<T>(lv.g, lv.ST<T>(), wd, cur, bl, oth, d, cf.c1[j],
                                     cf.c2[j] * iw, st, nk));
      std::swap(cur, oth);
    };
    SPFD_LAUNCH(c, lvl_name(LVL_NAMES("cheb_first"), l), f32, 1, 4 * w * S, 2 * S,
                launch_cheb<T>(true, lv.S, wd, bl, d, cur, 0.0, cf.c2[0] * iw, st, nk));
    for (int j = 1; j < k; ++j) step(j);
    residual(cur, lv.R<T>());
    Level &cl = c->L[l + 1];
    const double Sc = (double)cl.S * nk;
    SPFD_LAUNCH(c, lvl_name(LVL_NAMES("restrict"), l), f32, 1,
                28 * w * Sc + w * S, 54 * Sc,
                launch_restrict<T>(lv.g, cl.g, cl.PP<T>(), lv.R<T>(), cl.B<T>(), st, nk,
                                   block_order(c, TF_RESTRICT, l)));
    T *ec = vcycle<T>(c, l + 1, cl.B<T>(), false, nk);
    SPFD_LAUNCH(c, lvl_name(LVL_NAMES("prolong"), l), f32, 1,
                (27.0 / 8.0 + 2.0) * w * S + w * Sc, 7 * S,
                launch_prolong<T>(lv.g, cl.g, lv.PC<T>(), ec, cur, st, nk,
                                  block_order(c, TF_PROLONG, l)));
    for (int j = 0; j < k; ++j) step(j);  // post-smoothing: the recurrence restarts
    return cur;
  }
  T *cur = lv.X<T>(), *oth = lv.Tt<T>();
  if (head)  // vcycle_head ran the projected first sweep already
    ;
  else if (proj)
    SPFD_LAUNCH(c, "jacobi_first_l0", f32, 1, 4 * w * S, 2 * S,
                launch_jacobi_first_proj<T>(lv.g, wd, bl, cur, c->sc, inv, st, nk,
                                            block_order(c, TF_JFIRST, l)));
  else
    SPFD_LAUNCH(c, lvl_name(LVL_NAMES("jacobi_first"), l), f32, 1,
                3 * w * S, S,
                launch_jacobi_first<T>(lv.g, wd, bl, cur, st, nk, block_order(c, TF_JFIRST, l)));
  auto sweep = [&](T *in, T *out) {
    if (l == 0)
      SPFD_LAUNCH(c, "jacobi7_l0", f32, 1, (5 * w + 3 * wc) * S, 16 * S,
                  (launch_jacobi7<T, typename Prec<T>::C7>(lv.g, Prec<T>::gx(lv),
                                                           lv.DIAG<T>(), wd, in, bl, out, st,
                                                           nk, block_order(c, TF_SMOOTH, l))));
    else
      SPFD_LAUNCH(c, lvl_name(LVL_NAMES("jacobi27"), l), f32, 1,
                  32 * w * S, 57 * S,
                  launch_jacobi27<T>(lv.g, lv.ST<T>(), wd, in, bl, out, st, nk,
                                     block_order(c, TF_SMOOTH, l)));
  };
  for (int s = 1; s < c->opts.nu_pre; ++s) { sweep(cur, oth); std::swap(cur, oth); }
  if (l == 0)
    SPFD_LAUNCH(c, "residual7_l0", f32, 1, (4 * w + 3 * wc) * S, 14 * S,
                (launch_residual7<T, typename Prec<T>::C7>(lv.g, Prec<T>::gx(lv),
                                                           lv.DIAG<T>(), cur, bl, lv.R<T>(), st,
                                                           nk, block_order(c, TF_RESID, l))));
  else
    SPFD_LAUNCH(c, lvl_name(LVL_NAMES("residual27"), l), f32, 1,
                30 * w * S, 55 * S,
                launch_residual27<T>(lv.g, lv.ST<T>(), cur, bl, lv.R<T>(), st, nk,
                                     block_order(c, TF_RESID, l)));
  Level &cl = c->L[l + 1];
  const double Sc = (double)cl.S * nk;
  SPFD_LAUNCH(c, lvl_name(LVL_NAMES("restrict"), l), f32, 1,
              28 * w * Sc + w * S, 54 * Sc,
              launch_restrict<T>(lv.g, cl.g, cl.PP<T>(), lv.R<T>(), cl.B<T>(), st, nk,
                                 block_order(c, TF_RESTRICT, l)));
  T *ec = vcycle<T>(c, l + 1, cl.B<T>(), false, nk);
  SPFD_LAUNCH(c, lvl_name(LVL_NAMES("prolong"), l), f32, 1,
              (27.0 / 8.0 + 2.0) * w * S + w * Sc, 7 * S,
              launch_prolong<T>(lv.g, cl.g, lv.PC<T>(), ec, cur, st, nk,
                                block_order(c, TF_PROLONG, l)));
  for (int s = 0; s < c->opts.nu_post; ++s) {
    if (rz && l == 0 && s + 1 == c->opts.nu_post)
      SPFD_LAUNCH(c, "jacobi7_l0", f32, 1, (5 * w + 3 * wc) * S, 20 * S,
                  (launch_jacobi7_rz<T, typename Prec<T>::C7>(
                      lv.g, Prec<T>::gx(lv), lv.DIAG<T>(), wd, cur, bl, oth, c->partials,
                      c->pstride, st, nk, block_order(c, TF_SMOOTH, l))));
    else
      sweep(cur, oth);
    std::swap(cur, oth);
  }
  return cur;
}

// ------------------------------------------------------------------ autotuner
// Chooses the block order (unit_rhs) of every batched kernel family on every
// level for nk right-hand sides: each order is timed on the context's own
// operators and level vectors (one warm-up launch, then two timed ones,
// CUDA events on the context's stream) and the faster is kept.  Tuning only
// rewrites scratch vectors that every solve initialises before use, and each
// kernel keeps zero vector entries at slots that are not unknowns, so it
// leaves no trace in later solves.  Order 1 is skipped where units * nk
// does not fit a one-dimensional grid.
template <typename T>
static spfd_status autotune_orders(spfd_ctx *c, int nk, std::vector<signed char> &tab) {
  using C7 = typename Prec<T>::C7;
  const int nl = (int)c->L.size();
  tab.assign((size_t)TF_COUNT * nl, 0);
  cudaStream_t st = c->stream;
  // every right-hand side is live while the kernels are timed (the CG
  // operator skips frozen ones); the solve sets the flags afresh
  TRY(batch_flags(c, 0, nk, 0, 0, -1));
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  struct Give {  // the events go back to the context's pool on every exit
    spfd_ctx *c;
    cudaEvent_t a, b;
    ~Give() {
      if (a) c->evpool.push_back(a);
      if (b) c->evpool.push_back(b);
    }
  } give{c, e0, e1};
  if (!e0 || !e1) return fail(SPFD_ECUDA, "autotuner events");
  auto timed = [&](const auto &launch, int order, float *ms) -> spfd_status {
    launch(order);
    CU(cudaEventRecord(e0, st));
    launch(order);
    launch(order);
    CU(cudaEventRecord(e1, st));
    CU(cudaEventSynchronize(e1));
    CU(cudaEventElapsedTime(ms, e0, e1));
    c->launch_count += 3;
    *ms *= 0.5f;
    return launch_check("autotune");
  };
  // SPFD_TUNE_FORCE=k keeps order k wherever it was timed (a test hook: all
  // orders give the same results, so a test can run each one)
  const char *force_env = getenv("SPFD_TUNE_FORCE");
  const int force = force_env ? atoi(force_env) : -1;
  // tile: whether the family has the right-hand-side tile (order 2)
  auto pick = [&](int fam, int l, int units, bool tile, const auto &launch) -> spfd_status {
    if (units <= 0 || !order1_fits(units, nk)) return SPFD_OK;
    float m[3] = {0.f, 0.f, -1.f};
    TRY(timed(launch, 0, &m[0]));
    TRY(timed(launch, 1, &m[1]));
    if (tile && nk >= RHS_TILE) TRY(timed(launch, 2, &m[2]));
    int best = m[1] < m[0] ? 1 : 0;
    if (m[2] >= 0.f && m[2] < m[best]) best = 2;
    if (force >= 0 && force <= 2 && m[force] >= 0.f) best = force;
    tab[(size_t)fam * nl + l] = (signed char)best;
    c->tune_log.push_back(TuneRecord{fam, l, nk, best, (double)m[0], (double)m[1], (double)m[2]});
    return SPFD_OK;
  };
  for (int l = 0; l + 1 < nl; ++l) {
    Level &lv = c->L[l], &cl = c->L[l + 1];
    const Grid &g = lv.g;
    const T *wd = lv.WDINV<T>();
    T *x = lv.X<T>(), *t = lv.Tt<T>(), *b = lv.B<T>(), *r = lv.R<T>();
    if (l == 0 && c->ncomp == 1)
      TRY(pick(TF_JFIRST, l, g.nb, false, [&](int o) {
        launch_jacobi_first_proj<T>(g, wd, b, x, c->sc, 0.0, st, nk, o);
      }));
    else
      TRY(pick(TF_JFIRST, l, g.nb, false, [&](int o) { launch_jacobi_first<T>(g, wd, b, x, st, nk, o); }));
    if (l == 0) {
      TRY(pick(TF_SMOOTH, l, g.nb, false, [&](int o) {
        launch_jacobi7<T, C7>(g, Prec<T>::gx(lv), lv.DIAG<T>(), wd, x, b, t, st, nk, o);
      }));
      TRY(pick(TF_RESID, l, g.nb, false, [&](int o) {
        launch_residual7<T, C7>(g, Prec<T>::gx(lv), lv.DIAG<T>(), x, b, r, st, nk, o);
      }));
      const T *opgx = sizeof(T) == 4 ? (const T *)lv.gx32 : (const T *)lv.gx;
      const T *opdiag = sizeof(T) == 4 ? (const T *)lv.diag32 : (const T *)lv.diag;
      TRY(pick(TF_APPLY, l, g.nb, false, [&](int o) {
        launch_apply_dot<T>(g, opgx, opdiag, x, r, c->sc, c->partials, st, nk, c->pstride, o);
      }));
    } else {
      TRY(pick(TF_SMOOTH, l, g.nb, true, [&](int o) {
        launch_jacobi27<T>(g, lv.ST<T>(), wd, x, b, t, st, nk, o);
      }));
      TRY(pick(TF_RESID, l, g.nb, true, [&](int o) {
        launch_residual27<T>(g, lv.ST<T>(), x, b, r, st, nk, o);
      }));
    }
    TRY(pick(TF_RESTRICT, l, cl.g.nb, true, [&](int o) {
      launch_restrict<T>(g, cl.g, cl.PP<T>(), r, cl.B<T>(), st, nk, o);
    }));
    TRY(pick(TF_PROLONG, l, (g.nb + 1) / 2, true, [&](int o) {
      launch_prolong<T>(g, cl.g, lv.PC<T>(), cl.X<T>(), x, st, nk, o);
    }));
  }
  return SPFD_OK;
}

// The block-order table for a batch of nk right-hand sides (tuned on first
// use when opts.autotune is set); nullptr keeps order 0.
static spfd_status batch_orders(spfd_ctx *c, int nk, const signed char **out) {
  *out = nullptr;
  if (nk <= 1 || !c->opts.autotune || c->ndof == 0) return SPFD_OK;
  auto it = c->tuned.find(nk);
  if (it == c->tuned.end()) {
    std::vector<signed char> tab;
    const bool mixed = c->opts.precision == SPFD_MIXED;
    TRY(mixed ? autotune_orders<float>(c, nk, tab) : autotune_orders<double>(c, nk, tab));
    it = c->tuned.emplace(nk, std::move(tab)).first;
  }
  *out = it->second.data();
  return SPFD_OK;
}

// ------------------------------------------------------------------ Krylov
// Per-right-hand-side flags and sums of the Scalars array, set on the device.
__global__ void k_batch_flags(Scalars *sc, int nk, int clear_rsum, int frozen, int restart) {
  pdl_entry();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nk) return;
  if (clear_rsum) {
    sc[j].rsum = 0.0;
    sc[j].rmean = 0.0;
    sc[j].rmean_f = 0.f;
  }
  if (frozen >= 0) sc[j].frozen = frozen;
  if (restart >= 0) sc[j].restart = restart;
}
spfd_status batch_flags(spfd_ctx *c, int j0, int nk, int clear_rsum, int frozen,
                        int restart) {
  if (nk <= 0) return SPFD_OK;
  SPFD_LAUNCH(c, "flags", false, 1, 0, 0,
              (pdl(k_batch_flags, (nk + 127) / 128, 128, c->stream)(c->sc + j0, nk, clear_rsum,
                                                                       frozen, restart)));
  return launch_check("batch flags");
}
// The residual about to enter the V-cycle already has zero mean: clear the
// sum and the means the fused projection reads.
static spfd_status zero_rsum(spfd_ctx *c, int j0 = 0, int nk = 1) {
  return batch_flags(c, j0, nk, 1, -1, -1);
}

// True relative residuals ||b - A x|| / ||b|| of the nk right-hand sides
// (level 0's r is the scratch).
static spfd_status true_residual(spfd_ctx *c, const double *bb, double *rel, int nk = 1) {
  Level &l0 = c->L[0];
  const double S = (double)l0.S * nk;
  SPFD_LAUNCH(c, "true_residual", false, 1, 56 * S, 14 * S,
              (launch_residual7<double, double>(l0.g, l0.gx, l0.diag, c->xk, c->bk, l0.r,
                                                c->stream, nk)));
  SPFD_LAUNCH(c, "true_residual", false, 1, 20 * S, 2 * S,
              launch_dot<double>(l0.g.nb, l0.r, l0.r, c->comp, c->sc, c->partials, 2,
                                 c->stream, nk, c->pstride));
  TRY(launch_check("true residual"));
  TRY(read_scalars(c, nk));
  for (int j = 0; j < nk; ++j)
    rel[j] = bb[j] > 0.0 ? std::sqrt(c->hsc[j].aux[2] / bb[j]) : 0.0;
  return SPFD_OK;
}

// z = M r (V-cycle on the projected residual), r.z and beta, then
// p = z + beta p, for the first nk right-hand sides; first = 1 on the first
// iteration (beta = 0).
template <typename T>
spfd_status precondition_step(spfd_ctx *c, T *r, T *p, int first, int nk, bool head) {
  const int nb = c->L[0].g.nb;
  const bool f32 = sizeof(T) == 4;
  const double w = sizeof(T), S = (double)c->L[0].S * nk;
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  const double *csum = c->ncomp > 1 ? c->csum : nullptr;
  cudaStream_t st = c->stream;
  // In FP32, r.z comes with the last level-0 sweep of the V-cycle when it
  // has one: that sweep is HBM-bound, so the products and warp sums are free
  // and a pass over r and z is saved.  The FP64 sweep is FP64-pipe-bound:
  // its warp sums cost more than the separate pass (0.29 against 0.18 ms per
  // sweep on the 2 mm body), so FP64 keeps k_dot_rz.
  const bool fused = f32 && c->L.size() > 1 && c->opts.nu_post >= 1 &&
                     c->opts.smoother == SPFD_SMOOTHER_JACOBI;
  T *z = vcycle<T>(c, 0, r, true, nk, fused, head);
  if (fused)
    SPFD_LAUNCH(c, "finish_rz", false, 1, 16.0 * jacobi7_rz_partials<T>(nb) * nk, 0,
                launch_finish_rz(jacobi7_rz_partials<T>(nb), c->partials,
                                 c->partials + (size_t)16 * nb, c->sc, first, st, nk,
                                 c->pstride, f32));
  else
    SPFD_LAUNCH(c, "dot_rz", f32, 1, (2 * w + 4) * S, 3 * S,
                launch_dot_rz<T>(nb, r, z, c->comp, c->sc, c->partials, first, st, nk,
                                 c->pstride));
  if (c->ncomp > 1)
    SPFD_LAUNCH(c, "project", f32, 3, 2 * (w + 4) * S, 12 * S,
                launch_comp_sum<T>(nb, z, c->comp, c->csum, c->ncomp, c->cstride, st, nk));
  SPFD_LAUNCH(c, "pupdate", f32, 1, (3 * w + 4) * S, 3 * S,
              launch_pupdate<T>(nb, p, z, c->comp, c->sc, csum, c->csize, inv, st, nk,
                                c->cstride));
  return launch_check("V-cycle");
}
template spfd_status precondition_step<double>(spfd_ctx *, double *, double *, int, int, bool);
template spfd_status precondition_step<float>(spfd_ctx *, float *, float *, int, int, bool);
template spfd_status project<double>(spfd_ctx *, double *, int, int);
template double *vcycle<double>(spfd_ctx *, int, double *, bool, int, bool, bool);

struct PcgResult {
  int iters = 0;
  bool conv = false;
  double rel_true = 0.0;
};

// Multigrid-preconditioned CG on level 0 for A x = r0, for nk right-hand
// sides at once (x = 0 on entry; r holds each r0 with zero mean on every
// component, and each right-hand side's Scalars hold rsum = 0).  Every
// right-hand side keeps its own recurrence, scalars and stopping decision;
// one that has stopped is frozen on the device (the x/r update skips it), so
// each reaches the iterate it would reach alone.  Launches cover the
// right-hand sides up to the last one still running.
// The level-0 V-cycle's first kernel, when it depends on nothing but r and
// the scalars update_xr left on the device (weighted Jacobi, one component,
// a coarser level below): the projected first sweep from the zero guess.
// The CG loop launches it right after the scalars' copy to the host, so the
// GPU runs it while the host waits for the copy and takes its decisions,
// instead of idling through that round trip; the V-cycle then starts with
// its residual.  It is the same launch as the V-cycle's own, so results are
// unchanged bit for bit; when the solve stops there, one sweep is spent.
template <typename T>
static bool vcycle_head_ok(const spfd_ctx *c) {
  return c->opts.smoother == SPFD_SMOOTHER_JACOBI && c->ncomp == 1 && c->L.size() > 1;
}
template <typename T>
static spfd_status vcycle_head(spfd_ctx *c, T *r, int nk) {
  Level &lv = c->L[0];
  const bool f32 = sizeof(T) == 4;
  const double w = sizeof(T), S = (double)lv.S * nk;
  const double inv = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  SPFD_LAUNCH(c, "jacobi_first_l0", f32, 1, 4 * w * S, 2 * S,
              launch_jacobi_first_proj<T>(lv.g, lv.WDINV<T>(), r, lv.X<T>(), c->sc, inv,
                                          c->stream, nk, block_order(c, TF_JFIRST, 0)));
  return launch_check("first sweep");
}

// T = double: the operator is the FP64 one and the stopping rule recomputes
// the true residual (restarting from it when the recursion has drifted).
// T = float: the inner solve of the refinement, stopped on the recursive
// residual.  bb[j] = |r0_j|^2; a right-hand side with bb[j] = 0 is solved
// by x = 0 and takes no iteration.
template <typename T>
static spfd_status pcg(spfd_ctx *c, T *x, T *r, T *p, T *q, const T *opgx,
                       const T *opdiag, const double *bb, const double *tolv,
                       const int *maxitv, PcgResult *res, int nk = 1) {
  Level &l0 = c->L[0];
  cudaStream_t st = c->stream;
  const int nb = l0.g.nb;
  const size_t S0 = l0.S;
  const bool f32 = sizeof(T) == 4;
  const double w = sizeof(T);
  std::vector<int> done(nk, 0);
  auto active_end = [&]() {
    int e = 0;
    for (int j = 0; j < nk; ++j)
      if (!done[j]) e = j + 1;
    return e;
  };
  CU(cudaMemsetAsync(p, 0, S0 * nk * sizeof(T), st));
  TRY(batch_flags(c, 0, nk, 0, 0, 0));
  for (int j = 0; j < nk; ++j) {
    res[j] = PcgResult{};
    if (!(bb[j] > 0.0)) {
      res[j].conv = true;
      done[j] = 2;
      TRY(batch_flags(c, j, 1, 0, 1, -1));
    }
  }
  int na = active_end();
  auto precondition = [&](int first, bool head) -> spfd_status {
    return precondition_step<T>(c, r, p, first, na, head);
  };
  const bool ahead = vcycle_head_ok<T>(c);
  if (na == 0) return SPFD_OK;
  TRY(precondition(1, false));
  // FP64 stopping: the recursive residual triggers a recomputation of the
  // true one; if that is still above tol, CG restarts from it (beta = 0).
  // Three restarts that fail to halve the best true residual mean the
  // rounding floor is reached: stop there (not converged).
  std::vector<double> best_true(nk, INFINITY), min_rrel(nk, INFINITY), rel(nk, 0.0);
  std::vector<int> stall(nk, 0), check, broke;
  int maxit_all = 0;
  for (int j = 0; j < nk; ++j) maxit_all = std::max(maxit_all, maxitv[j]);
  for (int it = 1; it <= maxit_all && na > 0; ++it) {
    // a right-hand side past its own iteration cap stops here
    bool capped = false;
    for (int j = 0; j < na; ++j)
      if (!done[j] && it > maxitv[j]) {
        TRY(batch_flags(c, j, 1, 0, 1, -1));
        done[j] = 2;
        capped = true;
      }
    if (capped) {
      na = active_end();
      if (na == 0) break;
    }
    const double S = (double)S0 * na;
    SPFD_LAUNCH(c, "apply_dot", f32, 1, (f32 ? 5 : 6) * w * S, (f32 ? 20 : 15) * S,
                launch_apply_dot<T>(l0.g, opgx, opdiag, p, q, c->sc, c->partials, st, na,
                                    c->pstride, block_order(c, TF_APPLY, 0)));
    SPFD_LAUNCH(c, "finish_pq", false, 1, 8.0 * nb * na, nb * na,
                launch_finish_pq(apply_dot_partials<T>(nb), c->partials,
                                 c->partials + (size_t)16 * nb, c->sc, st, na, c->pstride,
                                 f32));
    SPFD_LAUNCH(c, "update_xr", f32, 1, 6 * w * S, 7 * S,
                launch_update_xr<T>(nb, x, r, p, q, c->sc, c->partials, st, na, c->pstride));
    TRY(launch_check("CG update"));
    CU(cudaMemcpyAsync(c->hsc, c->sc, (size_t)na * sizeof(Scalars), cudaMemcpyDeviceToHost,
                       st));
    CU(cudaEventRecord(c->evsc, st));
    if (ahead) TRY(vcycle_head<T>(c, r, na));
    bool head = ahead;  // false once the host replaces an r (restart)
    {
      cudaError_t e = cudaEventSynchronize(c->evsc);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess)
        return fail(SPFD_ECUDA, "reading solver scalars: %s", cudaGetErrorString(e));
    }
    check.clear();
    broke.clear();
    for (int j = 0; j < na; ++j) {
      if (done[j]) continue;
      res[j].iters = it;
      const double tol = tolv[j];
      const double rrel = std::sqrt(c->hsc[j].rr / bb[j]);
      if (!std::isfinite(rrel) || rrel > 1e8 * std::max(min_rrel[j], tol)) {
        broke.push_back(j);  // breakdown: report the current iterate, not converged
        continue;
      }
      min_rrel[j] = std::min(min_rrel[j], rrel);
      if (rrel <= tol) {
        if (f32) { res[j].conv = true; done[j] = 1; }
        else check.push_back(j);
      }
    }
    if (!f32 && (!check.empty() || !broke.empty()))
      TRY(true_residual(c, bb, rel.data(), na));
    for (int j : broke) {
      if (!f32) res[j].rel_true = rel[j];
      done[j] = 1;
    }
    for (int j : check) {
      res[j].rel_true = rel[j];
      if (rel[j] <= tolv[j]) { res[j].conv = true; done[j] = 1; continue; }
      if (rel[j] < 0.5 * best_true[j]) { best_true[j] = rel[j]; stall[j] = 0; }
      else if (++stall[j] >= 3) { done[j] = 1; continue; }
      // restart from the true residual (left in level 0's r by true_residual)
      CU(cudaMemcpyAsync(r + (size_t)j * S0, l0.r + (size_t)j * S0, S0 * sizeof(T),
                         cudaMemcpyDeviceToDevice, st));
      TRY(project<T>(c, r + (size_t)j * S0, 1, j));
      TRY(batch_flags(c, j, 1, 1, -1, 1));
      if (head) {
        // the V-cycle runs the first sweep again: the other right-hand
        // sides' r were projected by the look-ahead sweep, so their means
        // are cleared and the sweep gives them the same values again
        TRY(batch_flags(c, 0, na, 1, -1, -1));
        head = false;
      }
    }
    for (int j = 0; j < na; ++j)
      if (done[j] == 1) {
        TRY(batch_flags(c, j, 1, 0, 1, -1));
        done[j] = 2;
      }
    na = active_end();
    if (na > 0) TRY(precondition(0, head));
  }
  return SPFD_OK;
}

// Right-hand sides of the nk solves: b = -G^T M a (or G^T gJ for the
// adjoint), projected; |b|^2 of each into bb.
static spfd_status prepare_rhs(spfd_ctx *c, const double *a_dev, double *bb, int nk = 1) {
  Level &l0 = c->L[0];
  const double S = (double)l0.S * nk;
  if (c->gJ_cur)
    SPFD_LAUNCH(c, "rhs", false, 1, 56 * S, 6 * S,
                launch_div_brick(l0.g, l0.diag, c->gJ_cur, c->bk, c->stream));
  else
    SPFD_LAUNCH(c, "rhs", false, 1, 56 * S, 12 * S,
                launch_rhs(l0.g, l0.gx, a_dev, c->bk, &c->sc->status, c->stream, nk));
  TRY(launch_check("rhs"));
  TRY(project<double>(c, c->bk, nk));
  SPFD_LAUNCH(c, "project", false, 1, 20 * S, 2 * S,
              launch_dot<double>(l0.g.nb, c->bk, c->bk, c->comp, c->sc, c->partials, 1,
                                 c->stream, nk, c->pstride));
  TRY(read_scalars(c, nk));
  if (c->hsc[0].status & DEV_BAD_A)  // one flag for the whole batch
    return fail(SPFD_EINVAL, "a holds a non-finite value on a conducting edge");
  for (int j = 0; j < nk; ++j) bb[j] = c->hsc[j].aux[1];
  return SPFD_OK;
}

static spfd_status solve_fp64(spfd_ctx *c, double tol, spfd_info *out, int nk = 1) {
  Level &l0 = c->L[0];
  const size_t S0 = l0.S;
  std::vector<double> bb(nk, 0.0), rel(nk, 0.0);
  std::vector<PcgResult> res(nk);
  TRY(prepare_rhs(c, c->a_cur, bb.data(), nk));
  CU(cudaMemsetAsync(c->xk, 0, S0 * nk * sizeof(double), c->stream));
  CU(cudaMemcpyAsync(c->rk, c->bk, S0 * nk * sizeof(double), cudaMemcpyDeviceToDevice,
                     c->stream));
  TRY(zero_rsum(c, 0, nk));  // b is projected
  std::vector<double> tolv(nk, tol);
  std::vector<int> maxitv(nk, c->opts.maxit);
  TRY(pcg<double>(c, c->xk, c->rk, c->pk, c->qk, l0.gx, l0.diag, bb.data(), tolv.data(),
                  maxitv.data(), res.data(), nk));
  TRY(project<double>(c, c->xk, nk));
  bool redo = false;
  for (int j = 0; j < nk; ++j) redo |= !res[j].conv;
  if (redo) {
    TRY(true_residual(c, bb.data(), rel.data(), nk));
    for (int j = 0; j < nk; ++j)
      if (!res[j].conv) res[j].rel_true = rel[j];
  }
  for (int j = 0; j < nk; ++j) {
    out[j].iters = res[j].iters;
    out[j].outer_iters = 0;
    out[j].converged = res[j].conv ? 1 : 0;
    out[j].rel_res_true = res[j].rel_true;
  }
  return SPFD_OK;
}

// FP64 iterative refinement around the FP32 multigrid-preconditioned CG,
// for nk right-hand sides at once.  Each right-hand side keeps its own outer
// state (scale, inner target, stall count, iteration budget) and leaves the
// loop on its own; the inner CG covers every one still refining in shared
// launches, each with its own recurrence, so each result is the one the
// right-hand side reaches alone.
static spfd_status solve_mixed(spfd_ctx *c, double tol, spfd_info *out, int nk = 1) {
  Level &l0 = c->L[0];
  cudaStream_t st = c->stream;
  const size_t S0 = l0.S;
  const double S = (double)S0;
  const int nb = l0.g.nb;
  const int max_outer = 30;
  std::vector<double> bb(nk, 0.0), nrm2(nk), rel(nk, 1.0), prev(nk, INFINITY), nr(nk);
  std::vector<double> rel_all(nk, 0.0), bb_in(nk), eta(nk);
  std::vector<int> total(nk, 0), stall(nk, 0), outer_of(nk, 0), active(nk, 0), cap(nk);
  std::vector<PcgResult> in(nk);
  TRY(prepare_rhs(c, c->a_cur, bb.data(), nk));
  CU(cudaMemsetAsync(c->xk, 0, S0 * nk * sizeof(double), st));
  for (int j = 0; j < nk; ++j) {
    out[j].iters = 0;
    out[j].outer_iters = 0;
    out[j].converged = 0;
    out[j].rel_res_true = 0.0;
    if (!(bb[j] > 0.0)) out[j].converged = 1;
    else active[j] = 1;
    nrm2[j] = bb[j];
  }
  CU(cudaMemcpyAsync(c->rk, c->bk, S0 * nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  for (int outer = 1;; ++outer) {
    // right-hand sides out of outer steps or inner iterations stop here
    int na = 0;
    for (int j = 0; j < nk; ++j) {
      if (!active[j]) continue;
      if (outer > max_outer || total[j] >= c->opts.maxit) {
        active[j] = 0;
        outer_of[j] = std::min(outer, max_outer);
        continue;
      }
      na = j + 1;
    }
    if (na == 0) break;
    CU(cudaMemsetAsync(c->dk32, 0, S0 * na * sizeof(float), st));
    for (int j = 0; j < na; ++j) {
      if (!active[j]) continue;
      nr[j] = std::sqrt(nrm2[j]);
      // inner target: what is still missing for tol, but no tighter than
      // what an FP32 solve reliably reaches
      eta[j] = std::min(0.5, std::max(0.5 * tol * std::sqrt(bb[j]) / nr[j], 1e-4));
      SPFD_LAUNCH(c, "convert", true, 1, 12 * S, S,
                  launch_scale_to_f32(nb, c->rk + (size_t)j * S0, 1.0 / nr[j],
                                      c->rk32 + (size_t)j * S0, c->sc + j,
                                      c->partials + (size_t)j * c->pstride, st));
    }
    SPFD_LAUNCH(c, "project", true, 1, 12 * S * na, 2 * S * na,
                launch_dot<float>(nb, c->rk32, c->rk32, c->comp, c->sc, c->partials, 3, st,
                                  na, c->pstride));
    TRY(read_scalars(c, na));
    for (int j = 0; j < na; ++j) {
      bb_in[j] = active[j] ? c->hsc[j].aux[3] : 0.0;  // 0: the inner CG skips it
      cap[j] = c->opts.maxit - total[j];
    }
    TRY(pcg<float>(c, c->dk32, c->rk32, c->pk32, c->qk32, l0.gx32, l0.diag32, bb_in.data(),
                   eta.data(), cap.data(), in.data(), na));
    for (int j = 0; j < na; ++j) {
      if (!active[j]) continue;
      total[j] += in[j].iters;
      SPFD_LAUNCH(c, "convert", false, 1, 20 * S, 2 * S,
                  launch_axpy_mixed(nb, c->xk + (size_t)j * S0, c->dk32 + (size_t)j * S0,
                                    nr[j], st));
    }
    TRY(true_residual(c, bb.data(), rel_all.data(), na));
    bool more = false;
    for (int j = 0; j < na; ++j) {
      if (!active[j]) continue;
      rel[j] = rel_all[j];
      bool stop = false;
      if (rel[j] <= tol) {
        out[j].converged = 1;
        stop = true;
      } else if (rel[j] > 0.5 * prev[j]) {
        if (++stall[j] >= 2) stop = true;
      } else {
        stall[j] = 0;
      }
      if (stop) {
        active[j] = 0;
        outer_of[j] = outer;
        continue;
      }
      prev[j] = std::min(prev[j], rel[j]);
      // the next correction solves for the true residual (in level 0's r)
      CU(cudaMemcpyAsync(c->rk + (size_t)j * S0, l0.r + (size_t)j * S0, S0 * sizeof(double),
                         cudaMemcpyDeviceToDevice, st));
      TRY(project<double>(c, c->rk + (size_t)j * S0, 1, j));
      SPFD_LAUNCH(c, "project", false, 1, 20 * S, 2 * S,
                  launch_dot<double>(nb, c->rk + (size_t)j * S0, c->rk + (size_t)j * S0,
                                     c->comp, c->sc + j, c->partials + (size_t)j * c->pstride,
                                     3, st));
      more = true;
    }
    if (more) {
      TRY(read_scalars(c, na));
      for (int j = 0; j < na; ++j)
        if (active[j]) nrm2[j] = c->hsc[j].aux[3];
    }
  }
  TRY(project<double>(c, c->xk, nk));
  for (int j = 0; j < nk; ++j) {
    if (!(bb[j] > 0.0)) continue;
    out[j].iters = total[j];
    out[j].outer_iters = outer_of[j];
    out[j].rel_res_true = rel[j];
  }
  return SPFD_OK;
}

// Grows the per-right-hand-side buffers to hold k right-hand sides: every
// level's x, b, r, t, the FP64 Krylov vectors, the scalars (each with
// inv_ndof), the reduction scratch and the component sums.  New vectors are
// zeroed (slots that are not unknowns must read 0).  Synchronises the stream.
static spfd_status ensure_batch(spfd_ctx *c, int k) {
  if (k <= c->kcap) return SPFD_OK;
  cudaStream_t st = c->stream;
  TRY(sync_check(c, "batch buffers"));
  auto grow = [&](double *&v, size_t n) -> spfd_status {
    dfree(c, v);
    TRY(dalloc(c, &v, n));
    CU(cudaMemsetAsync(v, 0, n * sizeof(double), st));
    return SPFD_OK;
  };
  auto grow32 = [&](float *&v, size_t n) -> spfd_status {
    dfree(c, v);
    TRY(dalloc(c, &v, n));
    CU(cudaMemsetAsync(v, 0, n * sizeof(float), st));
    return SPFD_OK;
  };
  const bool mixed = c->opts.precision == SPFD_MIXED;
  for (size_t l = 0; l < c->L.size(); ++l) {
    Level &lv = c->L[l];
    // the mixed solve runs its V-cycle in FP32; of the FP64 level vectors
    // it uses level 0's r only (true residuals)
    if (!mixed || l == 0)
      for (double **v : {&lv.x, &lv.b, &lv.r, &lv.t}) TRY(grow(*v, lv.S * k));
    if (mixed)
      for (float **v : {&lv.x32, &lv.b32, &lv.r32, &lv.t32}) TRY(grow32(*v, lv.S * k));
  }
  const size_t S0 = c->L[0].S;
  for (double **v : {&c->xk, &c->rk, &c->pk, &c->qk, &c->bk}) TRY(grow(*v, S0 * k));
  if (mixed)
    for (float **v : {&c->dk32, &c->rk32, &c->pk32, &c->qk32}) TRY(grow32(*v, S0 * k));
  TRY(grow(c->partials, c->pstride * k));
  if (c->ncomp > 1) TRY(grow(c->csum, (size_t)c->cstride * k));
  Scalars *sc = nullptr, *hsc = nullptr;
  TRY(dalloc(c, &sc, k));
  TRY(halloc(c, &hsc, k));
  memset(hsc, 0, (size_t)k * sizeof(Scalars));
  const double inv_ndof = c->ndof ? 1.0 / (double)c->ndof : 0.0;
  for (int j = 0; j < k; ++j) hsc[j].inv_ndof = inv_ndof;
  CU(cudaMemcpyAsync(sc, hsc, (size_t)k * sizeof(Scalars), cudaMemcpyHostToDevice, st));
  TRY(sync_check(c, "batch scalars"));
  dfree(c, c->sc);
  c->sc = sc;
  ++c->gen;  // solve buffers moved: captured graphs must be captured again
  c->hsc = hsc;
  c->kcap = k;
  return SPFD_OK;
}

// Solves the nk systems whose edge potentials are a_dev + j * 3 NN (NN
// nodes) into psi_dev + j * NN, in batched launches (FP64 CG, or the mixed
// refinement with a batched FP32 inner CG).
static spfd_status solve_device(spfd_ctx *c, const double *a_dev, double tol,
                                double *psi_dev, spfd_info *info, int nk = 1) {
  if (!(tol > 0.0)) tol = c->opts.tol;
  cudaStream_t st = c->stream;
  Level &l0 = c->L[0];
  const size_t NNs = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  std::vector<spfd_info> res(nk, c->info);
  const int64_t launches0 = c->launch_count;
  if (nk > 1 && c->ndof > 0) TRY(ensure_batch(c, nk));
  const signed char *orders = nullptr;
  TRY(batch_orders(c, nk, &orders));
  CU(cudaEventRecord(c->ev0, st));
  CU(cudaMemsetAsync(&c->sc->status, 0, sizeof(int), st));
  if (c->ndof == 0) {
    CU(cudaMemsetAsync(psi_dev, 0, NNs * nk * sizeof(double), st));
    for (auto &r : res) {
      r.iters = 0;
      r.outer_iters = 0;
      r.converged = 1;
      r.rel_res_true = 0.0;
    }
  } else {
    c->a_cur = a_dev;
    c->ord = orders;
    spfd_status s = c->opts.precision == SPFD_MIXED ? solve_mixed(c, tol, res.data(), nk)
                                                     : solve_fp64(c, tol, res.data(), nk);
    c->ord = nullptr;
    c->a_cur = nullptr;
    TRY(s);
    const double NN = (double)NNs * nk;
    SPFD_LAUNCH(c, "scatter", false, 1, 8 * NN + 12.0 * l0.S * nk, 0,
                launch_scatter<double>(l0.g, c->xk, c->comp, psi_dev, st, nk));
    TRY(launch_check("scatter"));
  }
  CU(cudaEventRecord(c->ev1, st));
  TRY(sync_check(c, "solve"));
  TRY(prof_flush(c));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  int bad = -1;
  for (int j = 0; j < nk; ++j) {
    res[j].ms_solve = ms;
    res[j].bytes_device = c->bytes;
    res[j].launches = c->launch_count - launches0;
    if (info) info[j] = res[j];
    if (!res[j].converged && bad < 0) bad = j;
  }
  c->info = res[nk - 1];
  if (c->opts.verbose)
    for (int j = 0; j < nk; ++j)
      fprintf(stderr, "[spfd] solve %d/%d: %d it (%d outer), rel %.3e, %.3f ms\n", j + 1, nk,
              res[j].iters, res[j].outer_iters, res[j].rel_res_true, ms);
  if (bad >= 0)
    return fail(SPFD_ENOTCONVERGED,
                "not converged: right-hand side %d at rel residual %.3e after %d iterations",
                bad, res[bad].rel_res_true, res[bad].iters);
  return SPFD_OK;
}

// Gradient of J = mean over conducting voxels of |E|^2 (Eq. 1, voxel
// averaged) with respect to a and the voxel conductivities, by one adjoint
// solve A lambda = G^T gJ with the context's operator and preconditioner.
extern "C" spfd_status spfd_energy_grad(spfd_ctx *ctx, const double *a_dev,
                                        const double *psi_dev, double omega, double tol,
                                        double *J_out, double *dJda_dev,
                                        double *dJdsigma_dev, spfd_info *info) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!a_dev || !psi_dev || !J_out || !dJda_dev || !dJdsigma_dev)
    return fail(SPFD_EINVAL, "a NULL argument");
  if (std::isnan(tol) || !std::isfinite(omega)) return fail(SPFD_EINVAL, "tol or omega invalid");
  spfd_ctx *c = ctx;
  cudaStream_t st = c->stream;
  Level &l0 = c->L[0];
  const size_t nv = (size_t)c->nx * c->ny * c->nz;
  const size_t NN = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  if (!c->ev_stage) TRY(dalloc(c, &c->ev_stage, 3 * nv));
  if (!c->gj_stage) TRY(dalloc(c, &c->gj_stage, 3 * NN));
  if (!c->lam_stage) TRY(dalloc(c, &c->lam_stage, NN));
  const double cf = omega / (4.0 * c->h);
  SPFD_LAUNCH(c, "energy", false, 1, 0, 0,
              launch_energy(c->mask, a_dev, psi_dev, c->nx, c->ny, c->nz, cf, c->ev_stage,
                            c->sc, c->partials, st));
  SPFD_LAUNCH(c, "energy", false, 1, 0, 0,
              launch_energy_gJ(c->mask, c->ev_stage, c->nx, c->ny, c->nz, cf, c->sc,
                               c->gj_stage, st));
  TRY(launch_check("energy"));
  CU(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  TRY(sync_check(c, "energy"));
  const double Jsum = c->hsc->aux[6], nc = c->hsc->aux[7];
  *J_out = nc > 0.0 ? Jsum / nc : 0.0;
  spfd_info res = c->info;
  spfd_status s = SPFD_OK;
  if (c->ndof == 0 || !(nc > 0.0)) {
    CU(cudaMemsetAsync(c->lam_stage, 0, NN * sizeof(double), st));
  } else {
    // the adjoint solve: same path as spfd_solve, right-hand side G^T gJ
    c->gJ_cur = c->gj_stage;
    s = solve_device(c, a_dev, tol, c->lam_stage, &res);
    c->gJ_cur = nullptr;
    if (s != SPFD_OK && s != SPFD_ENOTCONVERGED) return s;
  }
  SPFD_LAUNCH(c, "energy", false, 2, 0, 0,
              launch_energy_grads(l0.g, l0.gx, c->mask, a_dev, psi_dev, c->lam_stage,
                                  c->gj_stage, c->nx, c->ny, c->nz, c->h, dJda_dev,
                                  dJdsigma_dev, st));
  TRY(launch_check("energy gradients"));
  TRY(sync_check(c, "energy gradients"));
  if (info) *info = res;
  return s;
}

extern "C" spfd_status spfd_solve(spfd_ctx *ctx, const double *a_dev,
                                  double tol, double *psi_dev,
                                  spfd_info *info) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!a_dev || !psi_dev) return fail(SPFD_EINVAL, "a_dev / psi_dev is NULL");
  if (std::isnan(tol)) return fail(SPFD_EINVAL, "tol is NaN");
  return solve_device(ctx, a_dev, tol, psi_dev, info);
}

extern "C" spfd_status spfd_solve_batch(spfd_ctx *ctx, int nrhs, const double *a_dev,
                                        double tol, double *psi_dev, spfd_info *infos) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (nrhs < 1 || nrhs > 65535) return fail(SPFD_EINVAL, "nrhs must be in 1..65535");
  if (!a_dev || !psi_dev) return fail(SPFD_EINVAL, "a_dev / psi_dev is NULL");
  if (std::isnan(tol)) return fail(SPFD_EINVAL, "tol is NaN");
  return solve_device(ctx, a_dev, tol, psi_dev, infos, nrhs);
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
  const double nv = (double)ctx->nx * ctx->ny * ctx->nz;
  SPFD_LAUNCH(ctx, "efield", false, 1, 41 * nv, 40 * nv,
              launch_efield(ctx->mask, a_dev, psi_dev, ctx->nx, ctx->ny, ctx->nz,
                            ctx->h, omega, E_dev, ctx->stream));
  return launch_check("efield");
}

extern "C" spfd_status spfd_efield_complex(spfd_ctx *ctx, const double *a_re,
                                           const double *psi_re, const double *a_im,
                                           const double *psi_im, double omega,
                                           double *E_dev) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!a_re || !psi_re || !a_im || !psi_im || !E_dev) return fail(SPFD_EINVAL, "null array");
  if (!std::isfinite(omega)) return fail(SPFD_EINVAL, "omega must be finite");
  if (reinterpret_cast<uintptr_t>(E_dev) % 16)
    return fail(SPFD_EINVAL, "E_dev must be 16-byte aligned");
  const size_t nvox = (size_t)ctx->nx * ctx->ny * ctx->nz;
  const double nv = (double)nvox;
  double *E_im = nullptr;
  TRY(dalloc(ctx, &E_im, nvox));
  SPFD_LAUNCH(ctx, "efield", false, 1, 41 * nv, 40 * nv,
              launch_efield(ctx->mask, a_re, psi_re, ctx->nx, ctx->ny, ctx->nz, ctx->h, omega,
                            E_dev, ctx->stream));
  SPFD_LAUNCH(ctx, "efield", false, 1, 41 * nv, 40 * nv,
              launch_efield(ctx->mask, a_im, psi_im, ctx->nx, ctx->ny, ctx->nz, ctx->h, omega,
                            E_im, ctx->stream));
  SPFD_LAUNCH(ctx, "efield", false, 1, 24 * nv, 4 * nv,
              launch_efield_magnitude(nvox, E_dev, E_im, ctx->stream));
  // the block goes back to the context's spare list; later work that takes it
  // runs on the same stream, after the kernel above
  dfree(ctx, E_im);
  return launch_check("efield (complex)");
}

extern "C" spfd_status spfd_autotune_report(const spfd_ctx *ctx, spfd_tune_entry *entries,
                                            int max, int *n) {
  if (!ctx || !n || (max > 0 && !entries)) return fail(SPFD_EINVAL, "null argument");
  static const char *const names[TF_COUNT] = {"jacobi_first", "smooth", "residual",
                                              "restrict", "prolong", "apply_dot"};
  *n = (int)ctx->tune_log.size();
  for (int i = 0; i < max && i < *n; ++i) {
    const TuneRecord &r = ctx->tune_log[i];
    entries[i].family = names[r.fam];
    entries[i].level = r.level;
    entries[i].nrhs = r.nk;
    entries[i].order = r.order;
    entries[i].ms_order0 = r.ms0;
    entries[i].ms_order1 = r.ms1;
    entries[i].ms_order2 = r.ms2;
  }
  return SPFD_OK;
}

extern "C" spfd_status spfd_get_info(const spfd_ctx *ctx, spfd_info *info) {
  if (!ctx || !info) return fail(SPFD_EINVAL, "null argument");
  *info = ctx->info;
  info->bytes_device = ctx->bytes;
  return SPFD_OK;
}

extern "C" spfd_status spfd_kernel_stats(spfd_ctx *ctx, spfd_kernel_stat *stats,
                                         int max, int *n, int reset) {
  if (!ctx || !n || (max > 0 && !stats)) return fail(SPFD_EINVAL, "null argument");
  TRY(prof_flush(ctx));
  *n = (int)ctx->stats.size();
  for (int i = 0; i < max && i < *n; ++i) {
    const KernelStat &k = ctx->stats[i];
    stats[i].name = k.name.c_str();
    stats[i].launches = k.launches;
    stats[i].ms = k.ms;
    stats[i].bytes = k.bytes;
    stats[i].flops = k.flops;
  }
  if (reset)
    for (auto &k : ctx->stats) { k.launches = 0; k.ms = k.bytes = k.flops = 0.0; }
  return SPFD_OK;
}
