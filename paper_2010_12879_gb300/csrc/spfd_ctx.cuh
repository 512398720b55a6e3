// Host-side context of libspfd: levels, device buffers, profiling records.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <chrono>
#include <map>
#include <cstdlib>
#include <string>
#include <vector>

#include "spfd.h"
#include "spfd_internal.cuh"
#include "spfd_mem.cuh"

namespace spfd {

spfd_status fail(spfd_status s, const char *fmt, ...);
void set_error(const std::string &msg);
std::string last_error_copy();

#define CU(call)                                                            \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return ::spfd::fail(SPFD_ECUDA, "%s failed: %s (%s:%d)", #call,       \
                          cudaGetErrorString(e_), __FILE__, __LINE__);      \
  } while (0)

#define TRY(expr)                    \
  do {                               \
    spfd_status s_ = (expr);         \
    if (s_ != SPFD_OK) return s_;    \
  } while (0)

struct Level {
  Grid g{};                       // device view
  std::vector<int> hbmap;         // host brick map
  std::vector<int4> hbco;         // host brick coordinates
  size_t S = 0;                   // slots = nb * 512
  int64_t n_active = 0;
  double omega = 0.0, lmax = 0.0;
  // FP64 operator and transfer
  double *gx = nullptr;           // level 0: [3][S] +edge conductances
  double *st = nullptr;           // level >= 1: [27][S] Galerkin stencil
  double *P = nullptr;            // level >= 1: [27][S] interpolation from here to level-1
  double *Pc = nullptr;           // levels with a coarser level: [27][S/8] the same
                                  //   weights per fine cell (prolongation layout)
  double *diag = nullptr, *dinv = nullptr, *wdinv = nullptr;
  double *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
  // FP32 copies for the mixed-precision V-cycle
  float *gx32 = nullptr;          // level 0: [3][S] (inner CG operator)
  __nv_bfloat16 *gxbf = nullptr;  // level 0: [3][S] (V-cycle smoother)
  float *st32 = nullptr, *P32 = nullptr, *Pc32 = nullptr, *diag32 = nullptr,
        *wdinv32 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr, *t32 = nullptr;

  // accessors by precision
  template <typename T> T *X();
  template <typename T> T *B();
  template <typename T> T *R();
  template <typename T> T *Tt();
  template <typename T> const T *ST() const;
  template <typename T> const T *PP() const;
  template <typename T> const T *PC() const;
  template <typename T> const T *DIAG() const;
  template <typename T> const T *WDINV() const;
};
template <> inline double *Level::X<double>() { return x; }
template <> inline float *Level::X<float>() { return x32; }
template <> inline double *Level::B<double>() { return b; }
template <> inline float *Level::B<float>() { return b32; }
template <> inline double *Level::R<double>() { return r; }
template <> inline float *Level::R<float>() { return r32; }
template <> inline double *Level::Tt<double>() { return t; }
template <> inline float *Level::Tt<float>() { return t32; }
template <> inline const double *Level::ST<double>() const { return st; }
template <> inline const float *Level::ST<float>() const { return st32; }
template <> inline const double *Level::PP<double>() const { return P; }
template <> inline const float *Level::PP<float>() const { return P32; }
template <> inline const double *Level::PC<double>() const { return Pc; }
template <> inline const float *Level::PC<float>() const { return Pc32; }
template <> inline const double *Level::DIAG<double>() const { return diag; }
template <> inline const float *Level::DIAG<float>() const { return diag32; }
template <> inline const double *Level::WDINV<double>() const { return wdinv; }
template <> inline const float *Level::WDINV<float>() const { return wdinv32; }

// Kernel families whose block order the autotuner chooses per level
// (restriction and prolongation are indexed by their fine level).
enum TuneFam : int {
  TF_JFIRST = 0,   // first smoothing sweep from a zero guess
  TF_SMOOTH,       // weighted-Jacobi sweep (7-point on level 0, 27-point above)
  TF_RESID,        // residual
  TF_RESTRICT,     // restriction to the next coarser level
  TF_PROLONG,      // prolongation and correction from the next coarser level
  TF_APPLY,        // the CG operator with its dot product (level 0)
  TF_COUNT
};
struct TuneRecord {
  int fam, level, nk, order;
  double ms0, ms1, ms2;  // mean time per launch in orders 0, 1, 2 (-1: not timed)
};

struct KernelStat {
  std::string name;
  int64_t launches = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
};
struct ProfRec {
  int stat;
  cudaEvent_t a, b;
  double bytes, flops;
};

}  // namespace spfd

struct spfd_ctx {
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0;
  double h = 0.0;
  spfd_opts opts{};
  std::vector<spfd::Level> L;
  std::vector<void *> allocs;
  std::vector<size_t> alloc_bytes;  // block size of each entry of allocs
  // blocks released while the context lives: reused by its later requests
  // (ordered on its own stream), returned to the process cache at destroy
  std::vector<std::pair<void *, size_t>> spare;
  // pinned host blocks (staging, scalar mirror): returned to the process
  // cache at destroy, once no queued copy reads them
  std::vector<std::pair<void *, size_t>> hblocks;
  int64_t bytes = 0;
  int alloc_count = 0;
  double alloc_ms = 0.0;  // host time spent in cudaMalloc (verbose reports)
  // fine-level bookkeeping
  unsigned char *mask = nullptr;  // [nz][ny][nx] conducting voxel flags
  int *comp = nullptr;            // [S0] component id or -1
  int ncomp = 0;
  int64_t ndof = 0;
  int *csize = nullptr;           // [ncomp]
  // per-component sum workspace [kcap][cstride], cstride = 3 ncomp + 1
  // (only when ncomp > 1)
  double *csum = nullptr;
  int cstride = 0;
  // Krylov vectors (FP64) and the FP32 inner-solve vectors (mixed)
  double *xk = nullptr, *rk = nullptr, *pk = nullptr, *qk = nullptr, *bk = nullptr;
  float *dk32 = nullptr, *rk32 = nullptr, *pk32 = nullptr, *qk32 = nullptr;
  spfd::Scalars *sc = nullptr;    // device scalars, one per right-hand side
  spfd::Scalars *hsc = nullptr;   // pinned host mirror
  double *partials = nullptr;     // reduction scratch, pstride per right-hand side
  size_t pstride = 0;
  // right-hand sides the per-RHS buffers hold (level vectors, Krylov
  // vectors, scalars, partials, component sums); grown by batched solves
  int kcap = 1;
  // generation of the solve buffers: bumped whenever they are reallocated,
  // so that graphs captured over them know to capture again
  uint64_t gen = 0;
  // coarsest level
  int m = 0;
  int *cidx = nullptr;
  double *Binv = nullptr;
  // host-array staging; the edge potentials of the solve in progress
  double *a_stage = nullptr, *psi_stage = nullptr;
  const double *a_cur = nullptr;
  // adjoint solve: when set, the right-hand side is G^T gJ_cur instead of
  // -G^T M a_cur; scratch of spfd_energy_grad (allocated on first use)
  const double *gJ_cur = nullptr;
  double *ev_stage = nullptr, *gj_stage = nullptr, *lam_stage = nullptr;
  // scratch of spfd_percentile (allocated on first use, grown on demand):
  // per-group counters, digit histograms, the key segments, the chunk table
  // and its pinned host staging
  unsigned long long *pct_small = nullptr, *pct_keys = nullptr, *pct_cand = nullptr,
                     *pct_boff = nullptr;
  unsigned *pct_hist = nullptr, *pct_bcnt = nullptr;
  int *pct_candg = nullptr;
  long long *pct_chunks = nullptr, *pct_hstage = nullptr;
  long long pct_bcap = 0;
  int pct_gcap = 0, pct_chcap = 0;
  long long pct_keycap = 0, pct_nc = 0;  // pct_nc: conducting voxels seen last call
  size_t pct_hstage_n = 0;
  // block orders chosen by the autotuner for batched launches: per batch
  // size, TF_COUNT x (levels) entries of 0 or 1; ord points at the table of
  // the batched solve in progress (nullptr: order 0 everywhere)
  std::map<int, std::vector<signed char>> tuned;
  const signed char *ord = nullptr;
  std::vector<spfd::TuneRecord> tune_log;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t evsc = nullptr;  // the CG scalars' copy to the host
  spfd_info info{};
  // launch accounting and profiling
  int64_t launch_count = 0;
  std::vector<spfd::KernelStat> stats;
  std::vector<spfd::ProfRec> pending;
  std::vector<cudaEvent_t> evpool;
};

namespace spfd {

// Allocation with optional injected failure: SPFD_FAIL_ALLOC_AT=N makes the
// N-th device allocation of a context fail (counted from 1), so tests can
// check that every failure path releases what was already allocated.  With
// SPFD_POISON_ALLOC set, every block handed out is first filled with 0xff
// bytes (NaN in FP64 and FP32, -1 in integers) on the context's stream, so a
// test can show that no result depends on memory read before it is written.
template <typename T>
spfd_status dalloc(spfd_ctx *c, T **p, size_t count) {
  *p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  ++c->alloc_count;
  const char *inj = getenv("SPFD_FAIL_ALLOC_AT");
  if (inj && atoi(inj) == c->alloc_count)
    return fail(SPFD_ENOMEM, "injected allocation failure #%d", c->alloc_count);
  void *q = nullptr;
  size_t block = 0;
  // the context's own released blocks first (best fit, at most 25 % larger)
  int best = -1;
  for (size_t k = 0; k < c->spare.size(); ++k) {
    const size_t b = c->spare[k].second;
    if (b >= bytes && b <= bytes + bytes / 4 + 4096 &&
        (best < 0 || b < c->spare[best].second))
      best = (int)k;
  }
  if (best >= 0) {
    q = c->spare[best].first;
    block = c->spare[best].second;
    c->spare.erase(c->spare.begin() + best);
  } else {
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = spfd::mem_get(c->device, bytes, &q, &block);
    c->alloc_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? SPFD_ENOMEM : SPFD_ECUDA,
                  "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  if (getenv("SPFD_POISON_ALLOC")) {
    cudaError_t e = cudaMemsetAsync(q, 0xff, block, c->stream);
    if (e != cudaSuccess) {
      c->spare.emplace_back(q, block);
      return fail(SPFD_ECUDA, "poisoning a block failed: %s", cudaGetErrorString(e));
    }
  }
  c->allocs.push_back(q);
  c->alloc_bytes.push_back(block);
  c->bytes += (int64_t)block;
  *p = (T *)q;
  return SPFD_OK;
}

// Pinned host block held by the context until destroy.
template <typename T>
spfd_status halloc(spfd_ctx *c, T **p, size_t count) {
  *p = nullptr;
  void *q = nullptr;
  size_t block = 0;
  cudaError_t e = spfd::host_get(std::max<size_t>(count, 1) * sizeof(T), &q, &block);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SPFD_ENOMEM, "pinned host allocation failed: %s", cudaGetErrorString(e));
  }
  c->hblocks.emplace_back(q, block);
  *p = (T *)q;
  return SPFD_OK;
}

// Releases a buffer of the context to its spare list (no synchronisation:
// only this context's stream-ordered work can reuse it before destroy).
template <typename T>
void dfree(spfd_ctx *c, T *&p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), (void *)p);
  if (it != c->allocs.end()) {
    const size_t k = (size_t)(it - c->allocs.begin());
    c->bytes -= (int64_t)c->alloc_bytes[k];
    c->spare.emplace_back(*it, c->alloc_bytes[k]);
    c->alloc_bytes.erase(c->alloc_bytes.begin() + k);
    c->allocs.erase(it);
  }
  p = nullptr;
}

spfd_status sync_check(spfd_ctx *c, const char *what);
spfd_status launch_check(const char *what);
spfd_status read_scalars(spfd_ctx *c, int nk = 1);
spfd_status build_impl(spfd_ctx *c, const double *sigma);
void destroy_ctx(spfd_ctx *c);

// Profiling: event pair around a launch, resolved at the next flush.
int stat_index(spfd_ctx *c, const char *name, bool f32);
cudaEvent_t take_event(spfd_ctx *c);
void prof_push(spfd_ctx *c, int stat, cudaEvent_t a, cudaEvent_t b,
               double bytes, double flops);
spfd_status prof_flush(spfd_ctx *c);

}  // namespace spfd

// Block order of family fam on level l for the launch in progress.
inline int block_order(const spfd_ctx *c, int fam, int l) {
  return c->ord ? c->ord[fam * (int)c->L.size() + l] : 0;
}

// Solve steps shared by the host-driven solves (spfd_api.cu) and the
// captured, device-driven ones (spfd_graph.cu).  All of them only enqueue
// work on c->stream (no host synchronisation), so they can be captured.
// v -= per-component mean of v for nk right-hand sides starting at j0.
template <typename T>
spfd_status project(spfd_ctx *c, T *v, int nk = 1, int j0 = 0);
// V-cycle on level l for nk right-hand sides; returns the corrections.
// head: the level-0 cycle's first sweep already ran (vcycle_head).
template <typename T>
T *vcycle(spfd_ctx *c, int l, T *bl, bool proj, int nk, bool rz = false, bool head = false);
// z = M r, r.z, beta and p = z + beta p for the first nk right-hand sides.
template <typename T>
spfd_status precondition_step(spfd_ctx *c, T *r, T *p, int first, int nk, bool head = false);
// Per-right-hand-side flags (clear_rsum: 1 clears the residual sums; frozen,
// restart: >= 0 sets that flag) of the nk right-hand sides from j0.
spfd_status batch_flags(spfd_ctx *c, int j0, int nk, int clear_rsum, int frozen, int restart);

// Launch CALL (which starts NK kernels) on c->stream; with opts.profile the
// launch is bracketed by CUDA events and credited to family NAME with its
// algorithmic bytes and flops.
#define SPFD_LAUNCH(c, NAME, F32, NK, BYTES, FLOPS, CALL)                     \
  do {                                                                       \
    (c)->launch_count += (NK);                                               \
    if ((c)->opts.profile) {                                                 \
      cudaEvent_t e0_ = ::spfd::take_event(c), e1_ = ::spfd::take_event(c);  \
      cudaEventRecord(e0_, (c)->stream);                                     \
      CALL;                                                                  \
      cudaEventRecord(e1_, (c)->stream);                                     \
      ::spfd::prof_push((c), ::spfd::stat_index((c), NAME, F32), e0_, e1_,   \
                        (double)(BYTES), (double)(FLOPS));                   \
    } else {                                                                 \
      CALL;                                                                  \
    }                                                                        \
  } while (0)
