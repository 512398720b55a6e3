// Device-driven solves: the FP64 solve of Eq. 3 (Sec. II), or its
// mixed-precision refinement, captured as one CUDA graph whose loops run on
// the GPU, and groups of bodies (phantoms of different sizes) solved together
// by one launch of such a graph.
//
// The host-driven solve (spfd_api.cu) reads the CG scalars back after every
// iteration to decide whether to stop, check the true residual or restart.
// Here those decisions are taken by one-thread control kernels that set the
// handles of conditional graph nodes:
//
//   rhs, projection, |b|^2, x = 0, r = b, p = 0, control init, z = M r ...
//   WHILE (loop)
//     q = A p, p.q, x += alpha p, r -= alpha q, r.r
//     control: iteration count, breakdown, recursive residual <= tol?
//     IF (check)   true residual b - A x, |.|^2
//                  control: converged / stalled / restart?
//                  IF (restart)  r = b - A x, projected; beta = 0 next
//     control: stop at maxit or when done; loop and precondition flags
//     IF (precondition)  z = M r, r.z, beta, p = z + beta p
//   x projected; IF (not converged) true residual of the result; Psi
//
// The kernels and their order are those of the host-driven solve, and every
// decision compares the same FP64 values the host compares, so a graph solve
// returns the same Psi, bit for bit, with the same iteration count.
//
// The mixed-precision form nests the same pattern: a WHILE node over the FP64
// refinement steps (scale of the FP32 residual and inner target on the
// device), inside it a WHILE node over the FP32 CG iterations stopped on the
// recursive residual, then x += scale d, the true residual and the decision
// to refine again, exactly as the host-driven refinement takes them.
//
// A group captures one such branch per context, side by side in one graph,
// so the bodies' kernels share the GPU (small bodies fill what a large one
// leaves idle) and the whole group costs one graph launch and one host
// synchronisation.
#include <vector>

#include "spfd_ctx.cuh"

namespace spfd {

// Control state of one device-driven solve (device memory of the group).
struct GraphCtl {
  double tol;       // relative residual target (set per solve)
  double bb;        // |b|^2 of the projected right-hand side
  double best;      // best true relative residual seen by a check
  double min_rrel;  // smallest recursive relative residual
  double rel;       // last true relative residual
  int maxit;        // iteration cap (set per solve)
  int it, stall, done, conv, broke, bad;
  // mixed precision: FP64 refinement state and the FP32 inner CG's
  double nrm2;      // |r|^2 of the current FP64 residual
  double nr, inv_nr;  // its norm and 1 / norm (scale of the FP32 copy)
  double eta;       // inner relative target
  double prev;      // smallest true relative residual so far
  double bb_in;     // |r32|^2 of the scaled FP32 residual
  double min_rrel_in;
  int total;        // inner iterations so far
  int outer;        // refinement step in progress
  int outer_of;     // refinement steps taken when the solve stopped
  int it_in;        // inner iterations of this step
  int cap;          // inner iteration budget of this step
  int idone;        // the inner CG has stopped
};

namespace {

__global__ void k_ctl_init(GraphCtl *g, const Scalars *sc, cudaGraphConditionalHandle loop) {
  g->bb = sc->aux[1];
  g->best = INFINITY;
  g->min_rrel = INFINITY;
  g->rel = 0.0;
  g->it = 0;
  g->stall = 0;
  g->broke = 0;
  g->bad = (sc->status & DEV_BAD_A) != 0;
  const bool run = !g->bad && g->bb > 0.0;
  g->done = run ? 0 : 1;
  g->conv = (!g->bad && !(g->bb > 0.0)) ? 1 : 0;  // b = 0: x = 0 is exact
  cudaGraphSetConditional(loop, run ? 1u : 0u);
}

// After the x / r update of an iteration.
__global__ void k_ctl_iter(GraphCtl *g, const Scalars *sc, cudaGraphConditionalHandle check) {
  g->it += 1;
  const double rrel = sqrt(sc->rr / g->bb);
  unsigned chk = 0;
  if (!isfinite(rrel) || rrel > 1e8 * fmax(g->min_rrel, g->tol)) {
    g->broke = 1;  // breakdown: report the current iterate, not converged
    chk = 1;
  } else {
    g->min_rrel = fmin(g->min_rrel, rrel);
    if (rrel <= g->tol) chk = 1;
  }
  cudaGraphSetConditional(check, chk);
}

// After the true residual of a check (|b - A x|^2 in aux[2]).
__global__ void k_ctl_true(GraphCtl *g, const Scalars *sc, cudaGraphConditionalHandle restart) {
  const double rel = sqrt(sc->aux[2] / g->bb);
  g->rel = rel;
  unsigned rs = 0;
  if (g->broke) {
    g->done = 1;
  } else if (rel <= g->tol) {
    g->conv = 1;
    g->done = 1;
  } else {
    // three restarts that fail to halve the best true residual: the rounding
    // floor is reached
    if (rel < 0.5 * g->best) {
      g->best = rel;
      g->stall = 0;
    } else if (++g->stall >= 3) {
      g->done = 1;
    }
    rs = g->done ? 0u : 1u;
  }
  cudaGraphSetConditional(restart, rs);
}

// End of an iteration: stop at maxit, else precondition and go on.
__global__ void k_ctl_next(GraphCtl *g, Scalars *sc, cudaGraphConditionalHandle loop,
                           cudaGraphConditionalHandle prec) {
  if (!g->done && g->it >= g->maxit) g->done = 1;
  if (g->done) sc->frozen = 1;
  cudaGraphSetConditional(prec, g->done ? 0u : 1u);
  cudaGraphSetConditional(loop, g->done ? 0u : 1u);
}

// After the loop: recompute the true residual of a result that missed tol.
__global__ void k_ctl_after(const GraphCtl *g, cudaGraphConditionalHandle final_res) {
  cudaGraphSetConditional(final_res, (!g->conv && !g->bad && g->bb > 0.0) ? 1u : 0u);
}

__global__ void k_ctl_final(GraphCtl *g, const Scalars *sc) {
  g->rel = sqrt(sc->aux[2] / g->bb);
}

// ------------------------------------------- mixed precision (refinement)
__global__ void k_mctl_init(GraphCtl *g, const Scalars *sc, cudaGraphConditionalHandle outer) {
  g->bb = sc->aux[1];
  g->bad = (sc->status & DEV_BAD_A) != 0;
  const bool run = !g->bad && g->bb > 0.0;
  g->done = run ? 0 : 1;
  g->conv = (!g->bad && !(g->bb > 0.0)) ? 1 : 0;
  g->nrm2 = g->bb;
  g->prev = INFINITY;
  g->rel = 0.0;
  g->stall = 0;
  g->total = 0;
  g->outer = 0;
  g->outer_of = 0;
  cudaGraphSetConditional(outer, run ? 1u : 0u);
}

// Start of a refinement step: stop past 30 steps or the iteration budget,
// else the scale of the FP32 copy and the inner target.
__global__ void k_mctl_begin(GraphCtl *g, cudaGraphConditionalHandle outer,
                             cudaGraphConditionalHandle go) {
  g->outer += 1;
  const bool stop = g->outer > 30 || g->total >= g->maxit;
  if (stop) {
    g->done = 1;
    g->outer_of = min(g->outer, 30);
  } else {
    g->nr = sqrt(g->nrm2);
    g->inv_nr = 1.0 / g->nr;
    // what is still missing for tol, but no tighter than what an FP32 solve
    // reliably reaches
    g->eta = fmin(0.5, fmax(0.5 * g->tol * sqrt(g->bb) / g->nr, 1e-4));
  }
  cudaGraphSetConditional(outer, stop ? 0u : 1u);
  cudaGraphSetConditional(go, stop ? 0u : 1u);
}

// Inner CG start (|r32|^2 in aux[3]).
__global__ void k_ictl_init(GraphCtl *g, const Scalars *sc, cudaGraphConditionalHandle inner) {
  g->bb_in = sc->aux[3];
  g->it_in = 0;
  g->min_rrel_in = INFINITY;
  g->cap = g->maxit - g->total;
  g->idone = g->bb_in > 0.0 ? 0 : 1;
  cudaGraphSetConditional(inner, g->idone ? 0u : 1u);
}

// After an inner x / r update: stopped on the recursive residual.
__global__ void k_ictl_iter(GraphCtl *g, Scalars *sc, cudaGraphConditionalHandle inner,
                            cudaGraphConditionalHandle prec) {
  g->it_in += 1;
  const double rrel = sqrt(sc->rr / g->bb_in);
  if (!isfinite(rrel) || rrel > 1e8 * fmax(g->min_rrel_in, g->eta)) {
    g->idone = 1;
  } else {
    g->min_rrel_in = fmin(g->min_rrel_in, rrel);
    if (rrel <= g->eta) g->idone = 1;
  }
  if (!g->idone && g->it_in >= g->cap) g->idone = 1;
  if (g->idone) sc->frozen = 1;
  cudaGraphSetConditional(prec, g->idone ? 0u : 1u);
  cudaGraphSetConditional(inner, g->idone ? 0u : 1u);
}

__global__ void k_mctl_mid(GraphCtl *g) { g->total += g->it_in; }

// After the true residual of the refined x (|b - A x|^2 in aux[2]).
__global__ void k_mctl_check(GraphCtl *g, const Scalars *sc, cudaGraphConditionalHandle outer,
                             cudaGraphConditionalHandle next) {
  const double rel = sqrt(sc->aux[2] / g->bb);
  g->rel = rel;
  bool stop = false;
  if (rel <= g->tol) {
    g->conv = 1;
    stop = true;
  } else if (rel > 0.5 * g->prev) {
    if (++g->stall >= 2) stop = true;
  } else {
    g->stall = 0;
  }
  if (stop) {
    g->done = 1;
    g->outer_of = g->outer;
  } else {
    g->prev = fmin(g->prev, rel);
  }
  cudaGraphSetConditional(outer, stop ? 0u : 1u);
  cudaGraphSetConditional(next, stop ? 0u : 1u);
}

__global__ void k_mctl_nrm(GraphCtl *g, const Scalars *sc) { g->nrm2 = sc->aux[3]; }

// ---------------------------------------------------------------- capture
cudaGraph_t capture_graph(cudaStream_t s, const cudaGraphNode_t **deps, size_t *nd) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, deps, nullptr, nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return nullptr;
  return g;
}

spfd_status new_handle(cudaStream_t s, cudaGraphConditionalHandle *h) {
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraph_t g = capture_graph(s, &deps, &nd);
  if (!g) return fail(SPFD_ECUDA, "stream is not capturing");
  CU(cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault));
  return SPFD_OK;
}

// Appends a conditional node (after everything captured on s so far) and
// starts capturing its body on the stream body.
spfd_status cond_begin(cudaStream_t s, cudaGraphConditionalHandle h,
                       cudaGraphConditionalNodeType type, cudaStream_t body) {
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraph_t g = capture_graph(s, &deps, &nd);
  if (!g) return fail(SPFD_ECUDA, "stream is not capturing");
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CU(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  CU(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                         cudaStreamSetCaptureDependencies));
  CU(cudaStreamBeginCaptureToGraph(body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  return SPFD_OK;
}

spfd_status cond_end(cudaStream_t body) {
  cudaGraph_t g = nullptr;
  CU(cudaStreamEndCapture(body, &g));
  return SPFD_OK;
}

// The node captured last on s (the kernel just launched).
spfd_status last_node(cudaStream_t s, cudaGraphNode_t *out) {
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  if (!capture_graph(s, &deps, &nd) || nd != 1)
    return fail(SPFD_EINTERNAL, "could not identify a captured kernel node");
  *out = deps[0];
  return SPFD_OK;
}

// Points argument idx (a pointer) of an instantiated kernel node at val.
spfd_status patch_ptr(cudaGraphExec_t ex, cudaGraphNode_t node, int nargs, int idx,
                      const void *val) {
  cudaKernelNodeParams p{};
  CU(cudaGraphKernelNodeGetParams(node, &p));
  void *args[16];
  for (int i = 0; i < nargs; ++i) args[i] = p.kernelParams[i];
  const void *v = val;
  args[idx] = (void *)&v;
  p.kernelParams = args;
  CU(cudaGraphExecKernelNodeSetParams(ex, node, &p));
  return SPFD_OK;
}

// Argument positions of the pointers patched per solve:
// k_rhs(Grid, gx, a, b, status) and k_scatter<double>(Grid, x, comp, psi).
constexpr int RHS_NARGS = 5, RHS_ARG_A = 2;
constexpr int SCATTER_NARGS = 4, SCATTER_ARG_PSI = 3;

// True residual of x_k into level 0's r, |.|^2 into aux[2]; no host read.
spfd_status enqueue_true_residual(spfd_ctx *c) {
  Level &l0 = c->L[0];
  const double S = (double)l0.S;
  SPFD_LAUNCH(c, "true_residual", false, 1, 56 * S, 14 * S,
              (launch_residual7<double, double>(l0.g, l0.gx, l0.diag, c->xk, c->bk, l0.r,
                                                c->stream, 1)));
  SPFD_LAUNCH(c, "true_residual", false, 1, 20 * S, 2 * S,
              launch_dot<double>(l0.g.nb, l0.r, l0.r, c->comp, c->sc, c->partials, 2,
                                 c->stream, 1, c->pstride));
  return launch_check("true residual");
}

}  // namespace

// One branch: the whole FP64 solve of context c, captured on c->stream (a
// stream joined to a capture); body[0..2] are free streams for the bodies of
// the nested conditional nodes.  a and psi are the pointers of the capture;
// the nodes that read and write them are returned for patching.
spfd_status capture_solve_fp64(spfd_ctx *c, GraphCtl *ctl, const double *a, double *psi,
                               cudaStream_t body[3], cudaGraphNode_t *rhs_node,
                               cudaGraphNode_t *scatter_node) {
  Level &l0 = c->L[0];
  const size_t S0 = l0.S;
  const double S = (double)S0;
  const int nb = l0.g.nb;
  cudaStream_t s0 = c->stream;
  CU(cudaMemsetAsync(&c->sc->status, 0, sizeof(int), s0));
  // b = -G^T M a, projected; |b|^2 into aux[1]
  SPFD_LAUNCH(c, "rhs", false, 1, 56 * S, 12 * S,
              launch_rhs(l0.g, l0.gx, a, c->bk, &c->sc->status, s0, 1));
  TRY(launch_check("rhs"));
  TRY(last_node(s0, rhs_node));
  TRY(project<double>(c, c->bk, 1, 0));
  SPFD_LAUNCH(c, "project", false, 1, 20 * S, 2 * S,
              launch_dot<double>(nb, c->bk, c->bk, c->comp, c->sc, c->partials, 1, s0, 1,
                                 c->pstride));
  CU(cudaMemsetAsync(c->xk, 0, S0 * sizeof(double), s0));
  CU(cudaMemcpyAsync(c->rk, c->bk, S0 * sizeof(double), cudaMemcpyDeviceToDevice, s0));
  TRY(batch_flags(c, 0, 1, 1, -1, -1));  // b is projected: rsum = 0
  CU(cudaMemsetAsync(c->pk, 0, S0 * sizeof(double), s0));
  TRY(batch_flags(c, 0, 1, 0, 0, 0));
  cudaGraphConditionalHandle h_loop, h_final;
  TRY(new_handle(s0, &h_loop));
  TRY(new_handle(s0, &h_final));
  k_ctl_init<<<1, 1, 0, s0>>>(ctl, c->sc, h_loop);
  TRY(launch_check("control"));
  TRY(precondition_step<double>(c, c->rk, c->pk, 1, 1));

  // the CG loop
  TRY(cond_begin(s0, h_loop, cudaGraphCondTypeWhile, body[0]));
  {
    c->stream = body[0];
    cudaStream_t s1 = body[0];
    SPFD_LAUNCH(c, "apply_dot", false, 1, 6 * 8 * S, 15 * S,
                launch_apply_dot<double>(l0.g, l0.gx, l0.diag, c->pk, c->qk, c->sc,
                                         c->partials, s1, 1, c->pstride));
    SPFD_LAUNCH(c, "finish_pq", false, 1, 8.0 * nb, nb,
                launch_finish_pq(apply_dot_partials<double>(nb), c->partials,
                                 c->partials + (size_t)16 * nb, c->sc, s1, 1, c->pstride));
    SPFD_LAUNCH(c, "update_xr", false, 1, 6 * 8 * S, 7 * S,
                launch_update_xr<double>(nb, c->xk, c->rk, c->pk, c->qk, c->sc, c->partials,
                                         s1, 1, c->pstride));
    cudaGraphConditionalHandle h_check, h_prec;
    TRY(new_handle(s1, &h_check));
    TRY(new_handle(s1, &h_prec));
    k_ctl_iter<<<1, 1, 0, s1>>>(ctl, c->sc, h_check);
    TRY(launch_check("control"));
    TRY(cond_begin(s1, h_check, cudaGraphCondTypeIf, body[1]));
    {
      c->stream = body[1];
      cudaStream_t s2 = body[1];
      TRY(enqueue_true_residual(c));
      cudaGraphConditionalHandle h_restart;
      TRY(new_handle(s2, &h_restart));
      k_ctl_true<<<1, 1, 0, s2>>>(ctl, c->sc, h_restart);
      TRY(launch_check("control"));
      TRY(cond_begin(s2, h_restart, cudaGraphCondTypeIf, body[2]));
      {
        // restart from the true residual (left in level 0's r)
        c->stream = body[2];
        CU(cudaMemcpyAsync(c->rk, l0.r, S0 * sizeof(double), cudaMemcpyDeviceToDevice,
                           body[2]));
        TRY(project<double>(c, c->rk, 1, 0));
        TRY(batch_flags(c, 0, 1, 1, -1, 1));
      }
      TRY(cond_end(body[2]));
      c->stream = s2;
    }
    TRY(cond_end(body[1]));
    c->stream = s1;
    k_ctl_next<<<1, 1, 0, s1>>>(ctl, c->sc, h_loop, h_prec);
    TRY(launch_check("control"));
    TRY(cond_begin(s1, h_prec, cudaGraphCondTypeIf, body[1]));
    c->stream = body[1];
    TRY(precondition_step<double>(c, c->rk, c->pk, 0, 1));
    TRY(cond_end(body[1]));
    c->stream = s1;
  }
  TRY(cond_end(body[0]));
  c->stream = s0;

  TRY(project<double>(c, c->xk, 1, 0));
  k_ctl_after<<<1, 1, 0, s0>>>(ctl, h_final);
  TRY(launch_check("control"));
  TRY(cond_begin(s0, h_final, cudaGraphCondTypeIf, body[0]));
  c->stream = body[0];
  TRY(enqueue_true_residual(c));
  k_ctl_final<<<1, 1, 0, body[0]>>>(ctl, c->sc);
  TRY(launch_check("control"));
  TRY(cond_end(body[0]));
  c->stream = s0;
  const double NN = (double)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  SPFD_LAUNCH(c, "scatter", false, 1, 8 * NN + 12.0 * S, 0,
              launch_scatter<double>(l0.g, c->xk, c->comp, psi, s0, 1));
  TRY(launch_check("scatter"));
  TRY(last_node(s0, scatter_node));
  return SPFD_OK;
}

// One branch: the mixed-precision solve of context c (the steps of the
// host-driven refinement), captured on c->stream; body[0..3] are free
// streams for the nested conditional bodies.
spfd_status capture_solve_mixed(spfd_ctx *c, GraphCtl *ctl, const double *a, double *psi,
                                cudaStream_t body[4], cudaGraphNode_t *rhs_node,
                                cudaGraphNode_t *scatter_node) {
  Level &l0 = c->L[0];
  const size_t S0 = l0.S;
  const double S = (double)S0;
  const int nb = l0.g.nb;
  cudaStream_t s0 = c->stream;
  CU(cudaMemsetAsync(&c->sc->status, 0, sizeof(int), s0));
  SPFD_LAUNCH(c, "rhs", false, 1, 56 * S, 12 * S,
              launch_rhs(l0.g, l0.gx, a, c->bk, &c->sc->status, s0, 1));
  TRY(launch_check("rhs"));
  TRY(last_node(s0, rhs_node));
  TRY(project<double>(c, c->bk, 1, 0));
  SPFD_LAUNCH(c, "project", false, 1, 20 * S, 2 * S,
              launch_dot<double>(nb, c->bk, c->bk, c->comp, c->sc, c->partials, 1, s0, 1,
                                 c->pstride));
  CU(cudaMemsetAsync(c->xk, 0, S0 * sizeof(double), s0));
  CU(cudaMemcpyAsync(c->rk, c->bk, S0 * sizeof(double), cudaMemcpyDeviceToDevice, s0));
  cudaGraphConditionalHandle h_outer;
  TRY(new_handle(s0, &h_outer));
  k_mctl_init<<<1, 1, 0, s0>>>(ctl, c->sc, h_outer);
  TRY(launch_check("control"));
  TRY(cond_begin(s0, h_outer, cudaGraphCondTypeWhile, body[0]));
  {
    cudaStream_t s1 = body[0];
    c->stream = s1;
    cudaGraphConditionalHandle h_go;
    TRY(new_handle(s1, &h_go));
    k_mctl_begin<<<1, 1, 0, s1>>>(ctl, h_outer, h_go);
    TRY(launch_check("control"));
    TRY(cond_begin(s1, h_go, cudaGraphCondTypeIf, body[1]));
    {
      cudaStream_t s2 = body[1];
      c->stream = s2;
      CU(cudaMemsetAsync(c->dk32, 0, S0 * sizeof(float), s2));
      SPFD_LAUNCH(c, "convert", true, 1, 12 * S, S,
                  launch_scale_to_f32(nb, c->rk, 0.0, c->rk32, c->sc, c->partials, s2,
                                      &ctl->inv_nr));
      SPFD_LAUNCH(c, "project", true, 1, 12 * S, 2 * S,
                  launch_dot<float>(nb, c->rk32, c->rk32, c->comp, c->sc, c->partials, 3, s2,
                                    1, c->pstride));
      // the inner FP32 CG
      CU(cudaMemsetAsync(c->pk32, 0, S0 * sizeof(float), s2));
      TRY(batch_flags(c, 0, 1, 0, 0, 0));
      cudaGraphConditionalHandle h_inner, h_next;
      TRY(new_handle(s2, &h_inner));
      TRY(new_handle(s2, &h_next));
      k_ictl_init<<<1, 1, 0, s2>>>(ctl, c->sc, h_inner);
      TRY(launch_check("control"));
      TRY(precondition_step<float>(c, c->rk32, c->pk32, 1, 1));
      TRY(cond_begin(s2, h_inner, cudaGraphCondTypeWhile, body[2]));
      {
        cudaStream_t s3 = body[2];
        c->stream = s3;
        SPFD_LAUNCH(c, "apply_dot", true, 1, 5 * 4 * S, 20 * S,
                    launch_apply_dot<float>(l0.g, l0.gx32, l0.diag32, c->pk32, c->qk32, c->sc,
                                            c->partials, s3, 1, c->pstride));
        SPFD_LAUNCH(c, "finish_pq", false, 1, 8.0 * nb, nb,
                    launch_finish_pq(apply_dot_partials<float>(nb), c->partials,
                                     c->partials + (size_t)16 * nb, c->sc, s3, 1, c->pstride,
                                     true));
        SPFD_LAUNCH(c, "update_xr", true, 1, 6 * 4 * S, 7 * S,
                    launch_update_xr<float>(nb, c->dk32, c->rk32, c->pk32, c->qk32, c->sc,
                                            c->partials, s3, 1, c->pstride));
        cudaGraphConditionalHandle h_iprec;
        TRY(new_handle(s3, &h_iprec));
        k_ictl_iter<<<1, 1, 0, s3>>>(ctl, c->sc, h_inner, h_iprec);
        TRY(launch_check("control"));
        TRY(cond_begin(s3, h_iprec, cudaGraphCondTypeIf, body[3]));
        c->stream = body[3];
        TRY(precondition_step<float>(c, c->rk32, c->pk32, 0, 1));
        TRY(cond_end(body[3]));
        c->stream = s3;
      }
      TRY(cond_end(body[2]));
      c->stream = s2;
      k_mctl_mid<<<1, 1, 0, s2>>>(ctl);
      TRY(launch_check("control"));
      SPFD_LAUNCH(c, "convert", false, 1, 20 * S, 2 * S,
                  launch_axpy_mixed(nb, c->xk, c->dk32, 0.0, s2, &ctl->nr));
      TRY(enqueue_true_residual(c));
      k_mctl_check<<<1, 1, 0, s2>>>(ctl, c->sc, h_outer, h_next);
      TRY(launch_check("control"));
      TRY(cond_begin(s2, h_next, cudaGraphCondTypeIf, body[2]));
      {
        // the next correction solves for the true residual (in level 0's r)
        c->stream = body[2];
        CU(cudaMemcpyAsync(c->rk, l0.r, S0 * sizeof(double), cudaMemcpyDeviceToDevice,
                           body[2]));
        TRY(project<double>(c, c->rk, 1, 0));
        SPFD_LAUNCH(c, "project", false, 1, 20 * S, 2 * S,
                    launch_dot<double>(nb, c->rk, c->rk, c->comp, c->sc, c->partials, 3,
                                       body[2], 1, c->pstride));
        k_mctl_nrm<<<1, 1, 0, body[2]>>>(ctl, c->sc);
        TRY(launch_check("control"));
      }
      TRY(cond_end(body[2]));
      c->stream = s2;
    }
    TRY(cond_end(body[1]));
    c->stream = s1;
  }
  TRY(cond_end(body[0]));
  c->stream = s0;
  TRY(project<double>(c, c->xk, 1, 0));
  const double NN = (double)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  SPFD_LAUNCH(c, "scatter", false, 1, 8 * NN + 12.0 * S, 0,
              launch_scatter<double>(l0.g, c->xk, c->comp, psi, s0, 1));
  TRY(launch_check("scatter"));
  TRY(last_node(s0, scatter_node));
  return SPFD_OK;
}

}  // namespace spfd

using namespace spfd;

struct spfd_group {
  int device = 0;
  cudaStream_t stream = nullptr;        // launch stream (caller's)
  std::vector<spfd_ctx *> ctx;
  std::vector<uint64_t> gen;            // buffer generation of each context at capture
  std::vector<cudaStream_t> branch;     // capture stream per context
  cudaStream_t origin = nullptr, body[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> rhs_node, scatter_node;
  GraphCtl *dctl = nullptr, *hctl = nullptr;
  bool captured = false;
  int64_t launches = 0;                 // kernel launches recorded in the graph
};

namespace {

void release_graph(spfd_group *g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  g->captured = false;
}

// Captures the group's graph with the pointers of this call.
spfd_status capture_group(spfd_group *g, const double *const *a, double *const *psi) {
  release_graph(g);
  const int n = (int)g->ctx.size();
  g->rhs_node.assign(n, nullptr);
  g->scatter_node.assign(n, nullptr);
  std::vector<cudaStream_t> saved(n);
  std::vector<int> prof(n);
  std::vector<int64_t> l0(n);
  for (int i = 0; i < n; ++i) {
    saved[i] = g->ctx[i]->stream;
    prof[i] = g->ctx[i]->opts.profile;
    l0[i] = g->ctx[i]->launch_count;
  }
  // the captured kernels are launched plainly (the graph has no host gaps
  // to hide); restored on every exit
  struct PdlOff {
    bool was = pdl_allowed;
    PdlOff() { pdl_allowed = false; }
    ~PdlOff() { pdl_allowed = was; }
  } pdl_off;
  CU(cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeThreadLocal));
  spfd_status s = SPFD_OK;
  cudaError_t e = cudaEventRecord(g->fork, g->origin);
  for (int i = 0; i < n && s == SPFD_OK && e == cudaSuccess; ++i) {
    spfd_ctx *c = g->ctx[i];
    if (c->ndof == 0) continue;
    e = cudaStreamWaitEvent(g->branch[i], g->fork, 0);
    if (e != cudaSuccess) break;
    c->stream = g->branch[i];
    c->opts.profile = 0;  // no event nodes inside the graph
    s = c->opts.precision == SPFD_MIXED
            ? capture_solve_mixed(c, g->dctl + i, a[i], psi[i], g->body, &g->rhs_node[i],
                                  &g->scatter_node[i])
            : capture_solve_fp64(c, g->dctl + i, a[i], psi[i], g->body, &g->rhs_node[i],
                                 &g->scatter_node[i]);
    c->stream = saved[i];
    c->opts.profile = prof[i];
    if (s != SPFD_OK) break;
    e = cudaEventRecord(g->join[i], g->branch[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->origin, g->join[i], 0);
  }
  for (int i = 0; i < n; ++i) {
    g->ctx[i]->stream = saved[i];
    g->ctx[i]->opts.profile = prof[i];
  }
  // a failure inside a conditional body leaves that body's capture open
  for (cudaStream_t b : g->body) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(b, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(b, &tmp);  // the body graph belongs to its node
    }
  }
  cudaGetLastError();
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(g->origin, &graph);
  if (s != SPFD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(SPFD_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : ee));
  }
  g->graph = graph;
  CU(cudaGraphInstantiate(&g->exec, graph, 0));
  g->launches = 0;
  for (int i = 0; i < n; ++i) {
    g->launches += g->ctx[i]->launch_count - l0[i];
    g->ctx[i]->launch_count = l0[i];  // capture launched nothing
    g->gen[i] = g->ctx[i]->gen;
  }
  g->captured = true;
  return SPFD_OK;
}

void destroy_group(spfd_group *g) {
  if (!g) return;
  if (g->stream || g->origin) cudaStreamSynchronize(g->origin);
  release_graph(g);
  for (cudaStream_t s : g->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaStream_t s : g->body)
    if (s) cudaStreamDestroy(s);
  if (g->origin) cudaStreamDestroy(g->origin);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {g->fork, g->ev0, g->ev1})
    if (e) cudaEventDestroy(e);
  if (g->dctl) cudaFree(g->dctl);
  if (g->hctl) cudaFreeHost(g->hctl);
  delete g;
}

}  // namespace

extern "C" spfd_status spfd_group_create(spfd_ctx *const *ctxs, int n, void *stream,
                                         spfd_group **out) {
  if (!out) return fail(SPFD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1 || n > 4096) return fail(SPFD_EINVAL, "need 1..4096 contexts");
  int dev = -1;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(SPFD_EINVAL, "context %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(SPFD_EINVAL, "context %d appears twice", i);
    if (dev < 0) dev = ctxs[i]->device;
    if (ctxs[i]->device != dev) return fail(SPFD_EINVAL, "contexts on different devices");
  }
  CU(cudaSetDevice(dev));
  spfd_group *g = new spfd_group();
  g->device = dev;
  g->stream = (cudaStream_t)stream;
  g->ctx.assign(ctxs, ctxs + n);
  g->gen.assign(n, 0);
  g->branch.assign(n, nullptr);
  g->join.assign(n, nullptr);
  auto bad = [&](cudaError_t e) {
    destroy_group(g);
    return fail(SPFD_ECUDA, "group set-up failed: %s", cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking)) != cudaSuccess)
    return bad(e);
  for (int i = 0; i < 4; ++i)
    if ((e = cudaStreamCreateWithFlags(&g->body[i], cudaStreamNonBlocking)) != cudaSuccess)
      return bad(e);
  for (int i = 0; i < n; ++i) {
    if ((e = cudaStreamCreateWithFlags(&g->branch[i], cudaStreamNonBlocking)) != cudaSuccess)
      return bad(e);
    if ((e = cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming)) != cudaSuccess)
      return bad(e);
  }
  if ((e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreate(&g->ev0)) != cudaSuccess ||
      (e = cudaEventCreate(&g->ev1)) != cudaSuccess)
    return bad(e);
  if ((e = cudaMalloc(&g->dctl, (size_t)n * sizeof(GraphCtl))) != cudaSuccess) return bad(e);
  if ((e = cudaMallocHost(&g->hctl, (size_t)n * sizeof(GraphCtl))) != cudaSuccess) return bad(e);
  *out = g;
  return SPFD_OK;
}

extern "C" spfd_status spfd_group_solve(spfd_group *g, const double *const *a_devs,
                                        double tol, double *const *psi_devs,
                                        spfd_info *infos) {
  if (!g) return fail(SPFD_EINVAL, "group is NULL");
  if (!a_devs || !psi_devs) return fail(SPFD_EINVAL, "null array list");
  const int n = (int)g->ctx.size();
  for (int i = 0; i < n; ++i)
    if (!a_devs[i] || !psi_devs[i]) return fail(SPFD_EINVAL, "null array for context %d", i);
  CU(cudaSetDevice(g->device));
  cudaStream_t st = g->stream;
  // work already queued on the contexts' own streams comes first
  for (int i = 0; i < n; ++i) {
    CU(cudaEventRecord(g->join[i], g->ctx[i]->stream));
    CU(cudaStreamWaitEvent(st, g->join[i], 0));
  }
  int active = 0;
  for (int i = 0; i < n; ++i) active += g->ctx[i]->ndof > 0;
  bool recapture = active > 0 && !g->captured;
  for (int i = 0; i < n; ++i) recapture |= active > 0 && g->ctx[i]->gen != g->gen[i];
  if (recapture) {
    CU(cudaStreamSynchronize(st));
    TRY(capture_group(g, a_devs, psi_devs));
  }
  for (int i = 0; i < n; ++i) {
    spfd_ctx *c = g->ctx[i];
    GraphCtl &h = g->hctl[i];
    memset(&h, 0, sizeof h);
    h.tol = tol > 0.0 ? tol : c->opts.tol;
    h.maxit = c->opts.maxit;
    if (c->ndof == 0) continue;
    TRY(patch_ptr(g->exec, g->rhs_node[i], RHS_NARGS, RHS_ARG_A, a_devs[i]));
    TRY(patch_ptr(g->exec, g->scatter_node[i], SCATTER_NARGS, SCATTER_ARG_PSI, psi_devs[i]));
  }
  CU(cudaEventRecord(g->ev0, st));
  CU(cudaMemcpyAsync(g->dctl, g->hctl, (size_t)n * sizeof(GraphCtl), cudaMemcpyHostToDevice,
                     st));
  for (int i = 0; i < n; ++i)
    if (g->ctx[i]->ndof == 0) {
      const size_t NN = (size_t)(g->ctx[i]->nx + 1) * (g->ctx[i]->ny + 1) * (g->ctx[i]->nz + 1);
      CU(cudaMemsetAsync(psi_devs[i], 0, NN * sizeof(double), st));
    }
  if (active > 0) CU(cudaGraphLaunch(g->exec, st));
  CU(cudaMemcpyAsync(g->hctl, g->dctl, (size_t)n * sizeof(GraphCtl), cudaMemcpyDeviceToHost,
                     st));
  CU(cudaEventRecord(g->ev1, st));
  CU(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, g->ev0, g->ev1);
  int first_bad = -1, first_nc = -1;
  for (int i = 0; i < n; ++i) {
    spfd_ctx *c = g->ctx[i];
    const GraphCtl &h = g->hctl[i];
    spfd_info r = c->info;
    const bool empty = c->ndof == 0;
    const bool mixed = c->opts.precision == SPFD_MIXED;
    r.iters = empty ? 0 : (mixed ? h.total : h.it);
    r.outer_iters = empty || !mixed ? 0 : h.outer_of;
    r.converged = empty ? 1 : h.conv;
    r.rel_res_true = empty ? 0.0 : h.rel;
    r.ms_solve = ms;
    r.bytes_device = c->bytes;
    r.launches = g->launches;
    c->info = r;
    if (infos) infos[i] = r;
    if (!empty && h.bad && first_bad < 0) first_bad = i;
    if (!r.converged && first_nc < 0) first_nc = i;
  }
  if (first_bad >= 0)
    return fail(SPFD_EINVAL, "context %d: a holds a non-finite value on a conducting edge",
                first_bad);
  if (first_nc >= 0)
    return fail(SPFD_ENOTCONVERGED,
                "not converged: context %d at rel residual %.3e", first_nc,
                g->hctl[first_nc].rel);
  return SPFD_OK;
}

extern "C" void spfd_group_destroy(spfd_group *g) { destroy_group(g); }
