/*
 * spfd.h -- C ABI of the GB300 SPFD Poisson solver (libspfd.so).
 *
 * The library solves the discrete Poisson system of the Co-Simulation Scalar
 * Potential Finite Difference scheme (Haussmann et al., Eq. 3 in Sec. II)
 *
 *     G^T M_k G Psi = -G^T M_k a
 *
 * on the nodes of a voxel body model, by conjugate gradients preconditioned
 * with an operator-dependent geometric multigrid V-cycle, and evaluates the
 * voxel-averaged induced field of Eq. 1, |E| = |-j omega (a + G Psi)|
 * (Sec. III-E).  Every array argument is a plain pointer; no framework types
 * cross this boundary.
 *
 * Grid conventions
 *   voxels  [nz][ny][nx]          (x fastest), FP64 conductivity sigma in S/m
 *   nodes   [nz+1][ny+1][nx+1]    (voxel corners), FP64 Psi in V*s
 *   edges   [3][nz+1][ny+1][nx+1] component d in {x,y,z} holds the edge that
 *           leaves node (i,j,k) in +d; a in V*s (line integral of A); slots
 *           past the last node along d are ignored.
 *   h       voxel edge length in m; omega angular frequency in rad/s.
 *
 * Method choices the paper leaves open (Sec. II does not fix how M_k is
 * formed from the voxels; Sec. III-A keeps only conducting voxels):
 *   - edge conductance g_e = h * (sum of sigma of the <= 4 voxels around the
 *     edge) / 4, voxels outside the grid counting as air;
 *   - a node is an unknown iff an incident edge has g_e > 0; other nodes of
 *     the returned Psi are 0;
 *   - Psi is returned with zero mean on each connected conducting component
 *     (the system fixes it only up to one constant per component);
 *   - the relative residual is ||b - A Psi||_2 / ||b||_2, recomputed at exit.
 *
 * Ownership and streams
 *   Pointers named *_dev are caller-owned CUDA device pointers, contiguous in
 *   the layouts above; *_host pointers are caller-owned host memory (pinned
 *   memory gives the fastest copies).  The context owns every internal buffer
 *   and releases them in spfd_destroy.  All device work is ordered on the
 *   stream given to spfd_build; spfd_solve and spfd_solve_host synchronise
 *   that stream before returning (they report iteration counts), spfd_efield
 *   does not.
 *
 * Errors
 *   Every entry point returns a status code and never aborts the process.
 *   spfd_last_error() returns a thread-local description of the last failure.
 *   A context on which SPFD_ECUDA was returned must only be destroyed.
 */
#ifndef SPFD_H
#define SPFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPFD_OK = 0,
  SPFD_EINVAL = 1,         /* invalid argument (null, size, NaN/negative sigma, non-finite a) */
  SPFD_ENOMEM = 2,         /* a device or host allocation failed; nothing leaked */
  SPFD_ECUDA = 3,          /* a CUDA call or kernel failed */
  SPFD_ENOTCONVERGED = 4,  /* maxit reached or stagnated; Psi holds the last iterate */
  SPFD_EINTERNAL = 5       /* a bounded device loop hit its iteration cap */
} spfd_status;

/* Smoother of the V-cycle (both applied to D^-1 A, D the operator's
 * diagonal, on every level but the coarsest).
 *   SPFD_SMOOTHER_JACOBI:    weighted Jacobi, omega = 4 / (3 lambda_max),
 *                            nu_pre / nu_post sweeps (the default).
 *   SPFD_SMOOTHER_CHEBYSHEV: Chebyshev polynomial of degree cheb_degree
 *                            before and after the coarse correction, on the
 *                            eigenvalue interval [lambda_max / 8, lambda_max]
 *                            (three-term recurrence; each step costs one
 *                            residual); nu_pre / nu_post are not used. */
enum { SPFD_SMOOTHER_JACOBI = 0, SPFD_SMOOTHER_CHEBYSHEV = 1 };

/* Arithmetic of the solve.
 *   SPFD_FP64:  every operation (operator, V-cycle, Krylov) in FP64.
 *   SPFD_MIXED: FP64 iterative refinement around an FP32 preconditioned CG
 *               whose V-cycle keeps the finest-level conductances in BF16
 *               and accumulates in FP32; residuals, CG dot products and the
 *               coarsest-level solve stay FP64. */
enum { SPFD_FP64 = 0, SPFD_MIXED = 1 };

typedef struct {
  double tol;        /* default relative residual target (used when spfd_solve gets tol <= 0) */
  int maxit;         /* PCG iteration cap (default 200) */
  int nu_pre;        /* pre-smoothing sweeps per level (default 1) */
  int nu_post;       /* post-smoothing sweeps per level (default 1) */
  int smoother;      /* SPFD_SMOOTHER_JACOBI (default) or SPFD_SMOOTHER_CHEBYSHEV */
  int cheb_degree;   /* Chebyshev degree, 1 .. 8 (default 2; used with CHEBYSHEV only) */
  int precision;     /* SPFD_FP64 or SPFD_MIXED */
  int coarse_max;    /* stop coarsening at <= this many unknowns (default 512) */
  int max_levels;    /* hierarchy depth cap (default 12) */
  int verbose;       /* 0 = silent; 1 = one line per build/solve on stderr */
  int profile;       /* 1 = time every kernel launch with CUDA events (see
                        spfd_kernel_stats); adds ~2 us of host work per launch */
  int autotune;      /* 1 (default) = the first batched solve of each batch
                        size times the block orders of each batched kernel
                        family and level and keeps the fastest (see
                        spfd_autotune_report); 0 = fixed order 0 */
} spfd_opts;

typedef struct {
  int iters;              /* PCG iterations performed (inner iterations for SPFD_MIXED) */
  int outer_iters;        /* refinement steps (SPFD_MIXED), 0 for SPFD_FP64 */
  int converged;          /* 1 if rel_res_true <= tol */
  double rel_res_true;    /* ||b - A Psi|| / ||b|| recomputed in FP64 at exit */
  double ms_build;        /* device time of spfd_build */
  double ms_solve;        /* device time of the last solve */
  int64_t n_dof;          /* unknowns on the finest level */
  int n_comp;             /* connected conducting components */
  int n_levels;           /* multigrid levels */
  int64_t n_bricks;       /* active 8x8x8 node bricks on the finest level */
  int64_t bytes_device;   /* device memory held by the context */
  int64_t launches;       /* kernels launched by the last build / solve call */
} spfd_info;

/* Per-kernel-family timing collected while opts.profile is set. */
typedef struct {
  const char *name;       /* family, e.g. "jacobi7_l0" (static string) */
  int64_t launches;       /* launches timed since the last reset */
  double ms;              /* summed device time of those launches */
  double bytes;           /* algorithmic DRAM bytes of those launches */
  double flops;           /* FP64 (or FP32) operations of those launches */
} spfd_kernel_stat;

typedef struct spfd_ctx spfd_ctx;

/* Fill *opts with the defaults listed above. */
void spfd_opts_default(spfd_opts *opts);

/* Build the operator of Eq. 3 and its multigrid hierarchy.
 *   sigma_dev  [nz][ny][nx] FP64 conductivities (>= 0, finite), device.
 *   nx,ny,nz   voxel counts, each >= 1, with (nx+1)(ny+1)(nz+1) < 2^31.
 *   h          voxel edge length, > 0.
 *   opts       NULL for defaults.
 *   stream     cudaStream_t to order all work of this context on (NULL =
 *              the legacy default stream).
 *   out        receives the context (NULL on failure).
 * An all-air grid is valid: it yields a context with zero unknowns. */
spfd_status spfd_build(const double *sigma_dev, int nx, int ny, int nz,
                       double h, const spfd_opts *opts, void *stream,
                       spfd_ctx **out);

/* Solve Eq. 3 for the edge potentials a and write Psi.
 *   a_dev    [3][nz+1][ny+1][nx+1] FP64, device (finite on every edge that
 *            touches a conducting voxel).
 *   tol      relative residual target (> 0), or <= 0 for opts.tol.
 *   psi_dev  [nz+1][ny+1][nx+1] FP64 output, device.
 *   info     optional report (may be NULL).
 * Returns SPFD_ENOTCONVERGED (with Psi written) if tol was not reached. */
spfd_status spfd_solve(spfd_ctx *ctx, const double *a_dev, double tol,
                       double *psi_dev, spfd_info *info);

/* Solve Eq. 3 for nrhs source fields on the same body (e.g. coil positions
 * and orientations) in one call.
 *   nrhs     number of right-hand sides, 1..65535.
 *   a_dev    [nrhs][3][nz+1][ny+1][nx+1] FP64, device (as in spfd_solve).
 *   tol      relative residual target of every right-hand side (> 0), or
 *            <= 0 for opts.tol.
 *   psi_dev  [nrhs][nz+1][ny+1][nx+1] FP64 output, device.
 *   infos    optional array of nrhs reports (may be NULL); ms_solve and
 *            launches are those of the whole call.
 * With opts.precision = SPFD_FP64 the right-hand sides share every launch
 * (each kernel covers the batch, one host synchronisation per CG iteration
 * for all of them) while each keeps its own CG recurrence and stopping
 * decision, so each Psi is the one spfd_solve returns for it alone.  The
 * context grows its per-right-hand-side buffers on the first call with a
 * larger nrhs (about 10 FP64 vectors of the finest level per right-hand
 * side; with SPFD_MIXED also their FP32 copies) and keeps them.  With
 * SPFD_MIXED each right-hand side keeps its own FP64 refinement (scale,
 * inner target, stopping) while the FP32 inner CG covers all of them in
 * shared launches; each Psi again equals its spfd_solve result.  Returns
 * SPFD_ENOTCONVERGED (every Psi written) if any
 * right-hand side missed tol; a non-finite a on a conducting edge of any of
 * them gives SPFD_EINVAL. */
spfd_status spfd_solve_batch(spfd_ctx *ctx, int nrhs, const double *a_dev, double tol,
                             double *psi_dev, spfd_info *infos);

/* spfd_solve with host arrays: copies a to the device, solves, copies Psi
 * back, all on the context's stream.  Device staging buffers are allocated on
 * first use and kept by the context. */
spfd_status spfd_solve_host(spfd_ctx *ctx, const double *a_host, double tol,
                            double *psi_host, spfd_info *info);

/* Steps 4 and 5 of the pipeline (Sec. II-A) in one call with host arrays:
 * builds the operator of Eq. 3 for sigma, solves it for a to tol, evaluates
 * the voxel-averaged |E| of Eq. 1 and returns Psi and |E| in host memory
 * (spfd_build + spfd_solve + spfd_efield + spfd_destroy, with the copies).
 *   sigma_host  [nz][ny][nx] FP64 conductivities, host.
 *   a_host      [3][nz+1][ny+1][nx+1] FP64 edge potentials, host.  Only the
 *               edges of conducting voxels are read: in each row (fixed edge
 *               direction, y and z node index) the nodes from the first to
 *               one past the last conducting voxel of the voxel rows it
 *               touches; when the device can read the memory directly
 *               (pinned memory, or any memory where pageable-memory access
 *               is supported) they are pulled by the GPU while the operator
 *               is built, else a is copied whole.
 *   nx..h       as in spfd_build; tol as in spfd_solve; omega as in
 *               spfd_efield; opts NULL for defaults.
 *   stream      cudaStream_t (NULL = legacy default stream); a second stream
 *               of the call's own carries the copy of a and of Psi.
 *   psi_host    [nz+1][ny+1][nx+1] FP64 output, host.
 *   E_host      [nz][ny][nx] FP64 output in V/m, host.  When the device can
 *               write both directly, host threads of the call zero them
 *               during the solve and the GPU writes only the spans of the
 *               unknowns' node rows (Psi) and of the conducting voxels' rows
 *               (|E|); else they are copied whole.
 *   info        optional report of the solve; launches counts every kernel
 *               of the call.
 * With opts->verbose >= 2 the call prints its phase times to stderr.
 * Device buffers come from the library's block cache and are returned to it.
 * Synchronises.  Returns SPFD_ENOTCONVERGED (Psi and |E| written) if tol was
 * not reached.  Pinned host arrays give the fastest copies. */
spfd_status spfd_pipeline_host(const double *sigma_host, const double *a_host, int nx,
                               int ny, int nz, double h, double tol, double omega,
                               const spfd_opts *opts, void *stream, double *psi_host,
                               double *E_host, spfd_info *info);

/* Voxel-averaged |E| of Eq. 1: for each conducting voxel,
 *   E_d = omega / (4 h) * sum over its four d-edges of (a_e + Psi_head - Psi_tail),
 *   |E| = sqrt(E_x^2 + E_y^2 + E_z^2); air voxels get 0.
 *   a_dev    as in spfd_solve;  psi_dev  [nz+1][ny+1][nx+1] FP64, device.
 *   E_dev    [nz][ny][nx] FP64 output in V/m, device.
 * Asynchronous on the context's stream. */
spfd_status spfd_efield(spfd_ctx *ctx, const double *a_dev,
                        const double *psi_dev, double omega, double *E_dev);

/* |E| of a complex (phasor) source a = a_re + j a_im.  The operator of Eq. 3
 * is real, so Psi = psi_re + j psi_im comes from two real solves (for
 * instance one spfd_solve_batch of the two parts); the voxel-averaged field
 * of Eq. 1 is then E_re + j E_im, and this writes its magnitude
 *   |E| = sqrt(|E_re|^2 + |E_im|^2)
 * (a peak-phasor magnitude; a_im = psi_im = 0 gives spfd_efield's result).
 *   a_re, a_im       as a_dev of spfd_solve;  psi_re, psi_im as psi_dev.
 *   E_dev            [nz][ny][nx] FP64 output in V/m, device, 16-byte
 *                    aligned (SPFD_EINVAL otherwise).
 * A scratch array of the voxel grid's size comes from the context's block
 * cache.  Asynchronous on the context's stream. */
spfd_status spfd_efield_complex(spfd_ctx *ctx, const double *a_re, const double *psi_re,
                                const double *a_im, const double *psi_im, double omega,
                                double *E_dev);

/* Step 3 of the pipeline (Sec. II-A, step 3): the edge vector potentials a
 * from the magnetic facet fluxes b of Eq. 2, b = C a, by tree-cotree
 * gauging.  C (the discrete curl) annihilates every discrete gradient, so b
 * fixes a only up to one; the gauge sets a = 0 on the edges of a spanning
 * tree of the node grid, and the cotree edges then follow from b uniquely.
 * The tree is the comb on the root line (j, k) = (j0, k0): every z edge, the
 * y edges of the plane k = k0 and the x edges of the root line.  The result
 * differs from any other potential of the same b by a discrete gradient, so
 * spfd_solve and spfd_efield give the same |E| from it (gauge invariance of
 * Eq. 1 and Eq. 3).
 *   b_dev   [3][nz+1][ny+1][nx+1] FP64 facet fluxes in Wb, device: component
 *           d at node (i,j,k) is the flux through the square spanned by the
 *           two edges that leave that node along d1 = (d+1) mod 3 and
 *           d2 = (d+2) mod 3, with normal +d (its boundary run along d1
 *           first); slots of facets that would leave the grid are ignored.
 *           b must be divergence-free (zero net flux out of every voxel) for
 *           C a = b to hold on every facet; otherwise the facets z off the
 *           plane k0 absorb the mismatch.
 *   nx,ny,nz voxel counts (>= 1); j0 in 0..ny, k0 in 0..nz (a central root
 *           line keeps |a| smallest).
 *   stream  cudaStream_t to run on (NULL = the legacy default stream).
 *   a_dev   [3][nz+1][ny+1][nx+1] FP64 output in V*s (the layout of
 *           spfd_solve's a), device; every slot is written (0 on the tree
 *           and past the last node).  Must not overlap b_dev.
 * Needs no context and allocates nothing; asynchronous. */
spfd_status spfd_tree_cotree(const double *b_dev, int nx, int ny, int nz, int j0, int k0,
                             void *stream, double *a_dev);

/* Step 6 of the pipeline (Sec. II-A, step 6; Sec. III-E): the p-quantile
 * (p = 0.99 for the 99th percentile) of the voxel-averaged |E| per tissue and
 * over the whole body.  The quantile of n values is the nearest-rank value,
 * the k-th smallest with k the least integer >= p * n in exact arithmetic
 * (p read as its binary fraction; k >= 1), so no rounding decides the rank
 * and the result is one of the inputs, bit for bit.
 *   E_dev        [nz][ny][nx] FP64 |E| (e.g. from spfd_efield), device; only
 *                the context's conducting voxels (sigma > 0) are read, and
 *                there it must be finite and >= 0 (else SPFD_EINVAL).
 *   labels_dev   [nz][ny][nx] int32 tissue labels, device; a conducting
 *                voxel with label t in 0..n_labels-1 counts for tissue t, any
 *                other label for the whole body only.  May be NULL when
 *                n_labels = 0.
 *   n_labels     0..2048.
 *   p            in (0, 1].
 *   values_host  host output of n_labels + 1 entries: tissues 0..n_labels-1,
 *                then the whole body (NaN for a group without voxels).
 *   counts_host  optional host output of n_labels + 1 voxel counts.
 * Allocates scratch on first use (8 bytes per conducting voxel twice, 32 KB
 * per group) and keeps it; synchronises the stream. */
spfd_status spfd_percentile(spfd_ctx *ctx, const double *E_dev, const int32_t *labels_dev,
                            int n_labels, double p, double *values_host,
                            int64_t *counts_host);

/* Several bodies solved together by one launch of a captured CUDA graph.
 *
 * A group holds contexts built for different bodies (for example phantoms of
 * different sizes) and solves Eq. 3 (Sec. II) on all of them at once.  The
 * solve of each context (the same steps as spfd_solve, FP64 or mixed) is
 * captured as one branch of a single graph whose loops run on the GPU: control
 * kernels decide, between iterations, to check the true residual, restart or
 * stop, through the graph's conditional nodes, so the host launches the
 * graph once and synchronises once per group solve.  Each Psi equals what
 * spfd_solve returns for that context, bit for bit, with the same iteration
 * count.  The paper solves one body at a time (Sec. III); grouping is a
 * throughput form of the same solve.
 *
 * spfd_group_create
 *   ctxs    n distinct contexts (1..4096) on one device, of either precision
 *           (a SPFD_MIXED context's branch runs its refinement as nested
 *           device-driven loops).  The group keeps the pointers: destroy the
 *           group before any of its contexts.
 *   stream  cudaStream_t the group launches on (NULL = legacy default
 *           stream); work already queued on the contexts' streams runs
 *           first.
 * spfd_group_solve
 *   a_devs    n device pointers, a_devs[i] laid out as in spfd_solve for
 *             context i.
 *   tol       relative residual target (> 0), or <= 0 for each context's
 *             opts.tol; maxit is each context's opts.maxit.
 *   psi_devs  n device outputs, laid out as in spfd_solve.
 *   infos     optional array of n reports (ms_solve: the whole group).
 *   The first call captures and instantiates the graph (milliseconds);
 *   later calls only point its input and output nodes at the new arrays.  A
 *   call also captures again after a context has reallocated its solve
 *   buffers (e.g. a larger spfd_solve_batch).  Contexts must not be used on
 *   other streams while a group solve runs.  Synchronises.  Returns
 *   SPFD_ENOTCONVERGED (every Psi written) if any body missed tol and
 *   SPFD_EINVAL if any a is non-finite on a conducting edge.
 * spfd_group_destroy  releases the graph, streams and events; NULL is a
 *   no-op. */
typedef struct spfd_group spfd_group;
spfd_status spfd_group_create(spfd_ctx *const *ctxs, int n, void *stream, spfd_group **out);
spfd_status spfd_group_solve(spfd_group *group, const double *const *a_devs, double tol,
                             double *const *psi_devs, spfd_info *infos);
void spfd_group_destroy(spfd_group *group);

/* Report of the context (sizes, last solve); does not synchronise. */
spfd_status spfd_get_info(const spfd_ctx *ctx, spfd_info *info);

/* Kernel timing of a context built with opts.profile = 1.
 *   stats  caller array of at least max entries (may be NULL when max = 0).
 *   n      receives the number of families (may exceed max).
 *   reset  1 = clear the accumulated times after copying them out.
 * Synchronises the context's stream.  Algorithmic bytes count each array
 * element a kernel must read or write once (halo re-reads not counted). */
spfd_status spfd_kernel_stats(spfd_ctx *ctx, spfd_kernel_stat *stats, int max,
                              int *n, int reset);

/* Relative residual ||b - A psi||_2 / ||b||_2 of a node potential for the
 * system above (b = -G^T M_k a, A = G^T M_k G, summed over the conducting
 * nodes), computed directly from the voxel grid without a context and
 * without allocating any device memory.  The paper has no counterpart: this
 * is a service for callers that cannot allocate while they check a solution
 * -- processes whose device memory an allocator has reserved up front (a
 * framework's caching allocator, a fixed arena), real-time loops that must
 * not enter the allocator, or code that must not trigger the implicit
 * synchronisation a cudaMalloc or cudaFree can cause.
 *   sigma_dev, a_dev, psi_dev  as in spfd_build / spfd_solve (device, FP64).
 *   nx, ny, nz, h              the voxel grid; at most 134,217,728 nodes
 *                              ((nx+1)(ny+1)(nz+1)), else SPFD_EINVAL.
 *   stream                     cudaStream_t to run on (NULL = default stream);
 *                              it must not be capturing into a CUDA graph:
 *                              the call copies the result to host memory and
 *                              synchronises the stream before it returns.
 *   rel_res                    host output; 0 when b = 0.
 * The partial sums live in one fixed 256 KB device array of the library,
 * which every device that loads the library holds until the process exits.
 * The first call on a device looks up that array's device address (with
 * that device current) and keeps it; a cudaDeviceReset on that device
 * invalidates the kept address, so no call may follow one.  Every call
 * shares the array and it keeps the last call's contents (the counter that
 * must start at zero is cleared by each call): calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  b is not projected, so the value matches spfd_solve's
 * rel_res_true to rounding. */
spfd_status spfd_residual_noalloc(const double *sigma_dev, const double *a_dev,
                                  const double *psi_dev, int nx, int ny, int nz,
                                  double h, void *stream, double *rel_res);

/* Release every resource of the context.  NULL is a no-op.  The context's
 * device buffers are idle once its stream has been synchronised; they go to
 * a process-wide cache (per device) from which later spfd_build calls take
 * blocks of matching size instead of calling cudaMalloc again. */
void spfd_destroy(spfd_ctx *ctx);

/* Gradient of the field energy
 *   J = (1 / Nc) * sum over the Nc conducting voxels v of |E_v|^2,
 *   E_v,d = omega / (4h) * sum over the four d-edges e of v of u_e,
 *   u = a + G Psi
 * (Eq. 1 voxel-averaged as in spfd_efield, without the sqrt), where psi_dev
 * solves Eq. 3 for a_dev (from spfd_solve).  One adjoint solve
 * A lambda = G^T dJ/du with the context's operator, preconditioner and
 * precision gives
 *   dJda_dev[e]      = dJ/du_e - g_e (lambda_head - lambda_tail)   (edges,
 *                      layout of a_dev),
 *   dJdsigma_dev[v]  = h/4 * sum over the 12 edges of v of
 *                      -(lambda_head - lambda_tail) u_e             (voxels,
 *                      layout of sigma; 0 in air),
 * the derivative with respect to the conductivity of each conducting voxel
 * (the set of conducting voxels held fixed).  J_out is host memory;
 * dJda_dev and dJdsigma_dev are caller-owned device arrays.  tol applies to
 * the adjoint solve.  Allocates scratch on first use (3 voxel-grid and 4
 * node-grid arrays) and synchronises the stream.  Returns SPFD_ENOTCONVERGED
 * (with the gradients of the current iterate) when the adjoint solve stops
 * above tol.  Not in the paper: the adjoint of its Eq. 3 / Eq. 1 pipeline. */
spfd_status spfd_energy_grad(spfd_ctx *ctx, const double *a_dev, const double *psi_dev,
                             double omega, double tol, double *J_out, double *dJda_dev,
                             double *dJdsigma_dev, spfd_info *info);

/* One decision of the autotuner of batched solves (not in the paper: launch
 * tuning of this library).  A batched launch covers nk right-hand sides
 * over the bricks of a level in one of three block orders: 0 = the
 * right-hand sides one after the other, 1 = the nk blocks of each brick side
 * by side, so that they share the brick's operator entries through L2,
 * 2 = a tile of 4 right-hand sides per block, which reads the brick's
 * operator entries (27-point stencils, interpolation weights) into registers
 * once for the tile (the 27-point smoother and residual, restriction and
 * prolongation, for batches of 4 or more).  The first spfd_solve_batch of
 * each batch size (with opts.autotune set) times the orders of every batched
 * kernel family on every level and keeps the fastest; results are unchanged
 * whichever is kept. */
typedef struct {
  const char *family;  /* "jacobi_first", "smooth", "residual", "restrict",
                          "prolong" (fine level) or "apply_dot" (static) */
  int level;           /* multigrid level (0 = finest) */
  int nrhs;            /* batch size tuned for */
  int order;           /* the order kept (0, 1 or 2) */
  double ms_order0;    /* mean time of one launch in order 0 */
  double ms_order1;    /* mean time of one launch in order 1 */
  double ms_order2;    /* mean time of one launch in order 2, -1 if not timed */
} spfd_tune_entry;

/* The autotuner's decisions for this context, oldest first.
 *   entries  caller array of at least max entries (may be NULL when max = 0).
 *   n        receives the number of decisions recorded (may exceed max). */
spfd_status spfd_autotune_report(const spfd_ctx *ctx, spfd_tune_entry *entries, int max,
                                 int *n);

/* Give every cached device block back to the driver (cudaFree); the bytes
 * released go to *released if it is not NULL.  Safe at any time: contexts
 * alive keep their own buffers.  A cudaMalloc that fails for lack of memory
 * does the same once before it retries.  Not part of the paper's method:
 * memory management of this library. */
spfd_status spfd_release_cached_memory(size_t *released);

/* This GPU's FP64 fused multiply-add rate, measured (not part of the paper's
 * method: the denominator of the roofline of the library's FP64 kernels,
 * which are bound by the FP64 pipe).  Runs a kernel of independent FMA chains
 * on every resident warp six times and reports the fastest of the last five:
 *   stream   cudaStream_t to run on (NULL = legacy default stream).
 *   tflops   host output: 2 * FMAs / time, in TFLOP/s.
 *   ms       optional host output: that kernel's CUDA-event time.
 * Synchronises the stream. */
spfd_status spfd_fp64_fma_rate(void *stream, double *tflops, double *ms);

/* Thread-local message for the most recent failing call on this thread. */
const char *spfd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPFD_H */
