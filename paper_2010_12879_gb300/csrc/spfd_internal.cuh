// Internal declarations shared by the translation units of libspfd.
//
// Data layout.  Every multigrid level stores its node unknowns in 8x8x8-node
// bricks; only bricks that touch an unknown are allocated.  A level is
// described by its node dimensions (NX, NY, NZ), its brick-grid dimensions
// (MX, MY, MZ), a dense brick map [MZ][MY][MX] -> brick id (or -1) and the
// brick coordinates of each active brick.  Node (lx, ly, lz) of brick b lives
// at slot b*512 + (lz*8 + ly)*8 + lx of every per-node array.  Slots of nodes
// that are not unknowns (air, or past the grid edge) hold zero operator rows
// and zero vector entries, so kernels never branch on activity for
// correctness.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

namespace spfd {

constexpr int BE = 8;     // brick edge in nodes
constexpr int BV = 512;   // nodes per brick
constexpr int NT = 512;   // threads per brick-kernel block (one node each)

// Programmatic dependent launch.  The solve's kernels (the V-cycle, the
// Krylov updates and reductions) are launched by pdl() with programmatic
// stream serialization allowed: a kernel's blocks may be scheduled on the
// SMs while its predecessor on the stream is still finishing, which hides
// the launch gap between the solve's many short dependent kernels.  Every
// kernel launched that way calls pdl_entry() before it touches global
// memory: griddepcontrol.wait holds it until the predecessor grid has
// completed and its writes are visible (it returns at once for a kernel
// launched without the attribute), and griddepcontrol.launch_dependents
// then lets the next kernel's blocks be scheduled as this grid's blocks
// retire.  Every read and write thus happens in the order of plain stream
// launches, and results are unchanged bit for bit.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Whether pdl() sets the attribute on this host thread (cleared while a
// graph is captured: the captured solves launch from the graph, with no
// host gaps to hide).
extern thread_local bool pdl_allowed;
// pdl(kernel, grid, block, stream)(args...) launches kernel<<<grid, block,
// 0, stream>>>(args...) with programmatic stream serialization; the kernel
// must begin with pdl_entry().
template <typename... P>
struct PdlLaunch {
  void (*k)(P...);
  dim3 grid, block;
  cudaStream_t st;
  template <typename... A>
  cudaError_t operator()(A &&...args) const {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl_allowed ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
  }
};
template <typename... P>
inline PdlLaunch<P...> pdl(void (*k)(P...), dim3 grid, dim3 block, cudaStream_t st) {
  return PdlLaunch<P...>{k, grid, block, st};
}

// Stencil offset index of (dx, dy, dz) in {-1,0,1}^3; 13 is the centre.
__host__ __device__ __forceinline__ constexpr int sidx(int dx, int dy, int dz) {
  return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}

// First per-cell prolongation weight of parity class q (node 2c + u of a
// 2x2x2 cell, q = uz*4 + uy*2 + ux): sum over q' < q of 2^popcount(q').
__host__ __device__ __forceinline__ constexpr int pc_off(int q) {
  return q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 3 : q == 3 ? 5 : q == 4 ? 9
       : q == 5 ? 11 : q == 6 ? 15 : 19;
}

// Position of parent o among the parents o' <= u (bit sets) in ascending
// order: parent o of a class-u node is weight pc_off(u) + crank(u, o) of its
// cell.
__host__ __device__ __forceinline__ constexpr int crank(int u, int o) {
  int r = 0;
  for (int c = 0; c < o; ++c) r += (c & ~u) == 0;
  return r;
}

// Block order of a batched launch (nk right-hand sides over units of one
// or two bricks).  Order 0: blockIdx.x is the unit and blockIdx.y the
// right-hand side, so the right-hand sides run one after the other.  Order 1
// (a one-dimensional grid): block b covers unit b / nk of right-hand side
// b % nk, so the nk blocks of one unit run side by side and share its
// operator entries through L2.  The arithmetic of every block is the same
// in both orders; the autotuner picks one per kernel family and level.
// Order 2 (the 27-point smoother and residual, restriction, prolongation): a
// right-hand-side tile, blockIdx.y selects RHS_TILE consecutive right-hand
// sides that one block handles in turn with the unit's operator entries held
// in registers, so they are read from memory once per tile; rhs is then the
// tile's first.  Per right-hand side the arithmetic is again the same.
// The order is a template parameter, so that the order-0 instances compile to
// the same code as kernels without a batch order.
constexpr int RHS_TILE = 4;
template <int ORD>
constexpr int rhs_tile() { return ORD == 2 ? RHS_TILE : 1; }
template <int ORD>
__device__ __forceinline__ void unit_rhs(int nk, int &unit, int &rhs) {
  if constexpr (ORD == 1) {
    unit = (int)(blockIdx.x / (unsigned)nk);
    rhs = (int)(blockIdx.x % (unsigned)nk);
  } else if constexpr (ORD == 2) {
    unit = (int)blockIdx.x;
    rhs = (int)blockIdx.y * RHS_TILE;
  } else {
    unit = (int)blockIdx.x;
    rhs = (int)blockIdx.y;
  }
}
inline dim3 unit_grid(int order, int units, int nk) {
  if (order == 2) return dim3((unsigned)units, (unsigned)((nk + RHS_TILE - 1) / RHS_TILE));
  return order ? dim3((unsigned)units * (unsigned)nk) : dim3((unsigned)units, (unsigned)nk);
}
// Order 1 is available while units * nk fits a one-dimensional grid.
inline bool order1_fits(int units, int nk) {
  return (long long)units * nk <= 2147483647LL;
}

struct Grid {
  int NX, NY, NZ;       // nodes per axis
  int MX, MY, MZ;       // bricks per axis
  int nb;               // active bricks
  const int *bmap;      // [MZ][MY][MX] brick id or -1
  const int4 *bco;      // [nb] brick coordinates (x, y, z, 0)
  const int *nbr;       // [nb][27] ids of the bricks at offset sidx(dx,dy,dz), or -1
  const int *kid;       // coarse levels: [nb][27] ids of the finer-level bricks
                        //   2B + (o - 1), o in {0,1,2}^3 (index o.z*9+o.y*3+o.x), or -1
  const int *par;       // levels with a coarser level: [nb][8] ids of the coarser
                        //   bricks (B >> 1) + o, o in {0,1}^3 (index o.z*4+o.y*2+o.x), or -1
  const unsigned *act;  // levels >= 1: [nb][16], bit t of word w is set when slot
                        //   b*512 + 32w + t has a nonzero column of the interpolation
                        //   from the finer level, which every nonzero Galerkin row and
                        //   every nonzero restricted value needs; a clear bit
                        //   guarantees a zero 27-point row and a zero restriction
                        //   weight column (level 0: unused)
};


// The activity bits (Grid::act) of this thread's warp on brick bk, one node
// per thread: bit (thread & 31) is this thread's slot.
__device__ __forceinline__ unsigned act_word(const Grid &g, int bk) {
  return __ldg(&g.act[(size_t)bk * 16 + (threadIdx.x >> 5)]);
}

// The bit pattern of an FP64 value, through an opaque move: the compiler
// would otherwise fold integer tests of the bits back into FP64 comparisons,
// and on GB300 each of those takes a slot of the narrow FP64 pipe.
__device__ __forceinline__ unsigned long long f64_bits(double x) {
  unsigned long long u;
  asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
  return u;
}
// x is not +-0 (for x known to be +-0 or positive: x > 0), from its bits.
__device__ __forceinline__ bool f64_nonzero(double x) { return (f64_bits(x) << 1) != 0ull; }
// x is infinite or NaN, from its bits.
__device__ __forceinline__ bool f64_nonfinite(double x) {
  return ((f64_bits(x) >> 52) & 0x7ffull) == 0x7ffull;
}
// w > 0 for a non-negative weight w: a bit test in FP64, a comparison in FP32.
template <typename T>
__device__ __forceinline__ bool weight_pos(T w) {
  if constexpr (sizeof(T) == 8) return f64_nonzero(w);
  else return w > T(0);
}

// An FP64 value (bits u) rounded to nearest even to the format with 8
// exponent bits and P stored significand bits: binary32 (P = 23) or bfloat16
// (P = 7), returned as that format's bits.  Integer operations only, from
// the IEEE 754 encodings: GB300 issues its hardware conversions from FP64 on
// the narrow FP64 pipe, which the kernels running beside the build's
// conversions need.  Overflow gives infinity, NaN stays a (quiet) NaN, and
// results below the smallest normal are subnormal or zero, as the hardware
// conversion gives them.
template <int P>
__host__ __device__ __forceinline__ unsigned narrow_f64_bits(unsigned long long u) {
  constexpr int D = 52 - P;  // dropped significand bits of a normal result
  const unsigned sign = (unsigned)(u >> 63) << (8 + P);
  const int e = (int)((u >> 52) & 0x7ff);
  const unsigned long long m = u & ((1ull << 52) - 1ull);
  constexpr unsigned INF = 0xffu << P;
  if (e == 0x7ff) return sign | INF | (m ? ((1u << (P - 1)) | (unsigned)(m >> D)) : 0u);
  const int E = e - 896;  // the target's biased exponent (bias 127 against 1023)
  if (E >= 0xff) return sign | INF;
  unsigned long long sig, q;
  int shift;
  if (E > 0) {
    sig = m;
    shift = D;
  } else {  // subnormal target: units of 2^(-126 - P)
    sig = (e ? (1ull << 52) : 0ull) | m;
    shift = 949 - P - (e ? e : 1);
    if (shift >= 64) return sign;
  }
  q = sig >> shift;
  const unsigned long long rem = sig & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  // a carry out of the significand moves into the exponent field, as it should
  return sign | ((E > 0 ? (unsigned)E << P : 0u) + (unsigned)q);
}

// Active-slot compaction of one brick of a 27-point level.  The block that
// handles brick bk gives its n-th thread the brick's n-th active slot (set
// activity bit, in slot order), so warps past the brick's active count skip
// the stencil arithmetic: a warp instruction occupies the FP64 pipe whatever
// its lane mask, so only warps with no active slot save FP64 time.  FP64
// kernels use it; FP32 ones, bound by memory, keep one slot per thread.
template <typename T>
constexpr bool compact27() { return sizeof(T) == 8; }

struct ActList {
  unsigned w[16];  // the brick's activity words
  int pre[17];     // exclusive prefix counts of w; pre[16] = active slots
};

// Warp 0 stages brick bk's words and prefix counts (a barrier must follow
// before any thread reads them).
__device__ __forceinline__ void act_stage(const Grid &g, int bk, ActList &al) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned w = lane < 16 ? __ldg(&g.act[(size_t)bk * 16 + lane]) : 0u;
    const int c = __popc(w);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane < 16) {
      al.w[lane] = w;
      al.pre[lane] = incl - c;
    }
    if (lane == 15) al.pre[16] = incl;
  }
}

// Local slot (0..511) of the brick's n-th active slot, n < al.pre[16].
__device__ __forceinline__ int act_slot(const ActList &al, int n) {
  int j = 0;  // the last word whose prefix count is <= n (it holds slot n)
#pragma unroll
  for (int step = 8; step > 0; step >>= 1)
    if (al.pre[j + step] <= n) j += step;
  unsigned w = al.w[j];
  int k = n - al.pre[j], pos = 0;  // the k-th set bit of w, by halving
#pragma unroll
  for (int width = 16; width > 0; width >>= 1) {
    const unsigned lo = w & ((1u << width) - 1u);
    const int c = __popc(lo);
    if (k >= c) {
      k -= c;
      w >>= width;
      pos += width;
    } else {
      w = lo;
    }
  }
  return j * 32 + pos;
}

// Whether local slot t of the staged brick is active.
__device__ __forceinline__ bool act_on(const ActList &al, int t) {
  return (al.w[t >> 5] >> (t & 31)) & 1u;
}

// Brick id of node (i, j, k) or -1 (outside the grid or brick not stored).
__device__ __forceinline__ int brick_at(const Grid &g, int i, int j, int k) {
  if ((unsigned)i >= (unsigned)g.NX || (unsigned)j >= (unsigned)g.NY ||
      (unsigned)k >= (unsigned)g.NZ)
    return -1;
  return __ldg(&g.bmap[((k >> 3) * g.MY + (j >> 3)) * g.MX + (i >> 3)]);
}

// Slot of node (i, j, k) or -1.
__device__ __forceinline__ int slot_at(const Grid &g, int i, int j, int k) {
  int b = brick_at(g, i, j, k);
  if (b < 0) return -1;
  return (b << 9) | ((k & 7) << 6) | ((j & 7) << 3) | (i & 7);
}

// Slot of the neighbour (lx+dx, ly+dy, lz+dz) of a node of brick b at brick
// coordinates bc; inside the brick it is pure arithmetic.
__device__ __forceinline__ int slot_nb(const Grid &g, int b, int4 bc, int lx,
                                       int ly, int lz, int dx, int dy, int dz) {
  int x = lx + dx, y = ly + dy, z = lz + dz;
  if ((unsigned)(x | y | z) < 8u) return (b << 9) | (z << 6) | (y << 3) | x;
  return slot_at(g, bc.x * 8 + x, bc.y * 8 + y, bc.z * 8 + z);
}

// Device scalars of the Krylov loop, reduction scratch and status flags.
struct Scalars {
  double bb;        // ||b||^2
  double rr;        // ||r||^2
  double rz;        // r . z
  double rz_old;
  double pq;        // p . A p
  double alpha, beta;
  double zsum;      // sum of z over the single component (projection)
  double rsum;      // sum of r over the unknowns (projection of r)
  double inv_ndof;  // 1 / (number of unknowns), set by the build
  double zmean, rmean;  // zsum / n, rsum / n (formed once by the last block)
  float alpha_f, beta_f, zmean_f, rmean_f;  // FP32 copies for FP32 kernels
  double aux[8];    // misc results (power iteration, refinement)
  unsigned long long ustat[2];  // count of positive entries, max entry (bits)
  unsigned int ticket[8];  // last-block counters, one per reduction site
  int status;       // SPFD_DEV_* bits
  int frozen;       // batched solves: this right-hand side has stopped
  int restart;      // batched solves: the next beta of this right-hand side is 0
};

enum : int {
  DEV_BAD_SIGMA = 1,     // NaN / negative / infinite conductivity
  DEV_BAD_A = 2,         // non-finite edge potential on a conducting edge
  DEV_UF_CAP = 4,        // union-find loop hit its iteration cap
  DEV_BAD_PIVOT = 8,     // coarsest dense inverse met a non-positive pivot
  DEV_GRID_WAIT = 16,    // a grid-wide barrier hit its wait cap
};

// Grid-wide barrier of a cooperative launch (all blocks resident): arrive
// on a counter, the last block to arrive resets it and advances the
// generation, the others wait for the generation to change.  count and gen
// start at zero and are left so after every barrier, so one pair serves
// every launch on a stream.  The wait is bounded: after GRID_SPIN_LIMIT
// polls (far beyond any real wait) it sets DEV_GRID_WAIT and goes on, so the
// caller fails with an error instead of hanging.  (Polling gen with acquire
// loads and a shorter sleep instead of atomics made the coarsest inverse
// slower.)
constexpr long long GRID_SPIN_LIMIT = 1LL << 22;

__device__ __forceinline__ void grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks,
                                             int *status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = atomicAdd(gen, 0u);
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long spins = 0;
      while (atomicAdd(gen, 0u) == g) {
        if (++spins > GRID_SPIN_LIMIT) {
          atomicOr(status, DEV_GRID_WAIT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// ---------------------------------------------------------------- launchers
// Setup (spfd_setup.cu)
void launch_sigma_flags(const double *sigma, int nx, int ny, int nz, int MX,
                        int MY, unsigned char *flags, unsigned char *mask,
                        int *status, cudaStream_t st);
void launch_build_fine(const Grid &g, const double *sigma, int nx, int ny,
                       int nz, double h, double *gx, double *diag,
                       double *dinv, cudaStream_t st);
void launch_components(const Grid &g, const double *gx, int *parent,
                       int *status, cudaStream_t st);
void launch_root_counts(const Grid &g, const int *parent, int *counts,
                        cudaStream_t st);
void launch_assign_comp(const Grid &g, const int *parent, const int *offsets,
                        int *comp, cudaStream_t st);
// dst (device, 16-byte aligned) = bytes of src_mapped, pinned host memory
// mapped into the device's address space (16-byte aligned), read by the SMs.
void launch_pull(void *dst, const void *src_mapped, size_t bytes, cudaStream_t st);
// *p = v on the device.
void launch_set_f64(double *p, double v, cudaStream_t st);
// Brick tables from the brick maps and coordinates already on the device:
// nbr [nb][27] of level g; kid [gc.nb][27] of coarse level gc (fine bricks of
// level gf); par [gf.nb][8] of fine level gf (coarse bricks of level gc).
void launch_brick_nbr(const Grid &g, int *nbr, cudaStream_t st);
void launch_brick_kid(const Grid &gf, const Grid &gc, int *kid, cudaStream_t st);
void launch_brick_par(const Grid &gf, const Grid &gc, int *par, cudaStream_t st);
void launch_comp_sizes(const Grid &g, const int *comp, int *sizes,
                       cudaStream_t st);
// Multigrid hierarchy (spfd_hierarchy.cu).  Pc: the fine level's compact
// per-cell interpolation weights, [27][S/8] (row pc_off(q) + j, column
// brick*64 + cell).  T: scratch for the product A P, [ap_rows_per_cell()][S/8].
// stc / P: the coarse level's 27 Galerkin coefficients and 27 per-coarse-node
// transfer weights ([d][I] = P(2I + d, I)), [27][Sc] each.
int ap_rows_per_cell();
void launch_interp_weights(const Grid &gf, const double *gx, const double *st27,
                           const double *diag, double *Pc, cudaStream_t st);
// act: the coarse level's activity bits ([gc.nb][16], see Grid::act), written
// with P.
void launch_galerkin(const Grid &gf, const Grid &gc, const double *gx,
                     const double *st27f, const double *diagf, const double *Pc,
                     double *T, double *stc, double *P, unsigned *act, cudaStream_t st);
// ustat[0] += number of entries > 0 of d[0..n), ustat[1] = max(ustat[1], bits
// of the largest entry) (non-negative doubles order like their bit patterns).
void launch_diag_stats(const double *d, size_t n, unsigned long long *ustat,
                       cudaStream_t st);
// diag = stc's centre coefficient where it exceeds rel * (the double whose
// bits are *maxbits, as written by launch_diag_stats), else 0; dinv = 1/diag.
void launch_coarse_diag(const Grid &gc, const double *stc, const unsigned long long *maxbits,
                        double rel, double *diag, double *dinv, cudaStream_t st);
// The coarsest level's dense matrix A (m x m, zeroed beforehand) from its
// operator op (27-point stencil if k27, else 7-point conductances with
// diag), then, if cc is given, the component shifts mu[cc] and the diagonal
// shift (see setup_coarsest).
void launch_coarse_dense(const Grid &g, const double *op, bool k27, size_t S, const double *diag,
                         const int *idx, const int *rowof, int m, const int *cc,
                         const double *mu, double shift, double *A, cudaStream_t st);
// Inverse of the SPD matrix in buf0 (m x m, row-major) by blocked
// Gauss-Jordan sweeps; returns buf0 or buf1, whichever holds the result.
// bar: two zeroed unsigned ints.
double *launch_dense_inverse(double *buf0, double *buf1, int m, int *status, unsigned *bar,
                             cudaStream_t st);
int dense_inverse_launches(int m);

// V-cycle pieces (spfd_cycle.cu); T = vector type, C = 7-point coefficient type.
// nk right-hand sides per launch (blockIdx.y): the vectors of a level with S
// slots are nk consecutive blocks of S values; operators are shared.
template <typename T, typename C>
void launch_residual7(const Grid &g, const C *gx, const T *diag, const T *x,
                      const T *b, T *r, cudaStream_t st, int nk = 1, int order = 0);
template <typename T>
void launch_residual27(const Grid &g, const T *stc, const T *x, const T *b,
                       T *r, cudaStream_t st, int nk = 1, int order = 0);
template <typename T>
void launch_jacobi_first(const Grid &g, const T *wdinv, const T *b, T *x,
                         cudaStream_t st, int nk = 1, int order = 0);
// First level-0 sweep with the projection of the right-hand side fused in:
// b <- b - (sum b)/n on the unknowns (one component), then x = wdinv * b;
// sc holds one Scalars per right-hand side.
template <typename T>
void launch_jacobi_first_proj(const Grid &g, const T *wdinv, T *b, T *x,
                              const Scalars *sc, double inv_ndof,
                              cudaStream_t st, int nk = 1, int order = 0);
template <typename T, typename C>
void launch_jacobi7(const Grid &g, const C *gx, const T *diag, const T *wdinv,
                    const T *xin, const T *b, T *xout, cudaStream_t st, int nk = 1,
                    int order = 0);
// The same sweep as the last one of the V-cycle on level 0 (b = r, xout =
// z): also writes 2 partials (r.z, sum of z over the unknowns) per warp,
// jacobi7_rz_partials(nb) pairs per right-hand side, for launch_finish_rz.
template <typename T, typename C>
void launch_jacobi7_rz(const Grid &g, const C *gx, const T *diag, const T *wdinv,
                       const T *xin, const T *b, T *xout, double *partials, size_t pstride,
                       cudaStream_t st, int nk = 1, int order = 0);
template <typename T> int jacobi7_rz_partials(int nb);
// Adds n pairs of partials (scratch: at least 304 doubles, not overlapping)
// and sets rz, beta, zsum and zmean as launch_dot_rz does.
// pairs: the partials are FP32 (hi, lo) pairs (FP32 producers).
void launch_finish_rz(int n, const double *partials, double *scratch, Scalars *sc, int first,
                      cudaStream_t st, int nk = 1, size_t pstride = 0, bool pairs = false);
template <typename T>
void launch_jacobi27(const Grid &g, const T *stc, const T *wdinv, const T *xin,
                     const T *b, T *xout, cudaStream_t st, int nk = 1, int order = 0);
template <typename T>
void launch_restrict(const Grid &gf, const Grid &gc, const T *P, const T *rf,
                     T *bc, cudaStream_t st, int nk = 1, int order = 0);
template <typename T>
void launch_prolong(const Grid &gf, const Grid &gc, const T *P, const T *ec,
                    T *ef, cudaStream_t st, int nk = 1, int order = 0);
// One Chebyshev smoothing step on a level of S slots (nk right-hand sides,
// S apart): d = c1 d + c2w wdinv r, x += d; first (from a zero guess, r = b):
// d = c2w wdinv b, x = d.
template <typename T>
void launch_cheb(bool first, size_t S, const T *wdinv, const T *r, T *d, T *x, double c1,
                 double c2w, cudaStream_t st, int nk = 1);
// One Chebyshev step fused with its residual r = b - A xin:
// d = c1 d + c2w wdinv r, xout = xin + d (level 0: 7-point, conductances C;
// coarse levels: 27-point).
template <typename T, typename C>
void launch_cheb7(const Grid &g, const C *gx, const T *diag, const T *wdinv, const T *xin,
                  const T *b, T *xout, T *d, double c1, double c2w, cudaStream_t st,
                  int nk = 1);
template <typename T>
void launch_cheb27(const Grid &g, const T *stc, const T *wdinv, const T *xin, const T *b,
                   T *xout, T *d, double c1, double c2w, cudaStream_t st, int nk = 1);
// x[idx] = Binv b[idx] on the coarsest level (S slots per right-hand side).
template <typename T>
void launch_coarse_solve(int m, size_t S, const int *idx, const double *Binv,
                         const T *b, T *x, cudaStream_t st, int nk = 1);

// Krylov loop, RHS, scatter, |E| (spfd_krylov.cu).  nk right-hand sides per
// launch (blockIdx.y): level-0 vectors are nk blocks of S0 values, sc points
// at nk consecutive Scalars, partials at nk regions pstride apart, csum at nk
// blocks of ncomp sums; edge and node-grid arrays are nk blocks of 3 NN / NN.
template <typename T>
void launch_apply_dot(const Grid &g, const T *gx, const T *diag, const T *p,
                      T *q, Scalars *sc, double *partials, cudaStream_t st, int nk = 1,
                      size_t pstride = 0, int order = 0);
// Number of partial sums launch_apply_dot writes for nb bricks (one per warp,
// 8 per brick in FP64, 4 in FP32, where each is an FP32 (hi, lo) pair in its
// 8-byte slot); launch_finish_pq adds n of them (scratch: at least 152
// doubles, not overlapping; pairs for FP32 partials) and sets alpha = rz / pq.
template <typename T> int apply_dot_partials(int nb);
void launch_finish_pq(int n, const double *partials, double *scratch, Scalars *sc,
                      cudaStream_t st, int nk = 1, size_t pstride = 0, bool pairs = false);
// x += alpha p, r -= alpha q, r.r, sum r; right-hand sides whose Scalars are
// frozen are left as they are.
template <typename T>
void launch_update_xr(int nb, T *x, T *r, const T *p, const T *q, Scalars *sc,
                      double *partials, cudaStream_t st, int nk = 1, size_t pstride = 0);
// r.z and beta (0 when first, or when the right-hand side's restart flag is
// set; the flag is cleared).
template <typename T>
void launch_dot_rz(int nb, const T *r, const T *z, const int *comp,
                   Scalars *sc, double *partials, int first, cudaStream_t st, int nk = 1,
                   size_t pstride = 0);
// Per-component sums of v (several components), exact and order-independent:
// ws is a workspace of cstride >= 3 ncomp + 1 doubles per right-hand side
// (zeroed here), whose first ncomp entries receive the sums.  Four launches.
template <typename T>
void launch_comp_sum(int nb, const T *v, const int *comp, double *ws, int ncomp,
                     int cstride, cudaStream_t st, int nk = 1);
template <typename T>
void launch_pupdate(int nb, T *p, const T *z, const int *comp,
                    const Scalars *sc, const double *csum, const int *csize,
                    double inv_ndof, cudaStream_t st, int nk = 1, int cstride = 0);
template <typename T>
void launch_sub_mean(int nb, T *v, const int *comp, const Scalars *sc,
                     int aux_slot, const double *csum, const int *csize,
                     double inv_ndof, cudaStream_t st, int nk = 1, int cstride = 0);
template <typename T>
void launch_dot(int nb, const T *x, const T *y, const int *comp, Scalars *sc,
                double *partials, int slot, cudaStream_t st, int nk = 1, size_t pstride = 0);
template <typename T>
void launch_scatter(const Grid &g, const T *x, const int *comp, double *psi,
                    cudaStream_t st, int nk = 1);
void launch_rhs(const Grid &g, const double *gx, const double *a, double *b,
                int *status, cudaStream_t st, int nk = 1);
void launch_gather(const Grid &g, const double *psi, const int *comp, double *x,
                   cudaStream_t st);
// Adjoint of J = mean over conducting voxels of |E|^2 (spfd_krylov.cu).
// Ev: [3][nx*ny*nz] scratch; gJ, dJda: [3][NN]; lam: node grid; dJds: voxels.
void launch_energy(const unsigned char *mask, const double *a, const double *psi, int nx,
                   int ny, int nz, double c, double *Ev, Scalars *sc, double *partials,
                   cudaStream_t st);
void launch_energy_gJ(const unsigned char *mask, const double *Ev, int nx, int ny, int nz,
                      double c, const Scalars *sc, double *gJ, cudaStream_t st);
void launch_div_brick(const Grid &g, const double *diag, const double *gJ, double *b,
                      cudaStream_t st);
void launch_energy_grads(const Grid &g, const double *gx, const unsigned char *mask,
                         const double *a, const double *psi, const double *lam,
                         const double *gJ, int nx, int ny, int nz, double h, double *dJda,
                         double *dJds, cudaStream_t st);
void launch_efield(const unsigned char *mask, const double *a,
                   const double *psi, int nx, int ny, int nz, double h,
                   double omega, double *E, cudaStream_t st);
// E = sqrt(E^2 + E_im^2) elementwise over n values (16-byte aligned arrays).
void launch_efield_magnitude(size_t n, double *E, const double *E_im, cudaStream_t st);
template <typename T>
void launch_convert(size_t n, const double *src, double f, T *dst,
                    cudaStream_t st);
// x += f d (f from *fdev when fdev is not null: device-driven solves).
void launch_axpy_mixed(int nb, double *x, const float *d, double f,
                       cudaStream_t st, const double *fdev = nullptr);
// r32 = (float)(f r), sum(r32) into sc (f from *fdev when fdev is not null).
void launch_scale_to_f32(int nb, const double *r, double f, float *r32,
                         Scalars *sc, double *partials, cudaStream_t st,
                         const double *fdev = nullptr);
// One step w = D^-1 A v of the power iteration on a 27-point level, in FP32
// on FP32 copies of the coefficients and the inverse diagonal; sc->aux[4] =
// v.(A v), sc->aux[5] = v.(D v) (D from the centre coefficient), summed in FP64.
void launch_power_init_f32(int nb, const float *dinv, float *v, cudaStream_t st);
void launch_power27_f32(const Grid &g, const float *st27, const float *dinv, const float *v,
                        float *w, Scalars *sc, double *partials, cudaStream_t st);
void launch_scale(int nb, double *v, double f, cudaStream_t st);
// Jacobi weights of a 27-point level from its power iteration: lambda =
// sc->aux[4] / sc->aux[5] (2 if not a positive number), omega = 4 / (3 margin
// lambda), wdinv = omega * dinv; *lam_out = lambda.
void launch_jacobi_weights(int nb, const double *dinv, const Scalars *sc, double margin,
                           double *wdinv, double *lam_out, cudaStream_t st);
void launch_scaled_copy(int nb, const double *src, double f, double *dst,
                        cudaStream_t st);

}  // namespace spfd
