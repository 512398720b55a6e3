// Solve-path kernels: multigrid V-cycle pieces, fused Krylov updates with
// deterministic grid reductions, right-hand side, Psi scatter and |E|.
//
// Paper: Eq. 3 (Sec. II) is the system; Sec. II-A fixes double precision and
// a relative-residual stopping rule; Eq. 1 with the voxel averaging of
// Sec. III-E gives |E|.  Every kernel here is bandwidth- or FP64-pipe bound;
// none is a dense contraction, so no tensor-core path is used.
#include "spfd_internal.cuh"

namespace spfd {

// --------------------------------------------------------------- conversions
template <typename T> __device__ __forceinline__ T cv(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cv(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cv(__nv_bfloat16 v) {
  return (T)__bfloat162float(v);
}

#define BRICK_PROLOGUE(g)                                              \
  const size_t S = (size_t)(g).nb * BV;                                \
  const int bk = blockIdx.x, t = threadIdx.x;                          \
  const int s = bk * BV + t;                                           \
  const int4 bc = (g).bco[bk];                                         \
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;                \
  (void)S; (void)lx; (void)ly; (void)lz;

// (A x)_s for the 7-point level-0 operator.  FP64: diag*x_s - sum g x_nbr
// (fewest FP64-pipe operations).  FP32 (BF16 or FP32 g): sum g (x_s - x_nbr),
// which is exactly zero on constants, so rounded conductances keep the
// operator positive semidefinite.
template <typename T, typename C>
__device__ __forceinline__ T apply7(const Grid &g, const C *__restrict__ gx,
                                    const T *__restrict__ diag,
                                    const T *__restrict__ x, size_t S, int bk,
                                    int4 bc, int s, int lx, int ly, int lz) {
  int m;
  if constexpr (sizeof(T) == 4) {
    const T xs = x[s];
    T acc = 0;
    m = slot_nb(g, bk, bc, lx, ly, lz, 1, 0, 0);
    if (m >= 0) acc += cv<T>(gx[s]) * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, -1, 0, 0);
    if (m >= 0) acc += cv<T>(gx[m]) * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 1, 0);
    if (m >= 0) acc += cv<T>(gx[S + s]) * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, -1, 0);
    if (m >= 0) acc += cv<T>(gx[S + m]) * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, 1);
    if (m >= 0) acc += cv<T>(gx[2 * S + s]) * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, -1);
    if (m >= 0) acc += cv<T>(gx[2 * S + m]) * (xs - x[m]);
    return acc;
  }
  T acc = diag[s] * x[s];
  m = slot_nb(g, bk, bc, lx, ly, lz, 1, 0, 0);
  if (m >= 0) acc -= cv<T>(gx[s]) * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, -1, 0, 0);
  if (m >= 0) acc -= cv<T>(gx[m]) * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, 1, 0);
  if (m >= 0) acc -= cv<T>(gx[S + s]) * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, -1, 0);
  if (m >= 0) acc -= cv<T>(gx[S + m]) * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, 1);
  if (m >= 0) acc -= cv<T>(gx[2 * S + s]) * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, -1);
  if (m >= 0) acc -= cv<T>(gx[2 * S + m]) * x[m];
  return acc;
}

template <typename T>
__device__ __forceinline__ T apply27(const Grid &g, const T *__restrict__ st,
                                     const T *__restrict__ x, size_t S, int bk,
                                     int4 bc, int s, int lx, int ly, int lz) {
  T acc = 0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    int m = slot_nb(g, bk, bc, lx, ly, lz, dx, dy, dz);
    if (m >= 0) acc += st[(size_t)e * S + s] * x[m];
  }
  return acc;
}

// ------------------------------------------------------------ smoothers
template <typename T, typename C>
__global__ void __launch_bounds__(NT)
k_residual7(Grid g, const C *__restrict__ gx, const T *__restrict__ diag,
            const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ r) {
  BRICK_PROLOGUE(g);
  r[s] = b[s] - apply7<T, C>(g, gx, diag, x, S, bk, bc, s, lx, ly, lz);
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_residual27(Grid g, const T *__restrict__ st, const T *__restrict__ x,
             const T *__restrict__ b, T *__restrict__ r) {
  BRICK_PROLOGUE(g);
  r[s] = b[s] - apply27<T>(g, st, x, S, bk, bc, s, lx, ly, lz);
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_jacobi_first(const T *__restrict__ wdinv, const T *__restrict__ b,
               T *__restrict__ x) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  x[s] = wdinv[s] * b[s];
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_jacobi_first_proj(const T *__restrict__ wdinv, T *__restrict__ b,
                    T *__restrict__ x, const Scalars *sc, double inv_ndof) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const T w = wdinv[s];
  if (w > (T)0) {  // an unknown of level 0
    const T bv = (T)((double)b[s] - sc->rsum * inv_ndof);
    b[s] = bv;
    x[s] = w * bv;
  } else {
    x[s] = (T)0;
  }
}

template <typename T, typename C>
__global__ void __launch_bounds__(NT)
k_jacobi7(Grid g, const C *__restrict__ gx, const T *__restrict__ diag,
          const T *__restrict__ wdinv, const T *__restrict__ xin,
          const T *__restrict__ b, T *__restrict__ xout) {
  BRICK_PROLOGUE(g);
  T r = b[s] - apply7<T, C>(g, gx, diag, xin, S, bk, bc, s, lx, ly, lz);
  xout[s] = xin[s] + wdinv[s] * r;
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_jacobi27(Grid g, const T *__restrict__ st, const T *__restrict__ wdinv,
           const T *__restrict__ xin, const T *__restrict__ b,
           T *__restrict__ xout) {
  BRICK_PROLOGUE(g);
  T r = b[s] - apply27<T>(g, st, xin, S, bk, bc, s, lx, ly, lz);
  xout[s] = xin[s] + wdinv[s] * r;
}

// ------------------------------------------------------------ transfers
// Restriction r_c(I) = sum_d P[d][I] r_f(2I + d)  (P^T, the adjoint of the
// prolongation below).
template <typename T>
__global__ void __launch_bounds__(NT)
k_restrict(Grid gf, Grid gc, const T *__restrict__ P, const T *__restrict__ rf,
           T *__restrict__ bcoarse) {
  BRICK_PROLOGUE(gc);
  const int I = bc.x * 8 + lx, J = bc.y * 8 + ly, K = bc.z * 8 + lz;
  T acc = 0;
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    int n = slot_at(gf, 2 * I + dx, 2 * J + dy, 2 * K + dz);
    if (n >= 0) acc += P[(size_t)d * S + s] * rf[n];
  }
  bcoarse[s] = acc;
}

// Prolongation + correction e_f(n) += sum over the <= 8 coarse parents I of n
// of P[n - 2I][I] e_c(I).
template <typename T>
__global__ void __launch_bounds__(NT)
k_prolong(Grid gf, Grid gc, const T *__restrict__ P, const T *__restrict__ ec,
          T *__restrict__ ef) {
  BRICK_PROLOGUE(gf);
  const size_t Sc = (size_t)gc.nb * BV;
  const int i = bc.x * 8 + lx, j = bc.y * 8 + ly, k = bc.z * 8 + lz;
  const int ox = i & 1, oy = j & 1, oz = k & 1;
  T acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    if ((cx && !ox) || (cy && !oy) || (cz && !oz)) continue;
    // parent index and offset d = n - 2I on each axis
    const int I = (i >> 1) + cx, J = (j >> 1) + cy, K = (k >> 1) + cz;
    const int dx = i - 2 * I, dy = j - 2 * J, dz = k - 2 * K;
    int sc = slot_at(gc, I, J, K);
    if (sc >= 0) acc += P[(size_t)sidx(dx, dy, dz) * Sc + sc] * ec[sc];
  }
  ef[s] += acc;
}

// Coarsest level: x = B^{-1} b on the m listed unknowns (dense, FP64); one
// warp per row.  Unlisted slots must be zero beforehand.
template <typename T>
__global__ void k_coarse_solve(int m, const int *__restrict__ idx,
                               const double *__restrict__ Binv,
                               const T *__restrict__ b, T *__restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const double *row = Binv + (size_t)warp * m;
  double acc = 0.0;
  for (int j = lane; j < m; j += 32) acc += row[j] * (double)b[idx[j]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[idx[warp]] = (T)acc;
}

// ------------------------------------------------------------ launchers
template <typename T, typename C>
void launch_residual7(const Grid &g, const C *gx, const T *diag, const T *x,
                      const T *b, T *r, cudaStream_t st) {
  if (g.nb) k_residual7<T, C><<<g.nb, NT, 0, st>>>(g, gx, diag, x, b, r);
}
template <typename T>
void launch_residual27(const Grid &g, const T *stc, const T *x, const T *b,
                       T *r, cudaStream_t st) {
  if (g.nb) k_residual27<T><<<g.nb, NT, 0, st>>>(g, stc, x, b, r);
}
template <typename T>
void launch_jacobi_first(const Grid &g, const T *wdinv, const T *b, T *x,
                         cudaStream_t st) {
  if (g.nb) k_jacobi_first<T><<<g.nb, NT, 0, st>>>(wdinv, b, x);
}
template <typename T>
void launch_jacobi_first_proj(const Grid &g, const T *wdinv, T *b, T *x,
                              const Scalars *sc, double inv_ndof,
                              cudaStream_t st) {
  if (g.nb) k_jacobi_first_proj<T><<<g.nb, NT, 0, st>>>(wdinv, b, x, sc, inv_ndof);
}
template <typename T, typename C>
void launch_jacobi7(const Grid &g, const C *gx, const T *diag, const T *wdinv,
                    const T *xin, const T *b, T *xout, cudaStream_t st) {
  if (g.nb) k_jacobi7<T, C><<<g.nb, NT, 0, st>>>(g, gx, diag, wdinv, xin, b, xout);
}
template <typename T>
void launch_jacobi27(const Grid &g, const T *stc, const T *wdinv, const T *xin,
                     const T *b, T *xout, cudaStream_t st) {
  if (g.nb) k_jacobi27<T><<<g.nb, NT, 0, st>>>(g, stc, wdinv, xin, b, xout);
}
template <typename T>
void launch_restrict(const Grid &gf, const Grid &gc, const T *P, const T *rf,
                     T *bcoarse, cudaStream_t st) {
  if (gc.nb) k_restrict<T><<<gc.nb, NT, 0, st>>>(gf, gc, P, rf, bcoarse);
}
template <typename T>
void launch_prolong(const Grid &gf, const Grid &gc, const T *P, const T *ec,
                    T *ef, cudaStream_t st) {
  if (gf.nb) k_prolong<T><<<gf.nb, NT, 0, st>>>(gf, gc, P, ec, ef);
}
template <typename T>
void launch_coarse_solve(int m, const int *idx, const double *Binv, const T *b,
                         T *x, cudaStream_t st) {
  if (m <= 0) return;
  const int warps_per_block = 8;
  k_coarse_solve<T><<<(m + warps_per_block - 1) / warps_per_block,
                      32 * warps_per_block, 0, st>>>(m, idx, Binv, b, x);
}

#define INST_T(T)                                                             \
  template void launch_residual27<T>(const Grid &, const T *, const T *,      \
                                     const T *, T *, cudaStream_t);           \
  template void launch_jacobi_first<T>(const Grid &, const T *, const T *,    \
                                       T *, cudaStream_t);                    \
  template void launch_jacobi_first_proj<T>(const Grid &, const T *, T *,     \
                                            T *, const Scalars *, double,     \
                                            cudaStream_t);                    \
  template void launch_jacobi27<T>(const Grid &, const T *, const T *,        \
                                   const T *, const T *, T *, cudaStream_t);  \
  template void launch_restrict<T>(const Grid &, const Grid &, const T *,     \
                                   const T *, T *, cudaStream_t);             \
  template void launch_prolong<T>(const Grid &, const Grid &, const T *,      \
                                  const T *, T *, cudaStream_t);              \
  template void launch_coarse_solve<T>(int, const int *, const double *,      \
                                       const T *, T *, cudaStream_t);
INST_T(double)
INST_T(float)
#define INST_TC(T, C)                                                         \
  template void launch_residual7<T, C>(const Grid &, const C *, const T *,    \
                                       const T *, const T *, T *,             \
                                       cudaStream_t);                         \
  template void launch_jacobi7<T, C>(const Grid &, const C *, const T *,      \
                                     const T *, const T *, const T *, T *,    \
                                     cudaStream_t);
INST_TC(double, double)
INST_TC(float, float)
INST_TC(float, __nv_bfloat16)

}  // namespace spfd
