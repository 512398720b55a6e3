// Krylov-loop kernels with fused, deterministic grid reductions; the
// right-hand side of Eq. 3, the Psi scatter and the |E| of Eq. 1.
//
// Every reduction here finishes on the device: each block writes its partial
// sums, and the last block to arrive (ticket counter) adds the partials in a
// fixed order and updates the Krylov scalars in place, so the loop needs no
// host round trip except the convergence test.
#include "spfd_internal.cuh"

namespace spfd {

// ------------------------------------------------------------ reductions
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sm[32][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[w][k] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? sm[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
  }
  __syncthreads();
}

// Returns true in thread 0 of the last block, with tot[] = grid totals.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *partials, unsigned *ticket,
                         double (&tot)[NV]) {
  __shared__ bool last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned prev = atomicAdd(ticket, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double a[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) a[k] = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] += __ldcg(&partials[(size_t)i * NV + k]);
  block_sum<NV>(a);
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = a[k];
  *ticket = 0u;
  return true;
}

#define BRICK_PROLOGUE(g)                                              \
  const size_t S = (size_t)(g).nb * BV;                                \
  const int bk = blockIdx.x, t = threadIdx.x;                          \
  const int s = bk * BV + t;                                           \
  const int4 bc = (g).bco[bk];                                         \
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;                \
  (void)S; (void)lx; (void)ly; (void)lz; (void)bc;

template <typename T>
__device__ __forceinline__ T apply7k(const Grid &g, const T *__restrict__ gx,
                                     const T *__restrict__ diag,
                                     const T *__restrict__ x, size_t S, int bk,
                                     int4 bc, int s, int lx, int ly, int lz) {
  int m;
  if constexpr (sizeof(T) == 4) {  // difference form: exactly zero on constants
    const T xs = x[s];
    T acc = 0;
    m = slot_nb(g, bk, bc, lx, ly, lz, 1, 0, 0);
    if (m >= 0) acc += gx[s] * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, -1, 0, 0);
    if (m >= 0) acc += gx[m] * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 1, 0);
    if (m >= 0) acc += gx[S + s] * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, -1, 0);
    if (m >= 0) acc += gx[S + m] * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, 1);
    if (m >= 0) acc += gx[2 * S + s] * (xs - x[m]);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, -1);
    if (m >= 0) acc += gx[2 * S + m] * (xs - x[m]);
    return acc;
  }
  T acc = diag[s] * x[s];
  m = slot_nb(g, bk, bc, lx, ly, lz, 1, 0, 0);
  if (m >= 0) acc -= gx[s] * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, -1, 0, 0);
  if (m >= 0) acc -= gx[m] * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, 1, 0);
  if (m >= 0) acc -= gx[S + s] * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, -1, 0);
  if (m >= 0) acc -= gx[S + m] * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, 1);
  if (m >= 0) acc -= gx[2 * S + s] * x[m];
  m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, -1);
  if (m >= 0) acc -= gx[2 * S + m] * x[m];
  return acc;
}

// q = A p and p.q; the last block sets alpha = rz / pq.
template <typename T>
__global__ void __launch_bounds__(NT)
k_apply_dot(Grid g, const T *__restrict__ gx, const T *__restrict__ diag,
            const T *__restrict__ p, T *__restrict__ q, Scalars *sc,
            double *partials) {
  BRICK_PROLOGUE(g);
  T qs = apply7k<T>(g, gx, diag, p, S, bk, bc, s, lx, ly, lz);
  q[s] = qs;
  double v[1] = {(double)p[s] * (double)qs};
  double tot[1];
  if (grid_sum<1>(v, partials, &sc->ticket[0], tot)) {
    sc->pq = tot[0];
    sc->alpha = tot[0] > 0.0 ? sc->rz / tot[0] : 0.0;
  }
}

// x += alpha p; r -= alpha q; rr = r.r
template <typename T>
__global__ void __launch_bounds__(NT)
k_update_xr(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
            const T *__restrict__ q, Scalars *sc, double *partials) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const T alpha = (T)sc->alpha;
  x[s] += alpha * p[s];
  T rs = r[s] - alpha * q[s];
  r[s] = rs;
  // removed nodes hold r = 0, so the plain sum is the sum over the unknowns
  double v[2] = {(double)rs * (double)rs, (double)rs};
  double tot[2];
  if (grid_sum<2>(v, partials, &sc->ticket[1], tot)) {
    sc->rr = tot[0];
    sc->rsum = tot[1];
  }
}

// rz = r.z (new), beta = rz/rz_old, zsum = sum of z over the unknowns.
template <typename T>
__global__ void __launch_bounds__(NT)
k_dot_rz(const T *__restrict__ r, const T *__restrict__ z,
         const int *__restrict__ comp, Scalars *sc, double *partials,
         int first) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const double zs = (double)z[s];
  double v[2] = {(double)r[s] * zs, comp[s] >= 0 ? zs : 0.0};
  double tot[2];
  if (grid_sum<2>(v, partials, &sc->ticket[2], tot)) {
    double old = sc->rz;
    sc->rz_old = old;
    sc->rz = tot[0];
    sc->beta = (first || old == 0.0) ? 0.0 : tot[0] / old;
    sc->zsum = tot[1];
  }
}

// Per-component sums of v over the unknowns (several components): lanes that
// share a component are combined before one atomic per group.
template <typename T>
__global__ void __launch_bounds__(NT)
k_comp_sum(const T *__restrict__ v, const int *__restrict__ comp, double *csum) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const int c = comp[s];
  const unsigned grp = __match_any_sync(0xffffffffu, c);
  double x = c >= 0 ? (double)v[s] : 0.0;
  // sum within the group: walk the set bits (at most 32)
  double tot = 0.0;
  unsigned m = grp;
  while (m) {
    int src = __ffs(m) - 1;
    tot += __shfl_sync(grp, x, src);
    m &= m - 1;
  }
  if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&csum[c], tot);
}

// p = (z - mean_c(z)) + beta p on the unknowns.  With one component the mean
// comes from sc->zsum; otherwise from csum[c] / csize[c].
template <typename T>
__global__ void __launch_bounds__(NT)
k_pupdate(T *__restrict__ p, const T *__restrict__ z,
          const int *__restrict__ comp, const Scalars *sc,
          const double *__restrict__ csum, const int *__restrict__ csize,
          double inv_ndof) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const int c = comp[s];
  if (c < 0) { p[s] = (T)0; return; }
  const double mean = csum ? csum[c] / (double)csize[c] : sc->zsum * inv_ndof;
  p[s] = (T)((double)z[s] - mean) + (T)sc->beta * p[s];
}

// v -= mean_c(v) on the unknowns (single component: mean = sc->aux[slot]/n).
template <typename T>
__global__ void __launch_bounds__(NT)
k_sub_mean(T *__restrict__ v, const int *__restrict__ comp, const Scalars *sc,
           int aux_slot, const double *__restrict__ csum,
           const int *__restrict__ csize, double inv_ndof) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const int c = comp[s];
  if (c < 0) { v[s] = (T)0; return; }
  const double mean = csum ? csum[c] / (double)csize[c] : sc->aux[aux_slot] * inv_ndof;
  v[s] = (T)((double)v[s] - mean);
}

// aux[slot] = sum over unknowns of x*y (y = null: plain sum of x).
template <typename T>
__global__ void __launch_bounds__(NT)
k_dot(const T *__restrict__ x, const T *__restrict__ y,
      const int *__restrict__ comp, Scalars *sc, double *partials, int slot) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  double v[1] = {comp[s] >= 0 ? (double)x[s] * (y ? (double)y[s] : 1.0) : 0.0};
  double tot[1];
  if (grid_sum<1>(v, partials, &sc->ticket[3], tot)) sc->aux[slot] = tot[0];
}

// ------------------------------------------------------------ Eq. 3 RHS
// b_n = sum_{e leaving n} g_e a_e - sum_{e entering n} g_e a_e, from the
// full-grid edge array a[3][NZ][NY][NX]; non-finite a on a conducting edge
// raises DEV_BAD_A.
__global__ void __launch_bounds__(NT)
k_rhs(Grid g, const double *__restrict__ gx, const double *__restrict__ a,
      double *__restrict__ b, int *status) {
  BRICK_PROLOGUE(g);
  const int i = bc.x * 8 + lx, j = bc.y * 8 + ly, k = bc.z * 8 + lz;
  double acc = 0.0;
  bool bad = false;
  if (i < g.NX && j < g.NY && k < g.NZ) {
    const size_t NN = (size_t)g.NX * g.NY * g.NZ;
    const size_t n = ((size_t)k * g.NY + j) * g.NX + i;
    auto term = [&](double ge, size_t idx, double sign) {
      if (ge > 0.0) {
        double av = a[idx];
        if (!isfinite(av)) bad = true;
        acc += sign * ge * av;
      }
    };
    term(gx[s], n, 1.0);
    term(gx[S + s], NN + n, 1.0);
    term(gx[2 * S + s], 2 * NN + n, 1.0);
    int m;
    m = slot_nb(g, bk, bc, lx, ly, lz, -1, 0, 0);
    if (m >= 0) term(gx[m], n - 1, -1.0);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, -1, 0);
    if (m >= 0) term(gx[S + m], NN + n - g.NX, -1.0);
    m = slot_nb(g, bk, bc, lx, ly, lz, 0, 0, -1);
    if (m >= 0) term(gx[2 * S + m], 2 * NN + n - (size_t)g.NX * g.NY, -1.0);
  }
  b[s] = bad ? 0.0 : acc;
  if (bad) atomicOr(status, DEV_BAD_A);
}

// psi[n] = x[slot(n)] on the full node grid (0 where no unknown).
template <typename T>
__global__ void k_scatter(Grid g, const T *__restrict__ x,
                          const int *__restrict__ comp, double *__restrict__ psi) {
  const size_t NN = (size_t)g.NX * g.NY * g.NZ;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < NN;
       n += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(n % g.NX), j = (int)((n / g.NX) % g.NY),
        k = (int)(n / ((size_t)g.NX * g.NY));
    int s = slot_at(g, i, j, k);
    psi[n] = (s >= 0 && comp[s] >= 0) ? (double)x[s] : 0.0;
  }
}

// x[slot(n)] = psi[n] on the unknowns (warm start / host input).
__global__ void __launch_bounds__(NT)
k_gather(Grid g, const double *__restrict__ psi, const int *__restrict__ comp,
         double *__restrict__ x) {
  BRICK_PROLOGUE(g);
  const int i = bc.x * 8 + lx, j = bc.y * 8 + ly, k = bc.z * 8 + lz;
  double v = 0.0;
  if (comp[s] >= 0) v = psi[((size_t)k * g.NY + j) * g.NX + i];
  x[s] = v;
}

// ------------------------------------------------------------ Eq. 1 |E|
__global__ void k_efield(const unsigned char *__restrict__ mask,
                         const double *__restrict__ a,
                         const double *__restrict__ psi, int nx, int ny, int nz,
                         double c, double *__restrict__ E) {
  const size_t NV_ = (size_t)nx * ny * nz;
  const size_t NX = nx + 1, NY = ny + 1;
  const size_t NN = NX * NY * (size_t)(nz + 1);
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < NV_;
       v += (size_t)gridDim.x * blockDim.x) {
    if (!mask[v]) { E[v] = 0.0; continue; }
    size_t i = v % nx, j = (v / nx) % ny, k = v / ((size_t)nx * ny);
    size_t n000 = (k * NY + j) * NX + i;
    double ex = 0.0, ey = 0.0, ez = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        size_t tx = n000 + (q * NY + r) * NX;       // x edge at (i, j+r, k+q)
        ex += a[tx] + psi[tx + 1] - psi[tx];
        size_t ty = n000 + q * NY * NX + r;         // y edge at (i+r, j, k+q)
        ey += a[NN + ty] + psi[ty + NX] - psi[ty];
        size_t tz = n000 + q * NX + r;              // z edge at (i+r, j+q, k)
        ez += a[2 * NN + tz] + psi[tz + NX * NY] - psi[tz];
      }
    ex *= c; ey *= c; ez *= c;
    E[v] = sqrt(ex * ex + ey * ey + ez * ez);
  }
}

// ------------------------------------------------ smoother eigenvalue estimate
// Deterministic start vector on the unknowns for the power iteration.
__global__ void __launch_bounds__(NT)
k_power_init(const double *__restrict__ diag, double *__restrict__ v) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  unsigned h = (unsigned)s * 2654435761u;
  h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
  v[s] = diag[s] > 0.0 ? 0.5 + (double)(h & 0xffff) / 65536.0 : 0.0;
}

// w = D^{-1} A v given r = -A v; aux[4] = |w|^2.
__global__ void __launch_bounds__(NT)
k_power_step(const double *__restrict__ r, const double *__restrict__ dinv,
             double *__restrict__ w, Scalars *sc, double *partials) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  double ws = -dinv[s] * r[s];
  w[s] = ws;
  double v[1] = {ws * ws};
  double tot[1];
  if (grid_sum<1>(v, partials, &sc->ticket[4], tot)) sc->aux[4] = tot[0];
}

__global__ void __launch_bounds__(NT) k_scale(double *__restrict__ v, double f) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  v[s] *= f;
}

__global__ void __launch_bounds__(NT)
k_scaled_copy(const double *__restrict__ src, double f, double *__restrict__ dst) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  dst[s] = f * src[s];
}

// ------------------------------------------------ precision conversions
// dst = (T) (f * src) elementwise over n values.
template <typename T>
__global__ void k_convert(size_t n, const double *__restrict__ src, double f,
                          T *__restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (T)(f * src[i]);
}
template <>
__global__ void k_convert<__nv_bfloat16>(size_t n, const double *__restrict__ src,
                                         double f, __nv_bfloat16 *__restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __double2bfloat16(f * src[i]);
}

// x += f * d (FP64 accumulation of an FP32 correction) on level-0 slots.
__global__ void __launch_bounds__(NT)
k_axpy_mixed(double *__restrict__ x, const float *__restrict__ d, double f) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  x[s] += f * (double)d[s];
}

// r32 = (float)(f * r64); the sum of r32 lands in sc->rsum for the fused
// projection of the first V-cycle sweep.
__global__ void __launch_bounds__(NT)
k_scale_to_f32(const double *__restrict__ r, double f, float *__restrict__ r32,
               Scalars *sc, double *partials) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const float v = (float)(f * r[s]);
  r32[s] = v;
  double t[1] = {(double)v};
  double tot[1];
  if (grid_sum<1>(t, partials, &sc->ticket[5], tot)) sc->rsum = tot[0];
}

// ------------------------------------------------------------ launchers
template <typename T>
void launch_convert(size_t n, const double *src, double f, T *dst,
                    cudaStream_t st) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks == 0) return;
  k_convert<T><<<(int)blocks, 256, 0, st>>>(n, src, f, dst);
}
template void launch_convert<float>(size_t, const double *, double, float *, cudaStream_t);
template void launch_convert<__nv_bfloat16>(size_t, const double *, double,
                                            __nv_bfloat16 *, cudaStream_t);
void launch_axpy_mixed(int nb, double *x, const float *d, double f,
                       cudaStream_t st) {
  if (nb) k_axpy_mixed<<<nb, NT, 0, st>>>(x, d, f);
}
void launch_scale_to_f32(int nb, const double *r, double f, float *r32,
                         Scalars *sc, double *partials, cudaStream_t st) {
  if (nb) k_scale_to_f32<<<nb, NT, 0, st>>>(r, f, r32, sc, partials);
}
void launch_power_init(int nb, const double *diag, double *v, cudaStream_t st) {
  if (nb) k_power_init<<<nb, NT, 0, st>>>(diag, v);
}
void launch_power_step(int nb, const double *r, const double *dinv, double *w,
                       Scalars *sc, double *partials, cudaStream_t st) {
  if (nb) k_power_step<<<nb, NT, 0, st>>>(r, dinv, w, sc, partials);
}
void launch_scale(int nb, double *v, double f, cudaStream_t st) {
  if (nb) k_scale<<<nb, NT, 0, st>>>(v, f);
}
void launch_scaled_copy(int nb, const double *src, double f, double *dst,
                        cudaStream_t st) {
  if (nb) k_scaled_copy<<<nb, NT, 0, st>>>(src, f, dst);
}
template <typename T>
void launch_apply_dot(const Grid &g, const T *gx, const T *diag, const T *p,
                      T *q, Scalars *sc, double *partials, cudaStream_t st) {
  if (g.nb) k_apply_dot<T><<<g.nb, NT, 0, st>>>(g, gx, diag, p, q, sc, partials);
}
template <typename T>
void launch_update_xr(int nb, T *x, T *r, const T *p, const T *q, Scalars *sc,
                      double *partials, cudaStream_t st) {
  if (nb) k_update_xr<T><<<nb, NT, 0, st>>>(x, r, p, q, sc, partials);
}
template <typename T>
void launch_dot_rz(int nb, const T *r, const T *z, const int *comp,
                   Scalars *sc, double *partials, int first, cudaStream_t st) {
  if (nb) k_dot_rz<T><<<nb, NT, 0, st>>>(r, z, comp, sc, partials, first);
}
template <typename T>
void launch_comp_sum(int nb, const T *v, const int *comp, double *csum,
                     cudaStream_t st) {
  if (nb) k_comp_sum<T><<<nb, NT, 0, st>>>(v, comp, csum);
}
template <typename T>
void launch_pupdate(int nb, T *p, const T *z, const int *comp,
                    const Scalars *sc, const double *csum, const int *csize,
                    double inv_ndof, cudaStream_t st) {
  if (nb) k_pupdate<T><<<nb, NT, 0, st>>>(p, z, comp, sc, csum, csize, inv_ndof);
}
template <typename T>
void launch_sub_mean(int nb, T *v, const int *comp, const Scalars *sc,
                     int aux_slot, const double *csum, const int *csize,
                     double inv_ndof, cudaStream_t st) {
  if (nb)
    k_sub_mean<T><<<nb, NT, 0, st>>>(v, comp, sc, aux_slot, csum, csize, inv_ndof);
}
template <typename T>
void launch_dot(int nb, const T *x, const T *y, const int *comp, Scalars *sc,
                double *partials, int slot, cudaStream_t st) {
  if (nb) k_dot<T><<<nb, NT, 0, st>>>(x, y, comp, sc, partials, slot);
}
void launch_rhs(const Grid &g, const double *gx, const double *a, double *b,
                int *status, cudaStream_t st) {
  if (g.nb) k_rhs<<<g.nb, NT, 0, st>>>(g, gx, a, b, status);
}
template <typename T>
void launch_scatter(const Grid &g, const T *x, const int *comp, double *psi,
                    cudaStream_t st) {
  size_t NN = (size_t)g.NX * g.NY * g.NZ;
  size_t blocks = (NN + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks == 0) blocks = 1;
  k_scatter<T><<<(int)blocks, 256, 0, st>>>(g, x, comp, psi);
}
void launch_gather(const Grid &g, const double *psi, const int *comp, double *x,
                   cudaStream_t st) {
  if (g.nb) k_gather<<<g.nb, NT, 0, st>>>(g, psi, comp, x);
}
void launch_efield(const unsigned char *mask, const double *a,
                   const double *psi, int nx, int ny, int nz, double h,
                   double omega, double *E, cudaStream_t st) {
  size_t n = (size_t)nx * ny * nz;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks == 0) blocks = 1;
  k_efield<<<(int)blocks, 256, 0, st>>>(mask, a, psi, nx, ny, nz,
                                        omega / (4.0 * h), E);
}

#define INST_K(T)                                                              \
  template void launch_apply_dot<T>(const Grid &, const T *, const T *,        \
                                    const T *, T *, Scalars *, double *,       \
                                    cudaStream_t);                             \
  template void launch_update_xr<T>(int, T *, T *, const T *, const T *,       \
                                    Scalars *, double *, cudaStream_t);        \
  template void launch_dot_rz<T>(int, const T *, const T *, const int *,       \
                                 Scalars *, double *, int, cudaStream_t);      \
  template void launch_comp_sum<T>(int, const T *, const int *, double *,      \
                                   cudaStream_t);                              \
  template void launch_pupdate<T>(int, T *, const T *, const int *,            \
                                  const Scalars *, const double *,             \
                                  const int *, double, cudaStream_t);          \
  template void launch_sub_mean<T>(int, T *, const int *, const Scalars *,     \
                                   int, const double *, const int *, double,   \
                                   cudaStream_t);                              \
  template void launch_dot<T>(int, const T *, const T *, const int *,          \
                              Scalars *, double *, int, cudaStream_t);         \
  template void launch_scatter<T>(const Grid &, const T *, const int *,        \
                                  double *, cudaStream_t);
INST_K(double)
INST_K(float)

}  // namespace spfd
