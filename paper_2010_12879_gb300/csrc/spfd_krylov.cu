// Krylov-loop kernels with fused, deterministic reductions; the right-hand
// side of Eq. 3, the Psi scatter and the |E| of Eq. 1.
//
// Reductions finish on the device: blocks write partial sums, and either the
// last block to arrive (ticket counter) or a one-block finishing kernel adds
// them in a fixed order and updates the Krylov scalars in place, so the loop
// needs no host round trip except the convergence test.
//
// GB300's FP64 pipe retires about one FP64 operation per 11 bytes of HBM
// traffic, so FP32 kernels here keep every per-element operation in FP32:
// scalars arrive pre-converted (alpha_f, beta_f, ...) and dot products sum
// per thread in compensated (Kahan) FP32 before the FP64 tree across threads
// and blocks.
#include <algorithm>

#include "spfd_internal.cuh"
#include "spfd_tile.cuh"

namespace spfd {

// ------------------------------------------------------------ accumulators
// Per-thread running sum: FP64 for double kernels, compensated FP32 for float
// kernels (about FP64 accuracy over the few dozen terms a thread adds).
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// ------------------------------------------------------------ reductions
// Block sums of the threads' NV FP64 values, left in warp 0 (every lane),
// for blocks of at most NT threads.  The values pass through shared memory
// and warp 0 adds them (lane l the values of threads l, l + 32, ..., then a
// butterfly): NV * (warps + 4) FP64 warp instructions per block, against
// 5 NV per warp plus 5 NV for a butterfly in every warp, on GB300's narrow
// FP64 pipe.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sm[NV][NT];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k][t] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = sm[k][lane];
      for (int i = 1; i < nw; ++i) a += sm[k][lane + 32 * i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      v[k] = a;
    }
  }
  __syncthreads();
}

// The tail of the grid reductions, once thread 0 has written this block's NV
// partials: a ticket finds the last block, which adds every block's partials
// in a fixed order.  Returns true in thread 0 of the last block, with tot[] =
// grid totals.
template <int NV>
__device__ bool grid_finish(double *partials, unsigned *ticket, double (&tot)[NV]) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
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

template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *partials, unsigned *ticket,
                         double (&tot)[NV]) {
  block_sum<NV>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)blockIdx.x * NV + k] = v[k];
  return grid_finish<NV>(partials, ticket, tot);
}

// hi + lo += oh + ol with the rounding error of the high parts kept (TwoSum).
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float oh, float ol) {
  const float s = hi + oh, bb = s - hi;
  const float e = (hi - (s - bb)) + (oh - bb);
  hi = s;
  lo = lo + ol + e;
}

// grid_sum for per-thread FP32 pairs (value hi + lo): the warps and the block
// add them as TwoSum pairs in FP32, and only the block's total is widened to
// FP64 (in thread 0).  An FP64 conversion or addition takes a 16-clock slot
// of GB300's narrow FP64 pipe for its warp whatever its lane mask, so
// widening in every thread put an FP64 tail of several microseconds at the
// end of the FP32 reduction kernels.
template <int NV>
__device__ bool grid_sum_f32(float (&hi)[NV], float (&lo)[NV], double *partials,
                             unsigned *ticket, double (&tot)[NV]) {
  __shared__ float sh[32][NV], sl[32][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      two_sum_add(hi[k], lo[k], __shfl_xor_sync(0xffffffffu, hi[k], o),
                  __shfl_xor_sync(0xffffffffu, lo[k], o));
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      sh[w][k] = hi[k];
      sl[w][k] = lo[k];
    }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float h = lane < nw ? sh[lane][k] : 0.f, l = lane < nw ? sl[lane][k] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        two_sum_add(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
      if (lane == 0) partials[(size_t)blockIdx.x * NV + k] = (double)h + (double)l;
    }
  }
  return grid_finish<NV>(partials, ticket, tot);
}

// grid_sum of per-thread accumulators: FP64 sums directly, compensated FP32
// sums (value s - c) as FP32 pairs.
template <typename T, int NV>
__device__ bool grid_sum_acc(const Acc<T> (&a)[NV], double *partials, unsigned *ticket,
                             double (&tot)[NV]) {
  if constexpr (sizeof(T) == 8) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = a[k].s;
    return grid_sum<NV>(v, partials, ticket, tot);
  } else {
    float h[NV], l[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      h[k] = a[k].s;
      l[k] = -a[k].c;
    }
    return grid_sum_f32<NV>(h, l, partials, ticket, tot);
  }
}

// Grid-stride reduction kernels use at most RED_GRID blocks, so the ticket
// sees few same-address atomics.
constexpr int RED_GRID = 608;  // 4 resident 512-thread blocks on each of 152 SMs

// ------------------------------------------------------------ CG operator
// q = A p on one brick per block (row mapping, four nodes per thread); each
// warp writes its part of p.q, and k_finish_pq adds them.  A right-hand side
// that has converged (frozen) gets q = 0 and p.q = 0 without its operator
// work.  (Written as that warp-uniform branch, the FP64 operator also
// measured 8 % faster than the unconditional form, 193 against 211 us per
// launch on the 2 mm body.)
template <typename T, int ORD>
__global__ void __launch_bounds__(BV / row_n_apply<T>(), row_min_blocks_apply<T>())
k_apply_dot(Grid g, const T *__restrict__ gx, const T *__restrict__ diag,
            const T *__restrict__ p, T *__restrict__ q, const Scalars *sc,
            double *partials, size_t pstride, int nk) {
  pdl_entry();
  constexpr int N = row_n_apply<T>(), NW = BV / N / 32;
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, s0 = row_slot<N>(bk, t);
  p += (size_t)rhs * S;
  q += (size_t)rhs * S;
  partials += (size_t)rhs * pstride;
  Qv<T, N> pc, qv;
  if (__any_sync(0xffffffffu, !sc[rhs].frozen)) {
    apply7_row<T, T, false, N, sizeof(T) == 8>(g, gx, diag, p, S, bk, t, zqn<T, N>(), pc, qv);
  } else {
    pc = zqn<T, N>();
    qv = zqn<T, N>();
  }
  stqn<T, N>(q + s0, qv);
  if constexpr (sizeof(T) == 4) {
    // FP32 products summed without rounding error in (hi, lo) pairs
    // (TwoSum) over the thread's nodes and the warp, rounded to FP64 in the
    // storing lane only
    float pq[N];
#pragma unroll
    for (int i = 0; i < N; ++i) pq[i] = pc.v[i] * qv.v[i];
    const WarpSum<float> part = warp_total<float, N>(pq);
    if ((t & 31) == 0) part.put(&partials[(size_t)bk * NW + (t >> 5)]);
  } else {
    double a = pc.v[0] * qv.v[0];
#pragma unroll
    for (int i = 1; i < N; ++i) a += pc.v[i] * qv.v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((t & 31) == 0) partials[(size_t)bk * NW + (t >> 5)] = a;
  }
}

// Number of partials k_apply_dot writes for nb bricks.
template <typename T>
int apply_dot_partials(int nb) { return nb * (BV / row_n_apply<T>() / 32); }

// pq = sum of the n partials of k_apply_dot (blocks add contiguous chunks,
// the last block adds the block sums, fixed order); alpha = rz / pq.
// scratch must not overlap the partials.
template <bool PAIRS>
__global__ void __launch_bounds__(NT)
k_finish_pq(const double *__restrict__ partials, int n, double *scratch, Scalars *sc,
            size_t pstride) {
  pdl_entry();
  partials += (size_t)blockIdx.y * pstride;
  scratch += (size_t)blockIdx.y * pstride;
  sc += blockIdx.y;
  double a = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    a += pair_at<PAIRS>(partials, i);
  double v[1] = {a};
  double tot[1];
  if (grid_sum<1>(v, scratch, &sc->ticket[6], tot)) {
    sc->pq = tot[0];
    const double al = tot[0] > 0.0 ? sc->rz / tot[0] : 0.0;
    sc->alpha = al;
    sc->alpha_f = (float)al;
  }
}

// x += alpha p; r -= alpha q; rr = r.r and rsum = sum r (removed nodes hold
// r = 0); the last block also forms rmean = rsum / n.
template <typename T>
__global__ void __launch_bounds__(NT)
k_update_xr(int nb, T *__restrict__ x, T *__restrict__ r,
            const T *__restrict__ p, const T *__restrict__ q, Scalars *sc,
            double *partials, size_t pstride) {
  pdl_entry();
  constexpr int N = V16<T>::N;
  sc += blockIdx.y;
  if (sc->frozen) return;  // this right-hand side has converged
  {
    const size_t off = (size_t)blockIdx.y * nb * BV;
    x += off; r += off; p += off; q += off;
    partials += (size_t)blockIdx.y * pstride;
  }
  T alpha;
  if constexpr (sizeof(T) == 4) alpha = sc->alpha_f; else alpha = sc->alpha;
  Acc<T> rr, rs_sum;
  const size_t nv = (size_t)nb * BV / N;
  for (size_t vi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; vi < nv;
       vi += (size_t)gridDim.x * blockDim.x) {
    const size_t s0 = vi * N;
    V16<T> xv = ld16(x + s0), rv = ld16(r + s0);
    const V16<T> pv = ld16(p + s0), qv = ld16(q + s0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      xv.v[i] += alpha * pv.v[i];
      rv.v[i] -= alpha * qv.v[i];
      rr.add(rv.v[i] * rv.v[i]);
      rs_sum.add(rv.v[i]);
    }
    st16(x + s0, xv);
    st16(r + s0, rv);
  }
  const Acc<T> v[2] = {rr, rs_sum};
  double tot[2];
  if (grid_sum_acc<T, 2>(v, partials, &sc->ticket[1], tot)) {
    sc->rr = tot[0];
    sc->rsum = tot[1];
    sc->rmean = tot[1] * sc->inv_ndof;
    sc->rmean_f = (float)sc->rmean;
  }
}

// rz = r.z (new), beta = rz / rz_old, zsum = sum of z over the unknowns and
// zmean = zsum / n.
// rz = r.z (tot[0]) and the sum of z over the unknowns (tot[1]) into the
// Scalars: beta = rz / rz_old (0 on the first iteration or after a restart)
// and the mean of z for its projection.
__device__ __forceinline__ void set_rz(Scalars *sc, const double (&tot)[2], int first) {
  const double old = sc->rz;
  sc->rz_old = old;
  sc->rz = tot[0];
  const double beta = (first || sc->restart || old == 0.0) ? 0.0 : tot[0] / old;
  sc->restart = 0;
  sc->beta = beta;
  sc->beta_f = (float)beta;
  sc->zsum = tot[1];
  sc->zmean = tot[1] * sc->inv_ndof;
  sc->zmean_f = (float)sc->zmean;
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_dot_rz(int nb, const T *__restrict__ r, const T *__restrict__ z,
         const int *__restrict__ comp, Scalars *sc, double *partials,
         int first, size_t pstride) {
  pdl_entry();
  constexpr int N = V16<T>::N;
  {
    const size_t off = (size_t)blockIdx.y * nb * BV;
    r += off; z += off;
    sc += blockIdx.y;
    partials += (size_t)blockIdx.y * pstride;
  }
  Acc<T> rz, zsum;
  const size_t nv = (size_t)nb * BV / N;
  for (size_t vi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; vi < nv;
       vi += (size_t)gridDim.x * blockDim.x) {
    const size_t s0 = vi * N;
    const V16<T> rv = ld16(r + s0), zv = ld16(z + s0);
    int c[N];
    ld_ints<N>(comp + s0, c);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      rz.add(rv.v[i] * zv.v[i]);
      if (c[i] >= 0) zsum.add(zv.v[i]);
    }
  }
  const Acc<T> v[2] = {rz, zsum};
  double tot[2];
  if (grid_sum_acc<T, 2>(v, partials, &sc->ticket[2], tot)) set_rz(sc, tot, first);
}

// The same scalars from the partial pairs the level-0 post-smoother wrote
// (k_jacobi7 with RZ): grid-stride sums, then the ticketed block tree.
template <bool PAIRS>
__global__ void __launch_bounds__(NT)
k_finish_rz(const double *__restrict__ partials, int n, double *scratch, Scalars *sc,
            int first, size_t pstride) {
  pdl_entry();
  partials += (size_t)blockIdx.y * pstride;
  scratch += (size_t)blockIdx.y * pstride;
  sc += blockIdx.y;
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[0] += pair_at<PAIRS>(partials, 2 * (size_t)i);
    v[1] += pair_at<PAIRS>(partials, 2 * (size_t)i + 1);
  }
  double tot[2];
  if (grid_sum<2>(v, scratch, &sc->ticket[2], tot)) set_rz(sc, tot, first);
}

// Per-component sums of v over the unknowns (several components), exact and
// independent of the order of the atomics, so that repeated and batched
// solves are bit-identical.  The workspace of one right-hand side (cstride
// words) holds the FP64 sums [ncomp], 128-bit accumulators [ncomp][2] and the
// bits of max |v|.  k_absmax takes max |v|; k_comp_sum scales every value by
// the same power of two, 2^k with max |v| 2^k < 2^96, truncates it to an
// integer and adds it to its component's 128-bit two's-complement
// accumulator (two 64-bit words, the low word's carry-out counted by the
// atomic that caused it); up to 2^31 values cannot overflow 2^127.
// k_comp_finish turns the accumulators back into FP64.  Values below
// 2^-95 max |v| are lost to truncation, far under FP64 rounding of the sum.
__device__ __forceinline__ int sum_scale_exp(unsigned long long maxbits) {
  return 95 - ilogb(__longlong_as_double((long long)maxbits));
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_absmax(const T *__restrict__ v, const int *__restrict__ comp, double *ws, int cstride,
         int ncomp) {
  pdl_entry();
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  v += (size_t)blockIdx.y * gridDim.x * BV;
  ws += (size_t)blockIdx.y * cstride;
  unsigned long long m =
      comp[s] >= 0 ? (unsigned long long)__double_as_longlong(fabs((double)v[s])) : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
    m = q > m ? q : m;
  }
  __shared__ unsigned long long wm[NT / 32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) m = wm[w] > m ? wm[w] : m;
    // non-negative doubles order like their bit patterns
    if (m) atomicMax(reinterpret_cast<unsigned long long *>(ws + 3 * ncomp), m);
  }
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_comp_sum(const T *__restrict__ v, const int *__restrict__ comp, double *ws, int cstride,
           int ncomp) {
  pdl_entry();
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  v += (size_t)blockIdx.y * gridDim.x * BV;
  ws += (size_t)blockIdx.y * cstride;
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(ws + ncomp);
  const unsigned long long mb = *reinterpret_cast<const unsigned long long *>(ws + 3 * ncomp);
  const int c = comp[s];
  const unsigned grp = __match_any_sync(0xffffffffu, c);
  unsigned long long lo = 0ull, hi = 0ull;
  if (c >= 0 && mb) {
    const double x = (double)v[s];
    const double ax = scalbn(fabs(x), sum_scale_exp(mb));  // < 2^96, exact
    const double hd = floor(ax * 0x1p-64);                 // exact
    lo = (unsigned long long)(ax - hd * 0x1p64);           // exact difference, truncated
    hi = (unsigned long long)hd;
    if (x < 0.0) {  // two's complement negation of (hi, lo)
      lo = ~lo + 1ull;
      hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
  }
  unsigned long long tl = 0ull, th = 0ull;
  unsigned m = grp;
  while (m) {  // exact sum within the group: walk the set bits (at most 32)
    const int src = __ffs(m) - 1;
    const unsigned long long ol = __shfl_sync(grp, lo, src), oh = __shfl_sync(grp, hi, src);
    const unsigned long long nl = tl + ol;
    th += oh + (nl < tl ? 1ull : 0ull);
    tl = nl;
    m &= m - 1;
  }
  if (c >= 0 && mb && (int)(threadIdx.x & 31) == __ffs(grp) - 1) {
    const unsigned long long old = atomicAdd(&acc[2 * c], tl);
    atomicAdd(&acc[2 * c + 1], th + (old + tl < old ? 1ull : 0ull));
  }
}

__global__ void k_comp_finish(double *ws, int cstride, int ncomp) {
  pdl_entry();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  ws += (size_t)blockIdx.y * cstride;
  if (c >= ncomp) return;
  const unsigned long long mb = *reinterpret_cast<const unsigned long long *>(ws + 3 * ncomp);
  const unsigned long long *acc = reinterpret_cast<const unsigned long long *>(ws + ncomp);
  unsigned long long lo = acc[2 * c], hi = acc[2 * c + 1];
  if (!mb) { ws[c] = 0.0; return; }
  const bool neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  const double mag = (double)hi * 0x1p64 + (double)lo;
  ws[c] = scalbn(neg ? -mag : mag, -sum_scale_exp(mb));
}

// p = (z - mean_c(z)) + beta p on the unknowns.  One component: the mean is
// sc->zmean; several: csum[c] / csize[c].
template <typename T>
__global__ void __launch_bounds__(NT)
k_pupdate(T *__restrict__ p, const T *__restrict__ z,
          const int *__restrict__ comp, const Scalars *sc,
          const double *__restrict__ csum, const int *__restrict__ csize, int cstride) {
  pdl_entry();
  constexpr int N = V16<T>::N;
  const size_t s0 = (size_t)blockIdx.x * BV + threadIdx.x * N;
  {
    const size_t off = (size_t)blockIdx.y * gridDim.x * BV;
    p += off; z += off;
    sc += blockIdx.y;
    if (csum) csum += (size_t)blockIdx.y * cstride;
  }
  T mean1, beta;
  if constexpr (sizeof(T) == 4) { mean1 = sc->zmean_f; beta = sc->beta_f; }
  else { mean1 = sc->zmean; beta = sc->beta; }
  int c[N];
  ld_ints<N>(comp + s0, c);
  const V16<T> zv = ld16(z + s0);
  V16<T> pv = ld16(p + s0);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (c[i] < 0) { pv.v[i] = (T)0; continue; }
    const T mean = csum ? (T)(csum[c[i]] / (double)csize[c[i]]) : mean1;
    pv.v[i] = (zv.v[i] - mean) + beta * pv.v[i];
  }
  st16(p + s0, pv);
}

// v -= mean_c(v) on the unknowns (single component: mean = aux[slot] / n).
template <typename T>
__global__ void __launch_bounds__(NT)
k_sub_mean(T *__restrict__ v, const int *__restrict__ comp, const Scalars *sc,
           int aux_slot, const double *__restrict__ csum,
           const int *__restrict__ csize, int cstride) {
  pdl_entry();
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  v += (size_t)blockIdx.y * gridDim.x * BV;
  sc += blockIdx.y;
  if (csum) csum += (size_t)blockIdx.y * cstride;
  const int c = comp[s];
  if (c < 0) { v[s] = (T)0; return; }
  const T mean = csum ? (T)(csum[c] / (double)csize[c])
                      : (T)(sc->aux[aux_slot] * sc->inv_ndof);
  v[s] = v[s] - mean;
}

// aux[slot] = sum over unknowns of x*y (y = null: plain sum of x).
template <typename T>
__global__ void __launch_bounds__(NT)
k_dot(int nb, const T *__restrict__ x, const T *__restrict__ y,
      const int *__restrict__ comp, Scalars *sc, double *partials, int slot,
      size_t pstride) {
  pdl_entry();
  {
    const size_t off = (size_t)blockIdx.y * nb * BV;
    x += off;
    if (y) y += off;
    sc += blockIdx.y;
    partials += (size_t)blockIdx.y * pstride;
  }
  Acc<T> acc;
  for (int bk = blockIdx.x; bk < nb; bk += gridDim.x) {
    const size_t s = (size_t)bk * BV + threadIdx.x;
    if (comp[s] >= 0) acc.add(y ? x[s] * y[s] : x[s]);
  }
  const Acc<T> v[1] = {acc};
  double tot[1];
  if (grid_sum_acc<T, 1>(v, partials, &sc->ticket[3], tot)) sc->aux[slot] = tot[0];
}

// ------------------------------------------------------------ Eq. 3 RHS
// b_n = sum_{e leaving n} g_e a_e - sum_{e entering n} g_e a_e, from the
// full-grid edge array a[3][NZ][NY][NX]; non-finite a on a conducting edge
// raises DEV_BAD_A.  The tests of g_e > 0 (g_e is +0, -0 or positive) and of
// a finite a_e look at bit patterns, so each edge costs one FP64 multiply-add
// on GB300's narrow FP64 pipe.
__global__ void __launch_bounds__(NT)
k_rhs(Grid g, const double *__restrict__ gx, const double *__restrict__ a,
      double *__restrict__ b, int *status) {
  __shared__ int sn[27];
  const int bk = blockIdx.x, t = threadIdx.x;
  load_nbr(g, bk, sn);
  __syncthreads();
  const size_t S = (size_t)g.nb * BV, s = (size_t)bk * BV + t;
  a += (size_t)blockIdx.y * 3 * ((size_t)g.NX * g.NY * g.NZ);
  b += (size_t)blockIdx.y * S;
  const int4 bc = g.bco[bk];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  const int i = bc.x * 8 + lx, j = bc.y * 8 + ly, k = bc.z * 8 + lz;
  double acc = 0.0;
  bool bad = false;
  if (i < g.NX && j < g.NY && k < g.NZ) {
    const size_t NN = (size_t)g.NX * g.NY * g.NZ;
    const size_t n = ((size_t)k * g.NY + j) * g.NX + i;
    // ge: a conductance (+0, -0 or positive), subtracted for an entering edge
    auto term = [&](double ge, size_t idx, bool entering) {
      if (f64_nonzero(ge)) {
        const double av = a[idx];
        if (f64_nonfinite(av)) bad = true;
        acc = fma(entering ? -ge : ge, av, acc);
      }
    };
    term(gx[s], n, false);
    term(gx[S + s], NN + n, false);
    term(gx[2 * S + s], 2 * NN + n, false);
    // -edges: the +edge conductance of the neighbour node
    int nb;
    if (lx > 0) term(gx[s - 1], n - 1, true);
    else if ((nb = sn[sidx(-1, 0, 0)]) >= 0) term(gx[(size_t)nb * BV + t + 7], n - 1, true);
    if (ly > 0) term(gx[S + s - 8], NN + n - g.NX, true);
    else if ((nb = sn[sidx(0, -1, 0)]) >= 0)
      term(gx[S + (size_t)nb * BV + t + 56], NN + n - g.NX, true);
    if (lz > 0) term(gx[2 * S + s - 64], 2 * NN + n - (size_t)g.NX * g.NY, true);
    else if ((nb = sn[sidx(0, 0, -1)]) >= 0)
      term(gx[2 * S + (size_t)nb * BV + t + 448], 2 * NN + n - (size_t)g.NX * g.NY, true);
  }
  b[s] = bad ? 0.0 : acc;
  if (bad) atomicOr(status, DEV_BAD_A);
}

// psi[n] = x[slot(n)] on the full node grid (0 where no unknown).
template <typename T>
__global__ void k_scatter(Grid g, const T *__restrict__ x,
                          const int *__restrict__ comp, double *__restrict__ psi) {
  pdl_entry();
  const size_t NN = (size_t)g.NX * g.NY * g.NZ;
  x += (size_t)blockIdx.y * g.nb * BV;
  psi += (size_t)blockIdx.y * NN;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < NN;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % g.NX), j = (int)((n / g.NX) % g.NY),
              k = (int)(n / ((size_t)g.NX * g.NY));
    const int s = slot_at(g, i, j, k);
    psi[n] = (s >= 0 && comp[s] >= 0) ? (double)x[s] : 0.0;
  }
}

// x[slot(n)] = psi[n] on the unknowns (warm start / host input).
__global__ void __launch_bounds__(NT)
k_gather(Grid g, const double *__restrict__ psi, const int *__restrict__ comp,
         double *__restrict__ x) {
  const int bk = blockIdx.x, t = threadIdx.x;
  const size_t s = (size_t)bk * BV + t;
  const int4 bc = g.bco[bk];
  const int i = bc.x * 8 + (t & 7), j = bc.y * 8 + ((t >> 3) & 7), k = bc.z * 8 + (t >> 6);
  double v = 0.0;
  if (comp[s] >= 0) v = psi[((size_t)k * g.NY + j) * g.NX + i];
  x[s] = v;
}

// ------------------------------------------------------------ Eq. 1 |E|
// E_d of voxel (i, j, k) = c * sum over its four d-edges of
// (a_e + Psi_head - Psi_tail), c = omega / (4h); |E| = |(E_x, E_y, E_z)|.
// Each edge term is formed as (a_e + Psi_head) - Psi_tail and the four terms
// of an axis are added in the order (s, t) = (0,0), (0,1), (1,0), (1,1) of
// the edge offsets, with no contracted multiply-add, so the result is the
// correctly rounded evaluation of that fixed expression.
//
// Every edge term is formed once.  Warp w covers the node columns
// 31w .. 31w + 31 of the plane j < ny (flattened as col = j * (nx+1) + i):
// lane l < 31 owns voxel (i, j) of its column when i < nx, and lane 31 only
// supplies its column's terms to lane 30.  A column forms, per node layer k,
// its x-edge terms at rows j and j+1 (X0, X1, with Psi of column i+1 from the
// next lane) and its y-edge term (Y), and per voxel layer its two z-edge terms
// (Z0, Z1); voxel i takes the y and z terms of column i+1 from the next lane
// too.  Block y walks EF_KCHUNK voxel layers and carries the terms of layer
// k+1 into layer k+1's voxels, so a layer's terms are formed once.  Layers
// with no conducting voxel in the warp form nothing (their voxels get 0).
// Per voxel layer a column forms 5 terms (10 FP64 additions) against 16 when
// every voxel forms its own.
constexpr int EF_THREADS = 256;
constexpr int EF_KCHUNK = 16;
// 4 resident blocks per SM (at most 64 registers a thread): the kernel waits
// on memory between layers, and the FP64 pipe needs the warps to cover it.
constexpr int EF_MIN_BLOCKS = 4;

struct EfTerms {
  double p0, p1;  // Psi(i, j, k), Psi(i, j+1, k)
  double x0, x1;  // x-edge terms at (i, j, k), (i, j+1, k)
  double y;       // y-edge term at (i, j, k)
};

__device__ __forceinline__ double shfl_next(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}

// The terms of node layer k for the column at node offset nc (every lane of
// the warp calls it; lanes without a column get zeros).
__device__ __forceinline__ EfTerms ef_layer(const double *__restrict__ a,
                                            const double *__restrict__ psi, bool live,
                                            size_t n, size_t NX, size_t NN) {
  EfTerms T;
  T.p0 = live ? psi[n] : 0.0;
  T.p1 = live ? psi[n + NX] : 0.0;
  const double q0 = shfl_next(T.p0), q1 = shfl_next(T.p1);  // column i+1
  T.x0 = live ? __dadd_rn(__dadd_rn(a[n], q0), -T.p0) : 0.0;
  T.x1 = live ? __dadd_rn(__dadd_rn(a[n + NX], q1), -T.p1) : 0.0;
  T.y = live ? __dadd_rn(__dadd_rn(a[NN + n], T.p1), -T.p0) : 0.0;
  return T;
}

__global__ void __launch_bounds__(EF_THREADS, EF_MIN_BLOCKS)
k_efield(const unsigned char *__restrict__ mask, const double *__restrict__ a,
         const double *__restrict__ psi, int nx, int ny, int nz, double c,
         double *__restrict__ E) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * EF_THREADS + threadIdx.x) >> 5;
  const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1);
  const size_t NN = NXY * ((size_t)nz + 1);
  const long long ncol = (long long)NX * ny;
  if (warp * 31 >= ncol) return;  // the whole warp is past the plane
  const long long col = warp * 31 + lane;
  const bool live = col < ncol;
  const int i = live ? (int)(col % (long long)NX) : 0, j = live ? (int)(col / (long long)NX) : 0;
  const bool own = live && lane < 31 && i < nx;
  const size_t nc = (size_t)j * NX + i;
  const int kb = blockIdx.y * EF_KCHUNK, ke = min(kb + EF_KCHUNK, nz);
  EfTerms T{};
  bool have = false;  // T holds layer k's terms (warp-uniform)
  for (int k = kb; k < ke; ++k) {
    const size_t v = ((size_t)k * ny + j) * nx + i;
    const bool cond = own && mask[v];
    if (!__any_sync(0xffffffffu, cond)) {
      if (own) E[v] = 0.0;
      have = false;
      continue;
    }
    const size_t n = (size_t)k * NXY + nc;
    if (!have) T = ef_layer(a, psi, live, n, NX, NN);
    const EfTerms Tn = ef_layer(a, psi, live, n + NXY, NX, NN);
    const double z0 = live ? __dadd_rn(__dadd_rn(a[2 * NN + n], Tn.p0), -T.p0) : 0.0;
    const double z1 = live ? __dadd_rn(__dadd_rn(a[2 * NN + n + NX], Tn.p1), -T.p1) : 0.0;
    // the y and z terms of column i+1
    const double y0n = shfl_next(T.y), y1n = shfl_next(Tn.y);
    const double z0n = shfl_next(z0), z1n = shfl_next(z1);
    if (own) {
      double e = 0.0;
      if (cond) {
        const double ex = __dmul_rn(__dadd_rn(__dadd_rn(__dadd_rn(T.x0, Tn.x0), T.x1), Tn.x1), c);
        const double ey = __dmul_rn(__dadd_rn(__dadd_rn(__dadd_rn(T.y, Tn.y), y0n), y1n), c);
        const double ez = __dmul_rn(__dadd_rn(__dadd_rn(__dadd_rn(z0, z1), z0n), z1n), c);
        e = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
      }
      E[v] = e;
    }
    T = Tn;
    have = true;
  }
}

// ------------------------------------------------ adjoint of the field energy
// J = (1/Nc) sum over conducting voxels of |E_v|^2, E_v,d = c * sum over the
// voxel's four d-edges of u_e, u = a + G Psi, c = omega / (4h) (Eq. 1,
// voxel averaged).  Its gradient needs one extra solve A lambda = G^T gJ,
// gJ = dJ/du; then dJ/da = gJ - g (G lambda) and dJ/dg = -(G lambda) u,
// which the edge-conductance rule (g_e = h/4 * sum of the 4 voxels' sigma)
// turns into dJ/dsigma_v = h/4 * sum over the voxel's 12 edges of dJ/dg.

__device__ __forceinline__ void voxel_ijk(size_t v, int nx, int ny, int *i, int *j, int *k) {
  const size_t r = v / (size_t)nx;
  *i = (int)(v - r * nx);
  *j = (int)(r % (size_t)ny);
  *k = (int)(r / (size_t)ny);
}

// Ev[d][v] = E_v,d (0 in air); sc->aux[6] = sum |E_v|^2, sc->aux[7] = Nc.
__global__ void __launch_bounds__(NT)
k_energy(const unsigned char *__restrict__ mask, const double *__restrict__ a,
         const double *__restrict__ psi, int nx, int ny, int nz, double c,
         double *__restrict__ Ev, Scalars *sc, double *partials) {
  const size_t nv = (size_t)nx * ny * nz;
  const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1), NN = NXY * ((size_t)nz + 1);
  double sum = 0.0, cnt = 0.0;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv;
       v += (size_t)gridDim.x * blockDim.x) {
    double E[3] = {0.0, 0.0, 0.0};
    if (mask[v]) {
      int i, j, k;
      voxel_ijk(v, nx, ny, &i, &j, &k);
      const size_t n = (size_t)k * NXY + (size_t)j * NX + i;
#pragma unroll
      for (int st = 0; st < 4; ++st) {  // (s, t) = (0,0), (0,1), (1,0), (1,1)
        const int s_ = st >> 1, t_ = st & 1;
        const size_t tx = n + s_ * NX + t_ * NXY;   // x edge at (i, j+s, k+t)
        const size_t ty = n + s_ + t_ * NXY;        // y edge at (i+s, j, k+t)
        const size_t tz = n + s_ + t_ * NX;         // z edge at (i+s, j+t, k)
        E[0] += (a[tx] + psi[tx + 1]) - psi[tx];
        E[1] += (a[NN + ty] + psi[ty + NX]) - psi[ty];
        E[2] += (a[2 * NN + tz] + psi[tz + NXY]) - psi[tz];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        E[d] *= c;
        sum += E[d] * E[d];
      }
      cnt += 1.0;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Ev[d * nv + v] = E[d];
  }
  double vals[2] = {sum, cnt}, tot[2];
  if (grid_sum<2>(vals, partials, &sc->ticket[7], tot)) {
    sc->aux[6] = tot[0];
    sc->aux[7] = tot[1];
  }
}

// gJ_e = sum over the conducting voxels v at edge e of 2 c E_v,d(e) / Nc,
// in increasing voxel order; one thread per node and direction.
__global__ void __launch_bounds__(NT)
k_energy_gJ(const unsigned char *__restrict__ mask, const double *__restrict__ Ev,
            int nx, int ny, int nz, double c, const Scalars *sc, double *__restrict__ gJ) {
  const size_t nv = (size_t)nx * ny * nz;
  const size_t NX = (size_t)nx + 1, NY = (size_t)ny + 1, NN = NX * NY * ((size_t)nz + 1);
  const double nc = sc->aux[7];
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 3 * NN;
       q += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(q / NN);
    const size_t n = q - (size_t)d * NN;
    const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
    double acc = 0.0;
    // the up to 4 voxels at the edge, lowest voxel index first: offsets on
    // the two axes other than d, (-1,-1), (0,-1), (-1,0), (0,0)
    const bool on = (d == 0 ? i < nx : d == 1 ? j < ny : k < nz);
    if (on && nc > 0.0) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int p1 = (w & 1) - 1, p2 = (w >> 1) - 1;  // offsets -1/0
        int vi = i, vj = j, vk = k;
        if (d == 0) { vj += p1; vk += p2; }
        else if (d == 1) { vi += p1; vk += p2; }
        else { vi += p1; vj += p2; }
        if (vi < 0 || vj < 0 || vk < 0 || vi >= nx || vj >= ny || vk >= nz) continue;
        const size_t v = ((size_t)vk * ny + vj) * nx + vi;
        if (mask[v]) acc += 2.0 * c * Ev[d * nv + v] / nc;
      }
    }
    gJ[q] = acc;
  }
}

// b = G^T gJ on the level-0 unknowns (0 elsewhere):
// sum of the entering edges' gJ minus the leaving edges'.
__global__ void __launch_bounds__(NT)
k_div_brick(Grid g, const double *__restrict__ diag, const double *__restrict__ gJ,
            double *__restrict__ b) {
  const int bk = blockIdx.x, t = threadIdx.x;
  const size_t s = (size_t)bk * BV + t;
  const int4 bc = g.bco[bk];
  const int i = bc.x * 8 + (t & 7), j = bc.y * 8 + ((t >> 3) & 7), k = bc.z * 8 + (t >> 6);
  double acc = 0.0;
  if (i < g.NX && j < g.NY && k < g.NZ && diag[s] > 0.0) {
    const size_t NN = (size_t)g.NX * g.NY * g.NZ;
    const size_t n = ((size_t)k * g.NY + j) * g.NX + i;
    if (i > 0) acc += gJ[n - 1];
    if (j > 0) acc += gJ[NN + n - g.NX];
    if (k > 0) acc += gJ[2 * NN + n - (size_t)g.NX * g.NY];
    if (i + 1 < g.NX) acc -= gJ[n];
    if (j + 1 < g.NY) acc -= gJ[NN + n];
    if (k + 1 < g.NZ) acc -= gJ[2 * NN + n];
  }
  b[s] = acc;
}

// dJ/da_e = gJ_e - g_e (lambda_head - lambda_tail); g_e from the level-0
// conductances (0 where the brick is not stored).
__global__ void __launch_bounds__(NT)
k_energy_grad_a(Grid g, const double *__restrict__ gx, const double *__restrict__ lam,
                const double *__restrict__ gJ, double *__restrict__ dJda) {
  const size_t NX = g.NX, NY = g.NY, NN = NX * NY * (size_t)g.NZ;
  const size_t S = (size_t)g.nb * BV;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < NN;
       n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
    const int s = slot_at(g, i, j, k);
    const size_t head[3] = {n + 1, n + NX, n + NX * NY};
    const bool has[3] = {i + 1 < g.NX, j + 1 < g.NY, k + 1 < g.NZ};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double gl = has[d] ? lam[head[d]] - lam[n] : 0.0;
      const double ge = s >= 0 ? gx[(size_t)d * S + s] : 0.0;
      dJda[d * NN + n] = gJ[d * NN + n] - ge * gl;
    }
  }
}

// dJ/dsigma_v = h/4 * sum over the 12 edges e of conducting voxel v of
// -(lambda_head - lambda_tail) u_e (0 in air).
__global__ void __launch_bounds__(NT)
k_energy_grad_sigma(const unsigned char *__restrict__ mask, const double *__restrict__ a,
                    const double *__restrict__ psi, const double *__restrict__ lam,
                    int nx, int ny, int nz, double h, double *__restrict__ dJds) {
  const size_t nv = (size_t)nx * ny * nz;
  const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1), NN = NXY * ((size_t)nz + 1);
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv;
       v += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (mask[v]) {
      int i, j, k;
      voxel_ijk(v, nx, ny, &i, &j, &k);
      const size_t n = (size_t)k * NXY + (size_t)j * NX + i;
#pragma unroll
      for (int pq = 0; pq < 4; ++pq) {
        const int p = pq >> 1, q = pq & 1;
        const size_t t3[3] = {n + p * NX + q * NXY, n + p + q * NXY, n + p + q * NX};
        const size_t off[3] = {1, NX, NXY};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const size_t tl = t3[d], hd = tl + off[d];
          const double u = (a[d * NN + tl] + psi[hd]) - psi[tl];
          const double gl = lam[hd] - lam[tl];
          acc += -gl * u;
        }
      }
      acc *= 0.25 * h;
    }
    dJds[v] = acc;
  }
}

// ------------------------------------------------ smoother eigenvalue estimate
// Power iteration for the Jacobi weight of a 27-point level.  One step is
// w = D^-1 A v, with the generalized Rayleigh quotient terms v.(A v) and
// v.(D v) added into sc->aux[4] and sc->aux[5] (last-block reduction);
// bricks are grid-strided over at most RED_GRID blocks, v is staged in a
// full-halo tile per brick and every slot is handled by its thread.  The
// steps run in FP32 on the level's FP32 copies (the 27 coefficients and the
// inverse diagonal rounded from FP64): the weight is an estimate taken with a
// 5 % margin, so FP32 rounding (relative 1e-7 per operation) does not move
// it, and the iteration leaves GB300's narrow FP64 pipe to the kernels that
// run beside it; only the block totals are widened to FP64.
// Start vector: 0.5 + k / 65536 from a hash of the slot (exact in FP32), zero
// where dinv is zero.
__global__ void __launch_bounds__(NT)
k_power_init_f32(const float *__restrict__ dinv, float *__restrict__ v) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  unsigned h = (unsigned)s * 2654435761u;
  h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
  v[s] = dinv[s] != 0.f ? 0.5f + (float)(h & 0xffff) * (1.f / 65536.f) : 0.f;
}

// v.(D v) takes the centre coefficient for D: it equals the diagonal where
// dinv is nonzero, and v is zero where dinv is zero.
__global__ void __launch_bounds__(NT)
k_power27_f32(Grid g, const float *__restrict__ st, const float *__restrict__ dinv,
              const float *__restrict__ v, float *__restrict__ w, Scalars *sc,
              double *partials) {
  __shared__ float tl[10][10][10];
  __shared__ int sn[27];
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV;
  float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
  for (int bk = blockIdx.x; bk < g.nb; bk += gridDim.x) {
    __syncthreads();  // the previous brick's tile is no longer read
    load_nbr(g, bk, sn);
    __syncthreads();
    tile_full<float>(tl, v, bk, sn);
    __syncthreads();
    const size_t s = (size_t)bk * BV + t;
    const float av = apply27_tile<float>(tl, st, S, s, t);
    const float vs = tile_at(tl, t);
    w[s] = dinv[s] * av;
    two_sum_add(hi[0], lo[0], vs * av, 0.f);
    two_sum_add(hi[1], lo[1], vs * vs * st[13 * S + s], 0.f);
  }
  double tot[2];
  if (grid_sum_f32<2>(hi, lo, partials, &sc->ticket[4], tot)) {
    sc->aux[4] = tot[0];
    sc->aux[5] = tot[1];
  }
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

__global__ void __launch_bounds__(NT)
k_jacobi_weights(const double *__restrict__ dinv, const Scalars *sc, double margin,
                 double *__restrict__ wdinv, double *lam_out) {
  __shared__ double om;
  if (threadIdx.x == 0) {
    double lam = sc->aux[4] / sc->aux[5];
    if (!(lam > 0.0) || !isfinite(lam)) lam = 2.0;
    om = 4.0 / (3.0 * margin * lam);
    if (blockIdx.x == 0) *lam_out = lam;
  }
  __syncthreads();
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  wdinv[s] = om * dinv[s];
}

// ------------------------------------------------ precision conversions
// dst = (T)(f * src) elementwise over n values.  With SCALE false (f = 1,
// every conversion of the build) the values are read as bit patterns and
// rounded with integer operations (narrow_f64_bits): no FP64-pipe slot is
// spent, so the kernel runs at memory speed beside the FP64 work of the
// build (power iterations, coarsest inverse).
template <typename T, bool SCALE>
__global__ void k_convert(size_t n, const double *__restrict__ src, double f,
                          T *__restrict__ dst) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if constexpr (SCALE) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      const double v = f * src[i];
      if constexpr (sizeof(T) == 2) dst[i] = __double2bfloat16(v);
      else dst[i] = (T)v;
    }
  } else {
    // pairs: 16-byte loads (src and dst come from the allocator, 256-byte
    // aligned), then the odd last value
    const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src);
    const size_t n2 = n / 2;
#pragma unroll 4
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += stride) {
      const ulonglong2 u = __ldcs(&s2[i]);
      if constexpr (sizeof(T) == 2) {
        const unsigned lo = narrow_f64_bits<7>(u.x), hi = narrow_f64_bits<7>(u.y);
        reinterpret_cast<unsigned *>(dst)[i] = lo | (hi << 16);
      } else {
        reinterpret_cast<float2 *>(dst)[i] = make_float2(__uint_as_float(narrow_f64_bits<23>(u.x)),
                                                         __uint_as_float(narrow_f64_bits<23>(u.y)));
      }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long u = reinterpret_cast<const unsigned long long *>(src)[n - 1];
      if constexpr (sizeof(T) == 2)
        dst[n - 1] = __ushort_as_bfloat16((unsigned short)narrow_f64_bits<7>(u));
      else
        dst[n - 1] = __uint_as_float(narrow_f64_bits<23>(u));
    }
  }
}

// x += f * d (FP64 accumulation of an FP32 correction) on level-0 slots.
__global__ void __launch_bounds__(NT)
k_axpy_mixed(double *__restrict__ x, const float *__restrict__ d, double f,
             const double *__restrict__ fdev) {
  pdl_entry();
  if (fdev) f = *fdev;
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  x[s] += f * (double)d[s];
}

// r32 = (float)(f * r64); sum(r32) and its mean land in sc->rsum / rmean_f
// for the fused projection of the first V-cycle sweep.
__global__ void __launch_bounds__(NT)
k_scale_to_f32(int nb, const double *__restrict__ r, double f,
               const double *__restrict__ fdev, float *__restrict__ r32, Scalars *sc,
               double *partials) {
  pdl_entry();
  if (fdev) f = *fdev;
  Acc<float> acc;
  for (int bk = blockIdx.x; bk < nb; bk += gridDim.x) {
    const size_t s = (size_t)bk * BV + threadIdx.x;
    const float v = (float)(f * r[s]);
    r32[s] = v;
    acc.add(v);
  }
  const Acc<float> t[1] = {acc};
  double tot[1];
  if (grid_sum_acc<float, 1>(t, partials, &sc->ticket[5], tot)) {
    sc->rsum = tot[0];
    sc->rmean = tot[0] * sc->inv_ndof;
    sc->rmean_f = (float)sc->rmean;
  }
}

// ------------------------------------------------------------ launchers
template <typename T>
void launch_convert(size_t n, const double *src, double f, T *dst,
                    cudaStream_t st) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks == 0) return;
  if (f == 1.0) k_convert<T, false><<<(int)blocks, 256, 0, st>>>(n, src, f, dst);
  else k_convert<T, true><<<(int)blocks, 256, 0, st>>>(n, src, f, dst);
}
template void launch_convert<float>(size_t, const double *, double, float *, cudaStream_t);
template void launch_convert<__nv_bfloat16>(size_t, const double *, double,
                                            __nv_bfloat16 *, cudaStream_t);
void launch_axpy_mixed(int nb, double *x, const float *d, double f,
                       cudaStream_t st, const double *fdev) {
  if (nb) pdl(k_axpy_mixed, nb, NT, st)(x, d, f, fdev);
}
void launch_scale_to_f32(int nb, const double *r, double f, float *r32,
                         Scalars *sc, double *partials, cudaStream_t st, const double *fdev) {
  if (nb)
    pdl(k_scale_to_f32, std::min(nb, RED_GRID), NT, st)(nb, r, f, fdev, r32, sc, partials);
}
void launch_power_init_f32(int nb, const float *dinv, float *v, cudaStream_t st) {
  if (nb) k_power_init_f32<<<nb, NT, 0, st>>>(dinv, v);
}
void launch_power27_f32(const Grid &g, const float *st27, const float *dinv, const float *v,
                        float *w, Scalars *sc, double *partials, cudaStream_t st) {
  if (g.nb)
    k_power27_f32<<<std::min(g.nb, RED_GRID), NT, 0, st>>>(g, st27, dinv, v, w, sc, partials);
}
void launch_scale(int nb, double *v, double f, cudaStream_t st) {
  if (nb) k_scale<<<nb, NT, 0, st>>>(v, f);
}
void launch_jacobi_weights(int nb, const double *dinv, const Scalars *sc, double margin,
                           double *wdinv, double *lam_out, cudaStream_t st) {
  if (nb) k_jacobi_weights<<<nb, NT, 0, st>>>(dinv, sc, margin, wdinv, lam_out);
}
void launch_scaled_copy(int nb, const double *src, double f, double *dst,
                        cudaStream_t st) {
  if (nb) k_scaled_copy<<<nb, NT, 0, st>>>(src, f, dst);
}
template <typename T>
void launch_apply_dot(const Grid &g, const T *gx, const T *diag, const T *p,
                      T *q, Scalars *sc, double *partials, cudaStream_t st, int nk,
                      size_t pstride, int order) {
  if (!g.nb) return;
  if (order)
    pdl(k_apply_dot<T, 1>, unit_grid(1, g.nb, nk), BV / row_n_apply<T>(), st)(
        g, gx, diag, p, q, sc, partials, pstride, nk);
  else
    pdl(k_apply_dot<T, 0>, unit_grid(0, g.nb, nk), BV / row_n_apply<T>(), st)(
        g, gx, diag, p, q, sc, partials, pstride, nk);
}
void launch_finish_rz(int n, const double *partials, double *scratch, Scalars *sc, int first,
                      cudaStream_t st, int nk, size_t pstride, bool pairs) {
  if (n <= 0) return;
  const int blocks = std::min(152, (n + NT - 1) / NT);
  if (pairs)
    pdl(k_finish_rz<true>, dim3(blocks, nk), NT, st)(partials, n, scratch, sc, first, pstride);
  else
    pdl(k_finish_rz<false>, dim3(blocks, nk), NT, st)(partials, n, scratch, sc, first, pstride);
}
void launch_finish_pq(int n, const double *partials, double *scratch, Scalars *sc,
                      cudaStream_t st, int nk, size_t pstride, bool pairs) {
  if (n <= 0) return;
  const int blocks = std::min(152, (n + NT - 1) / NT);
  if (pairs)
    pdl(k_finish_pq<true>, dim3(blocks, nk), NT, st)(partials, n, scratch, sc, pstride);
  else
    pdl(k_finish_pq<false>, dim3(blocks, nk), NT, st)(partials, n, scratch, sc, pstride);
}
template <typename T>
void launch_update_xr(int nb, T *x, T *r, const T *p, const T *q, Scalars *sc,
                      double *partials, cudaStream_t st, int nk, size_t pstride) {
  if (nb)
    pdl(k_update_xr<T>, dim3(std::min(nb, RED_GRID), nk), NT, st)(nb, x, r, p, q, sc,
                                                                    partials, pstride);
}
template <typename T>
void launch_dot_rz(int nb, const T *r, const T *z, const int *comp,
                   Scalars *sc, double *partials, int first, cudaStream_t st, int nk,
                   size_t pstride) {
  if (nb)
    pdl(k_dot_rz<T>, dim3(std::min(nb, RED_GRID), nk), NT, st)(nb, r, z, comp, sc, partials,
                                                                 first, pstride);
}
template <typename T>
void launch_comp_sum(int nb, const T *v, const int *comp, double *ws, int ncomp,
                     int cstride, cudaStream_t st, int nk) {
  cudaMemsetAsync(ws, 0, (size_t)nk * cstride * sizeof(double), st);
  if (!nb) return;
  pdl(k_absmax<T>, dim3(nb, nk), NT, st)(v, comp, ws, cstride, ncomp);
  pdl(k_comp_sum<T>, dim3(nb, nk), NT, st)(v, comp, ws, cstride, ncomp);
  pdl(k_comp_finish, dim3((ncomp + 255) / 256, nk), 256, st)(ws, cstride, ncomp);
}
template <typename T>
void launch_pupdate(int nb, T *p, const T *z, const int *comp,
                    const Scalars *sc, const double *csum, const int *csize,
                    double, cudaStream_t st, int nk, int cstride) {
  if (nb) pdl(k_pupdate<T>, dim3(nb, nk), NT / V16<T>::N, st)(p, z, comp, sc, csum, csize, cstride);
}
template <typename T>
void launch_sub_mean(int nb, T *v, const int *comp, const Scalars *sc,
                     int aux_slot, const double *csum, const int *csize,
                     double, cudaStream_t st, int nk, int cstride) {
  if (nb) pdl(k_sub_mean<T>, dim3(nb, nk), NT, st)(v, comp, sc, aux_slot, csum, csize, cstride);
}
template <typename T>
void launch_dot(int nb, const T *x, const T *y, const int *comp, Scalars *sc,
                double *partials, int slot, cudaStream_t st, int nk, size_t pstride) {
  if (nb)
    pdl(k_dot<T>, dim3(std::min(nb, RED_GRID), nk), NT, st)(nb, x, y, comp, sc, partials,
                                                              slot, pstride);
}
void launch_rhs(const Grid &g, const double *gx, const double *a, double *b,
                int *status, cudaStream_t st, int nk) {
  if (g.nb) k_rhs<<<dim3(g.nb, nk), NT, 0, st>>>(g, gx, a, b, status);
}
template <typename T>
void launch_scatter(const Grid &g, const T *x, const int *comp, double *psi,
                    cudaStream_t st, int nk) {
  size_t NN = (size_t)g.NX * g.NY * g.NZ;
  size_t blocks = (NN + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks == 0) blocks = 1;
  pdl(k_scatter<T>, dim3((int)blocks, nk), 256, st)(g, x, comp, psi);
}
void launch_gather(const Grid &g, const double *psi, const int *comp, double *x,
                   cudaStream_t st) {
  if (g.nb) k_gather<<<g.nb, NT, 0, st>>>(g, psi, comp, x);
}
void launch_efield(const unsigned char *mask, const double *a,
                   const double *psi, int nx, int ny, int nz, double h,
                   double omega, double *E, cudaStream_t st) {
  if ((size_t)nx * ny * nz == 0) return;
  const long long ncol = (long long)(nx + 1) * ny;
  const long long warps = (ncol + 30) / 31;
  const dim3 grid((unsigned)((warps * 32 + EF_THREADS - 1) / EF_THREADS),
                  (unsigned)((nz + EF_KCHUNK - 1) / EF_KCHUNK));
  k_efield<<<grid, EF_THREADS, 0, st>>>(mask, a, psi, nx, ny, nz, omega / (4.0 * h), E);
}

// |E| of a complex source from the magnitudes of its real and imaginary
// parts: E = sqrt(E^2 + E_im^2) in place, each operation rounded on its own
// (no contracted multiply-add), 16-byte loads.
__global__ void __launch_bounds__(256)
k_efield_magnitude(size_t n, double *__restrict__ E, const double *__restrict__ E_im) {
  const size_t n2 = n / 2, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += stride) {
    double2 a = reinterpret_cast<const double2 *>(E)[i];
    const double2 b = reinterpret_cast<const double2 *>(E_im)[i];
    a.x = sqrt(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(b.x, b.x)));
    a.y = sqrt(__dadd_rn(__dmul_rn(a.y, a.y), __dmul_rn(b.y, b.y)));
    reinterpret_cast<double2 *>(E)[i] = a;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
    E[n - 1] = sqrt(__dadd_rn(__dmul_rn(E[n - 1], E[n - 1]), __dmul_rn(E_im[n - 1], E_im[n - 1])));
}

void launch_efield_magnitude(size_t n, double *E, const double *E_im, cudaStream_t st) {
  if (n == 0) return;
  const size_t blocks = std::min<size_t>((n / 2 + 255) / 256 + 1, 152 * 16);
  k_efield_magnitude<<<(unsigned)blocks, 256, 0, st>>>(n, E, E_im);
}

static int grid_for(size_t n) {
  size_t b = (n + NT - 1) / NT;
  return (int)std::max<size_t>(1, std::min<size_t>(b, RED_GRID));
}
void launch_energy(const unsigned char *mask, const double *a, const double *psi, int nx,
                   int ny, int nz, double c, double *Ev, Scalars *sc, double *partials,
                   cudaStream_t st) {
  const size_t nv = (size_t)nx * ny * nz;
  k_energy<<<grid_for(nv), NT, 0, st>>>(mask, a, psi, nx, ny, nz, c, Ev, sc, partials);
}
void launch_energy_gJ(const unsigned char *mask, const double *Ev, int nx, int ny, int nz,
                      double c, const Scalars *sc, double *gJ, cudaStream_t st) {
  const size_t NN = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  k_energy_gJ<<<(int)std::min<size_t>((3 * NN + NT - 1) / NT, 152 * 64), NT, 0, st>>>(
      mask, Ev, nx, ny, nz, c, sc, gJ);
}
void launch_div_brick(const Grid &g, const double *diag, const double *gJ, double *b,
                      cudaStream_t st) {
  if (g.nb) k_div_brick<<<g.nb, NT, 0, st>>>(g, diag, gJ, b);
}
void launch_energy_grads(const Grid &g, const double *gx, const unsigned char *mask,
                         const double *a, const double *psi, const double *lam,
                         const double *gJ, int nx, int ny, int nz, double h, double *dJda,
                         double *dJds, cudaStream_t st) {
  const size_t NN = (size_t)g.NX * g.NY * g.NZ, nv = (size_t)nx * ny * nz;
  k_energy_grad_a<<<(int)std::min<size_t>((NN + NT - 1) / NT, 152 * 64), NT, 0, st>>>(
      g, gx, lam, gJ, dJda);
  if (nv)
    k_energy_grad_sigma<<<(int)std::min<size_t>((nv + NT - 1) / NT, 152 * 64), NT, 0, st>>>(
        mask, a, psi, lam, nx, ny, nz, h, dJds);
}

#define INST_K(T)                                                              \
  template void launch_apply_dot<T>(const Grid &, const T *, const T *,        \
                                    const T *, T *, Scalars *, double *,       \
                                    cudaStream_t, int, size_t, int);           \
  template void launch_update_xr<T>(int, T *, T *, const T *, const T *,       \
                                    Scalars *, double *, cudaStream_t, int,    \
                                    size_t);                                   \
  template void launch_dot_rz<T>(int, const T *, const T *, const int *,       \
                                 Scalars *, double *, int, cudaStream_t, int,  \
                                 size_t);                                      \
  template void launch_comp_sum<T>(int, const T *, const int *, double *, int, \
                                   int, cudaStream_t, int);                    \
  template void launch_pupdate<T>(int, T *, const T *, const int *,            \
                                  const Scalars *, const double *,             \
                                  const int *, double, cudaStream_t, int,      \
                                  int);                                        \
  template void launch_sub_mean<T>(int, T *, const int *, const Scalars *,     \
                                   int, const double *, const int *, double,   \
                                   cudaStream_t, int, int);                    \
  template void launch_dot<T>(int, const T *, const T *, const int *,          \
                              Scalars *, double *, int, cudaStream_t, int,     \
                              size_t);                                         \
  template void launch_scatter<T>(const Grid &, const T *, const int *,        \
                                  double *, cudaStream_t, int);
template int apply_dot_partials<double>(int);
template int apply_dot_partials<float>(int);
INST_K(double)
INST_K(float)

}  // namespace spfd
