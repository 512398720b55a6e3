// Brick access patterns of the stencil kernels.
//
// 27-point stencils (coarse levels): a block handles one 8x8x8 brick with
// one thread per node, loads its brick's 27 neighbour ids once and stages
// the vector it reads into a 10x10x10 shared tile (the brick plus its full
// one-node halo), so that every stencil read is a shared-memory load.
// 7-point operator (level 0): the row mapping below, four nodes per thread
// and no shared memory.  Either way, neighbours in bricks that are not stored
// read as zero, which matches the zero operator rows and vector entries of
// nodes that are not unknowns.
#pragma once

#include "spfd_internal.cuh"

namespace spfd {

template <typename T> __device__ __forceinline__ T cvt(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cvt(float v) { return (T)v; }
// BF16 is the upper half of an IEEE binary32: widening is exact and needs
// only the bits moved into place (two integer operations for a pair).
__device__ __forceinline__ float bf16_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }
template <typename T> __device__ __forceinline__ T cvt(__nv_bfloat16 v) {
  return (T)bf16_lo((unsigned)__bfloat16_as_ushort(v));
}

// 16-byte vectors of T (4 floats or 2 doubles) for streaming kernels; slot
// offsets used with them are multiples of the vector length and arrays come
// from cudaMalloc, so every access is 16-byte aligned.
template <typename T>
struct alignas(16) V16 {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};
template <typename T>
__device__ __forceinline__ V16<T> ld16(const T *p) {
  V16<T> r;
  *reinterpret_cast<uint4 *>(&r) = *reinterpret_cast<const uint4 *>(p);
  return r;
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const V16<T> &r) {
  *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(&r);
}
// N consecutive ints (the component ids matching a V16<T>).
template <int N>
__device__ __forceinline__ void ld_ints(const int *p, int (&c)[N]) {
  if constexpr (N == 4) {
    const int4 q = *reinterpret_cast<const int4 *>(p);
    c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
  } else {
    const int2 q = *reinterpret_cast<const int2 *>(p);
    c[0] = q.x; c[1] = q.y;
  }
}

// Vector loads.  COH = false: plain loads (standalone kernels: what they
// read was written by earlier launches).  COH = true: L2-only loads
// (ld.global.cg), for a vector written by other blocks earlier in the same
// launch (the fused coarse cycle), of which this SM's L1 may hold a stale
// line.
template <bool COH, typename T>
__device__ __forceinline__ T ldv(const T *p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// Neighbour brick ids of brick bk into shared memory (threads 0..26).
__device__ __forceinline__ void load_nbr(const Grid &g, int bk, int *sn) {
  if (threadIdx.x < 27) sn[threadIdx.x] = g.nbr[(size_t)bk * 27 + threadIdx.x];
}

// Brick + full halo of x (27-point stencils): the brick itself as 16-byte
// vectors, the 488 halo values from the neighbour bricks one per thread
// (planes tz = 0 and 9, then ty = 0 and 9, then tx = 0 and 9).
template <typename T, bool COH = false>
__device__ __forceinline__ void tile_full(T (*tl)[10][10], const T *__restrict__ x,
                                          int bk, const int *sn) {
  constexpr int VN = 16 / (int)sizeof(T), VPB = BV / VN;
  const int t = threadIdx.x;
  if (t < VPB) {
    const int e0 = t * VN, lx = e0 & 7, ly = (e0 >> 3) & 7, lz = e0 >> 6;
    const T *p = x + (size_t)bk * BV + e0;
    V16<T> v;
    if constexpr (COH) *reinterpret_cast<uint4 *>(&v) = __ldcg(reinterpret_cast<const uint4 *>(p));
    else v = ld16(p);
    T *row = &tl[1 + lz][1 + ly][1 + lx];
#pragma unroll
    for (int i = 0; i < VN; ++i) row[i] = v.v[i];
  }
  for (int u = (t + NT - VPB) % NT; u < 488; u += NT) {
    int tz, ty, tx;
    if (u < 200) {
      tz = u < 100 ? 0 : 9;
      const int r = u % 100;
      ty = r / 10; tx = r % 10;
    } else if (u < 360) {
      const int v = u - 200, w = v % 20;
      tz = 1 + v / 20; ty = w < 10 ? 0 : 9; tx = w % 10;
    } else {
      const int v = u - 360, w = v % 16;
      tz = 1 + v / 16; ty = 1 + (w >> 1); tx = (w & 1) ? 9 : 0;
    }
    const int ox = tx == 0 ? -1 : (tx == 9 ? 1 : 0);
    const int oy = ty == 0 ? -1 : (ty == 9 ? 1 : 0);
    const int oz = tz == 0 ? -1 : (tz == 9 ? 1 : 0);
    const int nb = sn[sidx(ox, oy, oz)];
    tl[tz][ty][tx] = nb >= 0
        ? ldv<COH>(&x[(size_t)nb * BV + (((tz - 1) & 7) * 8 + ((ty - 1) & 7)) * 8 + ((tx - 1) & 7)])
        : T(0);
  }
}

// ----------------------------------------------- level-0 7-point operator
// Row mapping: the N consecutive x nodes N h .. N h + N - 1 of row y of plane
// z of one brick go to one thread (h < 8 / N; the 8 / N threads of a row are
// consecutive lanes).  Own values and conductances arrive as vector loads,
// the +-y/+-z neighbours as the vectors of the rows beside it (L1/L2 hits
// inside the brick), the +-x neighbours of the row ends from the neighbouring
// lanes by shuffle or from the x-neighbour brick.  No shared memory, no
// barrier.
// Nodes per thread along x: FP64 kernels take two (half the registers of
// four, so twice the resident warps hide the memory latency behind the FP64
// pipe), FP32 kernels four (16-byte vector accesses, memory-bound).
template <typename T>
constexpr int row_n() { return sizeof(T) == 8 ? 2 : 4; }
// The weighted-Jacobi sweep keeps four nodes per thread in FP64 too: with
// two it measured 4 % slower on the 2 mm body, the residual 11 % faster.
template <typename T>
constexpr int row_n_jacobi() { return 4; }
// The CG operator takes four nodes per thread in both precisions (in FP64
// with its neighbour lookups first: 193.5 us per launch on the 2 mm body,
// against 206.8 us with two nodes per thread over a list of the rows that
// hold an unknown).
template <typename T>
constexpr int row_n_apply() { return 4; }
// Threads per brick in the row mapping.
template <typename T>
constexpr int row_threads() { return BV / row_n<T>(); }
// Resident blocks per SM asked of the compiler for row kernels: FP32 kernels
// wait on memory and want many warps in flight (10 blocks of 128 threads);
// FP64 kernels take 4 blocks (of 256 threads: 64 registers; of 128: 128).
template <typename T>
constexpr int row_min_blocks() { return sizeof(T) == 4 ? 10 : 4; }
// The weighted-Jacobi sweep asks for 9 resident FP32 blocks (56 registers,
// no spills): 61.4 against 65.1 us per level-0 launch on the 2 mm body with
// 10 (48 registers and spills); the residual and the CG operator measured
// 2-3 % slower with 9 and keep 10.
template <typename T>
constexpr int row_min_blocks_jacobi() { return sizeof(T) == 4 ? 9 : 4; }
// The FP64 CG operator (four nodes per thread) asks for 5 resident blocks (96
// registers): 190 against 195 us per launch with 4 (108 registers); 6 (80
// registers and spills) gave 193 us.
template <typename T>
constexpr int row_min_blocks_apply() { return sizeof(T) == 4 ? 10 : 5; }

template <typename T, int N>
struct Qv {
  T v[N];
};

// N consecutive values at p (aligned to their total size, or to 4 bytes for
// two BF16 values), widened to T.
template <typename T, typename C, int N>
__device__ __forceinline__ Qv<T, N> ldqn(const C *__restrict__ p) {
  Qv<T, N> r;
  if constexpr (N == 4) {
    if constexpr (sizeof(C) == 4) {
      const float4 u = *reinterpret_cast<const float4 *>(p);
      r.v[0] = (T)u.x; r.v[1] = (T)u.y; r.v[2] = (T)u.z; r.v[3] = (T)u.w;
    } else if constexpr (sizeof(C) == 8) {
      const double2 u = reinterpret_cast<const double2 *>(p)[0];
      const double2 w = reinterpret_cast<const double2 *>(p)[1];
      r.v[0] = (T)u.x; r.v[1] = (T)u.y; r.v[2] = (T)w.x; r.v[3] = (T)w.y;
    } else {
      const uint2 u = *reinterpret_cast<const uint2 *>(p);
      r.v[0] = (T)bf16_lo(u.x); r.v[1] = (T)bf16_hi(u.x);
      r.v[2] = (T)bf16_lo(u.y); r.v[3] = (T)bf16_hi(u.y);
    }
  } else {
    static_assert(N == 2, "two or four nodes per thread");
    if constexpr (sizeof(C) == 4) {
      const float2 u = *reinterpret_cast<const float2 *>(p);
      r.v[0] = (T)u.x; r.v[1] = (T)u.y;
    } else if constexpr (sizeof(C) == 8) {
      const double2 u = *reinterpret_cast<const double2 *>(p);
      r.v[0] = (T)u.x; r.v[1] = (T)u.y;
    } else {
      const unsigned u = *reinterpret_cast<const unsigned *>(p);
      r.v[0] = (T)bf16_lo(u); r.v[1] = (T)bf16_hi(u);
    }
  }
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Qv<T, N> zqn() {
  Qv<T, N> r;
#pragma unroll
  for (int i = 0; i < N; ++i) r.v[i] = T(0);
  return r;
}
template <typename T, int N>
__device__ __forceinline__ void stqn(T *__restrict__ p, const Qv<T, N> &r) {
  if constexpr (N == 4) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
      reinterpret_cast<double2 *>(p)[0] = make_double2(r.v[0], r.v[1]);
      reinterpret_cast<double2 *>(p)[1] = make_double2(r.v[2], r.v[3]);
    }
  } else {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float2 *>(p) = make_float2(r.v[0], r.v[1]);
    else *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
  }
}

// First slot of this thread's N nodes in brick b: 8 / N threads per row,
// rows in (z, y) order.
template <int N>
__device__ __forceinline__ size_t row_slot(int b, int t) {
  constexpr int TPR = 8 / N;
  return (size_t)b * BV + (t / (8 * TPR)) * 64 + ((t / TPR) & 7) * 8 + N * (t % TPR);
}

// The vector beside the row at s0: at offset in_off when that stays in the
// brick, else the row `across` of the neighbour brick e (zero if that brick
// is not stored).
template <typename T, typename C, int N>
__device__ __forceinline__ Qv<T, N> ldq_nb(const C *__restrict__ v, size_t s0, bool inside,
                                           long long in_off, const Grid &g, int b, int e,
                                           size_t across) {
  if (inside) return ldqn<T, C, N>(v + (long long)s0 + in_off);
  const int nb = __ldg(&g.nbr[(size_t)b * 27 + e]);
  return nb >= 0 ? ldqn<T, C, N>(v + (size_t)nb * BV + across) : zqn<T, N>();
}

// The same with the neighbour brick's id already looked up (nb).
template <typename T, typename C, int N>
__device__ __forceinline__ Qv<T, N> ldq_nbi(const C *__restrict__ v, size_t s0, bool inside,
                                            long long in_off, int nb, size_t across) {
  if (inside) return ldqn<T, C, N>(v + (long long)s0 + in_off);
  return nb >= 0 ? ldqn<T, C, N>(v + (size_t)nb * BV + across) : zqn<T, N>();
}

// out = A x (RES = false) or base - A x (RES = true) at this thread's N
// nodes of brick b, and xc = x there.  FP64: diag*x - sum g x_nbr, with base
// folded into the first FMA (fewest FP64-pipe operations).  FP32: sum
// g (x - x_nbr), exactly zero on constants, so rounded (BF16/FP32)
// conductances keep the operator positive semidefinite.  The x-neighbours
// of the row ends come from the neighbouring lanes by shuffle (a row's
// threads are consecutive lanes), else from the x-neighbour brick.  All 32
// lanes of each warp must call it.
template <typename T, typename C, bool RES, int N, bool NBF = RES>
__device__ __forceinline__ void apply7_row(const Grid &g, const C *__restrict__ gx,
                                           const T *__restrict__ diag, const T *__restrict__ x,
                                           size_t S, int b, int t, const Qv<T, N> &base,
                                           Qv<T, N> &xc, Qv<T, N> &out) {
  constexpr int TPR = 8 / N;
  const int h = t % TPR, y = (t / TPR) & 7, z = t / (8 * TPR);
  const size_t s0 = row_slot<N>(b, t);
  const size_t rz = (size_t)z * 64 + N * h, ry = (size_t)y * 8 + N * h;
  // NBF: the (at most one per axis) neighbour bricks this thread reads from
  // are looked up before any load that needs one (7 % and 6 % faster FP64
  // sweep and residual, 4-5 % in FP32, 6 % faster FP64 CG operator); the FP32
  // CG operator measured 11 % slower that way and keeps the lookups at its
  // loads
  int nx = -1, ny = -1, nz = -1;
  if constexpr (NBF) {
    const int *nt = g.nbr + (size_t)b * 27;
    nx = __ldg(nt + (h == 0 ? sidx(-1, 0, 0) : sidx(1, 0, 0)));
    if (y == 0 || y == 7) ny = __ldg(nt + (y == 0 ? sidx(0, -1, 0) : sidx(0, 1, 0)));
    if (z == 0 || z == 7) nz = __ldg(nt + (z == 0 ? sidx(0, 0, -1) : sidx(0, 0, 1)));
  }
  xc = ldqn<T, T, N>(x + s0);
  const Qv<T, N> gpx = ldqn<T, C, N>(gx + s0), gpy = ldqn<T, C, N>(gx + S + s0),
                 gpz = ldqn<T, C, N>(gx + 2 * S + s0);
  Qv<T, N> xym, xyp, xzm, xzp, gmy, gmz;
  if constexpr (NBF) {
    xym = ldq_nbi<T, T, N>(x, s0, y > 0, -8, ny, rz + 56);
    xyp = ldq_nbi<T, T, N>(x, s0, y < 7, 8, ny, rz);
    xzm = ldq_nbi<T, T, N>(x, s0, z > 0, -64, nz, 448 + ry);
    xzp = ldq_nbi<T, T, N>(x, s0, z < 7, 64, nz, ry);
    gmy = ldq_nbi<T, C, N>(gx + S, s0, y > 0, -8, ny, rz + 56);
    gmz = ldq_nbi<T, C, N>(gx + 2 * S, s0, z > 0, -64, nz, 448 + ry);
  } else {
    xym = ldq_nb<T, T, N>(x, s0, y > 0, -8, g, b, sidx(0, -1, 0), rz + 56);
    xyp = ldq_nb<T, T, N>(x, s0, y < 7, 8, g, b, sidx(0, 1, 0), rz);
    xzm = ldq_nb<T, T, N>(x, s0, z > 0, -64, g, b, sidx(0, 0, -1), 448 + ry);
    xzp = ldq_nb<T, T, N>(x, s0, z < 7, 64, g, b, sidx(0, 0, 1), ry);
    gmy = ldq_nb<T, C, N>(gx + S, s0, y > 0, -8, g, b, sidx(0, -1, 0), rz + 56);
    gmz = ldq_nb<T, C, N>(gx + 2 * S, s0, z > 0, -64, g, b, sidx(0, 0, -1), 448 + ry);
  }
  // row ends: the neighbouring lanes' end values, else the x-neighbour brick
  const T prev_last = __shfl_up_sync(0xffffffffu, xc.v[N - 1], 1);
  const T prev_glast = __shfl_up_sync(0xffffffffu, gpx.v[N - 1], 1);
  const T next_first = __shfl_down_sync(0xffffffffu, xc.v[0], 1);
  T xl, xr, gl;
  if (h == 0) {
    const int nb = NBF ? nx : __ldg(&g.nbr[(size_t)b * 27 + sidx(-1, 0, 0)]);
    const size_t m = (size_t)nb * BV + (size_t)z * 64 + (size_t)y * 8 + 7;
    xl = nb >= 0 ? x[m] : T(0);
    gl = nb >= 0 ? cvt<T>(gx[m]) : T(0);
  } else {
    xl = prev_last;
    gl = prev_glast;
  }
  if (h == TPR - 1) {
    const int nb = NBF ? nx : __ldg(&g.nbr[(size_t)b * 27 + sidx(1, 0, 0)]);
    xr = nb >= 0 ? x[(size_t)nb * BV + (size_t)z * 64 + (size_t)y * 8] : T(0);
  } else {
    xr = next_first;
  }
  Qv<T, N> dg;
  if constexpr (sizeof(T) == 8) dg = ldqn<T, T, N>(diag + s0);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const T c = xc.v[i];
    const T left = i > 0 ? xc.v[i - 1] : xl, right = i < N - 1 ? xc.v[i + 1] : xr;
    const T gmx = i > 0 ? gpx.v[i - 1] : gl;
    if constexpr (sizeof(T) == 4) {
      const T ax = gpx.v[i] * (c - right) + gmx * (c - left) + gpy.v[i] * (c - xyp.v[i]) +
                   gmy.v[i] * (c - xym.v[i]) + gpz.v[i] * (c - xzp.v[i]) +
                   gmz.v[i] * (c - xzm.v[i]);
      out.v[i] = RES ? base.v[i] - ax : ax;
    } else if constexpr (RES) {
      T acc = base.v[i] - dg.v[i] * c;
      acc += gpx.v[i] * right;
      acc += gmx * left;
      acc += gpy.v[i] * xyp.v[i];
      acc += gmy.v[i] * xym.v[i];
      acc += gpz.v[i] * xzp.v[i];
      acc += gmz.v[i] * xzm.v[i];
      out.v[i] = acc;
    } else {
      T acc = dg.v[i] * c;
      acc -= gpx.v[i] * right;
      acc -= gmx * left;
      acc -= gpy.v[i] * xyp.v[i];
      acc -= gmy.v[i] * xym.v[i];
      acc -= gpz.v[i] * xzp.v[i];
      acc -= gmz.v[i] * xzm.v[i];
      out.v[i] = acc;
    }
  }
}

// 27-point stencil at local slot ts (global slot s) of the tiled brick, x
// in a full-halo tile.
template <typename T>
__device__ __forceinline__ T apply27_tile(const T (*tl)[10][10], const T *__restrict__ st,
                                          size_t S, size_t s, int ts) {
  const int lx = ts & 7, ly = (ts >> 3) & 7, lz = ts >> 6;
  T acc = 0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    acc += st[(size_t)e * S + s] * tl[lz + 1 + dz][ly + 1 + dy][lx + 1 + dx];
  }
  return acc;
}

// The tile's value at local slot ts of its brick.
template <typename T>
__device__ __forceinline__ T tile_at(const T (*tl)[10][10], int ts) {
  return tl[(ts >> 6) + 1][((ts >> 3) & 7) + 1][(ts & 7) + 1];
}

// Sum of the N values of every lane of the warp, held by every lane: an
// FP64 sum for double; for float, an error-free (TwoSum) FP32 pair over the
// thread's values and the warp.  get() rounds it to FP64.
template <typename T> struct WarpSum;
// put() stores the sum into one 8-byte partial slot: the FP64 value, or the
// FP32 pair (hi, lo) as is, for a finishing kernel that widens it (pair_at)
// so that the FP32 kernel itself issues no FP64 instruction.
template <> struct WarpSum<double> {
  double s;
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ void put(double *slot) const { *slot = s; }
};
template <> struct WarpSum<float> {
  float hi, lo;
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ void put(double *slot) const {
    *reinterpret_cast<float2 *>(slot) = make_float2(hi, lo);
  }
};
// The value of partial slot i: an FP64 value, or (PAIRS) an FP32 pair
// written by WarpSum<float>::put.
template <bool PAIRS>
__device__ __forceinline__ double pair_at(const double *p, size_t i) {
  if constexpr (PAIRS) {
    const float2 q = reinterpret_cast<const float2 *>(p)[i];
    return (double)q.x + (double)q.y;
  } else {
    return p[i];
  }
}
template <typename T, int N>
__device__ __forceinline__ WarpSum<T> warp_total(const T (&v)[N]) {
  if constexpr (sizeof(T) == 4) {
    float hi = v[0], lo = 0.f;
#pragma unroll
    for (int i = 1; i < N; ++i) {
      const float sh = hi + v[i], bb = sh - hi;
      lo += (hi - (sh - bb)) + (v[i] - bb);
      hi = sh;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
      const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
      const float sh = hi + oh, bb = sh - hi;
      const float e = (hi - (sh - bb)) + (oh - bb);
      hi = sh;
      lo = lo + ol + e;
    }
    return WarpSum<float>{hi, lo};
  } else {
    double a = v[0];
#pragma unroll
    for (int i = 1; i < N; ++i) a += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return WarpSum<double>{a};
  }
}

// The 27 entries e * S + s of a direction-major array (stencil coefficients
// or interpolation weights of one node) into registers.
template <typename T>
__device__ __forceinline__ void load27(const T *__restrict__ a, size_t S, size_t s, T (&v)[27]) {
#pragma unroll
  for (int e = 0; e < 27; ++e) v[e] = a[(size_t)e * S + s];
}

// apply27_tile with the coefficients in registers (same order of terms).
template <typename T>
__device__ __forceinline__ T apply27_regs(const T (*tl)[10][10], const T (&cf)[27], int ts) {
  const int lx = ts & 7, ly = (ts >> 3) & 7, lz = ts >> 6;
  T acc = 0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    acc += cf[e] * tl[lz + 1 + dz][ly + 1 + dy][lx + 1 + dx];
  }
  return acc;
}

}  // namespace spfd
