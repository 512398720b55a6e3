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
template <typename T> __device__ __forceinline__ T cvt(__nv_bfloat16 v) {
  return (T)__bfloat162float(v);
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

// Neighbour brick ids of brick bk into shared memory (threads 0..26).
__device__ __forceinline__ void load_nbr(const Grid &g, int bk, int *sn) {
  if (threadIdx.x < 27) sn[threadIdx.x] = g.nbr[(size_t)bk * 27 + threadIdx.x];
}

// Brick + full halo of x (27-point stencils).
template <typename T>
__device__ __forceinline__ void tile_full(T (*tl)[10][10], const T *__restrict__ x,
                                          int bk, const int *sn) {
  for (int q = threadIdx.x; q < 1000; q += NT) {
    const int tz = q / 100, ty = (q / 10) % 10, tx = q % 10;
    const int ox = tx == 0 ? -1 : (tx == 9 ? 1 : 0);
    const int oy = ty == 0 ? -1 : (ty == 9 ? 1 : 0);
    const int oz = tz == 0 ? -1 : (tz == 9 ? 1 : 0);
    const int nb = (ox | oy | oz) ? sn[sidx(ox, oy, oz)] : bk;
    tl[tz][ty][tx] = nb >= 0
        ? x[(size_t)nb * BV + (((tz - 1) & 7) * 8 + ((ty - 1) & 7)) * 8 + ((tx - 1) & 7)]
        : T(0);
  }
}

// ----------------------------------------------- level-0 7-point operator
// Row mapping: thread t of a 128-thread group covers the four nodes
// x = 4h .. 4h+3 (h = t & 1) of row y = (t >> 1) & 7 of plane z = t >> 4 of
// one brick.  Own values and conductances arrive as 16-byte vectors, the
// +-y/+-z neighbours as the vectors of the rows beside it (L1/L2 hits inside
// the brick), the +-x neighbours of the row ends from the other half-row by
// shuffle or from the x-neighbour brick.  No shared memory, no barrier.
constexpr int RT = 128;  // threads per brick in the row mapping
// Resident blocks per SM asked of the compiler for row kernels: FP32 kernels
// wait on memory and want many warps in flight (12 blocks = 48 warps caps
// them at 40 registers); FP64 kernels are bound by the FP64 pipe and keep
// their registers.
template <typename T>
constexpr int row_min_blocks() { return sizeof(T) == 4 ? 10 : 4; }

template <typename T>
struct Q4 {
  T v[4];
};

// Four consecutive values at p (16-byte aligned for float/double, 8-byte for
// BF16), widened to T.
template <typename T, typename C>
__device__ __forceinline__ Q4<T> ldq(const C *__restrict__ p) {
  Q4<T> r;
  if constexpr (sizeof(C) == 4) {
    const float4 u = *reinterpret_cast<const float4 *>(p);
    r.v[0] = (T)u.x; r.v[1] = (T)u.y; r.v[2] = (T)u.z; r.v[3] = (T)u.w;
  } else if constexpr (sizeof(C) == 8) {
    const double2 u = reinterpret_cast<const double2 *>(p)[0];
    const double2 w = reinterpret_cast<const double2 *>(p)[1];
    r.v[0] = (T)u.x; r.v[1] = (T)u.y; r.v[2] = (T)w.x; r.v[3] = (T)w.y;
  } else {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    r.v[0] = (T)fa.x; r.v[1] = (T)fa.y; r.v[2] = (T)fb.x; r.v[3] = (T)fb.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ Q4<T> zq() {
  Q4<T> r;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.v[i] = T(0);
  return r;
}
template <typename T>
__device__ __forceinline__ void stq(T *__restrict__ p, const Q4<T> &r) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
    reinterpret_cast<double2 *>(p)[0] = make_double2(r.v[0], r.v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(r.v[2], r.v[3]);
  }
}

// First slot of this thread's four nodes in brick b.
__device__ __forceinline__ size_t row_slot(int b, int t) {
  return (size_t)b * BV + (t >> 4) * 64 + ((t >> 1) & 7) * 8 + 4 * (t & 1);
}

// The vector beside the row at s0: at offset in_off when that stays in the
// brick, else the row `across` of the neighbour brick e (zero if that brick
// is not stored).
template <typename T, typename C>
__device__ __forceinline__ Q4<T> ldq_nb(const C *__restrict__ v, size_t s0, bool inside,
                                        long long in_off, const Grid &g, int b, int e,
                                        size_t across) {
  if (inside) return ldq<T>(v + (long long)s0 + in_off);
  const int nb = __ldg(&g.nbr[(size_t)b * 27 + e]);
  return nb >= 0 ? ldq<T>(v + (size_t)nb * BV + across) : zq<T>();
}

// out = A x (RES = false) or base - A x (RES = true) at this thread's four
// nodes of brick b, and xc = x there.  FP64: diag*x - sum g x_nbr, with base
// folded into the first FMA (fewest FP64-pipe operations).  FP32: sum
// g (x - x_nbr), exactly zero on constants, so rounded (BF16/FP32)
// conductances keep the operator positive semidefinite.  All 32 lanes of
// each warp must call it (row-end shuffles).
template <typename T, typename C, bool RES>
__device__ __forceinline__ void apply7_row(const Grid &g, const C *__restrict__ gx,
                                           const T *__restrict__ diag, const T *__restrict__ x,
                                           size_t S, int b, int t, const Q4<T> &base,
                                           Q4<T> &xc, Q4<T> &out) {
  const int h = t & 1, y = (t >> 1) & 7, z = t >> 4;
  const size_t s0 = row_slot(b, t);
  const size_t rz = (size_t)z * 64 + 4 * h, ry = (size_t)y * 8 + 4 * h;
  xc = ldq<T>(x + s0);
  const Q4<T> gpx = ldq<T>(gx + s0), gpy = ldq<T>(gx + S + s0), gpz = ldq<T>(gx + 2 * S + s0);
  const Q4<T> xym = ldq_nb<T>(x, s0, y > 0, -8, g, b, sidx(0, -1, 0), rz + 56);
  const Q4<T> xyp = ldq_nb<T>(x, s0, y < 7, 8, g, b, sidx(0, 1, 0), rz);
  const Q4<T> xzm = ldq_nb<T>(x, s0, z > 0, -64, g, b, sidx(0, 0, -1), 448 + ry);
  const Q4<T> xzp = ldq_nb<T>(x, s0, z < 7, 64, g, b, sidx(0, 0, 1), ry);
  const Q4<T> gmy = ldq_nb<T>(gx + S, s0, y > 0, -8, g, b, sidx(0, -1, 0), rz + 56);
  const Q4<T> gmz = ldq_nb<T>(gx + 2 * S, s0, z > 0, -64, g, b, sidx(0, 0, -1), 448 + ry);
  // row ends: the other half-row by shuffle, else the x-neighbour brick
  const T o_first = __shfl_xor_sync(0xffffffffu, xc.v[0], 1);
  const T o_last = __shfl_xor_sync(0xffffffffu, xc.v[3], 1);
  const T og_last = __shfl_xor_sync(0xffffffffu, gpx.v[3], 1);
  T xl, xr, gl;
  if (h == 0) {
    xr = o_first;
    const int nb = __ldg(&g.nbr[(size_t)b * 27 + sidx(-1, 0, 0)]);
    const size_t m = (size_t)nb * BV + (size_t)z * 64 + (size_t)y * 8 + 7;
    xl = nb >= 0 ? x[m] : T(0);
    gl = nb >= 0 ? cvt<T>(gx[m]) : T(0);
  } else {
    xl = o_last;
    gl = og_last;
    const int nb = __ldg(&g.nbr[(size_t)b * 27 + sidx(1, 0, 0)]);
    xr = nb >= 0 ? x[(size_t)nb * BV + (size_t)z * 64 + (size_t)y * 8] : T(0);
  }
  Q4<T> dg;
  if constexpr (sizeof(T) == 8) dg = ldq<T>(diag + s0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T c = xc.v[i];
    const T left = i > 0 ? xc.v[i - 1] : xl, right = i < 3 ? xc.v[i + 1] : xr;
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

// 27-point stencil at this thread's node, x in a full-halo tile.
template <typename T>
__device__ __forceinline__ T apply27_tile(const T (*tl)[10][10], const T *__restrict__ st,
                                          size_t S, size_t s) {
  const int t = threadIdx.x, lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  T acc = 0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    acc += st[(size_t)e * S + s] * tl[lz + 1 + dz][ly + 1 + dy][lx + 1 + dx];
  }
  return acc;
}

}  // namespace spfd
