// Shared-memory brick tiles for the stencil kernels.
//
// A block handles one 8x8x8 brick with one thread per node.  The block loads
// its brick's 27 neighbour ids once, then stages the vector it reads into a
// 10x10x10 tile (the brick plus a one-node halo: the six faces for the
// 7-point operator, all 26 neighbours for 27-point stencils), so that every
// stencil read is a shared-memory load and no thread computes neighbour
// addresses.  Halo entries of absent bricks are zero, which matches the zero
// operator rows and vector entries of nodes that are not unknowns.
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

// Brick + face halo of x (7-point stencils).
template <typename T>
__device__ __forceinline__ void tile_faces(T (*tl)[10][10], const T *__restrict__ x,
                                           int bk, const int *sn) {
  const int t = threadIdx.x, lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  tl[lz + 1][ly + 1][lx + 1] = x[(size_t)bk * BV + t];
  if (t < 384) {
    const int f = t >> 6, u = t & 7, v = (t >> 3) & 7;
    int e, sx, sy, sz, tx, ty, tz;
    switch (f) {
      case 0: e = sidx(-1, 0, 0); sx = 7; sy = u; sz = v; tx = 0; ty = u + 1; tz = v + 1; break;
      case 1: e = sidx(1, 0, 0);  sx = 0; sy = u; sz = v; tx = 9; ty = u + 1; tz = v + 1; break;
      case 2: e = sidx(0, -1, 0); sx = u; sy = 7; sz = v; tx = u + 1; ty = 0; tz = v + 1; break;
      case 3: e = sidx(0, 1, 0);  sx = u; sy = 0; sz = v; tx = u + 1; ty = 9; tz = v + 1; break;
      case 4: e = sidx(0, 0, -1); sx = u; sy = v; sz = 7; tx = u + 1; ty = v + 1; tz = 0; break;
      default: e = sidx(0, 0, 1); sx = u; sy = v; sz = 0; tx = u + 1; ty = v + 1; tz = 9; break;
    }
    const int nb = sn[e];
    tl[tz][ty][tx] = nb >= 0 ? x[(size_t)nb * BV + (sz * 8 + sy) * 8 + sx] : T(0);
  }
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

// Face halo only (the centre value is stored by its own thread).
template <typename T>
__device__ __forceinline__ void tile_face_halo(T (*tl)[10][10], const T *__restrict__ x,
                                               const int *sn) {
  const int t = threadIdx.x;
  if (t < 384) {
    const int f = t >> 6, u = t & 7, v = (t >> 3) & 7;
    int e, sx, sy, sz, tx, ty, tz;
    switch (f) {
      case 0: e = sidx(-1, 0, 0); sx = 7; sy = u; sz = v; tx = 0; ty = u + 1; tz = v + 1; break;
      case 1: e = sidx(1, 0, 0);  sx = 0; sy = u; sz = v; tx = 9; ty = u + 1; tz = v + 1; break;
      case 2: e = sidx(0, -1, 0); sx = u; sy = 7; sz = v; tx = u + 1; ty = 0; tz = v + 1; break;
      case 3: e = sidx(0, 1, 0);  sx = u; sy = 0; sz = v; tx = u + 1; ty = 9; tz = v + 1; break;
      case 4: e = sidx(0, 0, -1); sx = u; sy = v; sz = 7; tx = u + 1; ty = v + 1; tz = 0; break;
      default: e = sidx(0, 0, 1); sx = u; sy = v; sz = 0; tx = u + 1; ty = v + 1; tz = 9; break;
    }
    const int nb = sn[e];
    tl[tz][ty][tx] = nb >= 0 ? x[(size_t)nb * BV + (sz * 8 + sy) * 8 + sx] : T(0);
  }
}

// Level-0 7-point operator at one node, split so that every load that does
// not need the neighbour-brick ids is issued before the block's first
// barrier (prefetch), and only the -x/-y/-z conductances of nodes on the
// brick's low faces wait for them (resolve).
template <typename T, typename C>
struct Stencil7 {
  T gpx, gpy, gpz, gmx, gmy, gmz, dg;
  __device__ __forceinline__ void prefetch(const C *__restrict__ gx,
                                           const T *__restrict__ diag, size_t S,
                                           size_t s, int lx, int ly, int lz) {
    gpx = cvt<T>(gx[s]);
    gpy = cvt<T>(gx[S + s]);
    gpz = cvt<T>(gx[2 * S + s]);
    gmx = lx > 0 ? cvt<T>(gx[s - 1]) : T(0);
    gmy = ly > 0 ? cvt<T>(gx[S + s - 8]) : T(0);
    gmz = lz > 0 ? cvt<T>(gx[2 * S + s - 64]) : T(0);
    if constexpr (sizeof(T) == 8) dg = diag[s]; else dg = T(0);
  }
  __device__ __forceinline__ void resolve(const C *__restrict__ gx, size_t S, int t,
                                          int lx, int ly, int lz, const int *sn) {
    if (lx == 0) {
      const int nb = sn[sidx(-1, 0, 0)];
      if (nb >= 0) gmx = cvt<T>(gx[(size_t)nb * BV + t + 7]);
    }
    if (ly == 0) {
      const int nb = sn[sidx(0, -1, 0)];
      if (nb >= 0) gmy = cvt<T>(gx[S + (size_t)nb * BV + t + 56]);
    }
    if (lz == 0) {
      const int nb = sn[sidx(0, 0, -1)];
      if (nb >= 0) gmz = cvt<T>(gx[2 * S + (size_t)nb * BV + t + 448]);
    }
  }
  // FP64: diag*x - sum g x_nbr; FP32: sum g (x - x_nbr) (exactly zero on
  // constants, so rounded conductances keep the operator semidefinite)
  __device__ __forceinline__ T apply(const T (*tl)[10][10], int lx, int ly, int lz) const {
    const T xc = tl[lz + 1][ly + 1][lx + 1];
    const T xpx = tl[lz + 1][ly + 1][lx + 2], xmx = tl[lz + 1][ly + 1][lx];
    const T xpy = tl[lz + 1][ly + 2][lx + 1], xmy = tl[lz + 1][ly][lx + 1];
    const T xpz = tl[lz + 2][ly + 1][lx + 1], xmz = tl[lz][ly + 1][lx + 1];
    if constexpr (sizeof(T) == 4) {
      return gpx * (xc - xpx) + gmx * (xc - xmx) + gpy * (xc - xpy) + gmy * (xc - xmy) +
             gpz * (xc - xpz) + gmz * (xc - xmz);
    } else {
      T acc = dg * xc;
      acc -= gpx * xpx;
      acc -= gmx * xmx;
      acc -= gpy * xpy;
      acc -= gmy * xmy;
      acc -= gpz * xpz;
      acc -= gmz * xmz;
      return acc;
    }
  }
};

// (A x) at this thread's node for the level-0 7-point operator, x in the tile.
// FP64: diag*x - sum g x_nbr (fewest FP64-pipe operations).  FP32: sum
// g (x - x_nbr), exactly zero on constants, so rounded (BF16/FP32)
// conductances keep the operator positive semidefinite.
template <typename T, typename C>
__device__ __forceinline__ T apply7_tile(const T (*tl)[10][10], const C *__restrict__ gx,
                                         const T *__restrict__ diag, size_t S, int bk,
                                         const int *sn) {
  const int t = threadIdx.x, lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  const size_t s = (size_t)bk * BV + t;
  const T xc = tl[lz + 1][ly + 1][lx + 1];
  const T xpx = tl[lz + 1][ly + 1][lx + 2], xmx = tl[lz + 1][ly + 1][lx];
  const T xpy = tl[lz + 1][ly + 2][lx + 1], xmy = tl[lz + 1][ly][lx + 1];
  const T xpz = tl[lz + 2][ly + 1][lx + 1], xmz = tl[lz][ly + 1][lx + 1];
  const T gpx = cvt<T>(gx[s]), gpy = cvt<T>(gx[S + s]), gpz = cvt<T>(gx[2 * S + s]);
  // conductances of the -x/-y/-z edges are the +edges of the neighbour nodes
  T gmx, gmy, gmz;
  if (lx > 0) gmx = cvt<T>(gx[s - 1]);
  else { const int nb = sn[sidx(-1, 0, 0)]; gmx = nb >= 0 ? cvt<T>(gx[(size_t)nb * BV + t + 7]) : T(0); }
  if (ly > 0) gmy = cvt<T>(gx[S + s - 8]);
  else { const int nb = sn[sidx(0, -1, 0)]; gmy = nb >= 0 ? cvt<T>(gx[S + (size_t)nb * BV + t + 56]) : T(0); }
  if (lz > 0) gmz = cvt<T>(gx[2 * S + s - 64]);
  else { const int nb = sn[sidx(0, 0, -1)]; gmz = nb >= 0 ? cvt<T>(gx[2 * S + (size_t)nb * BV + t + 448]) : T(0); }
  if constexpr (sizeof(T) == 4) {
    return gpx * (xc - xpx) + gmx * (xc - xmx) + gpy * (xc - xpy) + gmy * (xc - xmy) +
           gpz * (xc - xpz) + gmz * (xc - xmz);
  } else {
    T acc = diag[s] * xc;
    acc -= gpx * xpx;
    acc -= gmx * xmx;
    acc -= gpy * xpy;
    acc -= gmy * xmy;
    acc -= gpz * xpz;
    acc -= gmz * xmz;
    return acc;
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
