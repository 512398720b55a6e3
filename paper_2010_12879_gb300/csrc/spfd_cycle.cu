// V-cycle kernels: smoothers, residuals, restriction, prolongation and the
// coarsest-level solve.
//
// Paper: Eq. 3 (Sec. II) is the system; the paper's own preconditioner is
// AmgX's algebraic multigrid (Sec. III).  These kernels implement the
// geometric operator-dependent V-cycle that replaces it.  All are
// bandwidth-bound stencil or transfer sweeps (the FP64 forms approach the
// FP64 pipe's rate); none is a dense contraction, so no tensor-core path is
// used.  One block handles one 8x8x8 brick: two (FP64) or four (FP32) nodes
// per thread without shared memory on level 0, one node per thread with a shared tile on the
// 27-point levels (spfd_tile.cuh).
#include "spfd_internal.cuh"
#include "spfd_tile.cuh"

namespace spfd {

// ------------------------------------------------------------ smoothers
// Level 0 (7-point): r = b - A x, and the weighted-Jacobi sweep
// x_out = x + omega D^-1 (b - A x), on the row mapping.  (The level-0 row
// list that k_apply_dot uses in FP64 made these two slower: they issue
// fewer FP64 instructions per row, and the extra dependent load of the list
// entry and the looser brick locality cost more than the skipped rows.)
template <typename T, typename C, int ORD>
__global__ void __launch_bounds__(row_threads<T>(), row_min_blocks<T>())
k_residual7(Grid g, const C *__restrict__ gx, const T *__restrict__ diag,
            const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ r,
            int nk) {
  pdl_entry();
  constexpr int N = row_n<T>();
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, s0 = row_slot<N>(bk, t);
  const size_t off = (size_t)rhs * S;
  x += off; b += off; r += off;
  const Qv<T, N> bv = ldqn<T, T, N>(b + s0);
  Qv<T, N> xc, rv;
  apply7_row<T, C, true, N>(g, gx, diag, x, S, bk, t, bv, xc, rv);
  stqn<T, N>(r + s0, rv);
}

// RZ: the last sweep of the V-cycle on level 0, where b is the CG residual r
// and xout the preconditioned z: each warp also writes its parts of r.z and
// of the sum of z over the unknowns (w > 0) to partials[2 (brick warp) + {0,1}]
// (right-hand side rhs at rhs * pstride), which launch_finish_rz adds.
template <typename T, typename C, int ORD, bool RZ = false>
__global__ void __launch_bounds__(BV / row_n_jacobi<T>(), row_min_blocks_jacobi<T>())
k_jacobi7(Grid g, const C *__restrict__ gx, const T *__restrict__ diag,
          const T *__restrict__ wdinv, const T *__restrict__ xin,
          const T *__restrict__ b, T *__restrict__ xout, int nk,
          double *__restrict__ partials = nullptr, size_t pstride = 0) {
  pdl_entry();
  constexpr int N = row_n_jacobi<T>();
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, s0 = row_slot<N>(bk, t);
  const size_t off = (size_t)rhs * S;
  xin += off; b += off; xout += off;
  const Qv<T, N> bv = ldqn<T, T, N>(b + s0), wv = ldqn<T, T, N>(wdinv + s0);
  Qv<T, N> xc, rv;
  apply7_row<T, C, true, N>(g, gx, diag, xin, S, bk, t, bv, xc, rv);
#pragma unroll
  for (int i = 0; i < N; ++i) xc.v[i] += wv.v[i] * rv.v[i];
  stqn<T, N>(xout + s0, xc);
  if constexpr (RZ) {
    T rz[N], zs[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      rz[i] = bv.v[i] * xc.v[i];
      zs[i] = weight_pos(wv.v[i]) ? xc.v[i] : (T)0;
    }
    const WarpSum<T> prz = warp_total<T, N>(rz), pzs = warp_total<T, N>(zs);
    if ((t & 31) == 0) {
      double *pp = partials + (size_t)rhs * pstride +
                   2 * ((size_t)bk * (BV / N / 32) + (t >> 5));
      prz.put(pp);
      pzs.put(pp + 1);
    }
  }
}

// This thread's slot in a 27-point kernel over the staged brick: with
// compaction (FP64) the brick's n-th active slot for thread n, else the
// thread's own slot.  mine: the thread computes the stencil at ts; idle: its
// own slot is inactive and gets the zero-row result.
struct SlotMap {
  int ts;
  bool mine, idle;
};
template <typename T>
__device__ __forceinline__ SlotMap slot_map(const ActList &al) {
  const int t = threadIdx.x;
  SlotMap m;
  m.idle = !act_on(al, t);
  if constexpr (compact27<T>()) {
    m.mine = t < al.pre[16];
    m.ts = m.mine ? act_slot(al, t) : 0;
  } else {
    m.mine = !m.idle;
    m.ts = t;
  }
  return m;
}

// r = b - A x on brick bk of a 27-point level; every thread of the
// NT-thread block calls it, and tl, sn and al are the caller's shared tile,
// neighbour table and activity list.  A zero row (clear activity bit) gets
// r = b - 0 = b without its 27 coefficients or any arithmetic.  FP64:
// thread n computes the brick's n-th active slot (compaction).
template <typename T, bool COH>
__device__ __forceinline__ void residual27_unit(const Grid &g, const T *__restrict__ st,
                                                const T *x, const T *b, T *r, int bk,
                                                T (*tl)[10][10], int *sn, ActList &al) {
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, base = (size_t)bk * BV;
  load_nbr(g, bk, sn);
  if constexpr (compact27<T>()) {
    act_stage(g, bk, al);
    __syncthreads();
    tile_full<T, COH>(tl, x, bk, sn);
    if (!act_on(al, t)) r[base + t] = ldv<COH>(b + base + t);
    __syncthreads();
    if (t < al.pre[16]) {
      const int ts = act_slot(al, t);
      const size_t s = base + ts;
      r[s] = ldv<COH>(b + s) - apply27_tile<T>(tl, st, S, s, ts);
    }
  } else {
    const bool on = (act_word(g, bk) >> (t & 31)) & 1u;
    __syncthreads();
    tile_full<T, COH>(tl, x, bk, sn);
    __syncthreads();
    const size_t s = base + t;
    r[s] = ldv<COH>(b + s) - (on ? apply27_tile<T>(tl, st, S, s, t) : T(0));
  }
}

template <typename T, int ORD>
__global__ void __launch_bounds__(NT)
k_residual27(Grid g, const T *__restrict__ st, const T *__restrict__ x,
             const T *__restrict__ b, T *__restrict__ r, int nk) {
  pdl_entry();
  __shared__ T tl[rhs_tile<ORD>()][10][10][10];
  __shared__ int sn[27];
  __shared__ ActList al;
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, base = (size_t)bk * BV;
  if constexpr (rhs_tile<ORD>() == 1) {
    const size_t off = (size_t)rhs * S;
    residual27_unit<T, false>(g, st, x + off, b + off, r + off, bk, tl[0], sn, al);
  } else {
    load_nbr(g, bk, sn);
    act_stage(g, bk, al);
    __syncthreads();
    // the tile's right-hand sides side by side: all their halo tiles are
    // loaded at once, then each uses the coefficients held in registers
    const SlotMap m = slot_map<T>(al);
    const size_t sa = base + m.ts;
    T cf[27];
    if (m.mine) load27(st, S, sa, cf);
    const int nr = min(rhs_tile<ORD>(), nk - rhs);
    for (int k = 0; k < nr; ++k) tile_full<T>(tl[k], x + (size_t)(rhs + k) * S, bk, sn);
    __syncthreads();
    for (int k = 0; k < nr; ++k) {
      const size_t off = (size_t)(rhs + k) * S;
      if (m.idle) r[off + base + t] = b[off + base + t];
      if (m.mine) r[off + sa] = b[off + sa] - apply27_regs<T>(tl[k], cf, m.ts);
    }
  }
}

// One weighted-Jacobi sweep xout = xin + omega D^-1 (b - A xin) on brick bk
// of a 27-point level (as residual27_unit; a zero row gets xin + w b).
template <typename T, bool COH>
__device__ __forceinline__ void jacobi27_unit(const Grid &g, const T *__restrict__ st,
                                              const T *__restrict__ wdinv, const T *xin,
                                              const T *b, T *xout, int bk, T (*tl)[10][10],
                                              int *sn, ActList &al) {
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, base = (size_t)bk * BV;
  load_nbr(g, bk, sn);
  if constexpr (compact27<T>()) {
    act_stage(g, bk, al);
    __syncthreads();
    tile_full<T, COH>(tl, xin, bk, sn);
    __syncthreads();
    if (!act_on(al, t))
      xout[base + t] = tile_at(tl, t) + wdinv[base + t] * ldv<COH>(b + base + t);
    if (t < al.pre[16]) {
      const int ts = act_slot(al, t);
      const size_t s = base + ts;
      const T r = ldv<COH>(b + s) - apply27_tile<T>(tl, st, S, s, ts);
      xout[s] = tile_at(tl, ts) + wdinv[s] * r;
    }
  } else {
    const bool on = (act_word(g, bk) >> (t & 31)) & 1u;
    __syncthreads();
    tile_full<T, COH>(tl, xin, bk, sn);
    __syncthreads();
    const size_t s = base + t;
    const T r = ldv<COH>(b + s) - (on ? apply27_tile<T>(tl, st, S, s, t) : T(0));
    xout[s] = tile_at(tl, t) + wdinv[s] * r;
  }
}

template <typename T, int ORD>
__global__ void __launch_bounds__(NT)
k_jacobi27(Grid g, const T *__restrict__ st, const T *__restrict__ wdinv,
           const T *__restrict__ xin, const T *__restrict__ b,
           T *__restrict__ xout, int nk) {
  pdl_entry();
  __shared__ T tl[rhs_tile<ORD>()][10][10][10];
  __shared__ int sn[27];
  __shared__ ActList al;
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const int t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, base = (size_t)bk * BV;
  if constexpr (rhs_tile<ORD>() == 1) {
    const size_t off = (size_t)rhs * S;
    jacobi27_unit<T, false>(g, st, wdinv, xin + off, b + off, xout + off, bk, tl[0], sn, al);
  } else {
    load_nbr(g, bk, sn);
    act_stage(g, bk, al);
    __syncthreads();
    const SlotMap m = slot_map<T>(al);
    const size_t sa = base + m.ts;
    T cf[27];
    if (m.mine) load27(st, S, sa, cf);
    const T wd = m.mine ? wdinv[sa] : T(0), wi = m.idle ? wdinv[base + t] : T(0);
    const int nr = min(rhs_tile<ORD>(), nk - rhs);
    for (int k = 0; k < nr; ++k) tile_full<T>(tl[k], xin + (size_t)(rhs + k) * S, bk, sn);
    __syncthreads();
    for (int k = 0; k < nr; ++k) {
      const size_t off = (size_t)(rhs + k) * S;
      if (m.idle) xout[off + base + t] = tile_at(tl[k], t) + wi * b[off + base + t];
      if (m.mine) {
        const T r = b[off + sa] - apply27_regs<T>(tl[k], cf, m.ts);
        xout[off + sa] = tile_at(tl[k], m.ts) + wd * r;
      }
    }
  }
}

// First sweep from a zero guess, x = omega D^-1 b: a streaming kernel, one
// brick per block, 16 bytes per thread access.
template <typename T, int ORD>
__global__ void __launch_bounds__(NT)
k_jacobi_first(const T *__restrict__ wdinv, const T *__restrict__ b,
               T *__restrict__ x, int nb, int nk) {
  pdl_entry();
  constexpr int N = V16<T>::N;
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const size_t s0 = (size_t)bk * BV + threadIdx.x * N;
  const size_t off = (size_t)rhs * nb * BV;
  b += off; x += off;
  const V16<T> w = ld16(wdinv + s0), bv = ld16(b + s0);
  V16<T> xv;
#pragma unroll
  for (int i = 0; i < N; ++i) xv.v[i] = w.v[i] * bv.v[i];
  st16(x + s0, xv);
}

// The same with the projection of b fused in: b <- b - mean(b) on the
// unknowns (mean formed by the preceding reduction), in place.
template <typename T, int ORD>
__global__ void __launch_bounds__(NT)
k_jacobi_first_proj(const T *__restrict__ wdinv, T *__restrict__ b,
                    T *__restrict__ x, const Scalars *sc, int nb, int nk) {
  pdl_entry();
  constexpr int N = V16<T>::N;
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const size_t s0 = (size_t)bk * BV + threadIdx.x * N;
  const size_t off = (size_t)rhs * nb * BV;
  b += off; x += off; sc += rhs;
  T mean;
  if constexpr (sizeof(T) == 4) mean = sc->rmean_f; else mean = sc->rmean;
  const V16<T> w = ld16(wdinv + s0);
  V16<T> bv = ld16(b + s0), xv;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (weight_pos(w.v[i])) {  // an unknown of level 0
      bv.v[i] -= mean;
      xv.v[i] = w.v[i] * bv.v[i];
    } else {
      xv.v[i] = (T)0;
    }
  }
  st16(b + s0, bv);
  st16(x + s0, xv);
}

// ------------------------------------------------------------ Chebyshev sweeps
// One Chebyshev step fused with its residual: with r = b - A xin,
// d = c1 d + c2w wdinv r (in place: a thread reads and writes only its own
// slots of d) and xout = xin + d.  Level 0 on the row mapping of k_jacobi7,
// the 27-point levels as jacobi27_unit (FP64 with the active-slot
// compaction; a zero row has r = b).
template <typename T, typename C>
__global__ void __launch_bounds__(BV / row_n_jacobi<T>(), row_min_blocks<T>())
k_cheb7(Grid g, const C *__restrict__ gx, const T *__restrict__ diag,
        const T *__restrict__ wdinv, const T *__restrict__ xin, const T *__restrict__ b,
        T *__restrict__ xout, T *__restrict__ d, T c1, T c2w) {
  pdl_entry();
  constexpr int N = row_n_jacobi<T>();
  const int bk = blockIdx.x, t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, s0 = row_slot<N>(bk, t);
  const size_t off = (size_t)blockIdx.y * S;
  xin += off; b += off; xout += off; d += off;
  const Qv<T, N> bv = ldqn<T, T, N>(b + s0), wv = ldqn<T, T, N>(wdinv + s0);
  Qv<T, N> dv = ldqn<T, T, N>(d + s0), xc, rv;
  apply7_row<T, C, true, N>(g, gx, diag, xin, S, bk, t, bv, xc, rv);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    dv.v[i] = c1 * dv.v[i] + c2w * wv.v[i] * rv.v[i];
    xc.v[i] += dv.v[i];
  }
  stqn<T, N>(xout + s0, xc);
  stqn<T, N>(d + s0, dv);
}

template <typename T>
__global__ void __launch_bounds__(NT)
k_cheb27(Grid g, const T *__restrict__ st, const T *__restrict__ wdinv,
         const T *__restrict__ xin, const T *__restrict__ b, T *__restrict__ xout,
         T *__restrict__ d, T c1, T c2w) {
  pdl_entry();
  __shared__ T tl[10][10][10];
  __shared__ int sn[27];
  __shared__ ActList al;
  const int bk = blockIdx.x, t = threadIdx.x;
  const size_t S = (size_t)g.nb * BV, base = (size_t)bk * BV;
  const size_t off = (size_t)blockIdx.y * S;
  xin += off; b += off; xout += off; d += off;
  load_nbr(g, bk, sn);
  act_stage(g, bk, al);
  __syncthreads();
  tile_full<T>(tl, xin, bk, sn);
  __syncthreads();
  const SlotMap m = slot_map<T>(al);
  auto update = [&](size_t s, int ts, T r) {
    const T dn = c1 * d[s] + c2w * wdinv[s] * r;
    d[s] = dn;
    xout[s] = tile_at(tl, ts) + dn;
  };
  if (m.idle) update(base + t, t, b[base + t]);
  if (m.mine) {
    const size_t s = base + m.ts;
    update(s, m.ts, b[s] - apply27_tile<T>(tl, st, S, s, m.ts));
  }
}

// ------------------------------------------------------------ Chebyshev step
// One step of the Chebyshev smoother (three-term recurrence on D^-1 A):
// d = c1 d + c2w wdinv r, x += d, or (FIRST, from a zero guess, r = b)
// d = c2w wdinv b, x = d.  wdinv = omega D^-1 holds the Jacobi weight, which
// c2w absorbs; slots that are not unknowns (wdinv = 0) keep d = x = 0.  A
// streaming kernel over the level's slots; the residual r comes from the
// residual kernels above.
template <typename T, bool FIRST>
__global__ void __launch_bounds__(NT)
k_cheb(size_t S, const T *__restrict__ wdinv, const T *__restrict__ r, T *__restrict__ d,
       T *__restrict__ x, T c1, T c2w) {
  pdl_entry();
  constexpr int N = V16<T>::N;
  const size_t off = (size_t)blockIdx.y * S;
  r += off; d += off; x += off;
  const size_t nv = S / N;
  for (size_t vi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; vi < nv;
       vi += (size_t)gridDim.x * blockDim.x) {
    const size_t s0 = vi * N;
    const V16<T> w = ld16(wdinv + s0), rv = ld16(r + s0);
    V16<T> dv, xv;
    if constexpr (!FIRST) {
      dv = ld16(d + s0);
      xv = ld16(x + s0);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if constexpr (FIRST) {
        dv.v[i] = c2w * w.v[i] * rv.v[i];
        xv.v[i] = dv.v[i];
      } else {
        dv.v[i] = c1 * dv.v[i] + c2w * w.v[i] * rv.v[i];
        xv.v[i] += dv.v[i];
      }
    }
    st16(d + s0, dv);
    st16(x + s0, xv);
  }
}

// ------------------------------------------------------------ transfers
// Restriction r_c(I) = sum_d P[d][I] r_f(2I + d) (P^T, the adjoint of the
// prolongation below).  A coarse brick B reads the 17^3 fine nodes
// 16B-1 .. 16B+15 (per axis) from the 27 fine bricks 2B-1 .. 2B+1.
// The 17^3 fine nodes of brick bk's children into fs (sk: the child table):
// the 8 child bricks (16^3 nodes, fs[1..16]^3) as 16-byte vectors, then the
// three planes fs[0][*][*], fs[1..16][0][*] and fs[1..16][1..16][0] from the
// bricks before them, one value per thread.
template <typename T, bool COH>
__device__ __forceinline__ void restrict_fill(T (*fs)[17][17], const T *src, const int *sk) {
  constexpr int VN = 16 / (int)sizeof(T);  // values per vector
  constexpr int VPB = BV / VN;             // vectors per brick
  for (int q = threadIdx.x; q < 8 * VPB; q += NT) {
    const int cb = q / VPB, e0 = (q % VPB) * VN;
    const int ox = cb & 1, oy = (cb >> 1) & 1, oz = cb >> 2;
    const int nb = sk[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    const int lx = e0 & 7, ly = (e0 >> 3) & 7, lz = e0 >> 6;
    V16<T> v;
    if (nb >= 0) {
      const T *p = src + (size_t)nb * BV + e0;
      if constexpr (COH) *reinterpret_cast<uint4 *>(&v) = __ldcg(reinterpret_cast<const uint4 *>(p));
      else v = ld16(p);
    } else {
#pragma unroll
      for (int i = 0; i < VN; ++i) v.v[i] = T(0);
    }
    T *row = &fs[1 + 8 * oz + lz][1 + 8 * oy + ly][1 + 8 * ox + lx];
#pragma unroll
    for (int i = 0; i < VN; ++i) row[i] = v.v[i];
  }
  for (int q = threadIdx.x; q < 289 + 272 + 256; q += NT) {
    int fz, fy, fx;
    if (q < 289) {
      fz = 0; fy = q / 17; fx = q % 17;
    } else if (q < 289 + 272) {
      const int u = q - 289;
      fz = 1 + u / 17; fy = 0; fx = u % 17;
    } else {
      const int u = q - 289 - 272;
      fz = 1 + u / 16; fy = 1 + u % 16; fx = 0;
    }
    const int nb = sk[((fz + 7) >> 3) * 9 + ((fy + 7) >> 3) * 3 + ((fx + 7) >> 3)];
    fs[fz][fy][fx] = nb >= 0
        ? ldv<COH>(&src[(size_t)nb * BV + (((fz - 1) & 7) * 8 + ((fy - 1) & 7)) * 8 +
                        ((fx - 1) & 7)])
        : T(0);
  }
}

// One coarse brick bk, one coarse node per thread (NT threads call it).  A
// coarse node whose interpolation column is zero (clear activity bit)
// restricts to exactly +0: its 27 weights are not read.
template <typename T, bool COH>
__device__ __forceinline__ void restrict_unit(const Grid &gc, size_t Sf, const T *__restrict__ P,
                                              const T *rf, T *bcoarse, int bk,
                                              T (*fs)[17][17], int *sk) {
  const int t = threadIdx.x;
  const size_t Sc = (size_t)gc.nb * BV, s = (size_t)bk * BV + t;
  const int cx = 2 * (t & 7) + 1, cy = 2 * ((t >> 3) & 7) + 1, cz = 2 * (t >> 6) + 1;
  if (t < 27) sk[t] = gc.kid[(size_t)bk * 27 + t];
  const bool on = (act_word(gc, bk) >> (t & 31)) & 1u;
  __syncthreads();
  restrict_fill<T, COH>(fs, rf, sk);
  __syncthreads();
  T acc = 0;
  if (on) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      acc += P[(size_t)d * Sc + s] * fs[cz + dz][cy + dy][cx + dx];
    }
  }
  bcoarse[s] = acc;
}

template <typename T, int ORD>
__global__ void __launch_bounds__(NT)
k_restrict(Grid gc, size_t Sf, const T *__restrict__ P, const T *__restrict__ rf,
           T *__restrict__ bcoarse, int nk) {
  pdl_entry();
  __shared__ T fs[17][17][17];
  __shared__ int sk[27];
  int bk, rhs;
  unit_rhs<ORD>(nk, bk, rhs);
  const int t = threadIdx.x;
  const size_t Sc = (size_t)gc.nb * BV, s = (size_t)bk * BV + t;
  if constexpr (rhs_tile<ORD>() == 1) {
    restrict_unit<T, false>(gc, Sf, P, rf + (size_t)rhs * Sf, bcoarse + (size_t)rhs * Sc, bk,
                            fs, sk);
  } else {
    const int cx = 2 * (t & 7) + 1, cy = 2 * ((t >> 3) & 7) + 1, cz = 2 * (t >> 6) + 1;
    if (t < 27) sk[t] = gc.kid[(size_t)bk * 27 + t];
    const bool on = (act_word(gc, bk) >> (t & 31)) & 1u;
    T w[27];
    if (on) load27(P, Sc, s, w);
    else
#pragma unroll
      for (int e = 0; e < 27; ++e) w[e] = T(0);
    const int nr = min(rhs_tile<ORD>(), nk - rhs);
    for (int k = 0; k < nr; ++k) {
      __syncthreads();  // sk is loaded / the previous tile is consumed
      restrict_fill<T, false>(fs, rf + (size_t)(rhs + k) * Sf, sk);
      __syncthreads();
      T acc = 0;
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        acc += w[d] * fs[cz + dz][cy + dy][cx + dx];
      }
      bcoarse[(size_t)(rhs + k) * Sc + s] = acc;
    }
  }
}

// Prolongation + correction e_f(n) += sum over the <= 8 parents I of n of
// P(n, I) e_c(I).  One thread per 2x2x2 cell of a fine brick (two bricks per
// 128 threads): it loads the cell's 27 weights (row j of Pc at column
// brick*64 + cell, coalesced across the warp), the 8 coarse corner values
// c + o (o in {0,1}^3; coarse bricks from the brick's parent table) and its
// 8 fine values as 2-vectors along x, then writes the 8 corrected values.
// No shared memory and no barrier: every load is independent.
// Pair `pair` of fine bricks, thread `tid` (0..127) of the pair's group;
// nr right-hand sides from rhs on (S apart on each level).
template <typename T, bool COH>
__device__ __forceinline__ void prolong_unit(const Grid &gf, const Grid &gc,
                                             const T *__restrict__ Pc, const T *ec, T *ef,
                                             int pair, int tid, int rhs, int nr) {
  const int bk = pair * 2 + (tid >> 6);
  if (bk >= gf.nb) return;
  const int cell = tid & 63;
  const int ccx = cell & 3, ccy = (cell >> 2) & 3, ccz = cell >> 4;
  const size_t NC = (size_t)gf.nb * 64, cid = (size_t)bk * 64 + cell;
  T w[27];
#pragma unroll
  for (int j = 0; j < 27; ++j) w[j] = Pc[(size_t)j * NC + cid];
  const int4 bc = gf.bco[bk];
  for (int k = 0; k < nr; ++k) {
    const T *ecj = ec + (size_t)(rhs + k) * gc.nb * BV;
    T *efj = ef + (size_t)(rhs + k) * gf.nb * BV;
    T e[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int gx_ = 4 * bc.x + ccx + (o & 1), gy_ = 4 * bc.y + ccy + ((o >> 1) & 1),
                gz_ = 4 * bc.z + ccz + (o >> 2);
      const int pb = (((gz_ >> 3) - (bc.z >> 1)) << 2) | (((gy_ >> 3) - (bc.y >> 1)) << 1) |
                     ((gx_ >> 3) - (bc.x >> 1));
      const int nb = __ldg(&gf.par[(size_t)bk * 8 + pb]);
      e[o] = nb >= 0 ? ldv<COH>(&ecj[(size_t)nb * BV + ((gz_ & 7) * 8 + (gy_ & 7)) * 8 +
                                     (gx_ & 7)])
                     : T(0);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {  // r = uz*2 + uy: one 2-vector (ux = 0, 1) per row
      const int uy = r & 1, uz = r >> 1;
      T *row = efj + (size_t)bk * BV + ((2 * ccz + uz) * 8 + 2 * ccy + uy) * 8 + 2 * ccx;
      T v[2];
      if constexpr (sizeof(T) == 4) {
        const float2 u = ldv<COH>(reinterpret_cast<const float2 *>(row));
        v[0] = u.x; v[1] = u.y;
      } else {
        const double2 u = ldv<COH>(reinterpret_cast<const double2 *>(row));
        v[0] = u.x; v[1] = u.y;
      }
#pragma unroll
      for (int ux = 0; ux < 2; ++ux) {
        const int q = uz * 4 + uy * 2 + ux;
#pragma unroll
        for (int o = 0; o < 8; ++o)
          if ((o & ~q) == 0) v[ux] += w[pc_off(q) + crank(q, o)] * e[o];
      }
      if constexpr (sizeof(T) == 4) *reinterpret_cast<float2 *>(row) = make_float2(v[0], v[1]);
      else *reinterpret_cast<double2 *>(row) = make_double2(v[0], v[1]);
    }
  }
}

template <typename T, int ORD>
__global__ void __launch_bounds__(128)
k_prolong(Grid gf, Grid gc, const T *__restrict__ Pc, const T *__restrict__ ec,
          T *__restrict__ ef, int nk) {
  pdl_entry();
  int pair, rhs;
  unit_rhs<ORD>(nk, pair, rhs);
  const int nr = rhs_tile<ORD>() == 1 ? 1 : min(rhs_tile<ORD>(), nk - rhs);
  prolong_unit<T, false>(gf, gc, Pc, ec, ef, pair, threadIdx.x, rhs, nr);
}

// Coarsest level: x = B^{-1} b on the m listed unknowns (dense, FP64); one
// warp per row.  Unlisted slots must be zero beforehand.
template <typename T>
__global__ void k_coarse_solve(int m, size_t S, const int *__restrict__ idx,
                               const double *__restrict__ Binv,
                               const T *__restrict__ b, T *__restrict__ x) {
  pdl_entry();
  b += (size_t)blockIdx.y * S;
  x += (size_t)blockIdx.y * S;
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
                      const T *b, T *r, cudaStream_t st, int nk, int order) {
  if (g.nb)
    if (order)
      pdl(k_residual7<T, C, 1>, unit_grid(1, g.nb, nk), row_threads<T>(), st)(g, gx, diag, x, b,
                                                                                r, nk);
    else
      pdl(k_residual7<T, C, 0>, unit_grid(0, g.nb, nk), row_threads<T>(), st)(g, gx, diag, x, b,
                                                                                r, nk);
}
template <typename T>
void launch_residual27(const Grid &g, const T *stc, const T *x, const T *b,
                       T *r, cudaStream_t st, int nk, int order) {
  if (!g.nb) return;
  if (order == 2) pdl(k_residual27<T, 2>, unit_grid(2, g.nb, nk), NT, st)(g, stc, x, b, r, nk);
  else if (order) pdl(k_residual27<T, 1>, unit_grid(1, g.nb, nk), NT, st)(g, stc, x, b, r, nk);
  else pdl(k_residual27<T, 0>, unit_grid(0, g.nb, nk), NT, st)(g, stc, x, b, r, nk);
}
template <typename T>
void launch_jacobi_first(const Grid &g, const T *wdinv, const T *b, T *x,
                         cudaStream_t st, int nk, int order) {
  if (g.nb)
    if (order)
      pdl(k_jacobi_first<T, 1>, unit_grid(1, g.nb, nk), NT / V16<T>::N, st)(wdinv, b, x, g.nb, nk);
    else
      pdl(k_jacobi_first<T, 0>, unit_grid(0, g.nb, nk), NT / V16<T>::N, st)(wdinv, b, x, g.nb, nk);
}
template <typename T>
void launch_jacobi_first_proj(const Grid &g, const T *wdinv, T *b, T *x,
                              const Scalars *sc, double inv_ndof,
                              cudaStream_t st, int nk, int order) {
  (void)inv_ndof;  // the mean comes from each right-hand side's Scalars
  if (g.nb)
  {
    if (order)
      pdl(k_jacobi_first_proj<T, 1>, unit_grid(1, g.nb, nk), NT / V16<T>::N, st)(
          wdinv, b, x, sc, g.nb, nk);
    else
      pdl(k_jacobi_first_proj<T, 0>, unit_grid(0, g.nb, nk), NT / V16<T>::N, st)(
          wdinv, b, x, sc, g.nb, nk);
  }
}
template <typename T, typename C>
void launch_jacobi7_rz(const Grid &g, const C *gx, const T *diag, const T *wdinv,
                       const T *xin, const T *b, T *xout, double *partials, size_t pstride,
                       cudaStream_t st, int nk, int order) {
  if (!g.nb) return;
  if (order)
    pdl(k_jacobi7<T, C, 1, true>, unit_grid(1, g.nb, nk), BV / row_n_jacobi<T>(), st)(
        g, gx, diag, wdinv, xin, b, xout, nk, partials, pstride);
  else
    pdl(k_jacobi7<T, C, 0, true>, unit_grid(0, g.nb, nk), BV / row_n_jacobi<T>(), st)(
        g, gx, diag, wdinv, xin, b, xout, nk, partials, pstride);
}
template <typename T>
int jacobi7_rz_partials(int nb) { return nb * (BV / row_n_jacobi<T>() / 32); }
template int jacobi7_rz_partials<double>(int);
template int jacobi7_rz_partials<float>(int);
template <typename T, typename C>
void launch_jacobi7(const Grid &g, const C *gx, const T *diag, const T *wdinv,
                    const T *xin, const T *b, T *xout, cudaStream_t st, int nk, int order) {
  if (g.nb)
  {
    if (order)
      pdl(k_jacobi7<T, C, 1>, unit_grid(1, g.nb, nk), BV / row_n_jacobi<T>(), st)(
          g, gx, diag, wdinv, xin, b, xout, nk, nullptr, (size_t)0);
    else
      pdl(k_jacobi7<T, C, 0>, unit_grid(0, g.nb, nk), BV / row_n_jacobi<T>(), st)(
          g, gx, diag, wdinv, xin, b, xout, nk, nullptr, (size_t)0);
  }
}
template <typename T>
void launch_jacobi27(const Grid &g, const T *stc, const T *wdinv, const T *xin,
                     const T *b, T *xout, cudaStream_t st, int nk, int order) {
  if (g.nb)
  {
    if (order == 2)
      pdl(k_jacobi27<T, 2>, unit_grid(2, g.nb, nk), NT, st)(g, stc, wdinv, xin, b, xout, nk);
    else if (order)
      pdl(k_jacobi27<T, 1>, unit_grid(1, g.nb, nk), NT, st)(g, stc, wdinv, xin, b, xout, nk);
    else
      pdl(k_jacobi27<T, 0>, unit_grid(0, g.nb, nk), NT, st)(g, stc, wdinv, xin, b, xout, nk);
  }
}
template <typename T>
void launch_restrict(const Grid &gf, const Grid &gc, const T *P, const T *rf,
                     T *bcoarse, cudaStream_t st, int nk, int order) {
  if (gc.nb)
  {
    if (order == 2)
      pdl(k_restrict<T, 2>, unit_grid(2, gc.nb, nk), NT, st)(gc, (size_t)gf.nb * BV, P, rf,
                                                               bcoarse, nk);
    else if (order)
      pdl(k_restrict<T, 1>, unit_grid(1, gc.nb, nk), NT, st)(gc, (size_t)gf.nb * BV, P, rf,
                                                               bcoarse, nk);
    else
      pdl(k_restrict<T, 0>, unit_grid(0, gc.nb, nk), NT, st)(gc, (size_t)gf.nb * BV, P, rf,
                                                               bcoarse, nk);
  }
}
template <typename T>
void launch_prolong(const Grid &gf, const Grid &gc, const T *P, const T *ec,
                    T *ef, cudaStream_t st, int nk, int order) {
  if (gf.nb)
  {
    if (order == 2)
      pdl(k_prolong<T, 2>, unit_grid(2, (gf.nb + 1) / 2, nk), 128, st)(gf, gc, P, ec, ef, nk);
    else if (order)
      pdl(k_prolong<T, 1>, unit_grid(1, (gf.nb + 1) / 2, nk), 128, st)(gf, gc, P, ec, ef, nk);
    else
      pdl(k_prolong<T, 0>, unit_grid(0, (gf.nb + 1) / 2, nk), 128, st)(gf, gc, P, ec, ef, nk);
  }
}
template <typename T, typename C>
void launch_cheb7(const Grid &g, const C *gx, const T *diag, const T *wdinv, const T *xin,
                  const T *b, T *xout, T *d, double c1, double c2w, cudaStream_t st, int nk) {
  if (g.nb)
    pdl(k_cheb7<T, C>, dim3(g.nb, nk), BV / row_n_jacobi<T>(), st)(g, gx, diag, wdinv, xin,
                                                                    b, xout, d, (T)c1, (T)c2w);
}
template <typename T>
void launch_cheb27(const Grid &g, const T *stc, const T *wdinv, const T *xin, const T *b,
                   T *xout, T *d, double c1, double c2w, cudaStream_t st, int nk) {
  if (g.nb)
    pdl(k_cheb27<T>, dim3(g.nb, nk), NT, st)(g, stc, wdinv, xin, b, xout, d, (T)c1, (T)c2w);
}
template <typename T>
void launch_cheb(bool first, size_t S, const T *wdinv, const T *r, T *d, T *x, double c1,
                 double c2w, cudaStream_t st, int nk) {
  if (S == 0) return;
  const size_t nv = S / V16<T>::N;
  const size_t want = (nv + NT - 1) / NT;
  const unsigned blocks = (unsigned)(want < 152 * 8 ? want : 152 * 8);
  if (first)
    pdl(k_cheb<T, true>, dim3(blocks, nk), NT, st)(S, wdinv, r, d, x, (T)c1, (T)c2w);
  else
    pdl(k_cheb<T, false>, dim3(blocks, nk), NT, st)(S, wdinv, r, d, x, (T)c1, (T)c2w);
}
template <typename T>
void launch_coarse_solve(int m, size_t S, const int *idx, const double *Binv,
                         const T *b, T *x, cudaStream_t st, int nk) {
  if (m <= 0) return;
  const int warps_per_block = 8;
  pdl(k_coarse_solve<T>, dim3((m + warps_per_block - 1) / warps_per_block, nk), 32 * warps_per_block, st)(m, S, idx, Binv, b, x);
}

#define INST_T(T)                                                             \
  template void launch_residual27<T>(const Grid &, const T *, const T *,      \
                                     const T *, T *, cudaStream_t, int, int); \
  template void launch_jacobi_first<T>(const Grid &, const T *, const T *,    \
                                       T *, cudaStream_t, int, int);          \
  template void launch_jacobi_first_proj<T>(const Grid &, const T *, T *,     \
                                            T *, const Scalars *, double,     \
                                            cudaStream_t, int, int);          \
  template void launch_jacobi27<T>(const Grid &, const T *, const T *,        \
                                   const T *, const T *, T *, cudaStream_t,   \
                                   int, int);                                 \
  template void launch_restrict<T>(const Grid &, const Grid &, const T *,     \
                                   const T *, T *, cudaStream_t, int, int);   \
  template void launch_prolong<T>(const Grid &, const Grid &, const T *,      \
                                  const T *, T *, cudaStream_t, int, int);    \
  template void launch_coarse_solve<T>(int, size_t, const int *,              \
                                       const double *, const T *, T *,        \
                                       cudaStream_t, int);                    \
  template void launch_cheb<T>(bool, size_t, const T *, const T *, T *, T *,  \
                               double, double, cudaStream_t, int);            \
  template void launch_cheb27<T>(const Grid &, const T *, const T *,          \
                                 const T *, const T *, T *, T *, double,      \
                                 double, cudaStream_t, int);
INST_T(double)
INST_T(float)
#define INST_TC(T, C)                                                         \
  template void launch_jacobi7_rz<T, C>(const Grid &, const C *, const T *,   \
                                        const T *, const T *, const T *, T *, \
                                        double *, size_t, cudaStream_t, int,  \
                                        int);                                 \
  template void launch_residual7<T, C>(const Grid &, const C *, const T *,    \
                                       const T *, const T *, T *,             \
                                       cudaStream_t, int, int);               \
  template void launch_jacobi7<T, C>(const Grid &, const C *, const T *,      \
                                     const T *, const T *, const T *, T *,    \
                                     cudaStream_t, int, int);
INST_TC(double, double)
INST_TC(float, float)
template void launch_cheb7<double, double>(const Grid &, const double *, const double *,
                                           const double *, const double *, const double *,
                                           double *, double *, double, double, cudaStream_t,
                                           int);
template void launch_cheb7<float, __nv_bfloat16>(const Grid &, const __nv_bfloat16 *,
                                                 const float *, const float *, const float *,
                                                 const float *, float *, float *, double, double,
                                                 cudaStream_t, int);
INST_TC(float, __nv_bfloat16)

}  // namespace spfd
