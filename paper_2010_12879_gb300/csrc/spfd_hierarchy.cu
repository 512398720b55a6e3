// Multigrid hierarchy: operator-dependent interpolation and Galerkin coarse
// operators A_c = P^T A P on the brick layout.
//
// The paper solves Eq. 3 with the algebraic multigrid of the AmgX library
// (Sec. III); this replaces it with a geometric hierarchy on the node grid
// whose transfer operators follow the fine operator (black-box multigrid):
// coarse node I sits on fine node 2I, and a fine node with odd indices on
// some axes is interpolated from its 2, 4 or 8 parents with the operator
// collapsed onto those axes.
//
// Compact per-cell storage.  A fine brick holds 64 cells of 2x2x2 nodes; node
// 2c + u of cell c (parity class u = (ux, uy, uz), q = uz*4 + uy*2 + ux) has
// the 2^|u| parents c + o, o <= u componentwise.  Pc[pc_off(q) + crank(q, o)]
// [col] (col = brick*64 + cell) is the weight of parent o, so the 27 weights
// of a cell hold every non-zero of P, and the threads of one class (two warps
// per 512-thread block) read consecutive columns.  The same layout carries
// the product A P: a node of class u reaches the coarse nodes base + t,
// base = c - 1 + u, t in [0, 3 - u) on each axis, so a cell holds
// 27 + 3*18 + 3*12 + 8 = 125 values of A P instead of 8 x 27.
//
// Every kernel maps thread t of a block to class t >> 6 and cell t & 63 and
// dispatches on the class at compile time, so the stencil offsets, the
// parents touched and the accumulator indices are constants and the
// accumulators stay in registers.  Zero tests
// of coefficients and weights look at bit patterns (f64_nonzero): on GB300 an
// FP64 comparison takes a slot of the narrow FP64 pipe, as a multiply-add
// does.
#include "spfd_internal.cuh"

namespace spfd {

namespace {

__host__ __device__ constexpr int popc3(int q) {
  return (q & 1) + ((q >> 1) & 1) + ((q >> 2) & 1);
}
// Rows of A P kept for class q, and the first of them.
__host__ __device__ constexpr int tsize(int q) {
  return (3 - (q & 1)) * (3 - ((q >> 1) & 1)) * (3 - (q >> 2));
}
__host__ __device__ constexpr int toff(int q) {
  int r = 0;
  for (int p = 0; p < q; ++p) r += tsize(p);
  return r;
}
static_assert(toff(8) == 125, "A P rows per cell");
static_assert(pc_off(7) + 8 == 27, "P rows per cell");

// One multigrid level seen as an operator: the 7-point form (three +edge
// conductances per node and the diagonal) on level 0, 27 Galerkin
// coefficients per node on coarser levels.
struct LevelOp {
  Grid g;
  const double *gx;    // [3][S] or null
  const double *st;    // [27][S] or null
  const double *diag;  // [S]
  size_t S, NC;        // slots, cells (S / 8)
};

// Column of the cell at local cell coordinates (x, y, z) of brick b, each in
// [-1, 4] (outside [0, 3] it lies in a face/edge/corner neighbour brick), or
// -1 if that brick is not stored.
__device__ __forceinline__ long long cell_col(const Grid &g, int b, int x, int y, int z) {
  const int ox = x >> 2, oy = y >> 2, oz = z >> 2;
  int bb = b;
  if (ox | oy | oz) {
    bb = __ldg(&g.nbr[(size_t)b * 27 + sidx(ox, oy, oz)]);
    if (bb < 0) return -1;
  }
  return (long long)bb * 64 + (((z & 3) * 4 + (y & 3)) * 4 + (x & 3));
}

// Slot of the class-(ux, uy, uz) node of cell column cc.
__device__ __forceinline__ size_t cell_slot(long long cc, int ux, int uy, int uz) {
  const int cell = (int)(cc & 63);
  const int lx = 2 * (cell & 3) + ux, ly = 2 * ((cell >> 2) & 3) + uy,
            lz = 2 * (cell >> 4) + uz;
  return (size_t)(cc >> 6) * BV + (lz * 8 + ly) * 8 + lx;
}

// A(n, n + e) for node n (slot s, class u, local cell c of brick b).  On the
// 7-point level the conductance of a -edge is stored at the lower node.
template <bool K27>
__device__ __forceinline__ double coef(const LevelOp &A, int e, size_t s, int b,
                                       int cx, int cy, int cz, int ux, int uy, int uz) {
  if (K27) return A.st[(size_t)e * A.S + s];
  if (e == 13) return A.diag[s];
  const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = e / 9 - 1;
  const int d = ex ? 0 : (ey ? 1 : 2);
  if (ex + ey + ez > 0) return -A.gx[(size_t)d * A.S + s];
  const long long mc = cell_col(A.g, b, cx + ((ux + ex) >> 1), cy + ((uy + ey) >> 1),
                                cz + ((uz + ez) >> 1));
  if (mc < 0) return 0.0;
  return -A.gx[(size_t)d * A.S + cell_slot(mc, (ux + ex) & 1, (uy + ey) & 1, (uz + ez) & 1)];
}

__device__ __forceinline__ constexpr bool in_stencil(bool k27, int e) {
  return k27 || ((e % 3 != 1) + ((e / 3) % 3 != 1) + (e / 9 != 1)) <= 1;
}

// ------------------------------------------------- interpolation weights
// Node n of class Q (|Q| >= 1) solves its own row of A u = 0 with the
// operator collapsed onto its odd axes: the couplings to n + e are summed
// onto n + p, p = e restricted to the odd axes of n; those with p = 0 form
// the denominator, the others couple n to nodes of lower classes whose
// weights are final.  Weights of neighbours that are not unknowns (air, or
// bricks that are not stored) are taken trilinear while the recursion runs,
// so that constants are reproduced; rows of nodes that are not unknowns are
// zero.  Rows whose collapsed diagonal vanishes fall back to trilinear.
template <int Q, bool K27>
__device__ __forceinline__ void interp_node(const LevelOp &A, double *__restrict__ Pc,
                                            int b, int4 bc, int cell) {
  constexpr int UX = Q & 1, UY = (Q >> 1) & 1, UZ = Q >> 2;
  constexpr int NW = 1 << popc3(Q);
  const Grid &g = A.g;
  const int cx = cell & 3, cy = (cell >> 2) & 3, cz = cell >> 4;
  const int i = bc.x * 8 + 2 * cx + UX, j = bc.y * 8 + 2 * cy + UY, k = bc.z * 8 + 2 * cz + UZ;
  const size_t s = (size_t)b * BV + ((2 * cz + UZ) * 8 + 2 * cy + UY) * 8 + 2 * cx + UX;
  const size_t col = (size_t)b * 64 + cell;
  const bool valid = i < g.NX && j < g.NY && k < g.NZ;
  const double dg = valid ? A.diag[s] : 0.0;
  double w[NW];
#pragma unroll
  for (int r = 0; r < NW; ++r) w[r] = 0.0;
  if (f64_nonzero(dg)) {  // dg >= 0
    if (Q == 0) {
      w[0] = 1.0;
    } else {
      double ac[27];
#pragma unroll
      for (int p = 0; p < 27; ++p) ac[p] = 0.0;
#pragma unroll
      for (int e = 0; e < 27; ++e) {
        if (!in_stencil(K27, e)) continue;
        const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = e / 9 - 1;
        ac[sidx(UX ? ex : 0, UY ? ey : 0, UZ ? ez : 0)] +=
            coef<K27>(A, e, s, b, cx, cy, cz, UX, UY, UZ);
      }
      double acc[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) acc[r] = 0.0;
#pragma unroll
      for (int p = 0; p < 27; ++p) {
        const int px = p % 3 - 1, py = (p / 3) % 3 - 1, pz = p / 9 - 1;
        if (p == 13 || (!UX && px) || (!UY && py) || (!UZ && pz)) continue;
        const double a = ac[p];
        if (!f64_nonzero(a)) continue;
        if (i + px >= g.NX || j + py >= g.NY || k + pz >= g.NZ) continue;
        // the neighbour is even where p is non-zero; its cell is ours moved
        // by one on the axes where p = +1
        const int MQ = Q & ~((px != 0) | ((py != 0) << 1) | ((pz != 0) << 2));
        const int MX = px == 1, MY = py == 1, MZ = pz == 1;
        const int NWM = 1 << popc3(MQ);
        double wm[8];
        if (MQ == 0) {
          wm[0] = 1.0;  // coincident nodes: 1 whether or not they are unknowns
        } else {
          const long long mc = cell_col(g, b, cx + MX, cy + MY, cz + MZ);
          bool stored = false;
          if (mc >= 0)
            stored = f64_nonzero(A.diag[cell_slot(mc, MQ & 1, (MQ >> 1) & 1, MQ >> 2)]);
#pragma unroll
          for (int r = 0; r < 8; ++r) wm[r] = 1.0 / NWM;
          if (stored) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
              if (r < NWM) wm[r] = Pc[(size_t)(pc_off(MQ) + r) * A.NC + mc];
          }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          if (o & ~MQ) continue;
          const int oo = o | MX | (MY << 1) | (MZ << 2);
          acc[crank(Q, oo)] += a * wm[crank(MQ, o)];
        }
      }
      const double den = ac[13];
      if (den > 1e-12 * dg) {
        const double inv = -1.0 / den;
#pragma unroll
        for (int r = 0; r < NW; ++r) w[r] = acc[r] * inv;
      } else {
#pragma unroll
        for (int r = 0; r < NW; ++r) w[r] = 1.0 / NW;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NW; ++r) Pc[(size_t)(pc_off(Q) + r) * A.NC + col] = w[r];
}

// Pass 1: classes 0 (coincident) and 1, 2, 4 (one odd axis); pass 2: classes
// with two odd axes; pass 3: class 7.  Each pass reads only classes of
// earlier passes, except class 0, whose weight a reader never loads.  A
// block holds only the pass's classes (64 threads each, one per cell) for
// interp_bricks<PASS>() bricks, so every launched warp has work.
template <int PASS>
constexpr int interp_classes() { return PASS == 1 ? 4 : (PASS == 2 ? 3 : 1); }
template <int PASS>
constexpr int interp_bricks() { return PASS == 3 ? 8 : 2; }
template <bool K27, int PASS>
__global__ void __launch_bounds__(NT) k_interp(LevelOp A, double *__restrict__ Pc) {
  constexpr int NCL = interp_classes<PASS>();
  const int cell = threadIdx.x & 63, grp = threadIdx.x >> 6;
  const int ci = grp % NCL, b = blockIdx.x * interp_bricks<PASS>() + grp / NCL;
  if (b >= A.g.nb) return;
  const int q = PASS == 1 ? (ci == 0 ? 0 : 1 << (ci - 1)) : (PASS == 2 ? 7 - (1 << ci) : 7);
  const int4 bc = A.g.bco[b];
  switch (q) {
    case 0: interp_node<0, K27>(A, Pc, b, bc, cell); break;
    case 1: interp_node<1, K27>(A, Pc, b, bc, cell); break;
    case 2: interp_node<2, K27>(A, Pc, b, bc, cell); break;
    case 3: interp_node<3, K27>(A, Pc, b, bc, cell); break;
    case 4: interp_node<4, K27>(A, Pc, b, bc, cell); break;
    case 5: interp_node<5, K27>(A, Pc, b, bc, cell); break;
    case 6: interp_node<6, K27>(A, Pc, b, bc, cell); break;
    default: interp_node<7, K27>(A, Pc, b, bc, cell); break;
  }
}

// ------------------------------------------------------- T = A P (stage 1)
// T(n, base(n) + t) = sum_e A(n, n + e) P(n + e, base(n) + t).
template <int Q, bool K27>
__device__ __forceinline__ void ap_node(const LevelOp &A, const double *__restrict__ Pc,
                                        double *__restrict__ T, int b, int4 bc, int cell) {
  constexpr int UX = Q & 1, UY = (Q >> 1) & 1, UZ = Q >> 2;
  constexpr int TX = 3 - UX, TY = 3 - UY, TZ = 3 - UZ, NTQ = TX * TY * TZ;
  const Grid &g = A.g;
  const int cx = cell & 3, cy = (cell >> 2) & 3, cz = cell >> 4;
  const int i = bc.x * 8 + 2 * cx + UX, j = bc.y * 8 + 2 * cy + UY, k = bc.z * 8 + 2 * cz + UZ;
  const size_t s = (size_t)b * BV + ((2 * cz + UZ) * 8 + 2 * cy + UY) * 8 + 2 * cx + UX;
  const size_t col = (size_t)b * 64 + cell;
  double acc[NTQ];
#pragma unroll
  for (int r = 0; r < NTQ; ++r) acc[r] = 0.0;
  if (i < g.NX && j < g.NY && k < g.NZ) {
#pragma unroll
    for (int e = 0; e < 27; ++e) {
      if (!in_stencil(K27, e)) continue;
      const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = e / 9 - 1;
      const double a = coef<K27>(A, e, s, b, cx, cy, cz, UX, UY, UZ);
      if (!f64_nonzero(a)) continue;
      const int mux = (UX + ex) & 1, muy = (UY + ey) & 1, muz = (UZ + ez) & 1;
      const int dcx = (UX + ex) >> 1, dcy = (UY + ey) >> 1, dcz = (UZ + ez) >> 1;
      const int MQ = mux | (muy << 1) | (muz << 2);
      const long long mc = (dcx | dcy | dcz) ? cell_col(g, b, cx + dcx, cy + dcy, cz + dcz)
                                             : (long long)col;
      if (mc < 0) continue;
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        if (o & ~MQ) continue;
        const int tx = dcx + (o & 1) + 1 - UX, ty = dcy + ((o >> 1) & 1) + 1 - UY,
                  tz = dcz + (o >> 2) + 1 - UZ;
        acc[(tz * TY + ty) * TX + tx] +=
            a * Pc[(size_t)(pc_off(MQ) + crank(MQ, o)) * A.NC + mc];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NTQ; ++r) T[(size_t)(toff(Q) + r) * A.NC + col] = acc[r];
}

// 7-point level: two resident blocks (at most 64 registers; 66 unbounded,
// which allowed one); 27-point levels keep one (92 registers).
template <bool K27>
__global__ void __launch_bounds__(NT, K27 ? 1 : 2) k_ap(LevelOp A, const double *__restrict__ Pc,
                                           double *__restrict__ T) {
  const int q = threadIdx.x >> 6, cell = threadIdx.x & 63, b = blockIdx.x;
  const int4 bc = A.g.bco[b];
  switch (q) {
    case 0: ap_node<0, K27>(A, Pc, T, b, bc, cell); break;
    case 1: ap_node<1, K27>(A, Pc, T, b, bc, cell); break;
    case 2: ap_node<2, K27>(A, Pc, T, b, bc, cell); break;
    case 3: ap_node<3, K27>(A, Pc, T, b, bc, cell); break;
    case 4: ap_node<4, K27>(A, Pc, T, b, bc, cell); break;
    case 5: ap_node<5, K27>(A, Pc, T, b, bc, cell); break;
    case 6: ap_node<6, K27>(A, Pc, T, b, bc, cell); break;
    default: ap_node<7, K27>(A, Pc, T, b, bc, cell); break;
  }
}

// ------------------------------------------------- A_c = P^T T (stage 2)
// One thread per coarse node I: A_c(I, I + D) = sum_d P(2I + d, I)
// T(2I + d, I + D) for the 14 offsets D with sidx(D) >= 13 (the others follow
// by symmetry, k_mirror), and P[d][I] = P(2I + d, I) for restriction and
// prolongation.  Fine node 2I + d lies in cell I + (d == -1) of class |d|
// and sees I as its parent (d == -1); its A P row starts at
// base = I - 1 + (d == +1), so t = D + 1 - (d == +1).
// The 9 terms d = (dx, dy, DZ) of one coarse node: P[d] written, the
// products with T accumulated into acc (offsets D with sidx(D) >= 13).
template <int DZ>
__device__ __forceinline__ void ptap_layer(const Grid &gf, const Grid &gc, size_t NCf,
                                           const double *__restrict__ Pc,
                                           const double *__restrict__ T, double *__restrict__ P,
                                           const int *kid, size_t Sc, size_t s, int X, int Y,
                                           int Z, int I, int J, int K, bool valid,
                                           double (&acc)[14], bool &any) {
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int d = (DZ + 1) * 9 + j;
    const int dx = j % 3 - 1, dy = j / 3 - 1, dz = DZ;
    const int ux = dx != 0, uy = dy != 0, uz = dz != 0;
    const int U = ux | (uy << 1) | (uz << 2);
    const int O = (dx < 0) | ((dy < 0) << 1) | ((dz < 0) << 2);
    // fine cell of 2I + d in cell coordinates local to fine brick 2B
    const int fx = X - (dx < 0), fy = Y - (dy < 0), fz = Z - (dz < 0);
    const int kb = kid[((fz >> 2) + 1) * 9 + ((fy >> 2) + 1) * 3 + ((fx >> 2) + 1)];
    double w = 0.0;
    long long col = -1;
    if (valid && kb >= 0 && 2 * I + dx < gf.NX && 2 * J + dy < gf.NY && 2 * K + dz < gf.NZ) {
      col = (long long)kb * 64 + (((fz & 3) * 4 + (fy & 3)) * 4 + (fx & 3));
      w = Pc[(size_t)(pc_off(U) + crank(U, O)) * NCf + col];
    }
    P[(size_t)d * Sc + s] = w;
    any |= f64_nonzero(w);
    if (f64_nonzero(w)) {
#pragma unroll
      for (int D = 13; D < 27; ++D) {
        const int Dx = D % 3 - 1, Dy = (D / 3) % 3 - 1, Dz = D / 9 - 1;
        const int tx = Dx + 1 - (dx > 0), ty = Dy + 1 - (dy > 0), tz = Dz + 1 - (dz > 0);
        if (tx < 0 || tx > 2 - ux || ty < 0 || ty > 2 - uy || tz < 0 || tz > 2 - uz) continue;
        acc[D - 13] +=
            w * T[(size_t)(toff(U) + (tz * (3 - uy) + ty) * (3 - ux) + tx) * NCf + col];
      }
    }
  }
}

// Each also writes the coarse level's activity bits (Grid::act): the bit of
// a coarse node is set when one of its 27 weights P[d] is not zero.
__global__ void __launch_bounds__(NT)
k_ptap(Grid gf, Grid gc, size_t NCf, const double *__restrict__ Pc,
       const double *__restrict__ T, double *__restrict__ stc, double *__restrict__ P,
       unsigned *__restrict__ act) {
  __shared__ int kid[27];
  const int b = blockIdx.x, t = threadIdx.x;
  if (t < 27) kid[t] = gc.kid[(size_t)b * 27 + t];
  __syncthreads();
  const size_t Sc = (size_t)gc.nb * BV, s = (size_t)b * BV + t;
  const int X = t & 7, Y = (t >> 3) & 7, Z = t >> 6;
  const int4 bc = gc.bco[b];
  const int I = bc.x * 8 + X, J = bc.y * 8 + Y, K = bc.z * 8 + Z;
  const bool valid = I < gc.NX && J < gc.NY && K < gc.NZ;
  double acc[14];
#pragma unroll
  for (int r = 0; r < 14; ++r) acc[r] = 0.0;
  bool any = false;
  ptap_layer<-1>(gf, gc, NCf, Pc, T, P, kid, Sc, s, X, Y, Z, I, J, K, valid, acc, any);
  ptap_layer<0>(gf, gc, NCf, Pc, T, P, kid, Sc, s, X, Y, Z, I, J, K, valid, acc, any);
  ptap_layer<1>(gf, gc, NCf, Pc, T, P, kid, Sc, s, X, Y, Z, I, J, K, valid, acc, any);
#pragma unroll
  for (int r = 0; r < 14; ++r) stc[(size_t)(13 + r) * Sc + s] = acc[r];
  const unsigned word = __ballot_sync(0xffffffffu, any);
  if ((t & 31) == 0) act[(size_t)b * 16 + (t >> 5)] = word;
}

// The same for small coarse levels, where one thread per coarse node leaves
// most SMs idle: three threads per coarse node, one per fine z-layer of its
// 27 points, in blocks of 3 x 128 threads over a quarter brick; the layers'
// sums are added in a fixed order (dz = -1, 0, +1).
constexpr int PT_Q = 128;
__global__ void __launch_bounds__(3 * PT_Q)
k_ptap3(Grid gf, Grid gc, size_t NCf, const double *__restrict__ Pc,
        const double *__restrict__ T, double *__restrict__ stc, double *__restrict__ P,
        unsigned *__restrict__ act) {
  __shared__ int kid[27];
  __shared__ double red[2][PT_Q][15];
  __shared__ bool anyp[2][PT_Q];
  const int b = blockIdx.x >> 2;
  const int part = threadIdx.x / PT_Q, nl = threadIdx.x % PT_Q;
  const int t = (blockIdx.x & 3) * PT_Q + nl;
  if (threadIdx.x < 27) kid[threadIdx.x] = gc.kid[(size_t)b * 27 + threadIdx.x];
  __syncthreads();
  const size_t Sc = (size_t)gc.nb * BV, s = (size_t)b * BV + t;
  const int X = t & 7, Y = (t >> 3) & 7, Z = t >> 6;
  const int4 bc = gc.bco[b];
  const int I = bc.x * 8 + X, J = bc.y * 8 + Y, K = bc.z * 8 + Z;
  const bool valid = I < gc.NX && J < gc.NY && K < gc.NZ;
  double acc[14];
#pragma unroll
  for (int r = 0; r < 14; ++r) acc[r] = 0.0;
  bool any = false;
  if (part == 0)
    ptap_layer<-1>(gf, gc, NCf, Pc, T, P, kid, Sc, s, X, Y, Z, I, J, K, valid, acc, any);
  else if (part == 1)
    ptap_layer<0>(gf, gc, NCf, Pc, T, P, kid, Sc, s, X, Y, Z, I, J, K, valid, acc, any);
  else
    ptap_layer<1>(gf, gc, NCf, Pc, T, P, kid, Sc, s, X, Y, Z, I, J, K, valid, acc, any);
  if (part > 0) {
#pragma unroll
    for (int r = 0; r < 14; ++r) red[part - 1][nl][r] = acc[r];
    anyp[part - 1][nl] = any;
  }
  __syncthreads();
  if (part == 0) {
#pragma unroll
    for (int r = 0; r < 14; ++r)
      stc[(size_t)(13 + r) * Sc + s] = (acc[r] + red[0][nl][r]) + red[1][nl][r];
    // part 0 is threads 0 .. PT_Q-1: whole warps, slots t in warp order
    const unsigned word = __ballot_sync(0xffffffffu, any || anyp[0][nl] || anyp[1][nl]);
    if ((nl & 31) == 0) act[(size_t)b * 16 + (t >> 5)] = word;
  }
}

// A_c(I, I + D) = A_c(I + D, I) for the 13 offsets with sidx(D) < 13.
__global__ void __launch_bounds__(NT) k_mirror(Grid g, double *__restrict__ stc) {
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const size_t s = (size_t)b * BV + t;
  const int4 bc = g.bco[b];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
#pragma unroll
  for (int e = 0; e < 13; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    const int m = slot_nb(g, b, bc, lx, ly, lz, dx, dy, dz);
    stc[(size_t)e * S + s] = m >= 0 ? stc[(size_t)(26 - e) * S + m] : 0.0;
  }
}

}  // namespace

int ap_rows_per_cell() { return toff(8); }

void launch_interp_weights(const Grid &gf, const double *gx, const double *st27,
                           const double *diag, double *Pc, cudaStream_t st) {
  if (gf.nb == 0) return;
  const LevelOp A{gf, gx, st27, diag, (size_t)gf.nb * BV, (size_t)gf.nb * 64};
  auto grid = [&](int bricks) { return (unsigned)((gf.nb + bricks - 1) / bricks); };
  constexpr int T1 = 64 * interp_classes<1>() * interp_bricks<1>();
  constexpr int T2 = 64 * interp_classes<2>() * interp_bricks<2>();
  constexpr int T3 = 64 * interp_classes<3>() * interp_bricks<3>();
  static_assert(T1 <= NT && T2 <= NT && T3 <= NT, "interp blocks");
  if (st27) {
    k_interp<true, 1><<<grid(interp_bricks<1>()), T1, 0, st>>>(A, Pc);
    k_interp<true, 2><<<grid(interp_bricks<2>()), T2, 0, st>>>(A, Pc);
    k_interp<true, 3><<<grid(interp_bricks<3>()), T3, 0, st>>>(A, Pc);
  } else {
    k_interp<false, 1><<<grid(interp_bricks<1>()), T1, 0, st>>>(A, Pc);
    k_interp<false, 2><<<grid(interp_bricks<2>()), T2, 0, st>>>(A, Pc);
    k_interp<false, 3><<<grid(interp_bricks<3>()), T3, 0, st>>>(A, Pc);
  }
}

void launch_galerkin(const Grid &gf, const Grid &gc, const double *gx,
                     const double *st27f, const double *diagf, const double *Pc,
                     double *T, double *stc, double *P, unsigned *act, cudaStream_t st) {
  if (gf.nb == 0 || gc.nb == 0) return;
  const LevelOp A{gf, gx, st27f, diagf, (size_t)gf.nb * BV, (size_t)gf.nb * 64};
  if (st27f) k_ap<true><<<gf.nb, NT, 0, st>>>(A, Pc, T);
  else k_ap<false><<<gf.nb, NT, 0, st>>>(A, Pc, T);
  // below a few waves of one-brick blocks, three threads per coarse node
  if (gc.nb < 1024) k_ptap3<<<gc.nb * 4, 3 * PT_Q, 0, st>>>(gf, gc, A.NC, Pc, T, stc, P, act);
  else k_ptap<<<gc.nb, NT, 0, st>>>(gf, gc, A.NC, Pc, T, stc, P, act);
  k_mirror<<<gc.nb, NT, 0, st>>>(gc, stc);
}

}  // namespace spfd
