// Setup kernels: conductances, unknowns, components, multigrid hierarchy.
//
// Paper: Eq. 3 (Sec. II) defines the operator G^T M_k G; M_k's edge
// conductances are the averaged conductivities of the voxels around each
// edge; Sec. III-A keeps only conducting nodes as unknowns.  The hierarchy
// (operator-dependent interpolation + Galerkin coarse operators) replaces the
// algebraic multigrid of the AmgX library the paper uses (Sec. III).
#include "spfd_internal.cuh"

namespace spfd {

// ------------------------------------------------------------ sigma -> bricks
__global__ void k_sigma_flags(const double *__restrict__ sigma, int nx, int ny,
                              int nz, int MX, int MY,
                              unsigned char *__restrict__ flags,
                              unsigned char *__restrict__ mask, int *status) {
  const long long n = (long long)nx * ny * nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int bad = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += stride) {
    double s = sigma[v];
    mask[v] = s > 0.0;
    if (!(s >= 0.0) || !isfinite(s)) { bad = 1; continue; }
    if (s > 0.0) {
      int i = (int)(v % nx);
      int j = (int)((v / nx) % ny);
      int k = (int)(v / ((long long)nx * ny));
      // the voxel's 8 corner nodes are unknowns; mark their bricks
      int i0 = i >> 3, i1 = (i + 1) >> 3, j0 = j >> 3, j1 = (j + 1) >> 3;
      int k0 = k >> 3, k1 = (k + 1) >> 3;
      flags[(k0 * MY + j0) * MX + i0] = 1;
      if (i1 != i0) flags[(k0 * MY + j0) * MX + i1] = 1;
      if (j1 != j0) flags[(k0 * MY + j1) * MX + i0] = 1;
      if (k1 != k0) flags[(k1 * MY + j0) * MX + i0] = 1;
      if (i1 != i0 && j1 != j0) flags[(k0 * MY + j1) * MX + i1] = 1;
      if (i1 != i0 && k1 != k0) flags[(k1 * MY + j0) * MX + i1] = 1;
      if (j1 != j0 && k1 != k0) flags[(k1 * MY + j1) * MX + i0] = 1;
      if (i1 != i0 && j1 != j0 && k1 != k0) flags[(k1 * MY + j1) * MX + i1] = 1;
    }
  }
  if (bad) atomicOr(status, DEV_BAD_SIGMA);
}

void launch_sigma_flags(const double *sigma, int nx, int ny, int nz, int MX,
                        int MY, unsigned char *flags, unsigned char *mask,
                        int *status, cudaStream_t st) {
  long long n = (long long)nx * ny * nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  k_sigma_flags<<<(int)blocks, 256, 0, st>>>(sigma, nx, ny, nz, MX, MY, flags,
                                              mask, status);
}

// ------------------------------------------------- conductances (Eq. 3, M_k)
__device__ __forceinline__ double sig_at(const double *__restrict__ s, int i,
                                         int j, int k, int nx, int ny, int nz) {
  if ((unsigned)i >= (unsigned)nx || (unsigned)j >= (unsigned)ny ||
      (unsigned)k >= (unsigned)nz)
    return 0.0;
  return __ldg(&s[((long long)k * ny + j) * nx + i]);
}

// g of the x/y/z edge leaving node (i,j,k): h/4 * sum of the 4 voxels around it.
__device__ __forceinline__ double g_edge(const double *s, int d, int i, int j,
                                         int k, int nx, int ny, int nz,
                                         double hq) {
  if (d == 0) {
    if (i < 0 || i >= nx) return 0.0;
    return hq * (sig_at(s, i, j - 1, k - 1, nx, ny, nz) + sig_at(s, i, j, k - 1, nx, ny, nz) +
                 sig_at(s, i, j - 1, k, nx, ny, nz) + sig_at(s, i, j, k, nx, ny, nz));
  } else if (d == 1) {
    if (j < 0 || j >= ny) return 0.0;
    return hq * (sig_at(s, i - 1, j, k - 1, nx, ny, nz) + sig_at(s, i, j, k - 1, nx, ny, nz) +
                 sig_at(s, i - 1, j, k, nx, ny, nz) + sig_at(s, i, j, k, nx, ny, nz));
  } else {
    if (k < 0 || k >= nz) return 0.0;
    return hq * (sig_at(s, i - 1, j - 1, k, nx, ny, nz) + sig_at(s, i, j - 1, k, nx, ny, nz) +
                 sig_at(s, i - 1, j, k, nx, ny, nz) + sig_at(s, i, j, k, nx, ny, nz));
  }
}

__global__ void __launch_bounds__(NT)
k_build_fine(Grid g, const double *__restrict__ sigma, int nx, int ny, int nz,
             double h, double *__restrict__ gx, double *__restrict__ diag,
             double *__restrict__ dinv) {
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const int4 bc = g.bco[b];
  const int i = bc.x * 8 + (t & 7), j = bc.y * 8 + ((t >> 3) & 7),
            k = bc.z * 8 + (t >> 6);
  const size_t s = (size_t)b * BV + t;
  double e[6] = {0, 0, 0, 0, 0, 0};
  if (i < g.NX && j < g.NY && k < g.NZ) {
    const double hq = h * 0.25;
    e[0] = g_edge(sigma, 0, i, j, k, nx, ny, nz, hq);      // +x
    e[1] = g_edge(sigma, 1, i, j, k, nx, ny, nz, hq);      // +y
    e[2] = g_edge(sigma, 2, i, j, k, nx, ny, nz, hq);      // +z
    e[3] = g_edge(sigma, 0, i - 1, j, k, nx, ny, nz, hq);  // -x
    e[4] = g_edge(sigma, 1, i, j - 1, k, nx, ny, nz, hq);  // -y
    e[5] = g_edge(sigma, 2, i, j, k - 1, nx, ny, nz, hq);  // -z
  }
  double d = ((e[3] + e[0]) + (e[4] + e[1])) + (e[5] + e[2]);
  gx[s] = e[0];
  gx[S + s] = e[1];
  gx[2 * S + s] = e[2];
  diag[s] = d;
  dinv[s] = d > 0.0 ? 1.0 / d : 0.0;
}

void launch_build_fine(const Grid &g, const double *sigma, int nx, int ny,
                       int nz, double h, double *gx, double *diag,
                       double *dinv, cudaStream_t st) {
  if (g.nb == 0) return;
  k_build_fine<<<g.nb, NT, 0, st>>>(g, sigma, nx, ny, nz, h, gx, diag, dinv);
}

// ------------------------------------------------ components (union-find)
// Lock-free union-find: roots are linked with atomicCAS (larger index under
// smaller), non-root pointers are only shortened.  Every loop is bounded and
// reports DEV_UF_CAP instead of spinning.
constexpr int UF_FIND_CAP = 1 << 16;
constexpr int UF_UNITE_CAP = 1 << 10;

__device__ int uf_find(int *parent, int x, int *capped) {
  volatile int *p = parent;
  for (int it = 0; it < UF_FIND_CAP; ++it) {
    int px = p[x];
    if (px == x) return x;
    int gp = p[px];
    if (gp != px) p[x] = gp;
    x = gp;
  }
  *capped = 1;
  return x;
}

__device__ void uf_unite(int *parent, int a, int b, int *capped) {
  for (int it = 0; it < UF_UNITE_CAP; ++it) {
    a = uf_find(parent, a, capped);
    b = uf_find(parent, b, capped);
    if (a == b || *capped) return;
    if (a < b) { int t = a; a = b; b = t; }
    if (atomicCAS(&parent[a], a, b) == a) return;
  }
  *capped = 1;
}

__global__ void __launch_bounds__(NT)
k_uf_init(Grid g, const double *__restrict__ gx, int *parent) {
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const size_t s = (size_t)b * BV + t;
  const int4 bc = g.bco[b];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  // active iff an incident edge conducts: own +edges or the neighbours' +edges
  bool act = gx[s] > 0 || gx[S + s] > 0 || gx[2 * S + s] > 0;
  if (!act) {
    int m = slot_nb(g, b, bc, lx, ly, lz, -1, 0, 0);
    act = m >= 0 && gx[m] > 0;
  }
  if (!act) {
    int m = slot_nb(g, b, bc, lx, ly, lz, 0, -1, 0);
    act = m >= 0 && gx[S + m] > 0;
  }
  if (!act) {
    int m = slot_nb(g, b, bc, lx, ly, lz, 0, 0, -1);
    act = m >= 0 && gx[2 * S + m] > 0;
  }
  parent[s] = act ? (int)s : -1;
}

__global__ void __launch_bounds__(NT)
k_uf_union(Grid g, const double *__restrict__ gx, int *parent, int *status) {
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const int s = b * BV + t;
  const int4 bc = g.bco[b];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  int capped = 0;
  if (gx[s] > 0) {
    int m = slot_nb(g, b, bc, lx, ly, lz, 1, 0, 0);
    if (m >= 0) uf_unite(parent, s, m, &capped);
  }
  if (gx[S + s] > 0) {
    int m = slot_nb(g, b, bc, lx, ly, lz, 0, 1, 0);
    if (m >= 0) uf_unite(parent, s, m, &capped);
  }
  if (gx[2 * S + s] > 0) {
    int m = slot_nb(g, b, bc, lx, ly, lz, 0, 0, 1);
    if (m >= 0) uf_unite(parent, s, m, &capped);
  }
  if (capped) atomicOr(status, DEV_UF_CAP);
}

__global__ void __launch_bounds__(NT)
k_uf_compress(Grid g, int *parent, int *status) {
  const int s = blockIdx.x * BV + threadIdx.x;
  int capped = 0;
  if (parent[s] >= 0) parent[s] = uf_find(parent, s, &capped);
  if (capped) atomicOr(status, DEV_UF_CAP);
}

void launch_components(const Grid &g, const double *gx, int *parent,
                       int *status, cudaStream_t st) {
  if (g.nb == 0) return;
  k_uf_init<<<g.nb, NT, 0, st>>>(g, gx, parent);
  k_uf_union<<<g.nb, NT, 0, st>>>(g, gx, parent, status);
  k_uf_compress<<<g.nb, NT, 0, st>>>(g, parent, status);
}

// Number of roots per brick (for deterministic component numbering).
__global__ void __launch_bounds__(NT)
k_root_counts(const int *__restrict__ parent, int *counts) {
  const int s = blockIdx.x * BV + threadIdx.x;
  int c = __syncthreads_count(parent[s] == s);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

void launch_root_counts(const Grid &g, const int *parent, int *counts,
                        cudaStream_t st) {
  if (g.nb == 0) return;
  k_root_counts<<<g.nb, NT, 0, st>>>(parent, counts);
}

// Component id of a root = offset of its brick + rank among the brick's roots.
__global__ void __launch_bounds__(NT)
k_root_ids(const int *__restrict__ parent, const int *__restrict__ offsets,
           int *comp) {
  __shared__ int warp_cnt[NT / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int s = blockIdx.x * BV + t;
  const bool root = parent[s] == s;
  unsigned m = __ballot_sync(0xffffffffu, root);
  if (lane == 0) warp_cnt[w] = __popc(m);
  __syncthreads();
  int before = 0;
  for (int q = 0; q < w; ++q) before += warp_cnt[q];
  before += __popc(m & ((1u << lane) - 1u));
  comp[s] = root ? offsets[blockIdx.x] + before : -1;
}

__global__ void __launch_bounds__(NT)
k_comp_from_root(const int *__restrict__ parent, int *comp) {
  const int s = blockIdx.x * BV + threadIdx.x;
  int p = parent[s];
  if (p >= 0 && p != s) comp[s] = comp[p];
}

void launch_assign_comp(const Grid &g, const int *parent, const int *offsets,
                        int *comp, cudaStream_t st) {
  if (g.nb == 0) return;
  k_root_ids<<<g.nb, NT, 0, st>>>(parent, offsets, comp);
  k_comp_from_root<<<g.nb, NT, 0, st>>>(parent, comp);
}

__global__ void __launch_bounds__(NT)
k_comp_sizes(const int *__restrict__ comp, int *sizes) {
  const int s = blockIdx.x * BV + threadIdx.x;
  const int c = comp[s];
  // group lanes holding the same component; the lowest lane adds the count
  unsigned grp = __match_any_sync(0xffffffffu, c);
  if (c >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1)
    atomicAdd(&sizes[c], __popc(grp));
}

void launch_comp_sizes(const Grid &g, const int *comp, int *sizes,
                       cudaStream_t st) {
  if (g.nb == 0) return;
  k_comp_sizes<<<g.nb, NT, 0, st>>>(comp, sizes);
}

// ------------------------------------------ fine-level stencil coefficients
// A(n, n+e) for stencil offset e.  Level 0 keeps the 7-point operator as the
// three +edge conductances per node plus the diagonal; coarser levels keep
// all 27 Galerkin coefficients.
struct Coef {
  Grid g;
  const double *gx;    // [3][S] (7-point level) or null
  const double *st;    // [27][S] (27-point level) or null
  const double *diag;  // [S]
  size_t S;
  __device__ double operator()(int s, int e) const {
    if (st) return st[(size_t)e * S + s];
    if (e == 13) return diag[s];
    int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    if ((dx != 0) + (dy != 0) + (dz != 0) != 1) return 0.0;
    int d = dx != 0 ? 0 : (dy != 0 ? 1 : 2);
    if (dx + dy + dz > 0) return -gx[(size_t)d * S + s];
    int b = s >> 9, t = s & 511;
    int m = slot_nb(g, b, g.bco[b], t & 7, (t >> 3) & 7, t >> 6, dx, dy, dz);
    return m >= 0 ? -gx[(size_t)d * S + m] : 0.0;
  }
};

// --------------------------------------------- interpolation weights (BoxMG)
// For every fine node n, W[c][n] (c = cz*4+cy*2+cx) is the weight of the
// coarse node floor(n/2) + c.  Nodes with an even index on every axis copy
// their coarse node; nodes with one odd index interpolate along that line
// with the operator collapsed onto it; nodes with two odd indices use the
// operator collapsed onto their plane and the already interpolated line
// nodes; nodes with three odd indices use the full stencil.  Inactive nodes
// (and rows whose collapsed diagonal vanishes) get trilinear weights while
// the recursion runs, so that neighbours still reproduce constants; the rows
// of inactive nodes are zeroed at the end.
__device__ __forceinline__ void trilinear(double w[8], int ox, int oy, int oz) {
  for (int c = 0; c < 8; ++c) {
    int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    double v = 1.0;
    v *= ox ? 0.5 : (cx == 0 ? 1.0 : 0.0);
    v *= oy ? 0.5 : (cy == 0 ? 1.0 : 0.0);
    v *= oz ? 0.5 : (cz == 0 ? 1.0 : 0.0);
    w[c] = v;
  }
}

__global__ void __launch_bounds__(NT)
k_interp_pass(Coef A, int pass, double *__restrict__ W) {
  const Grid &g = A.g;
  const size_t S = A.S;
  const int b = blockIdx.x, t = threadIdx.x;
  const int s = b * BV + t;
  const int4 bc = g.bco[b];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  const int i = bc.x * 8 + lx, j = bc.y * 8 + ly, k = bc.z * 8 + lz;
  const int ox = i & 1, oy = j & 1, oz = k & 1;
  const int type = ox + oy + oz;
  const bool valid = i < g.NX && j < g.NY && k < g.NZ;

  if (pass == 0) {  // initialise: coincident nodes copy their coarse node
    for (int c = 0; c < 8; ++c) W[c * S + s] = (c == 0 && type == 0) ? 1.0 : 0.0;
    return;
  }
  if (pass == 4) {  // drop the rows of nodes that are not unknowns
    if (!(valid && A.diag[s] > 0.0))
      for (int c = 0; c < 8; ++c) W[c * S + s] = 0.0;
    return;
  }
  if (type != pass || !valid) return;

  const double dg = A.diag[s];
  double w[8];
  bool ok = false;
  if (dg > 0.0) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double den = 0.0;
    for (int e = 0; e < 27; ++e) {
      int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
      double a = A(s, e);
      if (a == 0.0) continue;
      // collapse the offset onto the odd axes of n
      int px = ox ? dx : 0, py = oy ? dy : 0, pz = oz ? dz : 0;
      if (px == 0 && py == 0 && pz == 0) { den += a; continue; }
      int mi = i + px, mj = j + py, mk = k + pz;
      if ((unsigned)mi >= (unsigned)g.NX || (unsigned)mj >= (unsigned)g.NY ||
          (unsigned)mk >= (unsigned)g.NZ)
        continue;
      double wm[8];
      int m = slot_nb(g, b, bc, lx, ly, lz, px, py, pz);
      if (m >= 0) {
        for (int c = 0; c < 8; ++c) wm[c] = W[c * S + m];
      } else {
        trilinear(wm, mi & 1, mj & 1, mk & 1);  // not stored: a virtual node
      }
      // neighbour corner c' is our corner c' + (p == +1) on each axis
      for (int c = 0; c < 8; ++c) {
        if (wm[c] == 0.0) continue;
        int cx = (c & 1) + (px == 1), cy = ((c >> 1) & 1) + (py == 1),
            cz = (c >> 2) + (pz == 1);
        if (cx > 1 || cy > 1 || cz > 1) continue;
        acc[cz * 4 + cy * 2 + cx] += a * wm[c];
      }
    }
    if (den > 1e-12 * dg) {
      ok = true;
      double inv = -1.0 / den;
      for (int c = 0; c < 8; ++c) w[c] = acc[c] * inv;
    }
  }
  if (!ok) trilinear(w, ox, oy, oz);
  for (int c = 0; c < 8; ++c) W[c * S + s] = w[c];
}

void launch_interp_weights(const Grid &gf, const double *gx, const double *st27,
                           const double *diag, double *W, cudaStream_t st) {
  if (gf.nb == 0) return;
  Coef A{gf, gx, st27, diag, (size_t)gf.nb * BV};
  for (int pass = 0; pass <= 4; ++pass)
    k_interp_pass<<<gf.nb, NT, 0, st>>>(A, pass, W);
}

// -------------------------------------------------- Galerkin A_c = P^T A P
// One thread per coarse node I accumulates the 27 couplings
//   A_c(I, I+D) = sum_{n in supp I} P(n,I) sum_{e} A(n, n+e) P(n+e, I+D).
__global__ void __launch_bounds__(128)
k_galerkin(Coef A, Grid gc, const double *__restrict__ W,
           double *__restrict__ stc) {
  const Grid &gf = A.g;
  const size_t Sf = A.S, Sc = (size_t)gc.nb * BV;
  const long long sc = blockIdx.x * 128LL + threadIdx.x;
  if (sc >= (long long)Sc) return;
  const int b = (int)(sc >> 9), t = (int)(sc & 511);
  const int4 bc = gc.bco[b];
  const int I = bc.x * 8 + (t & 7), J = bc.y * 8 + ((t >> 3) & 7),
            K = bc.z * 8 + (t >> 6);
  double acc[27];
  for (int q = 0; q < 27; ++q) acc[q] = 0.0;
  if (I < gc.NX && J < gc.NY && K < gc.NZ) {
    for (int d = 0; d < 27; ++d) {
      int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      int n = slot_at(gf, 2 * I + dx, 2 * J + dy, 2 * K + dz);
      if (n < 0) continue;
      int c = (dz == -1) * 4 + (dy == -1) * 2 + (dx == -1);
      double w = W[c * Sf + n];
      if (w == 0.0) continue;
      int nbk = n >> 9, nt = n & 511;
      int4 nbc = gf.bco[nbk];
      int ni = nbc.x * 8 + (nt & 7), nj = nbc.y * 8 + ((nt >> 3) & 7),
          nk = nbc.z * 8 + (nt >> 6);
      for (int e = 0; e < 27; ++e) {
        double a = A(n, e);
        if (a == 0.0) continue;
        int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = e / 9 - 1;
        int m = slot_nb(gf, nbk, nbc, nt & 7, (nt >> 3) & 7, nt >> 6, ex, ey, ez);
        if (m < 0) continue;
        int mi = ni + ex, mj = nj + ey, mk = nk + ez;
        double wa = w * a;
        for (int c2 = 0; c2 < 8; ++c2) {
          double wm = W[c2 * Sf + m];
          if (wm == 0.0) continue;
          int DX = (mi >> 1) + (c2 & 1) - I, DY = (mj >> 1) + ((c2 >> 1) & 1) - J,
              DZ = (mk >> 1) + (c2 >> 2) - K;
          if (DX < -1 || DX > 1 || DY < -1 || DY > 1 || DZ < -1 || DZ > 1) continue;
          acc[sidx(DX, DY, DZ)] += wa * wm;
        }
      }
    }
  }
  for (int q = 0; q < 27; ++q) stc[q * Sc + sc] = acc[q];
}

void launch_galerkin(const Grid &gf, const Grid &gc, const double *gx,
                     const double *st27f, const double *diagf, const double *W,
                     double *stc, cudaStream_t st) {
  if (gc.nb == 0) return;
  Coef A{gf, gx, st27f, diagf, (size_t)gf.nb * BV};
  long long Sc = (long long)gc.nb * BV;
  k_galerkin<<<(int)((Sc + 127) / 128), 128, 0, st>>>(A, gc, W, stc);
}

// Average A_c(I,J) and A_c(J,I) so the coarse operator is exactly symmetric
// (the two sums above differ only in rounding order).
__global__ void __launch_bounds__(NT)
k_symmetrize(Grid g, double *__restrict__ stc) {
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const int s = b * BV + t;
  const int4 bc = g.bco[b];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  for (int e = 14; e < 27; ++e) {
    int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    int m = slot_nb(g, b, bc, lx, ly, lz, dx, dy, dz);
    double a = stc[(size_t)e * S + s];
    if (m < 0) {
      stc[(size_t)e * S + s] = 0.0;
      continue;
    }
    double c = stc[(size_t)(26 - e) * S + m];
    double v = 0.5 * (a + c);
    stc[(size_t)e * S + s] = v;
    stc[(size_t)(26 - e) * S + m] = v;
  }
}

void launch_symmetrize(const Grid &gc, double *stc, cudaStream_t st) {
  if (gc.nb == 0) return;
  k_symmetrize<<<gc.nb, NT, 0, st>>>(gc, stc);
}

// P stored per coarse node: P[d][I] = weight of coarse node I at fine node 2I+d.
__global__ void __launch_bounds__(NT)
k_pack_P(Grid gf, Grid gc, const double *__restrict__ W, double *__restrict__ P) {
  const size_t Sf = (size_t)gf.nb * BV, Sc = (size_t)gc.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const int s = b * BV + t;
  const int4 bc = gc.bco[b];
  const int I = bc.x * 8 + (t & 7), J = bc.y * 8 + ((t >> 3) & 7),
            K = bc.z * 8 + (t >> 6);
  for (int d = 0; d < 27; ++d) {
    int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    double w = 0.0;
    if (I < gc.NX && J < gc.NY && K < gc.NZ) {
      int n = slot_at(gf, 2 * I + dx, 2 * J + dy, 2 * K + dz);
      if (n >= 0) w = W[((dz == -1) * 4 + (dy == -1) * 2 + (dx == -1)) * Sf + n];
    }
    P[(size_t)d * Sc + s] = w;
  }
}

void launch_pack_P(const Grid &gf, const Grid &gc, const double *W, double *P,
                   cudaStream_t st) {
  if (gc.nb == 0) return;
  k_pack_P<<<gc.nb, NT, 0, st>>>(gf, gc, W, P);
}

// Diagonal, its inverse, and the level's largest diagonal (for a relative
// activity threshold).  Rows below 1e-13 * max diagonal are treated as not
// being unknowns (dinv = 0): they arise only from basis functions that are
// constant on a whole tiny component and carry no information.
__global__ void __launch_bounds__(NT)
k_coarse_diag(const double *__restrict__ stc, size_t S, double thresh,
              double *__restrict__ diag, double *__restrict__ dinv) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  double d = stc[13 * S + s];
  bool act = d > thresh;
  diag[s] = act ? d : 0.0;
  dinv[s] = act ? 1.0 / d : 0.0;
}

void launch_coarse_diag(const Grid &gc, const double *stc, double thresh,
                        double *diag, double *dinv, cudaStream_t st) {
  if (gc.nb == 0) return;
  k_coarse_diag<<<gc.nb, NT, 0, st>>>(stc, (size_t)gc.nb * BV, thresh, diag, dinv);
}

// Prolongation weights per fine cell.  A fine brick holds 64 cells of 2x2x2
// nodes; node 2c + u of cell c (u in {0,1}^3, parity class q = uz*4+uy*2+ux)
// has 2^(ux+uy+uz) parents c + o (o <= u componentwise).  Pc[pc_off(q) + j]
// [cell] is the weight of its j-th parent in (oz, oy, ox) loop order, so the
// threads of one parity class read consecutive entries.
__global__ void __launch_bounds__(NT)
k_pack_Pc(Grid gf, const double *__restrict__ W, double *__restrict__ Pc) {
  const size_t S = (size_t)gf.nb * BV, NC = S / 8;
  const int bk = blockIdx.x, t = threadIdx.x;
  const int q = t >> 6, cell = t & 63;
  const int ux = q & 1, uy = (q >> 1) & 1, uz = q >> 2;
  const int lx = 2 * (cell & 3) + ux, ly = 2 * ((cell >> 2) & 3) + uy, lz = 2 * (cell >> 4) + uz;
  const size_t s = (size_t)bk * BV + (lz * 8 + ly) * 8 + lx;
  const size_t cid = (size_t)bk * 64 + cell;
  int j = pc_off(q);
  for (int oz = 0; oz <= uz; ++oz)
    for (int oy = 0; oy <= uy; ++oy)
      for (int ox = 0; ox <= ux; ++ox)
        Pc[(size_t)(j++) * NC + cid] = W[(size_t)(oz * 4 + oy * 2 + ox) * S + s];
}

void launch_pack_Pc(const Grid &gf, const double *W, double *Pc, cudaStream_t st) {
  if (gf.nb) k_pack_Pc<<<gf.nb, NT, 0, st>>>(gf, W, Pc);
}

// ------------------------------------------------ coarsest dense inverse
// One Gauss-Jordan sweep of an SPD matrix on pivot k, read from A into B
// (m x m, row-major):  B[k][k] = 1/p,  B[k][j] = A[k][j]/p,
// B[i][k] = -A[i][k]/p,  B[i][j] = A[i][j] - A[i][k] A[k][j] / p  with
// p = A[k][k].  After sweeping every pivot once, B = A^-1.  Positive
// definiteness keeps every pivot (a Schur complement) positive, so no
// pivoting is needed; a non-positive pivot raises DEV_BAD_PIVOT.
__global__ void k_gj_sweep(const double *__restrict__ A, double *__restrict__ B,
                           int m, int k, int *status) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)m * m) return;
  const int i = (int)(idx / m), j = (int)(idx % m);
  const double p = A[(size_t)k * m + k];
  if (idx == 0 && !(p > 0.0)) atomicOr(status, DEV_BAD_PIVOT);
  const double inv = 1.0 / p;
  double v;
  if (i == k && j == k) v = inv;
  else if (i == k) v = A[(size_t)k * m + j] * inv;
  else if (j == k) v = -A[(size_t)i * m + k] * inv;
  else v = A[idx] - A[(size_t)i * m + k] * A[(size_t)k * m + j] * inv;
  B[idx] = v;
}

// Inverts the SPD matrix in buf0 (m x m); returns the buffer holding A^-1.
double *launch_dense_inverse(double *buf0, double *buf1, int m, int *status,
                             cudaStream_t st) {
  const size_t n = (size_t)m * m;
  const int threads = 256;
  const int blocks = (int)((n + threads - 1) / threads);
  double *a = buf0, *b = buf1;
  for (int k = 0; k < m; ++k) {
    k_gj_sweep<<<blocks, threads, 0, st>>>(a, b, m, k, status);
    double *tmp = a; a = b; b = tmp;
  }
  return a;
}

}  // namespace spfd
