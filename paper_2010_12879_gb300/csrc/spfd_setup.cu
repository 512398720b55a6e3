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
// One warp per voxel row (j, k): the row's conductivities are read as
// 16-byte pairs and classified by their bit patterns with integer operations
// (on this GPU an FP64 comparison costs a slot of the narrow FP64 pipe):
// conducting iff the value is > 0 (sign clear, not zero, exponent not all
// ones); invalid iff NaN or infinite (exponent all ones) or negative and not
// -0.  mask gets 1 per conducting voxel.  The bricks of the conducting
// voxels' corner nodes are flagged once per warp step: the lanes OR the
// x-bricks they touch into one word, and one lane per touched x-brick stores
// its flags for the row's (at most 4) brick rows, so a flag byte is not
// written once per voxel.
__device__ __forceinline__ unsigned char classify_sigma(unsigned long long u, int &bad) {
  const unsigned ex = (unsigned)(u >> 52) & 0x7ffu;
  const bool neg = (u >> 63) != 0;
  if (ex == 0x7ffu || (neg && (u << 1) != 0)) bad = 1;
  return (!neg && u != 0 && ex != 0x7ffu) ? 1 : 0;
}

__global__ void __launch_bounds__(256)
k_sigma_flags(const double *__restrict__ sigma, int nx, int ny, int nz, int MX, int MY,
              bool pairs, unsigned char *__restrict__ flags, unsigned char *__restrict__ mask,
              int *status) {
  const int lane = threadIdx.x & 31;
  const long long nrows = (long long)ny * nz;
  int bad = 0;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const int j0 = j >> 3, j1 = (j + 1) >> 3, k0 = k >> 3, k1 = (k + 1) >> 3;
    const double *row = sigma + (size_t)r * nx;
    unsigned char *mrow = mask + (size_t)r * nx;
    // pairs when every row starts on a 16-byte boundary (nx even and sigma
    // 16-byte aligned), else one value at a time; a step covers 64 (32)
    // voxels, whose corner nodes lie in 9 (5) x-bricks from c0 / 8 on
    const int step = pairs ? 64 : 32;
    for (int c0 = 0; c0 < nx; c0 += step) {
      const int base = c0 >> 3;
      unsigned bits = 0;
      if (pairs) {
        const int i = c0 + 2 * lane;
        if (i < nx) {  // nx is even, so i + 1 < nx
          const double2 p = *reinterpret_cast<const double2 *>(row + i);
          const unsigned char m0 = classify_sigma((unsigned long long)__double_as_longlong(p.x), bad);
          const unsigned char m1 = classify_sigma((unsigned long long)__double_as_longlong(p.y), bad);
          *reinterpret_cast<uchar2 *>(mrow + i) = make_uchar2(m0, m1);
          if (m0) bits |= (1u << ((i >> 3) - base)) | (1u << (((i + 1) >> 3) - base));
          if (m1) bits |= (1u << (((i + 1) >> 3) - base)) | (1u << (((i + 2) >> 3) - base));
        }
      } else {
        const int i = c0 + lane;
        if (i < nx) {
          const unsigned char m0 =
              classify_sigma((unsigned long long)__double_as_longlong(row[i]), bad);
          mrow[i] = m0;
          if (m0) bits |= (1u << ((i >> 3) - base)) | (1u << (((i + 1) >> 3) - base));
        }
      }
      bits = __reduce_or_sync(0xffffffffu, bits);
      if (lane < 9 && ((bits >> lane) & 1u)) {
        const int bx = base + lane;
        flags[((size_t)k0 * MY + j0) * MX + bx] = 1;
        if (j1 != j0) flags[((size_t)k0 * MY + j1) * MX + bx] = 1;
        if (k1 != k0) flags[((size_t)k1 * MY + j0) * MX + bx] = 1;
        if (j1 != j0 && k1 != k0) flags[((size_t)k1 * MY + j1) * MX + bx] = 1;
      }
    }
  }
  if (bad) atomicOr(status, DEV_BAD_SIGMA);
}

void launch_sigma_flags(const double *sigma, int nx, int ny, int nz, int MX,
                        int MY, unsigned char *flags, unsigned char *mask,
                        int *status, cudaStream_t st) {
  const long long rows = (long long)ny * nz;
  long long blocks = (rows + 7) / 8;  // 8 warps (rows) per block
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  const bool pairs = (nx & 1) == 0 && ((uintptr_t)sigma & 15) == 0;
  k_sigma_flags<<<(int)blocks, 256, 0, st>>>(sigma, nx, ny, nz, MX, MY, pairs, flags, mask,
                                              status);
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

// One brick per block.  The 9^3 voxels around the brick's nodes go to shared
// memory once; the sums of voxel pairs along y (py) and along x (px) are
// formed once there, and each +edge conductance of the nodes -1 .. 7 (per
// axis) is the sum of two such pairs times h/4 (the -edge of a node is the
// +edge of the node before it): a node costs about 8 FP64 operations for its
// six conductances, against 24 when each sums its own four voxels, which
// matters on GB300's narrow FP64 pipe.  The four voxels of an edge are
// added as (s00 + s01) + (s10 + s11).
__global__ void __launch_bounds__(NT)
k_build_fine(Grid g, const double *__restrict__ sigma, int nx, int ny, int nz,
             double h, double *__restrict__ gx, double *__restrict__ diag,
             double *__restrict__ dinv) {
  __shared__ double sv[9][9][9];  // voxels 8B - 1 .. 8B + 7 per axis (0 outside)
  __shared__ double py[9][8][9];  // sv[z][y][x] + sv[z][y + 1][x]
  __shared__ double px[9][9][8];  // sv[z][y][x] + sv[z][y][x + 1]
  __shared__ double ex[8][8][9];  // +x edge of node (lx, ly, lz), lx = -1 .. 7 at [lz][ly][lx + 1]
  __shared__ double ey[8][9][8];  // +y edge, ly = -1 .. 7 at [lz][ly + 1][lx]
  __shared__ double ez[9][8][8];  // +z edge, lz = -1 .. 7 at [lz + 1][ly][lx]
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const int4 bc = g.bco[b];
  const int x0 = bc.x * 8 - 1, y0 = bc.y * 8 - 1, z0 = bc.z * 8 - 1;
  for (int q = t; q < 729; q += NT) {
    const int vz = q / 81, vy = (q / 9) % 9, vx = q % 9;
    sv[vz][vy][vx] = sig_at(sigma, x0 + vx, y0 + vy, z0 + vz, nx, ny, nz);
  }
  __syncthreads();
  for (int q = t; q < 648; q += NT) {
    {
      const int vz = q / 72, vy = (q / 9) % 8, vx = q % 9;
      py[vz][vy][vx] = sv[vz][vy][vx] + sv[vz][vy + 1][vx];
    }
    {
      const int vz = q / 72, vy = (q / 8) % 9, vx = q % 8;
      px[vz][vy][vx] = sv[vz][vy][vx] + sv[vz][vy][vx + 1];
    }
  }
  __syncthreads();
  const double hq = h * 0.25;
  for (int q = t; q < 576; q += NT) {
    {  // x: index (lz, ly, lx + 1), voxels (lz..lz+1, ly..ly+1, xp)
      const int lz = q / 72, ly = (q / 9) % 8, xp = q % 9;
      ex[lz][ly][xp] = hq * (py[lz][ly][xp] + py[lz + 1][ly][xp]);
    }
    {  // y: index (lz, ly + 1, lx), voxels (lz..lz+1, yp, lx..lx+1)
      const int lz = q / 72, yp = (q / 8) % 9, lx = q % 8;
      ey[lz][yp][lx] = hq * (px[lz][yp][lx] + px[lz + 1][yp][lx]);
    }
    {  // z: index (lz + 1, ly, lx), voxels (zp, ly..ly+1, lx..lx+1)
      const int zp = q / 64, ly = (q / 8) % 8, lx = q % 8;
      ez[zp][ly][lx] = hq * (py[zp][ly][lx] + py[zp][ly][lx + 1]);
    }
  }
  __syncthreads();
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  const int i = bc.x * 8 + lx, j = bc.y * 8 + ly, k = bc.z * 8 + lz;
  const size_t s = (size_t)b * BV + t;
  double e[6] = {0, 0, 0, 0, 0, 0};
  if (i < g.NX && j < g.NY && k < g.NZ) {
    e[0] = ex[lz][ly][lx + 1];  // +x
    e[1] = ey[lz][ly + 1][lx];  // +y
    e[2] = ez[lz + 1][ly][lx];  // +z
    e[3] = ex[lz][ly][lx];      // -x
    e[4] = ey[lz][ly][lx];      // -y
    e[5] = ez[lz][ly][lx];      // -z
  }
  const double d = ((e[3] + e[0]) + (e[4] + e[1])) + (e[5] + e[2]);
  gx[s] = e[0];
  gx[S + s] = e[1];
  gx[2 * S + s] = e[2];
  diag[s] = d;
  // d is +0, -0 or positive: a bit test replaces the FP64 comparison
  dinv[s] = f64_nonzero(d) ? 1.0 / d : 0.0;
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

// Brick-local pass: the block links the edges inside its brick with the
// same lock-free union-find on a shared-memory forest, then writes each
// unknown's local root (the smallest slot of its local component) as its
// global parent.  A node is an unknown iff an incident edge conducts (its
// own +edges or the -edges that are its neighbours' +edges).
__device__ int uf_find_sh(int *p, int x, int *capped) {
  volatile int *q = p;
  for (int it = 0; it < UF_FIND_CAP; ++it) {
    const int px = q[x];
    if (px == x) return x;
    const int gp = q[px];
    if (gp != px) q[x] = gp;
    x = gp;
  }
  *capped = 1;
  return x;
}

__device__ void uf_unite_sh(int *p, int a, int b, int *capped) {
  for (int it = 0; it < UF_UNITE_CAP; ++it) {
    a = uf_find_sh(p, a, capped);
    b = uf_find_sh(p, b, capped);
    if (a == b || *capped) return;
    if (a < b) { const int t = a; a = b; b = t; }
    if (atomicCAS(&p[a], a, b) == a) return;
  }
  *capped = 1;
}

__global__ void __launch_bounds__(NT)
k_uf_local(Grid g, const double *__restrict__ gx, int *parent, int *status) {
  __shared__ int lp[BV];
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const size_t s = (size_t)b * BV + t;
  const int4 bc = g.bco[b];
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  const bool ex = f64_nonzero(gx[s]), ey = f64_nonzero(gx[S + s]),
             ez = f64_nonzero(gx[2 * S + s]);
  bool act = ex || ey || ez;
  if (!act) {
    const int m = slot_nb(g, b, bc, lx, ly, lz, -1, 0, 0);
    act = m >= 0 && f64_nonzero(gx[m]);
  }
  if (!act) {
    const int m = slot_nb(g, b, bc, lx, ly, lz, 0, -1, 0);
    act = m >= 0 && f64_nonzero(gx[S + m]);
  }
  if (!act) {
    const int m = slot_nb(g, b, bc, lx, ly, lz, 0, 0, -1);
    act = m >= 0 && f64_nonzero(gx[2 * S + m]);
  }
  lp[t] = act ? t : -1;
  __syncthreads();
  int capped = 0;
  if (ex && lx < 7) uf_unite_sh(lp, t, t + 1, &capped);
  if (ey && ly < 7) uf_unite_sh(lp, t, t + 8, &capped);
  if (ez && lz < 7) uf_unite_sh(lp, t, t + 64, &capped);
  __syncthreads();
  int r = -1;
  if (act) r = uf_find_sh(lp, t, &capped);
  parent[s] = act ? b * BV + r : -1;
  if (capped) atomicOr(status, DEV_UF_CAP);
}

// Links across the brick's +x/+y/+z faces (the edges the local pass left).
__global__ void __launch_bounds__(NT)
k_uf_union(Grid g, const double *__restrict__ gx, int *parent, int *status) {
  const size_t S = (size_t)g.nb * BV;
  const int b = blockIdx.x, t = threadIdx.x;
  const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
  if (lx != 7 && ly != 7 && lz != 7) return;
  const int s = b * BV + t;
  const int4 bc = g.bco[b];
  int capped = 0;
  if (lx == 7 && f64_nonzero(gx[s])) {
    const int m = slot_nb(g, b, bc, lx, ly, lz, 1, 0, 0);
    if (m >= 0) uf_unite(parent, s, m, &capped);
  }
  if (ly == 7 && f64_nonzero(gx[S + s])) {
    const int m = slot_nb(g, b, bc, lx, ly, lz, 0, 1, 0);
    if (m >= 0) uf_unite(parent, s, m, &capped);
  }
  if (lz == 7 && f64_nonzero(gx[2 * S + s])) {
    const int m = slot_nb(g, b, bc, lx, ly, lz, 0, 0, 1);
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
  k_uf_local<<<g.nb, NT, 0, st>>>(g, gx, parent, status);
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
  __shared__ int c0;
  const int s = blockIdx.x * BV + threadIdx.x;
  const int c = comp[s];
  // a brick inside one component (the common case) adds its count once
  if (threadIdx.x == 0) c0 = -1;
  __syncthreads();
  if (c >= 0) atomicMax(&c0, c);
  __syncthreads();
  const int n = __syncthreads_count(c >= 0);
  if (__syncthreads_and(c < 0 || c == c0)) {
    if (threadIdx.x == 0 && n > 0) atomicAdd(&sizes[c0], n);
    return;
  }
  // otherwise group the lanes holding the same component; the lowest lane adds
  const unsigned grp = __match_any_sync(0xffffffffu, c);
  if (c >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1)
    atomicAdd(&sizes[c], __popc(grp));
}

void launch_comp_sizes(const Grid &g, const int *comp, int *sizes,
                       cudaStream_t st) {
  if (g.nb == 0) return;
  k_comp_sizes<<<g.nb, NT, 0, st>>>(comp, sizes);
}

// Diagonal, its inverse, and the level's largest diagonal (for a relative
// activity threshold).  Rows below 1e-13 * max diagonal are treated as not
// being unknowns (dinv = 0): they arise only from basis functions that are
// constant on a whole tiny component and carry no information.
__global__ void __launch_bounds__(NT)
k_coarse_diag(const double *__restrict__ stc, size_t S, const unsigned long long *maxbits,
              double rel, double *__restrict__ diag, double *__restrict__ dinv) {
  const size_t s = (size_t)blockIdx.x * BV + threadIdx.x;
  const double thresh = rel * __longlong_as_double((long long)*maxbits);
  const double d = stc[13 * S + s];
  const bool act = d > thresh;
  diag[s] = act ? d : 0.0;
  dinv[s] = act ? 1.0 / d : 0.0;
}

void launch_coarse_diag(const Grid &gc, const double *stc, const unsigned long long *maxbits,
                        double rel, double *diag, double *dinv, cudaStream_t st) {
  if (gc.nb == 0) return;
  k_coarse_diag<<<gc.nb, NT, 0, st>>>(stc, (size_t)gc.nb * BV, maxbits, rel, diag, dinv);
}

__global__ void __launch_bounds__(NT)
k_diag_stats(const double *__restrict__ d, size_t n, unsigned long long *ustat) {
  __shared__ unsigned long long sc_[NT / 32], sm_[NT / 32];
  unsigned long long cnt = 0;
  double mx = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double v = d[i];
    if (v > 0.0) { ++cnt; mx = fmax(mx, v); }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sc_[w] = cnt;
    sm_[w] = (unsigned long long)__double_as_longlong(mx);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long c = 0, m = 0;
    for (int q = 0; q < NT / 32; ++q) { c += sc_[q]; m = sm_[q] > m ? sm_[q] : m; }
    atomicAdd(&ustat[0], c);
    atomicMax(&ustat[1], m);
  }
}

void launch_diag_stats(const double *d, size_t n, unsigned long long *ustat,
                       cudaStream_t st) {
  size_t blocks = (n + NT - 1) / NT;
  if (blocks > 608) blocks = 608;
  if (blocks == 0) return;
  k_diag_stats<<<(int)blocks, NT, 0, st>>>(d, n, ustat);
}

// ------------------------------------------------ coarsest dense matrix
// The dense matrix of the coarsest level's m unknowns (slots idx[a], row of
// slot u rowof[u] or -1), into A (zeroed beforehand), entry by entry as the
// operator stores it: 27-point levels A[a][rowof[u]] = 0 + st[e][idx[a]] for
// the neighbour u at offset e; the 7-point level (a single-level hierarchy)
// A[a][a] = diag and A[a][rowof[u]] = 0 - g for the six edges.
template <bool K27>
__global__ void k_coarse_scatter(Grid g, const double *__restrict__ op, size_t S,
                                 const double *__restrict__ diag, const int *__restrict__ idx,
                                 const int *__restrict__ rowof, int m, double *__restrict__ A) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 27LL * m) return;
  const int a = (int)(q / 27), e = (int)(q % 27);
  const int s = idx[a], b = s / BV, t = s % BV;
  const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
  if (!K27 && e == 13) {
    A[(size_t)a * m + a] = diag[s];
    return;
  }
  if (!K27 && (dx != 0) + (dy != 0) + (dz != 0) != 1) return;
  const int4 bc = g.bco[b];
  const int u = e == 13 ? s : slot_nb(g, b, bc, t & 7, (t >> 3) & 7, t >> 6, dx, dy, dz);
  if (u < 0) return;
  const int col = rowof[u];
  if (col < 0) return;
  if (K27) {
    A[(size_t)a * m + col] = 0.0 + op[(size_t)e * S + s];
  } else {
    const int ax = dx ? 0 : (dy ? 1 : 2);
    const double ge = dx + dy + dz > 0 ? op[(size_t)ax * S + s] : op[(size_t)ax * S + u];
    A[(size_t)a * m + col] = 0.0 - ge;
  }
}

// A[a][b] += mu[cc[a]] when a and b lie in one component of the coarsest
// graph, then A[a][a] += shift.
__global__ void k_coarse_regularise(double *__restrict__ A, int m, const int *__restrict__ cc,
                                    const double *__restrict__ mu, double shift) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)m * m) return;
  const int a = (int)(q / m), b = (int)(q % m);
  double v = A[q];
  if (cc[a] == cc[b]) v += mu[cc[a]];
  if (a == b) v += shift;
  A[q] = v;
}

void launch_coarse_dense(const Grid &g, const double *op, bool k27, size_t S, const double *diag,
                         const int *idx, const int *rowof, int m, const int *cc,
                         const double *mu, double shift, double *A, cudaStream_t st) {
  if (m <= 0) return;
  const unsigned nb1 = (unsigned)((27LL * m + 255) / 256);
  if (k27) k_coarse_scatter<true><<<nb1, 256, 0, st>>>(g, op, S, diag, idx, rowof, m, A);
  else k_coarse_scatter<false><<<nb1, 256, 0, st>>>(g, op, S, diag, idx, rowof, m, A);
  if (cc)
    k_coarse_regularise<<<(unsigned)(((long long)m * m + 255) / 256), 256, 0, st>>>(A, m, cc, mu,
                                                                                    shift);
}

// ------------------------------------------------ coarsest dense inverse
// Blocked Gauss-Jordan inversion of an SPD matrix (m x m, row-major).  A
// sweep takes the pivot set K = k0 .. k0+r-1 (r <= GJ_B) at once, reading
// the current matrix M and writing B (a principal pivot transform):
//   B[K,K] = D^-1,  B[K,j] = D^-1 M[K,j],  B[i,K] = -M[i,K] D^-1,
//   B[i,j] = M[i,j] - M[i,K] D^-1 M[K,j]   (i, j not in K),  D = M[K,K].
// After every pivot set has been swept once, B = A^-1.  D is inverted by
// scalar Gauss-Jordan in shared memory: its pivots are Schur complements of
// the SPD matrix, hence positive; a non-positive one raises DEV_BAD_PIVOT.
// Every block inverts D itself, forms W = D^-1 M[K, its columns] and
// updates its GJ_T x GJ_T tile; sweeps run one launch each (k_gj_block) or
// all in one cooperative launch with a grid barrier between them (k_gj_all).
// (Forming D^-1 and W once per column tile in a first phase of each sweep
// halves the FP64 work, but its second grid barrier per sweep made the
// inversion of the 2 mm body's 481 x 481 coarsest matrix slower: the sweeps
// are bound by latency, not by the FP64 pipe.)
constexpr int GJ_B = 16;   // pivots per sweep
constexpr int GJ_T = 32;   // tile edge
constexpr int GJ_NT = 256; // threads per block (GJ_B * GJ_B)

struct GjShared {
  double D[2][GJ_B][GJ_B + 1];
  double W[GJ_B][GJ_T];
  double U[GJ_T][GJ_B + 1];
  double C[GJ_B][GJ_T];
  double pinv[2];
};

// COH: read through L2 only (ld.global.cg), as the single-launch form must:
// what it reads was written by other blocks in the same launch, and a line
// cached in this SM's L1 by an earlier sweep would be stale.
template <bool COH>
__device__ __forceinline__ double gj_ld(const double *p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// D = M[K,K] (identity-padded to GJ_B) into sh.D[0] and its first pivot's
// reciprocal, and C = M[K, column tile j0] into sh.C.  A barrier follows.
template <bool COH>
__device__ __forceinline__ void gj_load_pivot_rows(GjShared &sh, const double *__restrict__ A,
                                                   int m, int k0, int r, int j0, int *status) {
  const int t = threadIdx.x;
  const int a = t / GJ_B, b = t % GJ_B;
  const double d0 =
      (a < r && b < r) ? gj_ld<COH>(&A[(size_t)(k0 + a) * m + k0 + b]) : (a == b ? 1.0 : 0.0);
  sh.D[0][a][b] = d0;
  if (t == 0) {
    if (!(d0 > 0.0)) atomicOr(status, DEV_BAD_PIVOT);
    sh.pinv[0] = d0 > 0.0 ? 1.0 / d0 : 0.0;
  }
  for (int q = t; q < GJ_T * GJ_B; q += GJ_NT) {
    const int l2 = q / GJ_T, jj = q % GJ_T;
    sh.C[l2][jj] =
        (l2 < r && j0 + jj < m) ? gj_ld<COH>(&A[(size_t)(k0 + l2) * m + j0 + jj]) : 0.0;
  }
}

// U = M[tile rows i0, K] into sh.U.  A barrier follows.
template <bool COH>
__device__ __forceinline__ void gj_load_pivot_cols(GjShared &sh, const double *__restrict__ A,
                                                   int m, int k0, int r, int i0) {
  for (int q = threadIdx.x; q < GJ_T * GJ_B; q += GJ_NT) {
    const int ii = q / GJ_B, l = q % GJ_B;
    sh.U[ii][l] = (l < r && i0 + ii < m) ? gj_ld<COH>(&A[(size_t)(i0 + ii) * m + k0 + l]) : 0.0;
  }
}

// D <- D^-1 in shared memory (after a barrier), one pivot per step,
// ping-pong between D[0] and D[1]: the thread that forms the next pivot also
// writes its reciprocal, so a step needs a single barrier.  The inverse ends
// in D[GJ_B & 1] = D[0]; W = D^-1 C then follows (each thread forms the
// entries (l, jj) and (l + 8, jj), its two sums interleaved, each in its own
// fixed order), and a barrier.
__device__ __forceinline__ void gj_invert_pivots(GjShared &sh, int *status) {
  auto &D = sh.D;
  auto &pinv = sh.pinv;
  const int t = threadIdx.x;
  const int a = t / GJ_B, b = t % GJ_B;
  for (int p = 0; p < GJ_B; ++p) {
    const double(*Dc)[GJ_B + 1] = D[p & 1];
    const double iv = pinv[p & 1];
    double v;
    if (a == p && b == p) v = iv;
    else if (a == p) v = Dc[p][b] * iv;
    else if (b == p) v = -Dc[a][p] * iv;
    else v = Dc[a][b] - Dc[a][p] * Dc[p][b] * iv;
    D[(p + 1) & 1][a][b] = v;
    if (a == p + 1 && b == p + 1) {
      if (!(v > 0.0)) atomicOr(status, DEV_BAD_PIVOT);
      pinv[(p + 1) & 1] = v > 0.0 ? 1.0 / v : 0.0;
    }
    __syncthreads();
  }
  const double(*Dinv)[GJ_B + 1] = D[GJ_B & 1];
  static_assert(GJ_B * GJ_T == 2 * GJ_NT && GJ_T * GJ_T == 4 * GJ_NT, "tile shape");
  {
    const int l = t / GJ_T, jj = t % GJ_T;
    double w0 = 0.0, w1 = 0.0;
#pragma unroll
    for (int l2 = 0; l2 < GJ_B; ++l2) {
      const double c = sh.C[l2][jj];
      w0 += Dinv[l][l2] * c;
      w1 += Dinv[l + GJ_NT / GJ_T][l2] * c;
    }
    sh.W[l][jj] = w0;
    sh.W[l + GJ_NT / GJ_T][jj] = w1;
  }
  __syncthreads();
}

// The tile (i0, j0) of B from M (A), with D^-1 in sh.D[0], W for the
// tile's columns in sh.W and U in sh.U: each thread updates rows ii0 + 8k
// (k = 0..3) of column jj, four independent chains, each subtracting its
// terms in order l = 0..15.
template <bool COH>
__device__ __forceinline__ void gj_update_tile(const GjShared &sh, const double *__restrict__ A,
                                               double *__restrict__ B, int m, int k0, int r,
                                               int i0, int j0) {
  const double(*Dinv)[GJ_B + 1] = sh.D[GJ_B & 1];
  constexpr int RS = GJ_NT / GJ_T;  // row stride between a thread's entries
  const int t = threadIdx.x;
  const int ii0 = t / GJ_T, jj = t % GJ_T, j = j0 + jj;
  const bool kj = j >= k0 && j < k0 + r;
  double v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + ii0 + RS * k;
    v[k] = (!kj && i < m && j < m) ? gj_ld<COH>(&A[(size_t)i * m + j]) : 0.0;
  }
#pragma unroll
  for (int l = 0; l < GJ_B; ++l) {
    const double mc = kj ? Dinv[l][j - k0] : sh.W[l][jj];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] -= sh.U[ii0 + RS * k][l] * mc;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int ii = ii0 + RS * k, i = i0 + ii;
    if (i >= m || j >= m) continue;
    const bool ki = i >= k0 && i < k0 + r;
    double out = v[k];
    if (ki) out = kj ? Dinv[i - k0][j - k0] : sh.W[i - k0][jj];
    B[(size_t)i * m + j] = out;
  }
}

// One sweep per launch: every block forms D^-1 and its W itself.
__global__ void __launch_bounds__(GJ_NT)
k_gj_block(const double *__restrict__ A, double *__restrict__ B, int m, int k0, int r,
           int *status) {
  __shared__ GjShared sh;
  const int i0 = blockIdx.y * GJ_T, j0 = blockIdx.x * GJ_T;
  gj_load_pivot_rows<false>(sh, A, m, k0, r, j0, status);
  gj_load_pivot_cols<false>(sh, A, m, k0, r, i0);
  __syncthreads();
  gj_invert_pivots(sh, status);
  gj_update_tile<false>(sh, A, B, m, k0, r, i0, j0);
}

// Every sweep in one cooperative launch: the same tiles and arithmetic as
// the per-sweep launches, with a grid barrier between sweeps (sweep k reads
// what sweep k-1 wrote).  bar[0..1]: barrier counter and generation, zero
// at launch.
__global__ void __launch_bounds__(GJ_NT)
k_gj_all(double *buf0, double *buf1, int m, int *status, unsigned *bar) {
  __shared__ GjShared sh;
  const unsigned nblocks = gridDim.x * gridDim.y;
  const int i0 = blockIdx.y * GJ_T, j0 = blockIdx.x * GJ_T;
  double *a = buf0, *b = buf1;
  for (int k0 = 0; k0 < m; k0 += GJ_B) {
    const int r = m - k0 < GJ_B ? m - k0 : GJ_B;
    gj_load_pivot_rows<true>(sh, a, m, k0, r, j0, status);
    gj_load_pivot_cols<true>(sh, a, m, k0, r, i0);
    __syncthreads();
    gj_invert_pivots(sh, status);
    gj_update_tile<true>(sh, a, b, m, k0, r, i0, j0);
    grid_barrier(&bar[0], &bar[1], nblocks, status);
    double *tmp = a; a = b; b = tmp;
  }
}

// Kernel launches of launch_dense_inverse for an m x m matrix: one when its
// tile grid fits on the device at once (a cooperative launch), else one per
// pivot set.
int dense_inverse_launches(int m) {
  const int nt = (m + GJ_T - 1) / GJ_T;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_all, GJ_NT, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    return (m + GJ_B - 1) / GJ_B;
  }
  return (coop && (long long)nt * nt <= (long long)per_sm * nsm) ? 1 : (m + GJ_B - 1) / GJ_B;
}

// Inverts the SPD matrix in buf0 (m x m); returns the buffer holding A^-1
// (buf0 or buf1, which serve as ping-pong buffers).  bar: two zeroed
// unsigned ints of device scratch for the cooperative form.
double *launch_dense_inverse(double *buf0, double *buf1, int m, int *status, unsigned *bar,
                             cudaStream_t st) {
  double *a = buf0, *b = buf1;
  const int nt = (m + GJ_T - 1) / GJ_T;
  if (dense_inverse_launches(m) == 1) {
    void *args[] = {&buf0, &buf1, &m, &status, &bar};
    if (cudaLaunchCooperativeKernel((const void *)k_gj_all, dim3(nt, nt), dim3(GJ_NT), args, 0,
                                    st) == cudaSuccess)
      return ((m + GJ_B - 1) / GJ_B) % 2 ? buf1 : buf0;
    cudaGetLastError();  // not launched: sweep launch by launch instead
  }
  for (int k0 = 0; k0 < m; k0 += GJ_B) {
    k_gj_block<<<dim3(nt, nt), GJ_NT, 0, st>>>(a, b, m, k0, m - k0 < GJ_B ? m - k0 : GJ_B,
                                              status);
    double *tmp = a; a = b; b = tmp;
  }
  return a;
}

// ------------------------------------------------------------ brick tables
// The neighbour, child and parent tables of the levels, from their brick maps
// and brick coordinates: data-parallel lookups, one thread per entry.
__global__ void k_brick_nbr(Grid g, int *__restrict__ nbr) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)g.nb * 27) return;
  const int b = (int)(q / 27), e = (int)(q % 27);
  const int4 bc = g.bco[b];
  const int x = bc.x + e % 3 - 1, y = bc.y + (e / 3) % 3 - 1, z = bc.z + e / 9 - 1;
  int v = -1;
  if (x >= 0 && y >= 0 && z >= 0 && x < g.MX && y < g.MY && z < g.MZ)
    v = g.bmap[((size_t)z * g.MY + y) * g.MX + x];
  nbr[q] = v;
}

// kid[B][o]: the fine brick 2B + o - 1 (o in {0,1,2}^3) of coarse brick B.
__global__ void k_brick_kid(Grid gf, Grid gc, int *__restrict__ kid) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)gc.nb * 27) return;
  const int b = (int)(q / 27), o = (int)(q % 27);
  const int4 bc = gc.bco[b];
  const int x = 2 * bc.x + o % 3 - 1, y = 2 * bc.y + (o / 3) % 3 - 1, z = 2 * bc.z + o / 9 - 1;
  int v = -1;
  if (x >= 0 && y >= 0 && z >= 0 && x < gf.MX && y < gf.MY && z < gf.MZ)
    v = gf.bmap[((size_t)z * gf.MY + y) * gf.MX + x];
  kid[q] = v;
}

// par[b][o]: the coarse brick (b >> 1) + o (o in {0,1}^3) of fine brick b.
__global__ void k_brick_par(Grid gf, Grid gc, int *__restrict__ par) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)gf.nb * 8) return;
  const int b = (int)(q / 8), o = (int)(q % 8);
  const int4 bc = gf.bco[b];
  const int x = (bc.x >> 1) + (o & 1), y = (bc.y >> 1) + ((o >> 1) & 1), z = (bc.z >> 1) + (o >> 2);
  int v = -1;
  if (x < gc.MX && y < gc.MY && z < gc.MZ) v = gc.bmap[((size_t)z * gc.MY + y) * gc.MX + x];
  par[q] = v;
}

static inline unsigned table_blocks(long long n) { return (unsigned)((n + 255) / 256); }

void launch_brick_nbr(const Grid &g, int *nbr, cudaStream_t st) {
  if (g.nb) k_brick_nbr<<<table_blocks((long long)g.nb * 27), 256, 0, st>>>(g, nbr);
}
void launch_brick_kid(const Grid &gf, const Grid &gc, int *kid, cudaStream_t st) {
  if (gc.nb) k_brick_kid<<<table_blocks((long long)gc.nb * 27), 256, 0, st>>>(gf, gc, kid);
}
void launch_brick_par(const Grid &gf, const Grid &gc, int *par, cudaStream_t st) {
  if (gf.nb) k_brick_par<<<table_blocks((long long)gf.nb * 8), 256, 0, st>>>(gf, gc, par);
}

// ------------------------------------------------------------ uploads
// dst = src for n16 16-byte words, src in pinned host memory read by the SMs
// over the chip-to-chip link (both 16-byte aligned), then the tail bytes.
__global__ void k_pull(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16,
                       const unsigned char *__restrict__ tsrc, unsigned char *__restrict__ tdst,
                       int ntail) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if (blockIdx.x == 0 && (int)threadIdx.x < ntail) tdst[threadIdx.x] = tsrc[threadIdx.x];
}

void launch_pull(void *dst, const void *src_mapped, size_t bytes, cudaStream_t st) {
  const size_t n16 = bytes / 16;
  const int ntail = (int)(bytes % 16);
  size_t blocks = (n16 + 255) / 256;
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (blocks == 0) blocks = 1;
  k_pull<<<(unsigned)blocks, 256, 0, st>>>(
      (const uint4 *)src_mapped, (uint4 *)dst, n16,
      (const unsigned char *)src_mapped + n16 * 16, (unsigned char *)dst + n16 * 16, ntail);
}

__global__ void k_set_f64(double *p, double v) { *p = v; }
void launch_set_f64(double *p, double v, cudaStream_t st) { k_set_f64<<<1, 1, 0, st>>>(p, v); }

}  // namespace spfd
