// spfd_tree_cotree: step 3 of the pipeline (Sec. II-A), the edge vector
// potentials a from the facet fluxes b of Eq. 2 (b = C a) by tree-cotree
// gauging.
//
// C has a null space (every discrete gradient), so b fixes a only up to a
// gradient.  Tree-cotree gauging removes it by setting a = 0 on the edges of
// a spanning tree of the node grid; the potentials of the remaining (cotree)
// edges then follow from b uniquely.  The tree used here is the comb on the
// root line (j, k) = (j0, k0):
//   every z edge,
//   the y edges of the plane k = k0,
//   the x edges of the line (j, k) = (j0, k0).
// With a_z = 0 the facet equations decouple into prefix sums:
//   facets z of the plane k0:  a_x(i, j+1, k0) = a_x(i, j, k0) - b_z(i, j, k0),
//                              a_x(i, j0, k0) = 0 (the root line);
//   facets y, along z:         a_x(i, j, k+1) = a_x(i, j, k) + b_y(i, j, k);
//   facets x, along z:         a_y(i, j, k+1) = a_y(i, j, k) - b_x(i, j, k),
//                              a_y(i, j, k0) = 0 (the tree plane);
// each run outward from the root (downward chains subtract the same terms).
// The facets z off the plane k0 are the redundant equations: they hold
// exactly when b is divergence-free (the net flux of every cell vanishes).
//
// One thread walks one node column (i, j) for one component (blockIdx.y:
// 0 = a_x from b_y, 1 = a_y from b_x and the zero a_z), loading U facet
// fluxes ahead of the dependent sums.  A warp covers 32 consecutive columns,
// so every load and store is a coalesced 256-byte row segment of one z plane.
// Per node the kernel reads 16 bytes (b_x, b_y) and writes 24 (a), plus the
// plane's b_z from L2.
#include "spfd_ctx.cuh"

namespace spfd {
namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_UNROLL = 8;

template <int COMP>
__device__ __forceinline__ void tc_column(const double *__restrict__ b, int nx, int ny,
                                          int nz, int j0, int k0, size_t col,
                                          int i, int j, double *__restrict__ a) {
  const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1);
  const size_t NN = NXY * ((size_t)nz + 1);
  double *__restrict__ out = a + (size_t)COMP * NN + col;
  // a_y also writes the zero a_z of its column (tree edges and the slots
  // past the last node)
  double *__restrict__ az = a + 2 * NN + col;
  const bool valid = COMP == 0 ? i < nx : j < ny;
  if (!valid) {  // slots past the last node along the edge's axis
    for (int k = 0; k <= nz; ++k) {
      out[(size_t)k * NXY] = 0.0;
      if (COMP == 1) az[(size_t)k * NXY] = 0.0;
    }
    return;
  }
  // a at (i, j, k0)
  double s0 = 0.0;
  if (COMP == 0) {
    const double *__restrict__ bz = b + 2 * NN + (size_t)k0 * NXY + i;
    if (j > j0)
      for (int jj = j0; jj < j; ++jj) s0 -= bz[(size_t)jj * NX];
    else
      for (int jj = j0 - 1; jj >= j; --jj) s0 += bz[(size_t)jj * NX];
  }
  // facet fluxes along the column: b_y for a_x, b_x for a_y
  const double *__restrict__ src = b + (COMP == 0 ? NN : 0) + col;
  out[(size_t)k0 * NXY] = s0;
  if (COMP == 1) az[(size_t)k0 * NXY] = 0.0;
  // upward: k0 -> nz
  double s = s0;
  for (int k = k0; k < nz; k += TC_UNROLL) {
    double v[TC_UNROLL];
#pragma unroll
    for (int u = 0; u < TC_UNROLL; ++u)
      v[u] = k + u < nz ? __ldcs(src + (size_t)(k + u) * NXY) : 0.0;
#pragma unroll
    for (int u = 0; u < TC_UNROLL; ++u) {
      if (k + u < nz) {
        s = COMP == 0 ? s + v[u] : s - v[u];
        const size_t o = (size_t)(k + u + 1) * NXY;
        __stcs(out + o, s);
        if (COMP == 1) __stcs(az + o, 0.0);
      }
    }
  }
  // downward: k0 -> 0
  s = s0;
  for (int k = k0 - 1; k >= 0; k -= TC_UNROLL) {
    double v[TC_UNROLL];
#pragma unroll
    for (int u = 0; u < TC_UNROLL; ++u)
      v[u] = k - u >= 0 ? __ldcs(src + (size_t)(k - u) * NXY) : 0.0;
#pragma unroll
    for (int u = 0; u < TC_UNROLL; ++u) {
      if (k - u >= 0) {
        s = COMP == 0 ? s - v[u] : s + v[u];
        const size_t o = (size_t)(k - u) * NXY;
        __stcs(out + o, s);
        if (COMP == 1) __stcs(az + o, 0.0);
      }
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS)
k_tree_cotree(const double *__restrict__ b, int nx, int ny, int nz, int j0, int k0,
              double *__restrict__ a) {
  const size_t NX = (size_t)nx + 1, NXY = NX * ((size_t)ny + 1);
  const size_t col = (size_t)blockIdx.x * TC_THREADS + threadIdx.x;
  if (col >= NXY) return;
  const int i = (int)(col % NX), j = (int)(col / NX);
  if (blockIdx.y == 0)
    tc_column<0>(b, nx, ny, nz, j0, k0, col, i, j, a);
  else
    tc_column<1>(b, nx, ny, nz, j0, k0, col, i, j, a);
}

}  // namespace
}  // namespace spfd

using namespace spfd;

extern "C" spfd_status spfd_tree_cotree(const double *b_dev, int nx, int ny, int nz, int j0,
                                        int k0, void *stream, double *a_dev) {
  if (!b_dev || !a_dev) return fail(SPFD_EINVAL, "null array");
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(SPFD_EINVAL, "voxel counts must be >= 1 (got %d %d %d)", nx, ny, nz);
  if (j0 < 0 || j0 > ny || k0 < 0 || k0 > nz)
    return fail(SPFD_EINVAL, "root line (j, k) = (%d, %d) outside the node grid", j0, k0);
  const size_t NXY = ((size_t)nx + 1) * ((size_t)ny + 1);
  const size_t NN = NXY * ((size_t)nz + 1);
  const char *bb = (const char *)b_dev, *ab = (const char *)a_dev;
  const size_t bytes = 3 * NN * sizeof(double);
  if (bb < ab + bytes && ab < bb + bytes)
    return fail(SPFD_EINVAL, "b and a overlap");
  const size_t blocks = (NXY + TC_THREADS - 1) / TC_THREADS;
  if (blocks > 0x7fffffffu) return fail(SPFD_EINVAL, "grid too large");
  cudaStream_t st = (cudaStream_t)stream;
  k_tree_cotree<<<dim3((unsigned)blocks, 2), TC_THREADS, 0, st>>>(b_dev, nx, ny, nz, j0, k0,
                                                                  a_dev);
  CU(cudaGetLastError());
  return SPFD_OK;
}
