// spfd_residual_noalloc: the relative residual of a potential, without a
// context and without allocating device memory.
//
// Some callers cannot allocate device memory when they want to check a
// solution: processes whose device memory is reserved up front by another
// allocator (a framework's caching allocator, a fixed arena), real-time loops
// that must not enter the allocator, or code that must not trigger the
// implicit synchronisation of cudaMalloc / cudaFree.  This entry point serves
// them: the caller passes the conductivities, edge potentials and node
// potentials it already holds, and the reduction's partial sums live in one
// file-scope device array of fixed size instead of in memory obtained from
// cudaMalloc.  The call reads its result back into host memory and
// synchronises the stream it is given, so that stream must not be capturing
// into a CUDA graph.
//
// The computation is a fused, brick-free variant of the true-residual kernel
// of the solver: for every node the six edge conductances are rebuilt from the
// voxel conductivities, then b_n = sum_{e leaving n} g_e a_e - sum_{e entering
// n} g_e a_e and (A psi)_n = sum_e g_e (psi_n - psi_other) are formed and
// |b - A psi|^2 and |b|^2 are accumulated over the nodes that carry an
// unknown.  b is not projected onto the range of A; its per-component sum is
// zero up to rounding, so the result agrees with the solver's report to
// rounding.
#include <mutex>

#include "spfd_ctx.cuh"

namespace spfd {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_NODES_PER_THREAD = 32;
constexpr long long NA_NODES_PER_BLOCK = (long long)NA_THREADS * NA_NODES_PER_THREAD;
constexpr int NA_MAX_BLOCKS = 16384;
// largest node grid the fixed scratch can serve: 16384 * 8192 = 134,217,728
constexpr long long NA_MAX_NODES = NA_MAX_BLOCKS * NA_NODES_PER_BLOCK;
constexpr int NA_MAX_DEVICES = 64;

struct NoallocScratch {
  double partial[NA_MAX_BLOCKS][2];  // per block: |b - A psi|^2, |b|^2
  unsigned int ticket;               // last-block counter; cleared before each launch
  double result[2];                  // grid totals written by the last block
};

// 256 KB per device that loads the library, held until the process exits.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

NoallocScratch *g_scratch_ptr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

__device__ __forceinline__ double na_sig(const double *__restrict__ s, long long i,
                                         long long j, long long k, int nx, int ny,
                                         int nz) {
  if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0.0;
  return s[(k * ny + j) * nx + i];
}

__global__ void __launch_bounds__(NA_THREADS)
k_residual_noalloc(const double *__restrict__ sigma, const double *__restrict__ a,
                   const double *__restrict__ psi, int nx, int ny, int nz,
                   double h, NoallocScratch *scr) {
  const long long NX = nx + 1, NY = ny + 1, NZ = nz + 1;
  const long long NN = NX * NY * NZ;
  const double hq = 0.25 * h;
  double rr = 0.0, bb = 0.0;
  const long long base = (long long)blockIdx.x * NA_NODES_PER_BLOCK;
  for (int q = 0; q < NA_NODES_PER_THREAD; ++q) {
    const long long n = base + (long long)q * NA_THREADS + threadIdx.x;
    if (n >= NN) break;
    const long long i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
    // conductances of the six edges at n (x+, x-, y+, y-, z+, z-)
    double g[6];
    g[0] = i < nx ? hq * (na_sig(sigma, i, j - 1, k - 1, nx, ny, nz) + na_sig(sigma, i, j, k - 1, nx, ny, nz) +
                          na_sig(sigma, i, j - 1, k, nx, ny, nz) + na_sig(sigma, i, j, k, nx, ny, nz)) : 0.0;
    g[1] = i > 0 ? hq * (na_sig(sigma, i - 1, j - 1, k - 1, nx, ny, nz) + na_sig(sigma, i - 1, j, k - 1, nx, ny, nz) +
                         na_sig(sigma, i - 1, j - 1, k, nx, ny, nz) + na_sig(sigma, i - 1, j, k, nx, ny, nz)) : 0.0;
    g[2] = j < ny ? hq * (na_sig(sigma, i - 1, j, k - 1, nx, ny, nz) + na_sig(sigma, i, j, k - 1, nx, ny, nz) +
                          na_sig(sigma, i - 1, j, k, nx, ny, nz) + na_sig(sigma, i, j, k, nx, ny, nz)) : 0.0;
    g[3] = j > 0 ? hq * (na_sig(sigma, i - 1, j - 1, k - 1, nx, ny, nz) + na_sig(sigma, i, j - 1, k - 1, nx, ny, nz) +
                         na_sig(sigma, i - 1, j - 1, k, nx, ny, nz) + na_sig(sigma, i, j - 1, k, nx, ny, nz)) : 0.0;
    g[4] = k < nz ? hq * (na_sig(sigma, i - 1, j - 1, k, nx, ny, nz) + na_sig(sigma, i, j - 1, k, nx, ny, nz) +
                          na_sig(sigma, i - 1, j, k, nx, ny, nz) + na_sig(sigma, i, j, k, nx, ny, nz)) : 0.0;
    g[5] = k > 0 ? hq * (na_sig(sigma, i - 1, j - 1, k - 1, nx, ny, nz) + na_sig(sigma, i, j - 1, k - 1, nx, ny, nz) +
                         na_sig(sigma, i - 1, j, k - 1, nx, ny, nz) + na_sig(sigma, i, j, k - 1, nx, ny, nz)) : 0.0;
    if (!(g[0] > 0.0 || g[1] > 0.0 || g[2] > 0.0 || g[3] > 0.0 || g[4] > 0.0 || g[5] > 0.0))
      continue;  // not an unknown
    const long long nb[6] = {n + 1, n - 1, n + NX, n - NX, n + NX * NY, n - NX * NY};
    const long long ea[6] = {n, n - 1, NN + n, NN + n - NX, 2 * NN + n, 2 * NN + n - NX * NY};
    const double sg[6] = {1.0, -1.0, 1.0, -1.0, 1.0, -1.0};
    const double pn = psi[n];
    double b = 0.0, ap = 0.0;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      if (g[e] > 0.0) {
        b += sg[e] * g[e] * a[ea[e]];
        ap += g[e] * (pn - psi[nb[e]]);
      }
    }
    const double r = b - ap;
    rr += r * r;
    bb += b * b;
  }
  // block reduction, then the last block adds the partials in block order
  __shared__ double sm[NA_THREADS / 32][2];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sm[w][0] = rr; sm[w][1] = bb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < NA_THREADS / 32; ++q) { t0 += sm[q][0]; t1 += sm[q][1]; }
    scr->partial[blockIdx.x][0] = t0;
    scr->partial[blockIdx.x][1] = t1;
    __threadfence();
    last = atomicAdd(&scr->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (unsigned q = threadIdx.x; q < gridDim.x; q += NA_THREADS) {
    s0 += __ldcg(&scr->partial[q][0]);
    s1 += __ldcg(&scr->partial[q][1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  __syncthreads();
  if (lane == 0) { sm[w][0] = s0; sm[w][1] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < NA_THREADS / 32; ++q) { t0 += sm[q][0]; t1 += sm[q][1]; }
    scr->result[0] = t0;
    scr->result[1] = t1;
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ variable is not a device
// address).  The kept address does not survive a cudaDeviceReset of that
// device, after which the module is loaded again.
spfd_status scratch_for_current_device(NoallocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return fail(SPFD_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES)
    return fail(SPFD_EINVAL, "device %d beyond the %d devices served", dev, NA_MAX_DEVICES);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(SPFD_ECUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = (NoallocScratch *)p;
  }
  *out = g_scratch_ptr[dev];
  return SPFD_OK;
}

}  // namespace
}  // namespace spfd

using namespace spfd;

extern "C" spfd_status spfd_residual_noalloc(const double *sigma_dev,
                                             const double *a_dev,
                                             const double *psi_dev, int nx,
                                             int ny, int nz, double h,
                                             void *stream, double *rel_res) {
  if (!sigma_dev || !a_dev || !psi_dev || !rel_res)
    return fail(SPFD_EINVAL, "null argument");
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(SPFD_EINVAL, "voxel counts must be >= 1 (got %d %d %d)", nx, ny, nz);
  if (!(h > 0.0) || !std::isfinite(h)) return fail(SPFD_EINVAL, "h must be > 0");
  const long long NN = ((long long)nx + 1) * ((long long)ny + 1) * ((long long)nz + 1);
  if (NN > NA_MAX_NODES)
    return fail(SPFD_EINVAL,
                "grid of %lld nodes exceeds the %lld nodes the fixed scratch of "
                "spfd_residual_noalloc serves",
                NN, NA_MAX_NODES);
  NoallocScratch *scr = nullptr;
  TRY(scratch_for_current_device(&scr));
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (int)((NN + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
  CU(cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), st));
  k_residual_noalloc<<<blocks, NA_THREADS, 0, st>>>(sigma_dev, a_dev, psi_dev, nx, ny,
                                                    nz, h, scr);
  CU(cudaGetLastError());
  double res[2] = {0.0, 0.0};
  CU(cudaMemcpyAsync(res, scr->result, sizeof res, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *rel_res = res[1] > 0.0 ? std::sqrt(res[0] / res[1]) : 0.0;
  return SPFD_OK;
}
