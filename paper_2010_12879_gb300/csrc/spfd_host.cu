// spfd_pipeline_host: steps 4 and 5 of the pipeline (Sec. II-A) in one call,
// from host arrays to host arrays.
//
// The caller hands over the voxel conductivities and the edge potentials in
// host memory and receives Psi (Eq. 3) and the voxel-averaged |E| (Eq. 1) in
// host memory.  On the device the call
//   1. copies sigma in (copy engine),
//   2. on a second stream, marks the voxel rows (j, k) that hold a conducting
//      voxel and pulls from host memory only the rows of a that contain an
//      edge of such a voxel (SM loads over the chip-to-chip link), zeroing
//      the others: the operator and |E| never read the rest, and on a body
//      phantom about half of the rows of a are skipped,
//   3. meanwhile builds the operator and hierarchy (spfd_build),
//   4. solves Eq. 3 once the rows of a have arrived (spfd_solve),
//   5. evaluates |E| (spfd_efield) while Psi goes back on the second stream,
//      then copies |E| back.
// The device buffers come from the library's block cache and go back to it,
// so repeated calls of one problem size do not call cudaMalloc.
//
// Host memory that the device can read directly (pinned, or any memory on a
// system with pageable-memory access) is pulled row by row; otherwise a
// is copied whole.
#include "spfd_ctx.cuh"

namespace spfd {
namespace {

// rowc[k * ny + j] = 1 iff voxel row (j, k) holds a voxel with sigma > 0; one
// warp per row.
__global__ void __launch_bounds__(256)
k_row_any(const double *__restrict__ sigma, int nx, int nrows, unsigned char *__restrict__ rowc) {
  const int lane = threadIdx.x & 31;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((long long)gridDim.x * blockDim.x) >> 5) {
    const double *row = sigma + (size_t)r * nx;
    bool any = false;
    for (int i = lane; i < nx; i += 32) any |= row[i] > 0.0;
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) rowc[r] = any ? 1 : 0;
  }
}

// Row (d, k, j) of a (the d-edges of node row (j, k), nx+1 slots) is needed
// iff one of its edges touches a conducting voxel:
//   x edges of node row (j, k): voxel rows (j-1..j, k-1..k),
//   y edges:                    voxel rows (j, k-1..k)   (none for j = ny),
//   z edges:                    voxel rows (j-1..j, k)   (none for k = nz).
__device__ __forceinline__ bool row_needed(const unsigned char *__restrict__ rowc, int ny,
                                           int nz, int d, int j, int k) {
  auto c = [&](int jj, int kk) {
    return jj >= 0 && jj < ny && kk >= 0 && kk < nz && rowc[(size_t)kk * ny + jj];
  };
  if (d == 0) return c(j - 1, k - 1) || c(j, k - 1) || c(j - 1, k) || c(j, k);
  if (d == 1) return c(j, k - 1) || c(j, k);
  return c(j - 1, k) || c(j, k);
}

// loads each lane has in flight per pass along a row (one pass covers 288
// slots, a whole row of the 2 mm body)
constexpr int PULL_PER_LANE = 9;

// One warp per row: the needed rows are loaded from host memory (every lane
// issues its loads before storing), the others zeroed.
__global__ void __launch_bounds__(256)
k_pull_rows(const double *__restrict__ a_host, const unsigned char *__restrict__ rowc, int nx,
            int ny, int nz, double *__restrict__ a_dev) {
  const int lane = threadIdx.x & 31;
  const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
  const long long nrows = 3LL * NZ * NY;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int d = (int)(r / ((long long)NZ * NY));
    const int rem = (int)(r % ((long long)NZ * NY));
    const int k = rem / NY, j = rem % NY;
    double *dst = a_dev + (size_t)r * NX;
    if (!row_needed(rowc, ny, nz, d, j, k)) {
      for (int i = lane; i < NX; i += 32) dst[i] = 0.0;
      continue;
    }
    const double *src = a_host + (size_t)r * NX;
    for (int i0 = 0; i0 < NX; i0 += 32 * PULL_PER_LANE) {
      double v[PULL_PER_LANE];
#pragma unroll
      for (int u = 0; u < PULL_PER_LANE; ++u) {
        const int i = i0 + u * 32 + lane;
        v[u] = i < NX ? src[i] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < PULL_PER_LANE; ++u) {
        const int i = i0 + u * 32 + lane;
        if (i < NX) dst[i] = v[u];
      }
    }
  }
}

// Device blocks from the library's cache, returned (after the streams have
// been synchronised) when the call ends.
struct Staging {
  int device = 0;
  std::vector<std::pair<void *, size_t>> blocks;
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    void *q = nullptr;
    size_t blk = 0;
    cudaError_t e = mem_get(device, count * sizeof(T), &q, &blk);
    if (e != cudaSuccess) return e;
    blocks.emplace_back(q, blk);
    *p = (T *)q;
    return cudaSuccess;
  }
  ~Staging() {
    for (auto &b : blocks) mem_put(device, b.first, b.second);
  }
};

// Streams and events of one call; synchronised and released on every exit.
struct CallStreams {
  cudaStream_t main = nullptr, side = nullptr;
  cudaEvent_t ev_sig = nullptr, ev_a = nullptr, ev_solved = nullptr;
  ~CallStreams() {
    cudaStreamSynchronize(main);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    if (ev_sig) cudaEventDestroy(ev_sig);
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_solved) cudaEventDestroy(ev_solved);
  }
};

// The device address through which a kernel may read host memory p, or
// nullptr if it cannot.
const double *device_view(const double *p, int device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer)
    return (const double *)at.devicePointer;
  cudaGetLastError();  // clear a lookup failure on unregistered memory
  int pageable = 0;
  if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device) ==
          cudaSuccess && pageable)
    return p;
  return nullptr;
}

}  // namespace
}  // namespace spfd

using namespace spfd;

extern "C" spfd_status spfd_pipeline_host(const double *sigma_host, const double *a_host,
                                          int nx, int ny, int nz, double h, double tol,
                                          double omega, const spfd_opts *opts, void *stream,
                                          double *psi_host, double *E_host, spfd_info *info) {
  if (!sigma_host || !a_host || !psi_host || !E_host) return fail(SPFD_EINVAL, "null array");
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(SPFD_EINVAL, "voxel counts must be >= 1 (got %d %d %d)", nx, ny, nz);
  if (((int64_t)nx + 1) * ((int64_t)ny + 1) * ((int64_t)nz + 1) >= ((int64_t)1 << 31))
    return fail(SPFD_EINVAL, "grid too large");
  if (!std::isfinite(omega)) return fail(SPFD_EINVAL, "omega must be finite");
  if (std::isnan(tol)) return fail(SPFD_EINVAL, "tol is NaN");
  const size_t nvox = (size_t)nx * ny * nz;
  const size_t NN = ((size_t)nx + 1) * ((size_t)ny + 1) * ((size_t)nz + 1);
  const int nrows = ny * nz;
  Staging stg;  // declared first: returned after the streams are synchronised
  CU(cudaGetDevice(&stg.device));
  CallStreams cs;
  cs.main = (cudaStream_t)stream;
  double *sig_d = nullptr, *a_d = nullptr, *psi_d = nullptr, *E_d = nullptr;
  unsigned char *rowc = nullptr;
  if (stg.get(&sig_d, nvox) != cudaSuccess || stg.get(&a_d, 3 * NN) != cudaSuccess ||
      stg.get(&psi_d, NN) != cudaSuccess || stg.get(&E_d, nvox) != cudaSuccess ||
      stg.get(&rowc, (size_t)nrows) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPFD_ENOMEM, "device staging buffers for the host pipeline");
  }
  CU(cudaStreamCreateWithFlags(&cs.side, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&cs.ev_sig, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&cs.ev_a, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&cs.ev_solved, cudaEventDisableTiming));
  // 1. sigma in
  CU(cudaMemcpyAsync(sig_d, sigma_host, nvox * sizeof(double), cudaMemcpyHostToDevice,
                     cs.main));
  CU(cudaEventRecord(cs.ev_sig, cs.main));
  // 2. the rows of a the solve and |E| read, beside the build
  CU(cudaStreamWaitEvent(cs.side, cs.ev_sig, 0));
  const double *a_view = device_view(a_host, stg.device);
  if (a_view) {
    k_row_any<<<(unsigned)std::min<long long>((nrows + 7) / 8, 152LL * 16), 256, 0, cs.side>>>(
        sig_d, nx, nrows, rowc);
    CU(cudaGetLastError());
    const long long arows = 3LL * (nz + 1) * (ny + 1);
    k_pull_rows<<<(unsigned)std::min<long long>((arows + 7) / 8, 152LL * 16), 256, 0,
                  cs.side>>>(a_view, rowc, nx, ny, nz, a_d);
    CU(cudaGetLastError());
  } else {
    CU(cudaMemcpyAsync(a_d, a_host, 3 * NN * sizeof(double), cudaMemcpyHostToDevice, cs.side));
  }
  CU(cudaEventRecord(cs.ev_a, cs.side));
  // 3. build
  spfd_ctx *ctx = nullptr;
  spfd_status s = spfd_build(sig_d, nx, ny, nz, h, opts, cs.main, &ctx);
  if (s != SPFD_OK) return s;
  struct CtxGuard {
    spfd_ctx *c;
    ~CtxGuard() { spfd_destroy(c); }
  } guard{ctx};
  const int64_t build_launches = ctx->info.launches;
  // 4. solve once a is in
  CU(cudaStreamWaitEvent(cs.main, cs.ev_a, 0));
  spfd_info inf{};
  s = spfd_solve(ctx, a_d, tol, psi_d, &inf);
  if (s != SPFD_OK && s != SPFD_ENOTCONVERGED) return s;
  const std::string msg = last_error_copy();
  // 5. Psi out beside |E|, then |E| out
  CU(cudaEventRecord(cs.ev_solved, cs.main));
  CU(cudaStreamWaitEvent(cs.side, cs.ev_solved, 0));
  CU(cudaMemcpyAsync(psi_host, psi_d, NN * sizeof(double), cudaMemcpyDeviceToHost, cs.side));
  TRY(spfd_efield(ctx, a_d, psi_d, omega, E_d));
  CU(cudaMemcpyAsync(E_host, E_d, nvox * sizeof(double), cudaMemcpyDeviceToHost, cs.main));
  CU(cudaStreamSynchronize(cs.side));
  CU(cudaStreamSynchronize(cs.main));
  if (info) {
    *info = inf;
    info->launches = build_launches + inf.launches + (a_view ? 2 : 0) + 1;
  }
  set_error(msg);
  return s;
}
