// spfd_pipeline_host: steps 4 and 5 of the pipeline (Sec. II-A) in one call,
// from host arrays to host arrays.
//
// The caller hands over the voxel conductivities and the edge potentials in
// host memory and receives Psi (Eq. 3) and the voxel-averaged |E| (Eq. 1) in
// host memory.  On the device the call
//   1. copies sigma in (copy engine),
//   2. on a second stream, finds in each voxel row (j, k) the span of its
//      conducting voxels and pulls from host memory only the part of each
//      row of a that holds an edge of such a voxel (SM loads over the
//      chip-to-chip link), zeroing the rest: the operator and |E| never read
//      it, and on a body phantom 54 % of the rows' nodes are pulled from 52 %
//      of the rows,
//   3. meanwhile builds the operator and hierarchy (spfd_build),
//   4. solves Eq. 3 once the rows of a have arrived (spfd_solve),
//   5. evaluates |E| (spfd_efield) while Psi goes back on the second stream,
//      then copies |E| back.  Where the device can write the output arrays
//      directly, host threads zero them while the GPU builds and solves, and
//      the GPU then writes only the spans of nonzero values (the unknowns'
//      node rows of Psi, the conducting voxels' rows of |E|): about a quarter
//      of the bytes cross the link.
// The device buffers come from the library's block cache and go back to it,
// so repeated calls of one problem size do not call cudaMalloc.
//
// Host memory that the device can read directly (pinned, or any memory on a
// system with pageable-memory access) is pulled row by row; otherwise a
// is copied whole.
#include <cstring>
#include <thread>

#include "spfd_ctx.cuh"

namespace spfd {
namespace {

// span[k * ny + j] = (first, last) x index of the conducting voxels
// (sigma > 0) of voxel row (j, k), or (-1, -1); one warp per row.
__global__ void __launch_bounds__(256)
k_row_span(const double *__restrict__ sigma, int nx, int nrows, int2 *__restrict__ span) {
  const int lane = threadIdx.x & 31;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((long long)gridDim.x * blockDim.x) >> 5) {
    const double *row = sigma + (size_t)r * nx;
    int lo = nx, hi = -1;
    for (int i = lane; i < nx; i += 32)
      if (row[i] > 0.0) {
        lo = min(lo, i);
        hi = i;
      }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) span[r] = hi >= 0 ? make_int2(lo, hi) : make_int2(-1, -1);
  }
}

// The nodes lo .. hi of row (d, k, j) of a (the d-edges of node row (j, k),
// nx+1 slots) that hold an edge of a conducting voxel: edges of nodes
// imin .. imax + 1 of the voxel rows they touch,
//   x edges of node row (j, k): voxel rows (j-1..j, k-1..k),
//   y edges:                    voxel rows (j, k-1..k)   (none for j = ny),
//   z edges:                    voxel rows (j-1..j, k)   (none for k = nz);
// hi < lo when none does.
__device__ __forceinline__ int2 row_nodes(const int2 *__restrict__ span, int ny, int nz, int d,
                                          int j, int k) {
  int lo = 1 << 30, hi = -1;
  auto take = [&](int jj, int kk) {
    if (jj < 0 || jj >= ny || kk < 0 || kk >= nz) return;
    const int2 q = span[(size_t)kk * ny + jj];
    if (q.y < 0) return;
    lo = min(lo, q.x);
    hi = max(hi, q.y + 1);
  };
  if (d == 0) {
    take(j - 1, k - 1); take(j, k - 1); take(j - 1, k); take(j, k);
  } else if (d == 1) {
    take(j, k - 1); take(j, k);
  } else {
    take(j - 1, k); take(j, k);
  }
  return make_int2(lo, hi);
}

// loads each lane has in flight per pass along a row (one pass covers 288
// slots, a whole row of the 2 mm body)
constexpr int PULL_PER_LANE = 9;

// One warp per row: the needed nodes are loaded from host memory (every lane
// issues its loads before storing), the others zeroed.
__global__ void __launch_bounds__(256)
k_pull_rows(const double *__restrict__ a_host, const int2 *__restrict__ span, int nx,
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
    const int2 nodes = row_nodes(span, ny, nz, d, j, k);
    const double *src = a_host + (size_t)r * NX;
    for (int i0 = 0; i0 < NX; i0 += 32 * PULL_PER_LANE) {
      double v[PULL_PER_LANE];
#pragma unroll
      for (int u = 0; u < PULL_PER_LANE; ++u) {
        const int i = i0 + u * 32 + lane;
        v[u] = (i >= nodes.x && i <= nodes.y) ? src[i] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < PULL_PER_LANE; ++u) {
        const int i = i0 + u * 32 + lane;
        if (i < NX) dst[i] = v[u];
      }
    }
  }
}

// The spans of rows of the node grid (Psi: node row (j, k), the nodes of
// its unknowns lie in row_nodes(..., 0, j, k)) or of the voxel grid (|E|:
// span[r], the conducting voxels) from device rows to host rows; the rest of
// each host row is left as it is (zeroed by the host beforehand).  One warp
// per row.
template <bool NODES>
__global__ void __launch_bounds__(256)
k_push_spans(const double *__restrict__ src, const int2 *__restrict__ span, int nx, int ny,
             int nz, double *__restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const size_t W = NODES ? (size_t)nx + 1 : (size_t)nx;
  const long long nrows = NODES ? (long long)(nz + 1) * (ny + 1) : (long long)nz * ny;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((long long)gridDim.x * blockDim.x) >> 5) {
    int2 q;
    if constexpr (NODES) q = row_nodes(span, ny, nz, 0, (int)(r % (ny + 1)), (int)(r / (ny + 1)));
    else q = span[r];
    // an empty row has q.y < 0 (voxel rows: (-1, -1); node rows: lo > hi)
    if (q.y < 0 || q.x > q.y) continue;
    const int lo = max(q.x, 0), hi = min(q.y, (int)W - 1);
    const double *s = src + (size_t)r * W;
    double *d = dst + (size_t)r * W;
    for (int i = lo + lane; i <= hi; i += 32) d[i] = s[i];
  }
}

// Host threads zeroing host arrays while the GPU works; joined before the
// GPU writes into them, and on every exit.
struct HostZero {
  std::vector<std::thread> t;
  void start(double *p, size_t n, int parts) {
    const size_t chunk = (n + parts - 1) / parts;
    for (size_t a = 0; a < n; a += chunk) {
      const size_t b = std::min(n, a + chunk);
      t.emplace_back([p, a, b] { std::memset(p + a, 0, (b - a) * sizeof(double)); });
    }
  }
  void join() {
    for (auto &x : t)
      if (x.joinable()) x.join();
    t.clear();
  }
  ~HostZero() { join(); }
};

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
// With opts.verbose >= 2 the call also times its phases (tm[]: start, sigma
// in, a in, built, solved, |E| done, end) and prints them.
struct CallStreams {
  cudaStream_t main = nullptr, side = nullptr;
  cudaEvent_t ev_sig = nullptr, ev_a = nullptr, ev_solved = nullptr;
  cudaEvent_t tm[7] = {};
  void mark(int i, cudaStream_t st) {
    if (tm[i]) cudaEventRecord(tm[i], st);
  }
  ~CallStreams() {
    cudaStreamSynchronize(main);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    if (ev_sig) cudaEventDestroy(ev_sig);
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_solved) cudaEventDestroy(ev_solved);
    for (cudaEvent_t e : tm)
      if (e) cudaEventDestroy(e);
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
  int2 *span = nullptr;
  if (stg.get(&sig_d, nvox) != cudaSuccess || stg.get(&a_d, 3 * NN) != cudaSuccess ||
      stg.get(&psi_d, NN) != cudaSuccess || stg.get(&E_d, nvox) != cudaSuccess ||
      stg.get(&span, (size_t)nrows) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPFD_ENOMEM, "device staging buffers for the host pipeline");
  }
  CU(cudaStreamCreateWithFlags(&cs.side, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&cs.ev_sig, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&cs.ev_a, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&cs.ev_solved, cudaEventDisableTiming));
  const bool timed = opts && opts->verbose >= 2;
  if (timed)
    for (cudaEvent_t &e : cs.tm) CU(cudaEventCreate(&e));
  cs.mark(0, cs.main);
  // output arrays the device can write: host threads zero them now, the GPU
  // writes the spans of nonzero values at the end
  double *psi_view = const_cast<double *>(device_view(psi_host, stg.device));
  double *E_view = const_cast<double *>(device_view(E_host, stg.device));
  const bool push = psi_view && E_view;
  HostZero zero;
  // 1. sigma in
  CU(cudaMemcpyAsync(sig_d, sigma_host, nvox * sizeof(double), cudaMemcpyHostToDevice,
                     cs.main));
  CU(cudaEventRecord(cs.ev_sig, cs.main));
  cs.mark(1, cs.main);

  // 2. the rows of a the solve and |E| read, beside the build
  CU(cudaStreamWaitEvent(cs.side, cs.ev_sig, 0));
  const double *a_view = device_view(a_host, stg.device);
  if (a_view || push) {
    k_row_span<<<(unsigned)std::min<long long>((nrows + 7) / 8, 152LL * 16), 256, 0,
                 cs.side>>>(sig_d, nx, nrows, span);
    CU(cudaGetLastError());
  }
  if (a_view) {
    const long long arows = 3LL * (nz + 1) * (ny + 1);
    // one block per SM: the pull is bound by the chip-to-chip link, and
    // more blocks only take SM slots from the build running beside it
    k_pull_rows<<<(unsigned)std::min<long long>((arows + 7) / 8, 152LL), 256, 0, cs.side>>>(
        a_view, span, nx, ny, nz, a_d);
    CU(cudaGetLastError());
  } else {
    CU(cudaMemcpyAsync(a_d, a_host, 3 * NN * sizeof(double), cudaMemcpyHostToDevice, cs.side));
  }
  CU(cudaEventRecord(cs.ev_a, cs.side));
  cs.mark(2, cs.side);
  // 3. build
  spfd_ctx *ctx = nullptr;
  // the build's own phase marks (verbose >= 2) synchronise its stream, which
  // would distort the call's phase times: the build gets verbose <= 1
  spfd_opts bopts;
  if (opts) {
    bopts = *opts;
    if (bopts.verbose > 1) bopts.verbose = 1;
  } else {
    spfd_opts_default(&bopts);
  }
  spfd_status s = spfd_build(sig_d, nx, ny, nz, h, &bopts, cs.main, &ctx);
  if (s != SPFD_OK) return s;
  struct CtxGuard {
    spfd_ctx *c;
    ~CtxGuard() { spfd_destroy(c); }
  } guard{ctx};
  const int64_t build_launches = ctx->info.launches;
  cs.mark(3, cs.main);
  if (push) {
    // the host zeroes the outputs during the solve, which uses neither host
    // memory nor the host's cores (beside the copies in and the build it
    // took memory bandwidth and cycles from them); two threads per array
    // finish well within the solve
    zero.start(psi_host, NN, 2);
    zero.start(E_host, nvox, 2);
  }
  // 4. solve once a is in
  CU(cudaStreamWaitEvent(cs.main, cs.ev_a, 0));
  spfd_info inf{};
  s = spfd_solve(ctx, a_d, tol, psi_d, &inf);
  if (s != SPFD_OK && s != SPFD_ENOTCONVERGED) return s;
  const std::string msg = last_error_copy();
  // 5. Psi out beside |E|, then |E| out
  cs.mark(4, cs.main);
  CU(cudaEventRecord(cs.ev_solved, cs.main));
  CU(cudaStreamWaitEvent(cs.side, cs.ev_solved, 0));
  if (!push)
    CU(cudaMemcpyAsync(psi_host, psi_d, NN * sizeof(double), cudaMemcpyDeviceToHost,
                       cs.side));
  TRY(spfd_efield(ctx, a_d, psi_d, omega, E_d));
  cs.mark(5, cs.main);
  if (push) {
    // after |E| (beside it the SM writes over the link slowed it down), one
    // block per SM (bound by the link)
    zero.join();  // the host's zeros are in before the GPU writes the spans
    const unsigned blocks =
        (unsigned)std::min<long long>(((long long)(nz + 1) * (ny + 1) + 7) / 8, 152LL);
    k_push_spans<true><<<blocks, 256, 0, cs.main>>>(psi_d, span, nx, ny, nz, psi_view);
    CU(cudaGetLastError());
    k_push_spans<false><<<blocks, 256, 0, cs.main>>>(E_d, span, nx, ny, nz, E_view);
    CU(cudaGetLastError());
  } else {
    CU(cudaMemcpyAsync(E_host, E_d, nvox * sizeof(double), cudaMemcpyDeviceToHost, cs.main));
  }
  CU(cudaStreamSynchronize(cs.side));
  CU(cudaStreamSynchronize(cs.main));
  if (timed) {  // both streams are idle: the mark's time is the end of the call's work
    cs.mark(6, cs.main);
    CU(cudaStreamSynchronize(cs.main));
    float t[7] = {};
    for (int i = 1; i < 7; ++i) cudaEventElapsedTime(&t[i], cs.tm[0], cs.tm[i]);
    fprintf(stderr,
            "[spfd] pipeline: sigma in %.3f ms, a in %.3f, built %.3f, solved %.3f, "
            "|E| %.3f, end %.3f (from the call's start)\n",
            t[1], t[2], t[3], t[4], t[5], t[6]);
  }
  if (info) {
    *info = inf;
    info->launches = build_launches + inf.launches + (a_view || push ? 1 : 0) +
                     (a_view ? 1 : 0) + (push ? 2 : 0) + 1;
  }
  set_error(msg);
  return s;
}
