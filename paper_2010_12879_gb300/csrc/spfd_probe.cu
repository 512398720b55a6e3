// spfd_fp64_fma_rate: this GPU's FP64 fused multiply-add rate, measured.
//
// The FP64 stencils of the library are bound by the FP64 pipe (on GB300 a
// handful of FP64 units per SM), so their roofline needs the pipe's rate.
// The kernel below keeps every resident warp busy with independent FMA
// chains and nothing else: 8 chains per thread (enough to cover the FMA
// latency), EFMA_STEPS steps each, no memory traffic inside the loop.  The
// rate is the FMA count (2 flops each) over the kernel's CUDA-event time of
// the fastest of several launches after a warm-up.
#include "spfd_ctx.cuh"

namespace spfd {
namespace {

constexpr int EFMA_THREADS = 256;
constexpr int EFMA_CHAINS = 8;
constexpr int EFMA_STEPS = 4096;

__global__ void __launch_bounds__(EFMA_THREADS)
k_fma_rate(double b, double c, double *out) {
  double a[EFMA_CHAINS];
#pragma unroll
  for (int i = 0; i < EFMA_CHAINS; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int k = 0; k < EFMA_STEPS; ++k) {
#pragma unroll
    for (int i = 0; i < EFMA_CHAINS; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < EFMA_CHAINS; ++i) s += a[i];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for b, c below
}

}  // namespace
}  // namespace spfd

using namespace spfd;

extern "C" spfd_status spfd_fp64_fma_rate(void *stream, double *tflops, double *ms) {
  if (!tflops) return fail(SPFD_EINVAL, "tflops is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0, per_sm = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate, EFMA_THREADS, 0));
  const int blocks = nsm * std::max(per_sm, 1);
  double *sink = nullptr;
  void *blk = nullptr;
  size_t bsz = 0;
  CU(mem_get(dev, sizeof(double), &blk, &bsz));
  sink = (double *)blk;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {
    err = cudaEventRecord(e0, st);
    // b slightly below 1 keeps the iterates bounded and normal
    k_fma_rate<<<blocks, EFMA_THREADS, 0, st>>>(0.999999, 1e-7, sink);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    if (err == cudaSuccess && rep > 0 && (best == 0.0f || t < best)) best = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  mem_put(dev, blk, bsz);
  if (err != cudaSuccess)
    return fail(SPFD_ECUDA, "FP64 rate probe failed: %s", cudaGetErrorString(err));
  const double fmas = (double)blocks * EFMA_THREADS * EFMA_CHAINS * EFMA_STEPS;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return SPFD_OK;
}
