// fp64_rate.cu -- throughput probe of the binary64 pipe (measurement only).
//
// The binary64 forward and adjoint sweeps are bound by the binary64 pipe, so
// their roofline is that pipe's rate, which this probe measures on the GPU in
// use: every thread runs kChains independent chains of fused multiply-adds
// (enough independent work per warp and enough warps per SM to cover the
// pipe's latency), and the rate is the number of fused multiply-adds over the
// kernel's CUDA-event time.  It is built into its own library, which only the
// benchmark loads; the advection library does not contain it.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_chains_kernel(double* sink, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = 1e-3 * (threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  // b < 1 keeps the chains bounded; the store keeps them alive
  if (s == -1.0) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

// Fused multiply-adds per second of the current device, in units of 1e9
// (*gops), and the timed kernel's duration in ms (*ms): one warm-up launch,
// then `reps` timed launches of blocks_per_sm * SMs CTAs of 256 threads, each
// thread doing kChains * iters fused multiply-adds.  Returns 0, or the CUDA
// error code of the first failing call.
extern "C" int advect_probe_fp64_fma_rate(int iters, int blocks_per_sm, int reps, double* gops, double* ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  if (iters < 1 || blocks_per_sm < 1 || reps < 1 || !gops || !ms) return (int)cudaErrorInvalidValue;
  const int blocks = sms * blocks_per_sm;
  double* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, z = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * blocks * kThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  const double b = 1.0 - 1.0 / 1048576.0, c = 1.0 / 1024.0;
  if (e == cudaSuccess) {
    dfma_chains_kernel<<<blocks, kThreads, 0, st>>>(sink, iters, b, c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    dfma_chains_kernel<<<blocks, kThreads, 0, st>>>(sink, iters, b, c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(z, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(z);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, z);
  if (e == cudaSuccess) {
    const double ops = (double)blocks * kThreads * kChains * (double)iters * reps;
    *ms = t / reps;
    *gops = ops / (t * 1e-3) / 1e9;
  }
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  return (int)e;
}
