// hgks_fp64_peak: the FP64 arithmetic rate of the device, measured.
//
// The residual kernels and the FP64 Krylov products are bound by the FP64 pipe,
// so their roofline is the rate at which the SMs retire double-precision fused
// multiply-adds. This measures it with the simplest kernel that keeps that pipe
// full: every thread runs kChains independent FMA recurrences x <- x a + b (no
// loads, no stores inside the loop), enough warps per SM to cover the FMA
// latency, a grid of whole waves over the SMs, timed with CUDA events on a
// stream of its own. A warm-up launch sizes the repeat count to the requested
// duration; the result is the best of the timed launches.
#include <algorithm>
#include <cmath>
#include "hgks_internal.h"

namespace hgks {
namespace {

constexpr int kChains = 8;       // independent recurrences per thread
constexpr int kPeakBlock = 256;

__global__ void __launch_bounds__(kPeakBlock) k_dfma_chains(double *__restrict__ sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = 1.0 + 1e-3 * k + 1e-9 * threadIdx.x;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  // a store the compiler cannot prove dead; the values stay near 1, so the
  // branch is never taken and no thread writes
  if (s == -1.0) sink[blockIdx.x * kPeakBlock + threadIdx.x] = s;
}

}  // namespace
}  // namespace hgks

using namespace hgks;

extern "C" hgks_status hgks_fp64_peak(int32_t device, double seconds, double *gflops_out) {
  if (!gflops_out) return fail_msg(HGKS_ERR_ARG, "gflops_out is NULL");
  *gflops_out = 0.0;
  if (!(seconds > 0.0) || seconds > 60.0) return fail_msg(HGKS_ERR_ARG, "seconds must be in (0, 60]");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail_msg(HGKS_ERR_ARG, "no such device");
  HGKS_ON_DEVICE(device);
  int sms = 0, per_sm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_chains, kPeakBlock, 0);
  if (e != cudaSuccess) return cuda_error(e, "device attributes");
  const int blocks = sms * std::max(per_sm, 1);   // one full wave of resident blocks
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  double *sink = nullptr;   // never written (see the kernel); a valid address all the same
  hgks_status status = HGKS_OK;
  auto done = [&](hgks_status s2) {
    if (st) cudaStreamSynchronize(st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    return s2;
  };
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess ||
      (e = cudaMalloc(&sink, sizeof(double) * (size_t)blocks * kPeakBlock)) != cudaSuccess)
    return done(cuda_error(e, "hgks_fp64_peak set-up"));
  const double ca = 1.0 - 1e-12, cb = 1e-12;   // x stays within [1, 1.01]
  auto timed = [&](int iters, float &ms) -> cudaError_t {
    cudaError_t r;
    if ((r = cudaEventRecord(a, st)) != cudaSuccess) return r;
    k_dfma_chains<<<blocks, kPeakBlock, 0, st>>>(sink, iters, ca, cb);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    if ((r = cudaEventRecord(b, st)) != cudaSuccess) return r;
    if ((r = cudaEventSynchronize(b)) != cudaSuccess) return r;
    return cudaEventElapsedTime(&ms, a, b);
  };
  float ms = 0.f;
  int iters = 1 << 12;
  if ((e = timed(iters, ms)) != cudaSuccess) return done(cuda_error(e, "hgks_fp64_peak"));
  // size one launch to about a tenth of the requested time (at most 2^24 iterations)
  const double target_ms = 100.0 * seconds;
  iters = (int)std::min<double>(1 << 24, std::max<double>(1 << 12, iters * target_ms / std::max(ms, 1e-3f)));
  const int reps = 10;
  double best = 0.0;
  for (int r = 0; r < reps; r++) {
    if ((e = timed(iters, ms)) != cudaSuccess) return done(cuda_error(e, "hgks_fp64_peak"));
    const double flops = 2.0 * kChains * (double)iters * blocks * kPeakBlock;
    best = std::max(best, flops / (ms * 1e-3) / 1e9);
  }
  *gflops_out = best;
  return done(status);
}
