// Throughput probes for the roofline denominators of the cell kernel: the
// MUFU ex2 rate (ex2.approx.ftz.f32, the exponential of every log-sum-exp
// term) and the FP32 FFMA rate, measured on all SMs of the current device,
// with the SM clock observed inside the kernels (clock64 against the
// global nanosecond timer).
#include <cuda_runtime.h>

#include "dd_common.cuh"
#include "domdec.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 16;

// Per block: [0] clock64 at start, [1] at end, [2] globaltimer ns at start, [3] at end.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// kProbeUnroll independent chains x <- 2^{-x} per thread (each ex2 takes the
// previous one's result, so nothing can be hoisted out of the loop; the
// values stay in [0.5, 0.71], no special cases).
__global__ void __launch_bounds__(kProbeThreads)
k_probe_ex2(int iters, float seed, float* sink, long long* clk) {
  float x[kProbeUnroll];
#pragma unroll
  for (int k = 0; k < kProbeUnroll; ++k) x[k] = seed + 0.01f * k + 1e-6f * threadIdx.x;
  __syncthreads();
  const long long c0 = clock64();
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(-x[k]));
  }
  __syncthreads();
  const long long c1 = clock64();
  const unsigned long long t1 = global_ns();
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeUnroll; ++k) acc += x[k];
  if (acc == 12345.f) sink[threadIdx.x] = acc;
  if (threadIdx.x == 0) {
    clk[4 * blockIdx.x + 0] = c0;
    clk[4 * blockIdx.x + 1] = c1;
    clk[4 * blockIdx.x + 2] = (long long)t0;
    clk[4 * blockIdx.x + 3] = (long long)t1;
  }
}

// kProbeUnroll independent FFMA chains x <- x a + b (a slightly below 1, so
// the values stay bounded).
__global__ void __launch_bounds__(kProbeThreads)
k_probe_ffma(int iters, float seed, float* sink, long long* clk) {
  float x[kProbeUnroll];
#pragma unroll
  for (int k = 0; k < kProbeUnroll; ++k) x[k] = seed + 0.001f * k + 1e-7f * threadIdx.x;
  const float a = 0.999999f, b = 1e-6f;
  __syncthreads();
  const long long c0 = clock64();
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) x[k] = fmaf(x[k], a, b);
  }
  __syncthreads();
  const long long c1 = clock64();
  const unsigned long long t1 = global_ns();
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeUnroll; ++k) acc += x[k];
  if (acc == 12345.f) sink[threadIdx.x] = acc;
  if (threadIdx.x == 0) {
    clk[4 * blockIdx.x + 0] = c0;
    clk[4 * blockIdx.x + 1] = c1;
    clk[4 * blockIdx.x + 2] = (long long)t0;
    clk[4 * blockIdx.x + 3] = (long long)t1;
  }
}

}  // namespace

extern "C" int domdec_probe_peaks(int iters, double out[8], void* stream) {
  if (!out || iters < 1) return DOMDEC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return DOMDEC_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_probe_ex2, kProbeThreads, 0) != cudaSuccess || bps < 1)
    return DOMDEC_ECUDA;
  bps = bps > 8 ? 8 : bps;   // 8 x 256 threads = 64 warps per SM
  const int grid = nsm * bps;
  float* sink = nullptr;
  long long* clk = nullptr;
  if (cudaMallocAsync(&sink, kProbeThreads * sizeof(float), st) != cudaSuccess) return DOMDEC_ENOMEM;
  if (cudaMallocAsync(&clk, 4 * (size_t)grid * sizeof(long long), st) != cudaSuccess) {
    cudaFreeAsync(sink, st);
    return DOMDEC_ENOMEM;
  }
  long long* hclk = new long long[4 * (size_t)grid];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = DOMDEC_OK;
  for (int which = 0; which < 2 && rc == DOMDEC_OK; ++which) {
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up, the second is timed
      cudaEventRecord(e0, st);
      if (which == 0) k_probe_ex2<<<grid, kProbeThreads, 0, st>>>(iters, 0.5f, sink, clk);
      else k_probe_ffma<<<grid, kProbeThreads, 0, st>>>(iters, 0.5f, sink, clk);
      cudaEventRecord(e1, st);
    }
    if (cudaMemcpyAsync(hclk, clk, 4 * (size_t)grid * sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = DOMDEC_ECUDA;
      break;
    }
    // SM clock: mean over blocks of cycles / ns
    double mhz = 0.0;
    for (int b = 0; b < grid; ++b) {
      const double dc = (double)(hclk[4 * b + 1] - hclk[4 * b]);
      const double dt = (double)(hclk[4 * b + 3] - hclk[4 * b + 2]);
      mhz += dt > 0.0 ? 1e3 * dc / dt : 0.0;
    }
    mhz /= grid;
    const double ops = (double)grid * kProbeThreads * (double)iters * kProbeUnroll;
    const double rate = ops / (ms * 1e-3);
    out[3 * which + 0] = rate;                          // ex2/s or FFMA/s
    out[3 * which + 1] = rate / (nsm * mhz * 1e6);      // per SM per clock
    out[3 * which + 2] = mhz;
  }
  out[6] = nsm;
  out[7] = grid;
  delete[] hclk;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  cudaFreeAsync(clk, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == DOMDEC_OK) rc = DOMDEC_ECUDA;
  return rc;
}

namespace {
__global__ void k_probe_log(const double* __restrict__ x, double* __restrict__ y, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = dd_log(x[i]);
}
}  // namespace

extern "C" int domdec_probe_log(const double* x, double* y, int n, void* stream) {
  if (!x || !y || n < 0) return DOMDEC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n) k_probe_log<<<(n + 255) / 256, 256, 0, st>>>(x, y, n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return DOMDEC_ECUDA;
  return DOMDEC_OK;
}
