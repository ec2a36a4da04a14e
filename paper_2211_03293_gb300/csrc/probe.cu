// Measurement utility: the FP64 FMA issue rate of the device, the denominator of
// the fast path's ALU roofline.  Not part of the method.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/mri_probe.h"
#include "fastmath.cuh"

namespace {

// Eight independent FMA chains per thread keep the FP64 pipe fed; the result is
// stored so the chains are not removed.
__global__ void dfma_chains(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// As dfma_chains, with only the first `active` lanes of every warp running the chains
// (the others return at once).
__global__ void dfma_chains_lanes(double* out, int iters, double a, double b, int active) {
  if ((int)(threadIdx.x & 31) >= active) return;
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// One warp, one dependent FMA chain: SM cycles per FMA.
__global__ void dfma_latency(double* out, long long* cycles, int iters, double a, double b) {
  double x = threadIdx.x * 1e-3;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) x = fma(x, a, b);
  const long long t1 = clock64();
  out[threadIdx.x] = x;
  if (threadIdx.x == 0) *cycles = t1 - t0;
}

struct Exp2Table {
  double v[mri::kExpTab];
};

__global__ void exp_probe_kernel(const double* x, double* y, long long n, Exp2Table tab) {
  __shared__ double s[mri::kExpTab];
  for (int i = threadIdx.x; i < mri::kExpTab; i += blockDim.x) s[i] = tab.v[i];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = mri::exp_tab(x[i], s);
}

__global__ void exp_pair_probe_kernel(const double* x, double* y, double* z, long long n, Exp2Table tab) {
  __shared__ double s[mri::kExpTab];
  for (int i = threadIdx.x; i < mri::kExpTab; i += blockDim.x) s[i] = tab.v[i];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    mri::exp_pair(x[i], s, y[i], z[i]);
}

struct LogTable {
  double v[mri::kLogTabDoubles];
};

__global__ void log_probe_kernel(const double* x, double* y, long long n, LogTable tab) {
  __shared__ double s[mri::kLogTabDoubles];
  for (int i = threadIdx.x; i < mri::kLogTabDoubles; i += blockDim.x) s[i] = tab.v[i];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = mri::log_tab(x[i], s);
}

}  // namespace

extern "C" int mri_probe_exp_pair(const double* x, double* y, double* z, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y || !z))) return -1;
  if (n == 0) return 0;
  Exp2Table tab;
  mri::fill_exp_table(tab.v);
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  exp_pair_probe_kernel<<<(int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, z, n, tab);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

extern "C" int mri_probe_log(const double* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return -1;
  if (n == 0) return 0;
  LogTable tab;
  mri::fill_log_table(tab.v);
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  log_probe_kernel<<<(int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n, tab);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

extern "C" int mri_probe_exp(const double* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return -1;
  if (n == 0) return 0;
  Exp2Table tab;
  mri::fill_exp_table(tab.v);
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  exp_probe_kernel<<<(int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n, tab);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

extern "C" int mri_probe_fp64_lanes(double* scratch, long long scratch_doubles, int iters, int active_lanes,
                                    int warps_per_sm, double* lane_fma_per_s, void* stream) {
  if (!scratch || !lane_fma_per_s || iters < 1 || active_lanes < 1 || active_lanes > 32 || warps_per_sm < 1 ||
      warps_per_sm > 32)
    return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return -3;
  const int threads = 32 * warps_per_sm, blocks = sms;
  if ((long long)threads * blocks > scratch_doubles) return -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -3;
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    dfma_chains_lanes<<<blocks, threads, 0, st>>>(scratch, iters, 0.9999999, 1e-7, active_lanes);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return -3; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *lane_fma_per_s = (double)active_lanes * warps_per_sm * blocks * (double)iters * 8.0 / (best * 1e-3);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

extern "C" int mri_probe_fp64_latency(double* scratch, long long scratch_doubles, int iters, double* cycles,
                                      void* stream) {
  if (!scratch || !cycles || iters < 1 || scratch_doubles < 40) return -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long* cyc = reinterpret_cast<long long*>(scratch + 32);
  dfma_latency<<<1, 32, 0, st>>>(scratch, cyc, iters, 0.9999999, 1e-7);
  long long h = 0;
  if (cudaMemcpyAsync(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -3;
  *cycles = (double)h / iters;
  return 0;
}

extern "C" int mri_probe_fp64_fma(double* scratch, long long scratch_doubles, int iters, double* fma_per_s,
                                  void* stream) {
  if (!scratch || !fma_per_s || iters < 1) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return -3;
  const int threads = 256, blocks = sms * 8;
  if ((long long)threads * blocks > scratch_doubles) return -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -3;
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    dfma_chains<<<blocks, threads, 0, st>>>(scratch, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return -3; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *fma_per_s = (double)threads * blocks * (double)iters * 8.0 / (best * 1e-3);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
