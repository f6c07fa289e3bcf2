// peaks.cu -- FMA throughput probes: the roofline denominator of the
// arithmetic-bound integrators (binary64 and binary32 CUDA-core FMA rates).
// Eight independent dependent chains per thread, every SM filled.
#include <cuda_runtime.h>

#include <string>

#include "../../include/odegpu.h"

namespace {

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
cudaError_t time_chains(int sms, int iters, double* fma_per_s) {
  const int threads = 256, blocks = sms * 4;
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(T));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, threads>>>(out, 8, (T)1.0000001, (T)1e-9);  // warm-up
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(out, iters, (T)1.0000001, (T)1e-9);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) *fma_per_s = (double)blocks * threads * iters * 16 * 8 / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return e;
}

// Cost of a binary64 cos, a general pow and a sqrt in units of the DFMA issue
// rate: four independent accumulation chains per thread with and without the
// call; the difference isolates the call.
template <int KIND>
__global__ void call_chains(double* out, int iters) {
  double x0 = 0.1 + threadIdx.x * 1e-5, x1 = x0 + 1.5, x2 = x0 + 3.0, x3 = x0 + 4.5;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int i = 0; i < iters; i++) {
    if (KIND == 1) {
      s0 += cos(x0); s1 += cos(x1); s2 += cos(x2); s3 += cos(x3);
    } else if (KIND == 2) {
      s0 += pow(x0, -0.2); s1 += pow(x1, -0.2); s2 += pow(x2, -0.2); s3 += pow(x3, -0.2);
    } else if (KIND == 3) {
      s0 += sqrt(x0); s1 += sqrt(x1); s2 += sqrt(x2); s3 += sqrt(x3);
    } else {
      s0 += x0; s1 += x1; s2 += x2; s3 += x3;
    }
    x0 += 0.0123; x1 += 0.0123; x2 += 0.0123; x3 += 0.0123;
    if (x0 > 6.0) x0 -= 5.9;
    if (x1 > 6.0) x1 -= 5.9;
    if (x2 > 6.0) x2 -= 5.9;
    if (x3 > 6.0) x3 -= 5.9;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s0 + s1 + s2 + s3;
}

template <int KIND>
cudaError_t time_calls(int sms, int iters, double* seconds) {
  const int threads = 256, blocks = sms * 4;
  double* out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  call_chains<KIND><<<blocks, threads>>>(out, 4);
  cudaEventRecord(e0);
  call_chains<KIND><<<blocks, threads>>>(out, iters);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) *seconds = ms * 1e-3 / ((double)blocks * threads * iters * 4);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return e;
}

}  // namespace

extern "C" int ode_probe_call_cost(int device, double* cos_dfma, double* pow_dfma, double* sqrt_dfma) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return ODE_ERR_CUDA;
  int sms = 0;
  double dfma = 0, t_cos = 0, t_pow = 0, t_sqrt = 0, t_loop = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = time_chains<double>(sms, 1000, &dfma);
  if (e == cudaSuccess) e = time_calls<1>(sms, 2000, &t_cos);
  if (e == cudaSuccess) e = time_calls<2>(sms, 500, &t_pow);
  if (e == cudaSuccess) e = time_calls<3>(sms, 2000, &t_sqrt);
  if (e == cudaSuccess) e = time_calls<0>(sms, 2000, &t_loop);
  // GPU seconds per call (all threads together) x DFMA per second of the GPU
  if (e == cudaSuccess) {
    if (cos_dfma) *cos_dfma = (t_cos - t_loop) * dfma;
    if (pow_dfma) *pow_dfma = (t_pow - t_loop) * dfma;
    if (sqrt_dfma) *sqrt_dfma = (t_sqrt - t_loop) * dfma;
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? ODE_OK : ODE_ERR_CUDA;
}

extern "C" int ode_probe_fma_peak(int device, double* dfma_per_s, double* ffma_per_s) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return ODE_ERR_CUDA;
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess && dfma_per_s) e = time_chains<double>(sms, 1000, dfma_per_s);
  if (e == cudaSuccess && ffma_per_s) e = time_chains<float>(sms, 20000, ffma_per_s);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? ODE_OK : ODE_ERR_CUDA;
}
