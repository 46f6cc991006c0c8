// FMA-chain microbenchmark that measures the FP32 / FP64 FMA-pipe peak of
// the device, the denominator of the |M|^2 kernels' roofline (they are bound
// by FMA-pipe arithmetic, not by HBM or tensor cores).
#include <cuda_runtime.h>

#include "../../include/qed.h"

namespace {

template <typename T, int CH>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int CH>
qed_status run(int iters, double* tflops, cudaStream_t st, T* buf, int blocks) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QED_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return QED_ECUDA; }
  for (int w = 0; w < 2; ++w) fma_chains<T, CH><<<blocks, 256, 0, st>>>(buf, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0, st);
  const int reps = 4;
  for (int r = 0; r < reps; ++r) fma_chains<T, CH><<<blocks, 256, 0, st>>>(buf, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return QED_ECUDA;
  *tflops = 2.0 * CH * (double)iters * blocks * 256.0 * reps / (ms * 1e-3) / 1e12;
  return QED_OK;
}

}  // namespace

extern "C" qed_status qed_measure_fma_peak(qed_precision precision, double* tflops, void* stream) {
  if (!tflops || (precision != QED_FP64 && precision != QED_MIXED)) return QED_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QED_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QED_ECUDA;
  const int blocks = sms * 8;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) return QED_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  qed_status s = precision == QED_MIXED
                     ? run<float, 8>(1 << 15, tflops, st, (float*)buf, blocks)
                     : run<double, 8>(1 << 10, tflops, st, (double*)buf, blocks);
  cudaFree(buf);
  return s;
}
