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

// Packed FP32 chains (two FMAs per instruction), the form of the |M|^2 joins.
template <int CH>
__global__ void __launch_bounds__(256) fma2_chains(float* out, int iters, float a, float b) {
  float2 x[CH];
  const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = __ffma2_rn(x[c], A, B);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FLOPs per thread of one launch and the launch itself, per kernel kind.
template <typename Launch>
qed_status run(Launch launch, double flop_per_launch, double* tflops, cudaStream_t st) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QED_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return QED_ECUDA; }
  for (int w = 0; w < 2; ++w) launch();
  cudaEventRecord(e0, st);
  const int reps = 4;
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return QED_ECUDA;
  *tflops = flop_per_launch * reps / (ms * 1e-3) / 1e12;
  return QED_OK;
}

}  // namespace

extern "C" qed_status qed_measure_fma_peak(qed_precision precision, double* tflops, void* stream) {
  if (!tflops || (precision != QED_FP64 && precision != QED_MIXED)) return QED_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QED_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QED_ECUDA;
  const int blocks = sms * 8;
  const double threads = (double)blocks * 256.0;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) return QED_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  qed_status s;
  if (precision == QED_MIXED) {
    // scalar and packed FMA chains; the larger rate is the FP32 peak
    const int it = 1 << 15;
    double scalar = 0.0, packed = 0.0;
    s = run([&] { fma_chains<float, 8><<<blocks, 256, 0, st>>>((float*)buf, it, 0.999999f, 1e-7f); },
            2.0 * 8 * it * threads, &scalar, st);
    if (s == QED_OK)
      s = run([&] { fma2_chains<8><<<blocks, 256, 0, st>>>((float*)buf, it / 2, 0.999999f, 1e-7f); },
              2.0 * 16 * (it / 2) * threads, &packed, st);
    *tflops = scalar > packed ? scalar : packed;
  } else {
    // about 0.3 s of FP64 chains per launch on B300
    const int it = 1 << 13;
    s = run([&] { fma_chains<double, 8><<<blocks, 256, 0, st>>>((double*)buf, it, 0.999999, 1e-7); },
            2.0 * 8 * it * threads, tflops, st);
  }
  cudaFree(buf);
  return s;
}
