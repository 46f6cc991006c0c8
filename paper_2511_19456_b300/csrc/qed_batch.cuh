// Work items, request table and persistent kernel of the batched evaluation
// (requests of different k in one launch; items taken from a device counter).
#pragma once

#include <cuda_runtime.h>

#include "qed_eval.cuh"

struct qed_plan_s;

namespace qed {

struct BatchItem {
  int32_t req;
  int32_t k;
  long long p0, p1;
};

struct BatchDesc {
  KParams kp;
};

// Up to 256 threads per block (the tuner's largest); registers up to 128
// (FP32) or 255 (FP64) per thread, the range the per-k paths need without
// spilling.
template <typename Real>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 2 : 1)
qed_batch_kernel(const BatchDesc* __restrict__ reqs, const BatchItem* __restrict__ items, int n_items,
                 unsigned* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const KParams& kp = reqs[item.req].kp;
    switch (item.k) {
#define QED_BATCH_CASE(KK)                                                                       \
  case KK: {                                                                                     \
    constexpr int T = 1 << (KK + 1);                                                             \
    eval_range<KK, true, Real, T, 1>(kp, item.p0, item.p1, (long long)(blockDim.x / T), smem);   \
    break;                                                                                       \
  }
      QED_BATCH_CASE(1) QED_BATCH_CASE(2) QED_BATCH_CASE(3) QED_BATCH_CASE(4) QED_BATCH_CASE(5)
#undef QED_BATCH_CASE
      default: break;
    }
    __syncthreads();
  }
}

using BatchFn = void (*)(const BatchDesc*, const BatchItem*, int, unsigned*);

// The specialised form of the batched kernel (generated with the
// straight-line forward kernels): the same work-item loop, with the
// straight-line point evaluation of every k.
BatchFn batch_spec_kernel(bool mixed);

// The batched kernel of a form (QED_KERNEL_TABLE or QED_KERNEL_SPECIALISED),
// and the shared memory per team of a plan's points in that form (the
// specialised kernel's own layout where it has one, else the plan's table
// layout); both defined in qed_batch.cu.
BatchFn batch_fn(bool mixed, int form);
int team_bytes_of(const qed_plan_s* P, int form);

// The largest dynamic shared memory a launch of fn may ask for: the device's
// opt-in maximum less the kernel's static shared memory.
inline cudaError_t max_dynamic_smem(const void* fn, int dev_smem, int* out) {
  cudaFuncAttributes fa{};
  const cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  *out = dev_smem - (int)fa.sharedSizeBytes;
  return e;
}

}  // namespace qed
