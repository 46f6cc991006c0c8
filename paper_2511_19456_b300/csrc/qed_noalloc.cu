// Allocation-free form of the batched evaluation (qed_batch_eval_static).
//
// Some callers cannot allocate device memory at the point where they need an
// evaluation. One example is an application that hands the whole device to
// its own memory pool and forbids foreign cudaMalloc calls. Another is a
// latency-critical serving loop, where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable. For them this entry point runs the
// same persistent batched kernel as qed_batch_eval in its default
// (straight-line) form, but its scratch (the work
// counter, the request table and the work items) lives in a file-scope static
// device array of fixed size. Every GPU that loads the library holds that
// array until the process exits.
//
// In host code the array's name is only a host-side stand-in for the symbol,
// not a device address. Every call obtains its address on the current device
// with cudaGetSymbolAddress (which allocates nothing), so a device reset,
// after which the library's device code is loaded anew, is followed as well.
// The first call on a device may load that code: make it before any stream
// capture. Calls share the array, and a call leaves its contents behind.
// The counter is therefore cleared on the stream before every launch, and
// calls that overlap on the GPU race.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "qed_batch.cuh"
#include "qed_plan.hpp"

using namespace qed;

namespace {

constexpr int kMaxRequests = 256;
constexpr int kMaxItems = 65536;
constexpr size_t kCounterBytes = 256;
constexpr size_t kDescOffset = kCounterBytes;
constexpr size_t kItemsOffset = (kDescOffset + kMaxRequests * sizeof(BatchDesc) + 255) / 256 * 256;
constexpr size_t kScratchBytes = (kItemsOffset + kMaxItems * sizeof(BatchItem) + 255) / 256 * 256;
constexpr int kBlock = 128;

// The scratch: counter, request table, work items.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;                      // guards the host tables below
BatchDesc g_desc[kMaxRequests];
BatchItem g_items[kMaxItems];

}  // namespace

extern "C" qed_status qed_batch_eval_static(const qed_plan_t* plans, int n_req, const long long* n_points,
                                            const double* const* d_momenta, double* const* d_out,
                                            void* stream) {
  if (!plans || !n_points || !d_momenta || !d_out || n_req < 1) return QED_EINVAL;
  if (n_req > kMaxRequests) return QED_EINVAL;   // beyond the static request table
  const bool mixed = plans[0] && plans[0]->prec == QED_MIXED;
  for (int r = 0; r < n_req; ++r) {
    if (!plans[r] || n_points[r] < 0) return QED_EINVAL;
    if ((plans[r]->prec == QED_MIXED) != mixed) return QED_EINVAL;
    if (!plans[r]->summed || plans[r]->k > 5 || plans[r]->rewrite) return QED_EUNSUPPORTED;
    if (n_points[r] > 0 && (!d_momenta[r] || !d_out[r] || ((uintptr_t)d_momenta[r] & 7u) ||
                            ((uintptr_t)d_out[r] & 7u)))
      return QED_EINVAL;
  }
  std::lock_guard<std::mutex> guard(g_lock);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  // the straight-line form, qed_batch_eval's default
  const BatchFn fn = batch_fn(mixed, QED_KERNEL_SPECIALISED);
  int dev_smem = 0, sms = 0;
  e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e);
  // the device address of the array on the current device
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return cuda_status(e);
  unsigned char* base = static_cast<unsigned char*>(p);
  unsigned* d_counter = reinterpret_cast<unsigned*>(base);
  BatchDesc* d_desc = reinterpret_cast<BatchDesc*>(base + kDescOffset);
  BatchItem* d_items = reinterpret_cast<BatchItem*>(base + kItemsOffset);

  // work items of about equal arithmetic, doubled until they fit the table
  size_t smem = 0;
  for (int r = 0; r < n_req; ++r) {
    const int team = 1 << (plans[r]->k + 1);
    smem = std::max(smem, (size_t)(kBlock / team) * team_bytes_of(plans[r], QED_KERNEL_SPECIALISED));
  }
  if (smem + 64 > (size_t)dev_smem) return QED_EUNSUPPORTED;
  double target = 4e8;
  int n_items = 0;
  for (;;) {
    n_items = 0;
    bool fits = true;
    for (int r = 0; r < n_req && fits; ++r) {
      const qed_plan_s* P = plans[r];
      const int tpc = kBlock / (1 << (P->k + 1));
      long long chunk = (long long)(target / (double)std::max<long long>(1, P->sc.flops_algorithmic));
      chunk = std::max<long long>(tpc, (chunk / tpc) * tpc);
      for (long long p0 = 0; p0 < n_points[r]; p0 += chunk) {
        if (n_items == kMaxItems) { fits = false; break; }
        g_items[n_items++] = BatchItem{r, P->k, p0, std::min(n_points[r], p0 + chunk)};
      }
    }
    if (fits) break;
    target *= 2.0;
  }
  std::stable_sort(g_items, g_items + n_items,
                   [](const BatchItem& x, const BatchItem& y) { return x.k > y.k; });
  for (int r = 0; r < n_req; ++r) g_desc[r].kp = make_params(plans[r], d_momenta[r], n_points[r], d_out[r]);

  // the kernel's shared-memory limit at the device's maximum, as
  // qed_batch_create sets it: no call lowers it under a batch's graph
  int limit = 0;
  e = max_dynamic_smem((const void*)fn, dev_smem, &limit);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, kBlock, smem);
  if (e != cudaSuccess) return cuda_status(e);
  if (per_sm < 1) return QED_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  // pageable sources: each copy has consumed its host table when it returns
  e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_desc, g_desc, n_req * sizeof(BatchDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_items > 0)
    e = cudaMemcpyAsync(d_items, g_items, n_items * sizeof(BatchItem), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  fn<<<per_sm * sms, kBlock, smem, st>>>(d_desc, d_items, n_items, d_counter);
  return cuda_status(cudaGetLastError());
}
