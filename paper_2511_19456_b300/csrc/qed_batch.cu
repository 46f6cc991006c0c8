// Batched evaluation: requests of different k (spin-summed, k = 1..5) with
// uneven point counts in ONE persistent launch.
//
// The host cuts every request into work items (request, point range), sized
// so that items carry about the same arithmetic, and orders them most
// expensive k first.  Persistent CTAs take items from a device counter
// (atomicAdd; no CTA ever waits on another) and evaluate the item's points
// with teams of the item's k (eval_range, the same code as the standalone
// forward kernel).  A counter reset plus the launch are captured once in a
// CUDA graph and replayed; per call only the request table (device pointers
// of momenta and outputs) is copied.  Two kernel forms, as for a plan: the
// table-driven point evaluation for every k, or the straight-line
// specialised one (generated at build time).  qed_batch_tune times every form, block size and item size
// of a small grid on the caller's buffers and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "qed_batch.cuh"
#include "qed_plan.hpp"

using namespace qed;

struct qed_batch_s {
  std::vector<qed_plan_t> plans;
  std::vector<long long> n;
  bool mixed = false;
  int form = QED_KERNEL_SPECIALISED;   // qed_kernel_form of the batched kernel
  int block = 128;
  double work_target = 4e8;      // algorithmic FLOPs per item
  std::vector<BatchDesc> h_desc;
  std::vector<BatchItem> h_items;
  BatchDesc* d_desc = nullptr;
  BatchItem* d_items = nullptr;
  size_t items_cap = 0;
  unsigned* d_counter = nullptr;
  size_t smem = 0;
  int grid = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace qed {

BatchFn batch_fn(bool mixed, int form) {
  if (form == QED_KERNEL_SPECIALISED) return batch_spec_kernel(mixed);
  return mixed ? qed_batch_kernel<float> : qed_batch_kernel<double>;
}

// Shared memory per team of a request's points in a form: the specialised
// kernel's own layout where it has one, else the plan's table kernel layout.
int team_bytes_of(const qed_plan_s* P, int form) {
  if (form == QED_KERNEL_SPECIALISED) {
    const SpecKernel sk = spec_forward_kernel(P->k, P->prec == QED_MIXED);
    if (sk.fn) return sk.team_bytes;
  }
  return P->team_bytes;
}

}  // namespace qed

namespace {

constexpr int kMaxBatchK = 5;

void destroy_graph(qed_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void free_batch(qed_batch_s* b) {
  if (!b) return;
  destroy_graph(b);
  cudaFree(b->d_desc);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// Work list, launch shape and graph for the current (block, work_target).
qed_status configure(qed_batch_s* b) {
  const int nreq = (int)b->plans.size();
  b->h_items.clear();
  size_t smem = 0;
  for (int r = 0; r < nreq; ++r) {
    const qed_plan_s* P = b->plans[r];
    const int team = 1 << (P->k + 1);
    if (b->block < team) return QED_EINVAL;
    const int tpc = b->block / team;
    smem = std::max(smem, (size_t)tpc * team_bytes_of(P, b->form));
    const double fl = (double)std::max<long long>(1, P->sc.flops_algorithmic);
    long long chunk = (long long)(b->work_target / fl);
    chunk = std::max<long long>(tpc, (chunk / tpc) * tpc);
    for (long long p0 = 0; p0 < b->n[r]; p0 += chunk)
      b->h_items.push_back(BatchItem{r, P->k, p0, std::min(b->n[r], p0 + chunk)});
  }
  std::stable_sort(b->h_items.begin(), b->h_items.end(),
                   [](const BatchItem& x, const BatchItem& y) { return x.k > y.k; });
  int dev_smem = 0, sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (smem + 64 > (size_t)dev_smem) return QED_EUNSUPPORTED;
  BatchFn fn = batch_fn(b->mixed, b->form);
  // the limit at the device's maximum, for every batch and for
  // qed_batch_eval_static alike: none of them lowers it under another's graph
  int limit = 0;
  e = max_dynamic_smem((const void*)fn, dev_smem, &limit);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, b->block, smem);
  if (e != cudaSuccess) return cuda_status(e);
  if (per_sm < 1) return QED_EUNSUPPORTED;
  b->smem = smem;
  b->grid = per_sm * sms;
  if (b->h_items.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    e = device_alloc((void**)&b->d_items, b->h_items.size() * sizeof(BatchItem));
    if (e != cudaSuccess) return cuda_status(e);
    b->items_cap = b->h_items.size();
  }
  if (!b->h_items.empty())
    e = cudaMemcpy(b->d_items, b->h_items.data(), b->h_items.size() * sizeof(BatchItem),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  // graph: counter reset + the persistent launch
  destroy_graph(b);
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), b->cap);
  fn<<<b->grid, b->block, b->smem, b->cap>>>(b->d_desc, b->d_items, (int)b->h_items.size(),
                                              b->d_counter);
  e = cudaStreamEndCapture(b->cap, &b->graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  return cuda_status(e);
}

qed_status set_pointers(qed_batch_s* b, const double* const* d_momenta, double* const* d_out) {
  if (!d_momenta || !d_out) return QED_EINVAL;
  for (size_t r = 0; r < b->plans.size(); ++r) {
    if (b->n[r] > 0 && (!d_momenta[r] || !d_out[r] || ((uintptr_t)d_momenta[r] & 7u) ||
                        ((uintptr_t)d_out[r] & 7u)))
      return QED_EINVAL;
    b->h_desc[r].kp.mom = d_momenta[r];
    b->h_desc[r].kp.out = d_out[r];
  }
  return QED_OK;
}

}  // namespace

extern "C" {

qed_status qed_batch_create(const qed_plan_t* plans, int n_req, const long long* n_points,
                            qed_batch_t* out) {
  if (!plans || !n_points || !out || n_req < 1) return QED_EINVAL;
  const bool mixed = plans[0] && plans[0]->prec == QED_MIXED;
  for (int r = 0; r < n_req; ++r) {
    if (!plans[r] || n_points[r] < 0) return QED_EINVAL;
    if ((plans[r]->prec == QED_MIXED) != mixed) return QED_EINVAL;
    if (!plans[r]->summed || plans[r]->k > kMaxBatchK || plans[r]->rewrite) return QED_EUNSUPPORTED;
  }
  qed_batch_s* b = new (std::nothrow) qed_batch_s();
  if (!b) return QED_ENOMEM;
  b->plans.assign(plans, plans + n_req);
  b->n.assign(n_points, n_points + n_req);
  b->mixed = mixed;
  b->h_desc.resize(n_req);
  for (int r = 0; r < n_req; ++r) b->h_desc[r].kp = make_params(plans[r], nullptr, n_points[r], nullptr);
  cudaError_t e = device_alloc((void**)&b->d_desc, n_req * sizeof(BatchDesc));
  if (e == cudaSuccess) e = device_alloc((void**)&b->d_counter, 256);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) { free_batch(b); return cuda_status(e); }
  qed_status s = configure(b);
  if (s != QED_OK) { free_batch(b); return s; }
  *out = b;
  return QED_OK;
}

qed_status qed_batch_eval(qed_batch_t b, const double* const* d_momenta, double* const* d_out,
                          void* stream) {
  if (!b) return QED_EINVAL;
  qed_status s = set_pointers(b, d_momenta, d_out);
  if (s != QED_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc.data(), b->h_desc.size() * sizeof(BatchDesc),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
  return cuda_status(e);
}

qed_status qed_batch_tune(qed_batch_t b, const double* const* d_momenta, double* const* d_out,
                          void* stream, double* best_ms) {
  if (!b) return QED_EINVAL;
  qed_status s = set_pointers(b, d_momenta, d_out);
  if (s != QED_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QED_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return QED_ECUDA; }
  const int blocks[] = {64, 128, 256};
  const double targets[] = {1e8, 4e8, 1.6e9};
  int best_block = b->block, best_form = b->form;
  double best_target = b->work_target, best = 1e300;
  for (int form : {QED_KERNEL_TABLE, QED_KERNEL_SPECIALISED})
  for (int blk : blocks) {
    for (double tgt : targets) {
      b->form = form;
      b->block = blk;
      b->work_target = tgt;
      if (configure(b) != QED_OK) continue;
      cudaMemcpyAsync(b->d_desc, b->h_desc.data(), b->h_desc.size() * sizeof(BatchDesc),
                      cudaMemcpyHostToDevice, st);
      cudaGraphLaunch(b->exec, st);   // warm-up
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 2; ++rep) cudaGraphLaunch(b->exec, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 2 < best) { best = ms / 2; best_block = blk; best_target = tgt; best_form = form; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->form = best_form;
  b->block = best_block;
  b->work_target = best_target;
  s = configure(b);
  if (s == QED_OK && best_ms) *best_ms = best;
  if (s == QED_OK && cudaGetLastError() != cudaSuccess) s = QED_ECUDA;
  return s;
}

qed_status qed_batch_info(qed_batch_t b, int* block, double* work_target, long long* n_items) {
  if (!b) return QED_EINVAL;
  if (block) *block = b->block;
  if (work_target) *work_target = b->work_target;
  if (n_items) *n_items = (long long)b->h_items.size();
  return QED_OK;
}

qed_status qed_batch_set_kernel_form(qed_batch_t b, int form) {
  if (!b || (form != QED_KERNEL_TABLE && form != QED_KERNEL_SPECIALISED)) return QED_EINVAL;
  const int old = b->form;
  b->form = form;
  qed_status s = configure(b);
  if (s != QED_OK) {
    b->form = old;
    configure(b);
  }
  return s;
}

qed_status qed_batch_kernel_form(qed_batch_t b, int* form) {
  if (!b || !form) return QED_EINVAL;
  *form = b->form;
  return QED_OK;
}

void qed_batch_destroy(qed_batch_t b) { free_batch(b); }

}  // extern "C"
