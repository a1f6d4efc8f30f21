// batch.cu -- many holograms per step, and the block-shape autotuner.
//
// cgh_batch: a set of plans (one per hologram, any sizes) whose fused steps are captured
// once into a single CUDA graph -- one branch per hologram, forked from and joined back to
// one origin stream -- and replayed with one cudaGraphLaunch per step.  Independent
// branches let the small holograms' kernels fill the SMs that a large hologram leaves idle,
// and the per-kernel launch cost is paid once at capture.  (The paper optimises one
// hologram at a time; batching is this library's addition.)  The sequential mode issues the
// same steps one after another on the caller's stream, as separate launches.
//
// cgh_autotune: times cgh_step for every valid (column block, row block, FFT kernel family)
// on the caller's data and keeps the fastest.
//
// cgh_adam_step_table: Adam over any number of parameter groups described by a device
// table, in one launch (the per-hologram groups of a whole batch).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "cgh_internal.h"

struct cgh_batch {
  std::vector<cgh_plan*> plans;
  std::vector<cgh_params> params;
  std::vector<cgh_grads> grads;
  std::vector<const float*> targets;
  std::vector<float*> losses;
  std::vector<char> bound;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches_per_replay = 0;
  PersistState* persist = nullptr;  // the persistent step's descriptors (persist.cu)
};

static void batch_release_graph(cgh_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

extern "C" cgh_status cgh_batch_create(cgh_plan* const* plans, int32_t count, cgh_batch** out) {
  if (!plans || !out || count < 1) return cgh_record_error(CGH_ERR_ARG, "plans/out NULL or count < 1");
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return cgh_record_error(CGH_ERR_ARG, "NULL plan in batch");
  cgh_batch* b = new (std::nothrow) cgh_batch();
  if (!b) return cgh_record_error(CGH_ERR_ARG, "out of host memory");
  b->plans.assign(plans, plans + count);
  b->params.resize(count);
  b->grads.resize(count);
  b->targets.assign(count, nullptr);
  b->losses.assign(count, nullptr);
  b->bound.assign(count, 0);
  b->streams.assign(count, nullptr);
  b->done.assign(count, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cgh_batch_destroy(b);
    return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = b;
  return CGH_OK;
}

extern "C" cgh_status cgh_batch_destroy(cgh_batch* b) {
  if (!b) return CGH_OK;
  batch_release_graph(b);
  persist_release(b->persist);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto ev : b->done)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
  return CGH_OK;
}

extern "C" cgh_status cgh_batch_bind(cgh_batch* b, int32_t i, const cgh_params* params,
                                     const float* target, float* loss_out,
                                     const cgh_grads* grads) {
  if (!b || i < 0 || i >= (int)b->plans.size()) return cgh_record_error(CGH_ERR_ARG, "bad batch index");
  if (!params || !target || !loss_out || !grads) return cgh_record_error(CGH_ERR_ARG, "NULL argument");
  b->params[i] = *params;
  b->grads[i] = *grads;
  b->targets[i] = target;
  b->losses[i] = loss_out;
  b->bound[i] = 1;
  batch_release_graph(b);  // pointers changed: capture again on the next graph step
  persist_invalidate(b->persist);  // ... and rebuild the persistent step's descriptors
  return CGH_OK;
}

static cgh_status batch_issue(cgh_batch* b, cudaStream_t origin, bool branches) {
  const int n = (int)b->plans.size();
  if (branches) {
    cudaError_t e = cudaEventRecord(b->fork, origin);
    if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  }
  for (int i = 0; i < n; ++i) {
    cudaStream_t s = origin;
    if (branches) {
      s = b->streams[i];
      cudaError_t e = cudaStreamWaitEvent(s, b->fork, 0);
      if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
    }
    cgh_status st = cgh_step(b->plans[i], &b->params[i], b->targets[i], b->losses[i],
                             &b->grads[i], (void*)s);
    if (st != CGH_OK) return st;
    if (branches) {
      cudaError_t e = cudaEventRecord(b->done[i], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, b->done[i], 0);
      if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  return CGH_OK;
}

extern "C" cgh_status cgh_batch_step(cgh_batch* b, int32_t use_graph, void* stream) {
  if (!b) return cgh_record_error(CGH_ERR_ARG, "batch is NULL");
  for (char x : b->bound)
    if (!x) return cgh_record_error(CGH_ERR_ARG, "every hologram must be bound (cgh_batch_bind)");
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return batch_issue(b, s, false);
  if (!b->exec) {
    // capture on the batch's own origin stream (the caller's stream may be the legacy
    // default stream, which cannot be captured), then replay on the caller's stream
    const long long before = cgh_launch_count();
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
    cgh_status st = batch_issue(b, b->origin, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->origin, &g);
    if (st != CGH_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      batch_release_graph(b);
      return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
    }
    b->launches_per_replay = cgh_launch_count() - before;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  return CGH_OK;
}

extern "C" int64_t cgh_batch_kernels_per_step(const cgh_batch* b) {
  return b ? b->launches_per_replay : 0;
}

extern "C" cgh_status cgh_batch_step_persistent(cgh_batch* b, void* stream) {
  if (!b) return cgh_record_error(CGH_ERR_ARG, "batch is NULL");
  for (char x : b->bound)
    if (!x) return cgh_record_error(CGH_ERR_ARG, "every hologram must be bound (cgh_batch_bind)");
  cgh_status st = persist_prepare(&b->persist, b->plans.data(), b->params.data(), b->grads.data(),
                                  b->targets.data(), b->losses.data(), (int)b->plans.size());
  if (st != CGH_OK) return st;
  return persist_launch(b->persist, (cudaStream_t)stream);
}

extern "C" cgh_status cgh_batch_persistent_status(cgh_batch* b, int32_t* timed_out, void* stream) {
  if (!b) return cgh_record_error(CGH_ERR_ARG, "batch is NULL");
  return persist_status(b->persist, timed_out, (cudaStream_t)stream);
}

extern "C" cgh_status cgh_batch_persistent_test(cgh_batch* b, int32_t skip_barrier,
                                                double timeout_s) {
  if (!b) return cgh_record_error(CGH_ERR_ARG, "batch is NULL");
  if (!b->persist) {
    cgh_status st = persist_prepare(&b->persist, b->plans.data(), b->params.data(),
                                    b->grads.data(), b->targets.data(), b->losses.data(),
                                    (int)b->plans.size());
    if (st != CGH_OK) return st;
  }
  long long budget = 0;
  if (timeout_s > 0.0) {
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    budget = (long long)(timeout_s * (khz > 0 ? khz : 2000000) * 1000.0);
    if (budget < 1) budget = 1;
  }
  persist_set_test(b->persist, skip_barrier, budget);
  return CGH_OK;
}

extern "C" int32_t cgh_batch_persistent_grid(const cgh_batch* b) {
  return b ? persist_grid(b->persist) : 0;
}

// ------------------------------------------------------------------ autotuner
extern "C" cgh_status cgh_autotune(cgh_plan* plan, const cgh_params* params, const float* target,
                                   const cgh_grads* grads, float* loss_out, int32_t iters,
                                   void* stream, cgh_tuning* best_out) {
  if (!plan || !params || !target || !grads || !loss_out)
    return cgh_record_error(CGH_ERR_ARG, "NULL argument");
  if (iters < 1) iters = 1;
  cudaStream_t s = (cudaStream_t)stream;
  cgh_tuning orig;
  cgh_plan_get_tuning(plan, &orig);
  static const int cbs[] = {1, 2, 4, 8};
  static const int rbs[] = {1, 2, 3, 4, 8};
  static const int kinds[] = {1, 2};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cgh_record_error(CGH_ERR_CUDA, "event creation failed");
  float best_ms = 1e30f;
  cgh_tuning best = orig;
  for (int kind : kinds)
    for (int cb : cbs)
      for (int rb : rbs) {
        cgh_tuning t = orig;
        t.col_block = cb;
        t.row_block = rb;
        t.fft_kernels = kind;
        t.pair_capacity_per_gaussian = 0;
        if (cgh_plan_set_tuning(plan, &t) != CGH_OK) continue;
        // warm-up (also sets kernel attributes), then time
        if (cgh_step(plan, params, target, loss_out, grads, s) != CGH_OK) continue;
        cudaEventRecord(e0, s);
        bool ok = true;
        for (int i = 0; i < iters && ok; ++i)
          ok = cgh_step(plan, params, target, loss_out, grads, s) == CGH_OK;
        cudaEventRecord(e1, s);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          cgh_plan_get_tuning(plan, &best);
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  best.pair_capacity_per_gaussian = 0;
  cgh_plan_set_tuning(plan, &best);
  if (best_out) cgh_plan_get_tuning(plan, best_out);
  return best_ms < 1e29f ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, "no tuning candidate ran");
}

// ------------------------------------------------------------------ table-driven Adam
namespace {
__global__ void k_adam_table(const cgh_adam_group* __restrict__ groups,
                             const long long* __restrict__ offsets, int ngroups, long long total,
                             float bc1, float inv_sqrt_bc2, float b1, float b2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = ngroups - 1;  // group with offsets[g] <= i < offsets[g + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const cgh_adam_group& gr = groups[lo];
    const long long j = i - offsets[lo];
    const float g = gr.grad[j];
    const float m = fmaf(b1, gr.exp_avg[j], (1.f - b1) * g);
    const float v = fmaf(b2, gr.exp_avg_sq[j], (1.f - b2) * g * g);
    gr.exp_avg[j] = m;
    gr.exp_avg_sq[j] = v;
    gr.param[j] -= (gr.lr / bc1) * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
  }
}
}  // namespace

extern "C" cgh_status cgh_adam_step_table(const cgh_adam_group* groups_dev,
                                          const int64_t* offsets_dev, int32_t num_groups,
                                          int64_t total, int32_t step, float beta1,
                                          float beta2, float eps, float lr_scale, void* stream) {
  if (!groups_dev || !offsets_dev || num_groups < 1 || total < 0 || step < 1 || !(lr_scale >= 0.f))
    return cgh_record_error(CGH_ERR_ARG, "bad Adam table arguments");
  // the learning-rate scale is folded into the first-moment bias correction (lr / bc1)
  const double bc1 = (1.0 - pow((double)beta1, (double)step)) / (lr_scale > 0.f ? lr_scale : 1.0);
  if (lr_scale == 0.f) return CGH_OK;
  const double bc2 = 1.0 - pow((double)beta2, (double)step);
  if (total == 0) return CGH_OK;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ADAM, s);
  k_adam_table<<<(unsigned)blocks, 256, 0, s>>>(groups_dev, (const long long*)offsets_dev,
                                                 num_groups, (long long)total, (float)bc1,
                                                 (float)(1.0 / sqrt(bc2)), beta1, beta2, eps);
  prof_end(KID_ADAM, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
}
