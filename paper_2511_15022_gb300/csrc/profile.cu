// profile.cu -- CUDA-event timing of every libcgh kernel launch (opt-in) and the launch
// counter.  Events are recorded on the launch's own stream, so the measured duration is
// that kernel's time on the stream that ran it.
#include <cuda_runtime.h>
#include <stdlib.h>

#include "cgh_internal.h"

namespace {
constexpr int kSlots = 65536;
struct Profiler {
  bool enabled = false;
  cudaEvent_t* ev = nullptr;  // 2 per slot
  int* kid = nullptr;
  int used = 0;
  int open = -1;
};
Profiler g_prof;
const char* kNames[KID_COUNT] = {
    "k_preprocess", "k_scan_tiles", "k_emit", "k_raster_fwd", "k_raster_bwd",
    "k_grad_finalize", "k_rows_pad_fwd", "k_cols_fwd_planes", "k_rows_loss",
    "k_cols_bwd_planes", "k_rows_inv_crop", "k_loss_pointwise", "k_loss_finalize", "k_adam",
    "k_encoder", "k_poh", "k_batch_persistent"};
}  // namespace

void prof_begin(int kid, cudaStream_t s) {
  cgh_count_launch(1);
  if (!g_prof.enabled || g_prof.used >= kSlots) return;
  g_prof.open = g_prof.used;
  g_prof.kid[g_prof.used] = kid;
  cudaEventRecord(g_prof.ev[2 * g_prof.used], s);
}

void prof_end(int kid, cudaStream_t s) {
  (void)kid;
  if (!g_prof.enabled || g_prof.open < 0) return;
  cudaEventRecord(g_prof.ev[2 * g_prof.open + 1], s);
  g_prof.used = g_prof.open + 1;
  g_prof.open = -1;
}

extern "C" cgh_status cgh_profile_enable(int32_t enable) {
  if (enable && !g_prof.ev) {
    g_prof.ev = (cudaEvent_t*)calloc(2 * kSlots, sizeof(cudaEvent_t));
    g_prof.kid = (int*)calloc(kSlots, sizeof(int));
    if (!g_prof.ev || !g_prof.kid) return CGH_ERR_ARG;
    for (int i = 0; i < 2 * kSlots; ++i)
      if (cudaEventCreate(&g_prof.ev[i]) != cudaSuccess) return CGH_ERR_CUDA;
  }
  g_prof.enabled = enable != 0;
  g_prof.used = 0;
  g_prof.open = -1;
  return CGH_OK;
}

extern "C" cgh_status cgh_profile_collect(double* total_ms, int64_t* launches) {
  if (!total_ms || !launches) return CGH_ERR_ARG;
  for (int k = 0; k < KID_COUNT; ++k) { total_ms[k] = 0.0; launches[k] = 0; }
  for (int i = 0; i < g_prof.used; ++i) {
    if (cudaEventSynchronize(g_prof.ev[2 * i + 1]) != cudaSuccess) return CGH_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]) != cudaSuccess)
      return CGH_ERR_CUDA;
    total_ms[g_prof.kid[i]] += ms;
    launches[g_prof.kid[i]] += 1;
  }
  g_prof.used = 0;
  g_prof.open = -1;
  return CGH_OK;
}

extern "C" int32_t cgh_kernel_count(void) { return KID_COUNT; }

extern "C" const char* cgh_kernel_name(int32_t id) {
  return (id >= 0 && id < KID_COUNT) ? kNames[id] : "";
}
