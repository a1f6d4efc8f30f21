// noalloc.cu -- forward rasterisation for callers that cannot allocate device memory.
//
// cgh_raster_fwd needs a plan and a caller-provided workspace for its binning scratch
// (per-Gaussian records, per-tile counts and starts, the (Gaussian, tile) lists).  Some
// callers cannot provide either: an application that reserves all device memory at start-up
// and forbids later allocations, or a latency-critical loop where cudaMalloc's implicit
// device-wide synchronisation is not acceptable.  This entry point keeps that scratch in a
// fixed file-scope device array instead, so it allocates nothing; the caller still passes
// the parameters and the output field.  The array stays resident on every device that
// loads the library until the process exits.
#include <cuda_runtime.h>
#include <stdio.h>

#include "cgh_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB per device
constexpr int kMaxGaussians = 65536;
constexpr int kMaxTiles = 16384;                    // e.g. 2048 x 2048 pixels in 16x16 tiles
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device (host code cannot use the
// symbol itself as a device pointer).
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" cgh_status cgh_raster_fwd_noalloc(int32_t H, int32_t W, int32_t C, float cutoff,
                                             const cgh_params* params, void* U_out,
                                             void* stream) {
  if (!params || !U_out) return cgh_record_error(CGH_ERR_ARG, "NULL argument");
  if (H < 1 || W < 1) return cgh_record_error(CGH_ERR_ARG, "H and W must be >= 1");
  if (C < 1 || C > CGH_MAX_C) return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE, "C must be 1..4");
  if (!(cutoff >= 0.f) || !(cutoff < 0.99f))
    return cgh_record_error(CGH_ERR_ARG, "cutoff must be in [0, 0.99)");
  if (params->N < 0) return cgh_record_error(CGH_ERR_ARG, "N must be >= 0");
  if (params->N > kMaxGaussians)
    return cgh_record_error(CGH_ERR_CAPACITY,
                            "cgh_raster_fwd_noalloc: N exceeds the fixed scratch limit of 65536");
  if (params->N > 0 && (!params->xy_raw || !params->s_raw || !params->theta || !params->amp ||
                        !params->phase || !params->alpha_raw))
    return cgh_record_error(CGH_ERR_ARG, "NULL parameter array");
  const int tiles_x = (W + CGH_TILE - 1) / CGH_TILE, tiles_y = (H + CGH_TILE - 1) / CGH_TILE;
  if ((long long)tiles_x * tiles_y > kMaxTiles)
    return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE,
                            "cgh_raster_fwd_noalloc: more than 16384 16x16 tiles");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return cgh_record_error(CGH_ERR_ARG, "device index too large");
  if (!g_scratch_addr[dev]) {  // first call on this device: look up the array's address
    void* addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_scratch);
    if (e != cudaSuccess || !addr)
      return cgh_record_error(CGH_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                             : "scratch address is NULL");
    g_scratch_addr[dev] = addr;
  }

  // A plan-shaped view of the scratch for the shared raster launcher: same carve-up as a
  // plan's workspace, the (Gaussian, tile) list takes whatever space is left.
  cgh_plan view = {};
  view.H = H; view.W = W; view.C = C; view.L = 1; view.pad = 1;
  view.cutoff = cutoff;
  view.max_gaussians = kMaxGaussians;
  view.tiles_x = tiles_x; view.tiles_y = tiles_y;
  const size_t N = (size_t)kMaxGaussians, T = (size_t)kMaxTiles;
  size_t o = 0;
  view.off_rec = o;        o = align256(o + N * CGH_REC_F4 * sizeof(float4));
  view.off_rect = o;       o = align256(o + N * sizeof(int4));
  view.off_raw = o;        // unused by the forward pass
  view.off_tile_count = o; o = align256(o + T * CGH_COUNT_STRIDE * sizeof(int));
  view.off_tile_start = o; o = align256(o + (T + 1) * sizeof(int));
  view.off_status = o;     o = align256(o + ST_COUNT * sizeof(int));
  view.off_pairs = o;
  view.pair_capacity = (int64_t)((kScratchBytes - o) / sizeof(int));
  view.ws = (char*)g_scratch_addr[dev];
  view.ws_bytes = kScratchBytes;

  e = launch_raster_fwd(&view, params, (float2*)U_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  return CGH_OK;
}
