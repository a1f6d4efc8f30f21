// persist.cu -- the batched step as one persistent kernel per step.
//
// Every hologram of a batch (any sizes, channel and plane counts) goes through the same
// sequence of phases as cgh_step: clear, preprocess, tile scan, tile emit, raster forward,
// row pass, identity-plane loss, column pass, loss row pass, adjoint column pass, crop row
// pass, raster backward, gradient finalize (+ loss sum).  One cooperative launch runs all
// phases for all holograms: in each phase the CTAs draw work items -- (hologram, Gaussian
// block), (hologram, tile), (hologram, row), (hologram, column) -- from an atomic work queue
// over the concatenated items of every hologram, so small and large holograms share the SMs;
// a grid barrier separates the phases.
//
// The barrier spins with a bounded budget of clock64 cycles (about a second by default):
// a CTA whose wait runs out sets the batch's error word and returns, every other CTA sees
// the word at its next wait and returns too, and the host reads CGH_ERR_TIMEOUT from
// cgh_batch_persistent_status.  No wait is unbounded, so a barrier that can never complete
// (a CTA that does not arrive) ends the kernel instead of hanging the GPU.  A host-set test
// hook makes CTA 0 skip its arrival at one chosen barrier to exercise exactly that path.
//
// Items run the same device functions as the planned kernels: the rasteriser's
// per-Gaussian / per-tile functions (raster.cuh) and the generic runtime-length FFT passes
// with one row or one column per item (blasm_generic.cuh).  (The paper optimises one
// hologram at a time; batching many in one launch is this library's addition.)
#include <cuda_runtime.h>
#include <string.h>

#include <vector>

// Workspace data is written and read within this one launch: every such load goes to L2
// (ld.global.cg), never to an SM's L1 or read-only cache that may hold an earlier phase's
// copy; the grid barrier's fences order the phases.  Only the item functions are taken from
// the headers, not their planned kernels.
#define CGH_ITEMS_ONLY
#define CGH_WS_LOAD(p) __ldcg(p)
#define CGH_RW_LOAD(p) __ldcg(p)
#define CGH_FIELD_LOAD(p) __ldcg(p)
#include "blasm_generic.cuh"
#include "raster.cuh"

namespace cgh {
namespace pst {

enum Phase {
  PH_ZERO = 0, PH_PRE, PH_SCAN, PH_EMIT, PH_RFWD, PH_ROWS, PH_IDENT, PH_COLS, PH_LOSS,
  PH_COLSB, PH_ROWSI, PH_RBWD, PH_FIN, PH_COUNT
};

constexpr int kThreads = 256;
constexpr int kZero = 4096;       // words cleared per item of the clearing phase
constexpr int kPScanChunk = 8192;  // tiles per staged chunk of the per-hologram scan

// One hologram of the batch (device copy).
struct Holo {
  RasterConsts rc;
  int C, N, T, H, Nx;
  cgh_params prm;
  cgh_grads g;
  const float* target;
  float* loss_out;
  float4* rec;
  int4* rect;
  float* raw;
  int* tile_count;
  int* tile_start;
  int* pairs;
  int* status;
  float* partials;
  float2* U0;
  float2* Y;
  float2* V;
  FFTDesc fx, fy;
  int bsx, bsy;               // shared-memory strides of one row / one column transform
  const BlasmDev* bl;         // every plane (identity planes' loss: masks and targets)
  const BlasmDev* blp;        // the propagated planes
  int Lp, ident;
  unsigned ident_mask;
  float gscale;               // 4 / (Ltot C H W)
  double inv_norm;            // 1 / (Ltot C H W)
  int n_partials;             // loss partials: H Lp C rows + H C identity rows
  int zc, zr;                 // clearing items: tile counters, raw moments (+ 1 status item)
};

struct Ctl {
  int nh;
  const Holo* holos;
  const int* offsets;          // [PH_COUNT][nh + 1]: prefix sums of each phase's items
  int* queue;                  // [PH_COUNT] work-queue counters, zero at launch
  unsigned* bar_count;         // CTAs arrived at the current barrier, zero at launch
  unsigned* bar_gen;           // barrier generation (any value at launch)
  int* error;                  // 0: ok; 1: a barrier wait ran out (zero at launch)
  long long spin_budget;       // clock64 cycles one barrier wait may take
  int skip_barrier;            // test hook: CTA 0 does not arrive at this barrier (-1: none)
};

// Grid barrier with a bounded wait.  Returns false when this CTA must stop: its own wait
// ran out, or another CTA's did (the error word is set).
__device__ bool grid_sync(const Ctl& c, int k) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = c.bar_gen;
    volatile int* err = c.error;
    const unsigned g0 = *gen;
    __threadfence();  // this CTA's writes are visible before its arrival
    bool released = false;
    if (!(k == c.skip_barrier && blockIdx.x == 0)) {
      if (atomicAdd(c.bar_count, 1u) + 1u == gridDim.x) {
        atomicExch(c.bar_count, 0u);  // reset before any CTA can arrive at the next barrier
        __threadfence();
        atomicAdd(c.bar_gen, 1u);
        released = true;
      }
    }
    int ok = 1;
    if (!released) {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (*err != 0 || clock64() - t0 > c.spin_budget) {
          atomicExch(c.error, 1);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    if (*err != 0) ok = 0;
    __threadfence();  // the other CTAs' writes before the barrier are visible after it
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int C>
__device__ void rfwd_item(const Holo& h, int t, unsigned char* dsm) {
  float4* srec = reinterpret_cast<float4*>(dsm);
  unsigned char* smask = dsm + sizeof(float4) * 256 * CGH_REC_F4;
  unsigned char(*slist)[256] = reinterpret_cast<unsigned char(*)[256]>(smask + 256);
  raster_fwd_tile<C>(h.rc, h.rec, h.rect, h.tile_start, h.pairs, h.U0, t % h.rc.tiles_x,
                     t / h.rc.tiles_x, srec, smask, slist);
}

template <int C>
__device__ void rbwd_item(const Holo& h, int t, unsigned char* dsm) {
  float4* srec = reinterpret_cast<float4*>(dsm);
  int* sgid = reinterpret_cast<int*>(dsm + sizeof(float4) * 256 * CGH_REC_F4);
  float2(*sdu)[CGH_TILE * CGH_TILE] =
      reinterpret_cast<float2(*)[CGH_TILE * CGH_TILE]>(sgid + 256);
  raster_bwd_tile<C>(h.rc, h.rec, h.rect, h.tile_start, h.pairs, h.U0, h.raw,
                     t % h.rc.tiles_x, t / h.rc.tiles_x, srec, sgid, sdu);
}

template <int MAXB>
__device__ void run_item(int ph, const Holo& h, int i, unsigned char* dsm) {
  const int tid = threadIdx.x;
  float2* sm = reinterpret_cast<float2*>(dsm);
  switch (ph) {
    case PH_ZERO: {
      int* dst;
      long long n, base;
      if (i < h.zc) {
        dst = h.tile_count; n = (long long)h.T * CGH_COUNT_STRIDE; base = (long long)i * kZero;
      } else if (i < h.zc + h.zr) {
        dst = reinterpret_cast<int*>(h.raw); n = (long long)h.N * CGH_RAW_STRIDE;
        base = (long long)(i - h.zc) * kZero;
      } else {
        dst = h.status; n = ST_COUNT; base = 0;
      }
      for (long long k = base + tid; k < n && k < base + kZero; k += kThreads) dst[k] = 0;
      break;
    }
    case PH_PRE: {
      const int n = i * kThreads + tid;
      if (n < h.N) {
        switch (h.C) {
          case 1: preprocess_one<1>(h.rc, h.prm, h.rec, h.rect, h.tile_count, h.status, n); break;
          case 2: preprocess_one<2>(h.rc, h.prm, h.rec, h.rect, h.tile_count, h.status, n); break;
          case 3: preprocess_one<3>(h.rc, h.prm, h.rec, h.rect, h.tile_count, h.status, n); break;
          default: preprocess_one<4>(h.rc, h.prm, h.rec, h.rect, h.tile_count, h.status, n); break;
        }
      }
      break;
    }
    case PH_SCAN: {
      long long* warp_sums = reinterpret_cast<long long*>(dsm);
      int* stage = reinterpret_cast<int*>(dsm + 32 * sizeof(long long));
      scan_tiles_cta(h.T, h.rc.cap, h.tile_count, h.tile_start, h.status, stage, warp_sums,
                     kPScanChunk);
      break;
    }
    case PH_EMIT:
      emit_warp(h.rc, h.rect, h.tile_start, h.tile_count, h.pairs, i * kThreads + tid);
      break;
    case PH_RFWD:
      switch (h.C) {
        case 1: rfwd_item<1>(h, i, dsm); break;
        case 2: rfwd_item<2>(h, i, dsm); break;
        case 3: rfwd_item<3>(h, i, dsm); break;
        default: rfwd_item<4>(h, i, dsm); break;
      }
      break;
    case PH_ROWS:  // item = c * H + y
      rows_pad_fwd_item<MAXB>(*h.blp, h.fx, 1, 1, h.bsx, i / h.H, i % h.H, h.U0, h.Y, sm);
      break;
    case PH_IDENT: {  // item = c * H + y; partials after the loss rows'
      __shared__ float red[32];
      ident_loss_item(*h.bl, h.ident_mask, h.gscale, h.U0, h.target, h.partials,
                      h.n_partials - h.C * h.H + i, 1, i % h.H, i / h.H, red);
      break;
    }
    case PH_COLS:  // item = c * Nx + column
      cols_fwd_planes_item<MAXB>(*h.blp, h.fy, 1, h.bsy, i / h.Nx, i % h.Nx, h.Y, h.V, sm);
      break;
    case PH_LOSS: {  // item = (l C + c) H + y over the propagated planes
      __shared__ float red[32];
      rows_loss_item<MAXB>(*h.blp, h.fx, 1, 1, h.bsx, i / h.H, i % h.H, h.V, h.target,
                           h.partials, i, 1, sm, red);
      break;
    }
    case PH_COLSB:
      cols_bwd_planes_item<MAXB>(*h.blp, h.fy, 1, h.bsy, i / h.Nx, i % h.Nx, h.V, h.Y, sm);
      break;
    case PH_ROWSI:
      rows_inv_crop_item<MAXB>(*h.blp, h.fx, 1, 1, h.bsx, i / h.H, i % h.H, h.Y, h.U0,
                               h.ident, sm);
      break;
    case PH_RBWD:
      switch (h.C) {
        case 1: rbwd_item<1>(h, i, dsm); break;
        case 2: rbwd_item<2>(h, i, dsm); break;
        case 3: rbwd_item<3>(h, i, dsm); break;
        default: rbwd_item<4>(h, i, dsm); break;
      }
      break;
    case PH_FIN: {
      const int nfin = (h.N + kThreads - 1) / kThreads;
      if (i < nfin) {
        const int n = i * kThreads + tid;
        if (n < h.N) {
          switch (h.C) {
            case 1: grad_finalize_one<1>(h.rc, h.prm, h.raw, h.g, nullptr, n); break;
            case 2: grad_finalize_one<2>(h.rc, h.prm, h.raw, h.g, nullptr, n); break;
            case 3: grad_finalize_one<3>(h.rc, h.prm, h.raw, h.g, nullptr, n); break;
            default: grad_finalize_one<4>(h.rc, h.prm, h.raw, h.g, nullptr, n); break;
          }
        }
      } else {  // the loss: sum of the partials in FP64, fixed order
        __shared__ double dred[kThreads / 32];
        double acc = 0.0;
        for (int k = tid; k < h.n_partials; k += kThreads) acc += (double)h.partials[k];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) dred[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
          double t = 0.0;
          for (int w = 0; w < kThreads / 32; ++w) t += dred[w];
          h.loss_out[0] = (float)(t * h.inv_norm);
        }
      }
      break;
    }
    default:
      break;
  }
}

// Copy `bytes` (a multiple of 4) from global to shared memory with the whole CTA.
__device__ __forceinline__ void cta_copy(void* dst, const void* src, int bytes) {
  const int* s = static_cast<const int*>(src);
  int* d = static_cast<int*>(dst);
  for (int k = threadIdx.x; k < bytes / 4; k += blockDim.x) d[k] = __ldcg(&s[k]);
}

template <int MAXB>
__global__ void __launch_bounds__(kThreads) k_batch_persistent(Ctl c) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_item;
  // the current hologram's descriptor and plane maps, staged once per change of hologram so
  // the items read them (sizes, transfer-function constants) from shared memory
  __shared__ Holo s_holo;
  __shared__ BlasmDev s_bl[2];
  int cur = -1;
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    if (ph > 0 && !grid_sync(c, ph - 1)) return;
    const int* off = c.offsets + ph * (c.nh + 1);
    const int total = off[c.nh];
    while (true) {
      if (threadIdx.x == 0) s_item = atomicAdd(&c.queue[ph], 1);
      __syncthreads();
      const int it = s_item;
      __syncthreads();  // every thread has read s_item before thread 0 may replace it
      if (it >= total) break;
      int lo = 0, hi = c.nh - 1;  // the hologram whose items hold `it`
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= it) lo = mid; else hi = mid - 1;
      }
      if (lo != cur) {
        cta_copy(&s_holo, &c.holos[lo], sizeof(Holo));
        cta_copy(&s_bl[0], c.holos[lo].bl, sizeof(BlasmDev));
        cta_copy(&s_bl[1], c.holos[lo].blp, sizeof(BlasmDev));
        __syncthreads();
        if (threadIdx.x == 0) {
          s_holo.bl = &s_bl[0];
          s_holo.blp = &s_bl[1];
        }
        __syncthreads();
        cur = lo;
      }
      run_item<MAXB>(ph, s_holo, it - off[lo], dsm);
      __syncthreads();  // the item's shared memory is free before the next item
    }
  }
}

}  // namespace pst
}  // namespace cgh

using namespace cgh;

// Host side of the persistent step: descriptors built from the batch's plans and bindings.
struct PersistState {
  int device = -1;
  void* dev = nullptr;  // one allocation: control words, queue, offsets, holos, plane maps
  size_t dev_bytes = 0;
  pst::Ctl ctl = {};
  size_t smem = 0;
  int maxb = 1;
  int grid = 0;
  size_t ctl_bytes = 0;  // bytes cleared before each launch (queue, barrier count, error)
  long long spin_budget = 0;
  int skip_barrier = -1;
  bool ready = false;
};

void persist_release(PersistState* ps) {
  if (!ps) return;
  if (ps->dev) cudaFree(ps->dev);
  delete ps;
}

static size_t pad256(size_t x) { return (x + 255) & ~(size_t)255; }

// Builds the descriptors (host) and uploads them once per binding.
cgh_status persist_prepare(PersistState** pps, cgh_plan* const* plans, const cgh_params* prm,
                           const cgh_grads* grads, const float* const* targets,
                           float* const* losses, int nh) {
  using namespace pst;
  PersistState* ps = *pps;
  if (!ps) {
    ps = new (std::nothrow) PersistState();
    if (!ps) return cgh_record_error(CGH_ERR_ARG, "out of host memory");
    *pps = ps;
  }
  if (ps->ready) return CGH_OK;
  std::vector<Holo> holos(nh);
  std::vector<BlasmDev> bls(2 * (size_t)nh);
  std::vector<int> offsets((size_t)PH_COUNT * (nh + 1), 0);
  size_t smem = 0;
  int maxbf = 0;
  for (int i = 0; i < nh; ++i) {
    cgh_plan* p = plans[i];
    if (!p->ws) return cgh_record_error(CGH_ERR_WORKSPACE, "a plan of the batch has no workspace");
    if (prm[i].N > p->max_gaussians) return cgh_record_error(CGH_ERR_CAPACITY, "N exceeds max_gaussians");
    Holo& h = holos[i];
    memset(&h, 0, sizeof(h));
    const int T = p->tiles_x * p->tiles_y;
    h.rc.H = p->H; h.rc.W = p->W; h.rc.C = p->C; h.rc.N = prm[i].N;
    h.rc.tiles_x = p->tiles_x; h.rc.tiles_y = p->tiles_y; h.rc.cutoff = p->cutoff;
    h.rc.cap = p->pair_capacity;
    h.C = p->C; h.N = prm[i].N; h.T = T; h.H = p->H; h.Nx = p->bl.Nx;
    h.prm = prm[i]; h.g = grads[i]; h.target = targets[i]; h.loss_out = losses[i];
    h.rec = (float4*)(p->ws + p->off_rec);
    h.rect = (int4*)(p->ws + p->off_rect);
    h.raw = (float*)(p->ws + p->off_raw);
    h.tile_count = (int*)(p->ws + p->off_tile_count);
    h.tile_start = (int*)(p->ws + p->off_tile_start);
    h.pairs = (int*)(p->ws + p->off_pairs);
    h.status = (int*)(p->ws + p->off_status);
    h.partials = (float*)(p->ws + p->off_loss);
    h.U0 = (float2*)(p->ws + p->off_U0);
    h.Y = (float2*)(p->ws + p->off_Y);
    h.V = (float2*)(p->ws + p->off_V);
    h.fx = p->fx; h.fy = p->fy;
    h.bsx = fft_smem_stride(p->fx.n);
    h.bsy = fft_smem_stride(p->fy.n);
    const bool ident = p->use_ident && p->n_ident > 0;
    bls[2 * i] = p->bl;
    bls[2 * i + 1] = ident ? p->bl_prop : p->bl;
    h.Lp = bls[2 * i + 1].L;
    h.ident = ident ? 1 : 0;
    h.ident_mask = ident ? p->ident_mask : 0u;
    const double norm = (double)p->L * p->C * p->H * p->W;
    h.gscale = (float)(4.0 / norm);
    h.inv_norm = 1.0 / norm;
    h.n_partials = p->H * h.Lp * p->C + (ident ? p->H * p->C : 0);
    if (h.n_partials > p->loss_slots)
      return cgh_record_error(CGH_ERR_WORKSPACE, "loss partials exceed the plan's slots");
    h.zc = (int)(((long long)T * CGH_COUNT_STRIDE + kZero - 1) / kZero);
    h.zr = (int)(((long long)h.N * CGH_RAW_STRIDE + kZero - 1) / kZero);
    const int nblk = (h.N + kThreads - 1) / kThreads;
    const int items[PH_COUNT] = {
        h.zc + h.zr + 1, nblk, 1, nblk, T,
        h.Lp > 0 ? p->H * p->C : 0,
        ident ? p->H * p->C : 0,
        h.Lp > 0 ? h.Nx * p->C : 0,
        p->H * h.Lp * p->C,
        h.Lp > 0 ? h.Nx * p->C : 0,
        h.Lp > 0 ? p->H * p->C : 0,
        T, nblk + 1};
    for (int ph = 0; ph < PH_COUNT; ++ph)
      offsets[(size_t)ph * (nh + 1) + i + 1] = offsets[(size_t)ph * (nh + 1) + i] + items[ph];
    // shared memory of the largest item, butterflies per thread of the longest pass
    const size_t rast = sizeof(float4) * 256 * CGH_REC_F4 + 256 + 8 * 256 + 256 * sizeof(int) +
                        sizeof(float2) * CGH_MAX_C * CGH_TILE * CGH_TILE;
    const size_t scan = 32 * sizeof(long long) + sizeof(int) * ((size_t)kPScanChunk + kPScanChunk / 32 + 1);
    const size_t rows = sizeof(float2) * (size_t)h.bsx;
    const size_t cols = sizeof(float2) * (size_t)h.bsy * 2;
    for (size_t v : {rast, scan, rows, cols}) smem = v > smem ? v : smem;
    for (const FFTDesc* d : {&p->fx, &p->fy})
      for (int q = 0; q < d->npass; ++q) maxbf = d->n / d->radix[q] > maxbf ? d->n / d->radix[q] : maxbf;
    p->bin_valid = 0;  // the persistent step rebins in this plan's workspace
  }
  const int maxb = (maxbf + kThreads - 1) / kThreads;
  if (maxb > 2)
    return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE,
                            "persistent step: a transform pass needs more than 2 butterflies per thread");
  smem = pad256(smem);
  // device layout: [queue PH_COUNT][bar_count][error] | bar_gen | offsets | holos | plane maps
  const size_t ctl_bytes = sizeof(int) * (PH_COUNT + 2);
  const size_t o_gen = pad256(ctl_bytes);
  const size_t o_off = o_gen + 256;
  const size_t o_holo = o_off + pad256(sizeof(int) * offsets.size());
  const size_t o_bl = o_holo + pad256(sizeof(Holo) * nh);
  const size_t total = o_bl + sizeof(BlasmDev) * bls.size();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (!ps->dev || ps->dev_bytes < total || ps->device != dev)) {
    if (ps->dev) cudaFree(ps->dev);
    ps->dev = nullptr;
    e = cudaMalloc(&ps->dev, total);
    ps->dev_bytes = total;
    ps->device = dev;
  }
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  char* base = (char*)ps->dev;
  for (int i = 0; i < nh; ++i) {  // plane maps referenced by device address
    holos[i].bl = (const BlasmDev*)(base + o_bl) + 2 * i;
    holos[i].blp = (const BlasmDev*)(base + o_bl) + 2 * i + 1;
  }
  e = cudaMemcpy(base + o_off, offsets.data(), sizeof(int) * offsets.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + o_holo, holos.data(), sizeof(Holo) * nh, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + o_bl, bls.data(), sizeof(BlasmDev) * bls.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(base, 0, o_gen + 256);
  // co-resident grid for the cooperative launch
  int sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void (*kern)(Ctl) = maxb == 1 ? k_batch_persistent<1> : k_batch_persistent<2>;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  if (per_sm < 1) return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE, "persistent step does not fit an SM");
  if (ps->spin_budget <= 0) {
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    ps->spin_budget = (long long)(khz > 0 ? khz : 2000000) * 1000LL;  // about one second
  }
  Ctl& c = ps->ctl;
  c.nh = nh;
  c.holos = (const Holo*)(base + o_holo);
  c.offsets = (const int*)(base + o_off);
  c.queue = (int*)base;
  c.bar_count = (unsigned*)(base + sizeof(int) * PH_COUNT);
  c.error = (int*)(base + sizeof(int) * (PH_COUNT + 1));
  c.bar_gen = (unsigned*)(base + o_gen);
  ps->ctl_bytes = ctl_bytes;
  ps->smem = smem;
  ps->maxb = maxb;
  ps->grid = sms * per_sm;
  ps->ready = true;
  return CGH_OK;
}

void persist_invalidate(PersistState* ps) {
  if (ps) ps->ready = false;
}

cgh_status persist_launch(PersistState* ps, cudaStream_t s) {
  using namespace pst;
  if (!ps || !ps->ready) return cgh_record_error(CGH_ERR_ARG, "persistent step not prepared");
  cudaError_t e = cudaMemsetAsync(ps->dev, 0, ps->ctl_bytes, s);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  Ctl c = ps->ctl;
  c.spin_budget = ps->spin_budget;
  c.skip_barrier = ps->skip_barrier;
  void* args[] = {&c};
  void (*kern)(Ctl) = ps->maxb == 1 ? k_batch_persistent<1> : k_batch_persistent<2>;
  prof_begin(KID_PERSIST, s);
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(ps->grid), dim3(kThreads), args, ps->smem, s);
  prof_end(KID_PERSIST, s);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  return CGH_OK;
}

cgh_status persist_status(PersistState* ps, int32_t* timed_out, cudaStream_t s) {
  int err = 0;
  if (ps && ps->ready) {
    cudaError_t e = cudaMemcpyAsync(&err, ps->ctl.error, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  }
  if (timed_out) *timed_out = err;
  return err ? cgh_record_error(CGH_ERR_TIMEOUT, "a grid barrier of the persistent step timed out")
             : CGH_OK;
}

void persist_set_test(PersistState* ps, int skip_barrier, long long budget) {
  if (!ps) return;
  ps->skip_barrier = skip_barrier;
  if (budget > 0) ps->spin_budget = budget;
  else ps->spin_budget = 0, ps->ready = false;  // default budget recomputed at prepare
}

int persist_grid(const PersistState* ps) { return ps && ps->ready ? ps->grid : 0; }
