// api.cu -- C ABI of libcgh (declared in include/cgh.h): plan construction, workspace
// layout, the entry points that sequence the kernels of raster.cu and blasm.cu, and the
// fused multi-group Adam update.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "blasm_spec.h"
#include "cgh_internal.h"

static thread_local char g_err[512] = "";
// process-wide: autograd runs backward passes on its own thread, and their launches count
static std::atomic<long long> g_launches{0};

void cgh_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static cgh_status fail(cgh_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

cgh_status cgh_record_error(cgh_status st, const char* msg) { return fail(st, "%s", msg); }

static cgh_status cuda_fail(cudaError_t e, const char* where) {
  return fail(CGH_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CGH_TRY(expr, where)                         \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

// ------------------------------------------------------------------ plan construction
// Radices with register codelets (fft.cuh).  A length is split into passes by exhaustive
// search: fewest passes first, then the largest smallest radix (fewest butterflies per
// pass), then the smallest largest radix (fewest registers).
static const int kRadixSet[] = {24, 20, 16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

static void search(int m, int depth, int* cur, int* best, int* best_n, int max_depth) {
  if (m == 1) {
    auto score = [](const int* r, int n, long long* a, long long* b, long long* c) {
      int mn = 1 << 30, mx = 0;
      for (int i = 0; i < n; ++i) { mn = r[i] < mn ? r[i] : mn; mx = r[i] > mx ? r[i] : mx; }
      *a = n; *b = -mn; *c = mx;
    };
    long long a0, b0, c0, a1, b1, c1;
    score(cur, depth, &a0, &b0, &c0);
    if (*best_n > 0) {
      score(best, *best_n, &a1, &b1, &c1);
      if (a0 > a1 || (a0 == a1 && (b0 > b1 || (b0 == b1 && c0 >= c1)))) return;
    }
    for (int i = 0; i < depth; ++i) best[i] = cur[i];
    *best_n = depth;
    return;
  }
  if (depth >= max_depth) return;
  for (int r : kRadixSet) {
    if (m % r) continue;
    if (depth > 0 && r > cur[depth - 1]) continue;  // non-increasing order: no duplicates
    cur[depth] = r;
    search(m / r, depth + 1, cur, best, best_n, max_depth);
  }
}

static bool factorise(int n, FFTDesc* d) {
  d->n = n;
  d->npass = 0;
  if (n == 1) return true;
  int cur[CGH_MAX_PASSES], best[CGH_MAX_PASSES], best_n = 0;
  search(n, 0, cur, best, &best_n, CGH_MAX_PASSES);
  if (best_n == 0) return false;
  for (int i = 0; i < best_n; ++i) d->radix[i] = best[i];
  d->npass = best_n;
  return true;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void layout(cgh_plan* p) {
  const size_t N = (size_t)(p->max_gaussians > 0 ? p->max_gaussians : 1);
  const size_t T = (size_t)p->tiles_x * p->tiles_y;
  p->pair_capacity = (int64_t)p->pair_cap_mult * (int64_t)N + 256;
  if (p->pair_capacity > 0x7fffffffLL) p->pair_capacity = 0x7fffffffLL;
  const size_t HW = (size_t)p->H * p->W;
  const size_t half = (size_t)p->H * p->bl.Nx;
  // loss partials: one per CTA of the loss row pass (at most H L C), plus those of the
  // identity planes' pass: one per tile (fused into the forward raster) or one per row and
  // channel (the persistent batched step)
  p->loss_slots = p->H * p->L * p->C + p->H * p->C + (int)T + 1024;
  size_t o = 0;
  p->off_rec = o;        o = align256(o + N * CGH_REC_F4 * sizeof(float4));
  p->off_rect = o;       o = align256(o + N * sizeof(int4));
  p->off_raw = o;        o = align256(o + N * CGH_RAW_STRIDE * sizeof(float));
  p->off_tile_count = o; o = align256(o + T * CGH_COUNT_STRIDE * sizeof(int));
  p->off_tile_start = o; o = align256(o + (T + 1) * sizeof(int));
  p->off_pairs = o;      o = align256(o + (size_t)p->pair_capacity * sizeof(int));
  p->off_status = o;     o = align256(o + ST_COUNT * sizeof(int));
  p->off_loss = o;       o = align256(o + (size_t)p->loss_slots * sizeof(float));
  p->off_U0 = o;         o = align256(o + (size_t)p->C * HW * sizeof(float2));
  p->off_Y = o;          o = align256(o + (size_t)p->C * half * sizeof(float2));
  p->off_V = o;          o = align256(o + (size_t)p->L * p->C * half * sizeof(float2));
  // the identity planes' gradient seed, later dL/dU(0) (plans with such planes only)
  p->off_S = o;          o = align256(o + (p->n_ident > 0 ? (size_t)p->C * HW * sizeof(float2) : 0));
  p->ws_needed = o;
}

extern "C" cgh_status cgh_plan_create(int32_t H, int32_t W, int32_t C, int32_t L,
                                      int32_t pad_factor, const double* lambda_m,
                                      double pitch_m, const double* z_m, double aperture,
                                      float cutoff, int32_t max_gaussians,
                                      cgh_plan** out_plan) {
  if (!out_plan) return fail(CGH_ERR_ARG, "out_plan is NULL");
  *out_plan = nullptr;
  if (H < 1 || W < 1) return fail(CGH_ERR_ARG, "H and W must be >= 1 (got %d x %d)", H, W);
  if (C < 1 || C > CGH_MAX_C) return fail(CGH_ERR_UNSUPPORTED_SIZE, "C must be in 1..%d", CGH_MAX_C);
  if (L < 1 || L > CGH_MAX_L) return fail(CGH_ERR_UNSUPPORTED_SIZE, "L must be in 1..%d", CGH_MAX_L);
  if (pad_factor < 1) return fail(CGH_ERR_ARG, "pad_factor must be >= 1");
  if (!lambda_m || !z_m) return fail(CGH_ERR_ARG, "lambda_m and z_m must be host arrays");
  if (!(pitch_m > 0.0) || !isfinite(pitch_m)) return fail(CGH_ERR_ARG, "pitch must be > 0");
  if (!(cutoff >= 0.f) || !(cutoff < 0.99f)) return fail(CGH_ERR_ARG, "cutoff must be in [0, 0.99)");
  if (max_gaussians < 0) return fail(CGH_ERR_ARG, "max_gaussians must be >= 0");
  if (!(aperture >= 0.0)) return fail(CGH_ERR_ARG, "aperture must be >= 0");
  const long long Ny = (long long)pad_factor * H, Nx = (long long)pad_factor * W;
  if (Ny > 16384 || Nx > 16384)
    return fail(CGH_ERR_UNSUPPORTED_SIZE, "padded grid %lld x %lld exceeds 16384", Ny, Nx);
  cgh_plan* p = new (std::nothrow) cgh_plan();
  if (!p) return fail(CGH_ERR_ARG, "out of host memory");
  p->H = H; p->W = W; p->C = C; p->L = L; p->pad = pad_factor;
  p->pitch = pitch_m; p->aperture = aperture; p->cutoff = cutoff;
  p->max_gaussians = max_gaussians;
  for (int c = 0; c < C; ++c) {
    if (!(lambda_m[c] > 0.0) || !isfinite(lambda_m[c])) { delete p; return fail(CGH_ERR_ARG, "lambda[%d] must be > 0", c); }
    p->lambda[c] = lambda_m[c];
  }
  for (int l = 0; l < L; ++l) {
    if (!isfinite(z_m[l])) { delete p; return fail(CGH_ERR_ARG, "z[%d] not finite", l); }
    p->z[l] = z_m[l];
  }
  p->tiles_x = (W + CGH_TILE - 1) / CGH_TILE;
  p->tiles_y = (H + CGH_TILE - 1) / CGH_TILE;
  p->col_block = (Nx % 4 == 0) ? 4 : (Nx % 2 == 0 ? 2 : 1);
  p->row_block = 2;
  p->fft_threads = 256;
  p->pair_cap_mult = 16;
  if (!factorise((int)Nx, &p->fx) || !factorise((int)Ny, &p->fy)) {
    delete p;
    return fail(CGH_ERR_UNSUPPORTED_SIZE,
                "padded sizes %lld x %lld must factor into 2, 3, 5 with at most %d passes", Ny,
                Nx, CGH_MAX_PASSES);
  }
  BlasmDev& bl = p->bl;
  memset(&bl, 0, sizeof(bl));
  bl.H = H; bl.W = W; bl.C = C; bl.L = L; bl.Ltot = L;
  for (int l = 0; l < L; ++l) bl.plane[l] = l;
  bl.Ny = (int)Ny; bl.Nx = (int)Nx;
  bl.oy = (int)((Ny - H) / 2); bl.ox = (int)((Nx - W) / 2);
  bl.inv_ntot = (float)(1.0 / ((double)Ny * (double)Nx));
  bl.aperture2 = (float)(aperture * aperture);
  bl.series_ok = 1;
  bl.loss_kind = 0;
  bl.recon_mask = nullptr;
  for (int c = 0; c < C; ++c) {  // largest q = lambda^2 (fx^2 + fy^2) on the padded grid
    const double fxn = (double)(Nx / 2) / ((double)Nx * pitch_m);
    const double fyn = (double)(Ny / 2) / ((double)Ny * pitch_m);
    const double qmax = lambda_m[c] * lambda_m[c] * (fxn * fxn + fyn * fyn);
    if (!(qmax < 0.04)) bl.series_ok = 0;
  }
  const double Lx = (double)Nx * pitch_m, Ly = (double)Ny * pitch_m;
  for (int c = 0; c < C; ++c) {
    const double lam = p->lambda[c];
    for (int l = 0; l < L; ++l) {
      const double d = p->z[l];
      TFConst& t = bl.tf[c * L + l];
      // band limit of Algorithm 3, evaluated exactly as |f| < f_max reads
      const double fxmax = 1.0 / (lam * sqrt((2.0 * d / Lx) * (2.0 * d / Lx) + 1.0));
      const double fymax = 1.0 / (lam * sqrt((2.0 * d / Ly) * (2.0 * d / Ly) + 1.0));
      int kxm = -1, kym = -1;
      for (long long s = 0; s <= Nx / 2; ++s)
        if (fabs((double)s / Lx) < fxmax) kxm = (int)s;
      for (long long s = 0; s <= Ny / 2; ++s)
        if (fabs((double)s / Ly) < fymax) kym = (int)s;
      t.kx_max = kxm;
      t.ky_max = kym;
      const double D = d / lam;  // propagation distance in wavelengths
      t.turns0 = (float)(D - nearbyint(D));
      const double qx = (lam / Lx) * (lam / Lx), qy = (lam / Ly) * (lam / Ly);
      t.qx = (float)qx;
      t.qy = (float)qy;
      t.ax = (float)(D * qx);
      t.ay = (float)(D * qy);
    }
  }
  // Planes whose propagation is the identity: distance exactly 0 and no aperture, with every
  // frequency bin of every channel inside the band (Algorithm 3 at d = 0: the phase k_z d is
  // 0 and f_max = 1/lambda, so H = 1 on the whole grid and U(d) = crop(IFFT(FFT(pad U))) = U).
  p->n_ident = 0;
  p->ident_mask = 0u;
  p->use_ident = 1;
  p->bl_prop = bl;
  p->bl_prop.L = 0;
  for (int l = 0; l < L; ++l) {
    bool ident = p->z[l] == 0.0 && aperture == 0.0;
    for (int c = 0; c < C && ident; ++c) {
      const TFConst& t = bl.tf[c * L + l];
      ident = t.kx_max >= (int)(Nx / 2) && t.ky_max >= (int)(Ny / 2);
    }
    if (ident) {
      p->ident_mask |= 1u << l;
      ++p->n_ident;
    } else {
      p->bl_prop.plane[p->bl_prop.L++] = l;
    }
  }
  // twiddle tables tw[m] = exp(-2 pi i m / n), FP64 on the host
  const size_t tbytes = sizeof(float2) * (size_t)(Nx + Ny);
  float2* host_tw = (float2*)malloc(tbytes);
  if (!host_tw) { delete p; return fail(CGH_ERR_ARG, "out of host memory"); }
  for (int which = 0; which < 2; ++which) {
    const int n = which == 0 ? (int)Nx : (int)Ny;
    float2* dst = host_tw + (which == 0 ? 0 : Nx);
    for (int m = 0; m < n; ++m) {
      const double ang = -2.0 * 3.14159265358979323846 * (double)m / (double)n;
      dst[m] = make_float2((float)cos(ang), (float)sin(ang));
    }
  }
  cudaError_t e = cudaMalloc(&p->tables_dev, tbytes);
  if (e == cudaSuccess) e = cudaMemcpy(p->tables_dev, host_tw, tbytes, cudaMemcpyHostToDevice);
  free(host_tw);
  if (e != cudaSuccess) {
    if (p->tables_dev) cudaFree(p->tables_dev);
    delete p;
    return cuda_fail(e, "cgh_plan_create (twiddle tables)");
  }
  p->tables_bytes = tbytes;
  p->fx.tw = (const float2*)p->tables_dev;
  p->fy.tw = (const float2*)p->tables_dev + Nx;
  // prefer block shapes with compile-time specialised kernels
  p->use_spec = 1;
  {
    static const int cbs[] = {4, 2, 8, 1};
    static const int rbs[] = {4, 2, 1, 8};
    bool done = false;
    for (int cb : cbs) {
      if (done || Nx % cb ||
          !spec_cols(0, (int)Ny, cb, nullptr, nullptr, nullptr, nullptr, 0, nullptr, true))
        continue;
      for (int rb : rbs) {
        if (spec_rows(0, (int)Nx, rb, cb, nullptr, nullptr, 0, nullptr, true)) {
          p->col_block = cb;
          p->row_block = rb;
          done = true;
          break;
        }
      }
    }
  }
  // largest column / row blocks (<= 4 / 2) whose transforms fit one CTA
  while (p->col_block > 1 && !fft_shape(p, p->fy, p->col_block, 2).ok) p->col_block /= 2;
  while (p->row_block > 1 && !fft_shape(p, p->fx, p->row_block, 1).ok) p->row_block /= 2;
  if (!fft_shape(p, p->fy, p->col_block, 2).ok || !fft_shape(p, p->fx, p->row_block, 1).ok) {
    cudaFree(p->tables_dev);
    delete p;
    return fail(CGH_ERR_UNSUPPORTED_SIZE, "padded sizes %lld x %lld need more than %d threads "
                "per transform", Ny, Nx, 2 * kMaxFFTThreads);
  }
  layout(p);
  *out_plan = p;
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_destroy(cgh_plan* plan) {
  if (!plan) return CGH_OK;
  if (plan->tables_dev) cudaFree(plan->tables_dev);
  delete plan;
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_workspace_bytes(const cgh_plan* plan, size_t* out_bytes) {
  if (!plan || !out_bytes) return fail(CGH_ERR_ARG, "NULL argument");
  *out_bytes = plan->ws_needed;
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_set_workspace(cgh_plan* plan, void* workspace, size_t bytes) {
  if (!plan) return fail(CGH_ERR_ARG, "plan is NULL");
  if (!workspace) return fail(CGH_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)workspace) % 256 != 0) return fail(CGH_ERR_ARG, "workspace must be 256-byte aligned");
  if (bytes < plan->ws_needed)
    return fail(CGH_ERR_WORKSPACE, "workspace of %zu bytes < required %zu", bytes, plan->ws_needed);
  // status words start at zero (the loss pass's CTA ticket relies on it)
  cudaError_t e = cudaMemset((char*)workspace + plan->off_status, 0, sizeof(int) * ST_COUNT);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(CGH_ERR_CUDA, "%s", cudaGetErrorString(e));
  plan->ws = (char*)workspace;
  plan->ws_bytes = bytes;
  plan->bin_valid = 0;  // a new workspace holds no binning
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_set_tuning(cgh_plan* plan, const cgh_tuning* t) {
  if (!plan || !t) return fail(CGH_ERR_ARG, "NULL argument");
  if (t->col_block) {
    if (t->col_block != 1 && t->col_block != 2 && t->col_block != 4 && t->col_block != 8)
      return fail(CGH_ERR_ARG, "col_block must be 1, 2, 4 or 8");
    if (plan->bl.Nx % t->col_block) return fail(CGH_ERR_ARG, "col_block must divide Nx");
    if (!fft_shape(plan, plan->fy, t->col_block, 2).ok)
      return fail(CGH_ERR_ARG, "col_block %d does not fit one CTA", t->col_block);
    plan->col_block = t->col_block;
  }
  if (t->row_block) {
    if (t->row_block < 1 || t->row_block > 8) return fail(CGH_ERR_ARG, "row_block must be 1..8");
    if (!fft_shape(plan, plan->fx, t->row_block, 1).ok)
      return fail(CGH_ERR_ARG, "row_block %d does not fit one CTA", t->row_block);
    plan->row_block = t->row_block;
  }
  if (t->fft_threads) {
    if (t->fft_threads < 64 || t->fft_threads > kMaxFFTThreads || t->fft_threads % 32)
      return fail(CGH_ERR_ARG, "fft_threads must be a multiple of 32 in 64..%d", kMaxFFTThreads);
    plan->fft_threads = t->fft_threads;
  }
  if (t->fft_kernels) {
    if (t->fft_kernels != 1 && t->fft_kernels != 2) return fail(CGH_ERR_ARG, "fft_kernels must be 1 or 2");
    plan->use_spec = t->fft_kernels == 1;
  }
  if (t->identity_planes) {
    if (t->identity_planes != 1 && t->identity_planes != 2)
      return fail(CGH_ERR_ARG, "identity_planes must be 1 or 2");
    plan->use_ident = t->identity_planes == 1;
  }
  if (t->pair_capacity_per_gaussian) {
    if (t->pair_capacity_per_gaussian < 1) return fail(CGH_ERR_ARG, "pair capacity must be >= 1");
    plan->pair_cap_mult = t->pair_capacity_per_gaussian;
    const size_t before = plan->ws_needed;
    layout(plan);
    plan->bin_valid = 0;  // the carve-up moved
    if (plan->ws && plan->ws_needed > plan->ws_bytes) {
      plan->ws = nullptr;
      plan->ws_bytes = 0;
      (void)before;
    } else if (plan->ws) {
      cudaError_t e = cudaMemset(plan->ws + plan->off_status, 0, sizeof(int) * ST_COUNT);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return fail(CGH_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
  }
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_get_tuning(const cgh_plan* plan, cgh_tuning* out) {
  if (!plan || !out) return fail(CGH_ERR_ARG, "NULL argument");
  out->col_block = plan->col_block;
  out->row_block = plan->row_block;
  out->fft_threads = plan->fft_threads;
  out->pair_capacity_per_gaussian = plan->pair_cap_mult;
  out->fft_kernels = plan->use_spec ? 1 : 2;
  out->identity_planes = plan->use_ident ? 1 : 2;
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_band_limits(const cgh_plan* plan, int32_t* kx_max,
                                           int32_t* ky_max) {
  if (!plan || !kx_max || !ky_max) return fail(CGH_ERR_ARG, "NULL argument");
  for (int i = 0; i < plan->C * plan->L; ++i) {
    kx_max[i] = plan->bl.tf[i].kx_max;
    ky_max[i] = plan->bl.tf[i].ky_max;
  }
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_identity_planes(const cgh_plan* plan, uint32_t* mask_out) {
  if (!plan || !mask_out) return fail(CGH_ERR_ARG, "NULL argument");
  *mask_out = plan->ident_mask;
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_set_loss(cgh_plan* plan, int32_t kind, const uint8_t* recon_mask) {
  if (!plan) return fail(CGH_ERR_ARG, "plan is NULL");
  if (kind != CGH_LOSS_MSE && kind != CGH_LOSS_RECON) return fail(CGH_ERR_ARG, "unknown loss kind");
  if (kind == CGH_LOSS_MSE && recon_mask) return fail(CGH_ERR_ARG, "a depth mask needs CGH_LOSS_RECON");
  plan->bl.loss_kind = kind;
  plan->bl.recon_mask = recon_mask;
  plan->bl_prop.loss_kind = kind;  // the plane map of the fused step carries the same loss
  plan->bl_prop.recon_mask = recon_mask;
  return CGH_OK;
}

extern "C" cgh_status cgh_plan_status(cgh_plan* plan, int64_t* pairs_needed, int32_t* overflow,
                                      int32_t* nonfinite, void* stream) {
  if (!plan) return fail(CGH_ERR_ARG, "plan is NULL");
  if (!plan->ws) return fail(CGH_ERR_WORKSPACE, "no workspace attached");
  int st[ST_COUNT];
  cudaStream_t s = (cudaStream_t)stream;
  CGH_TRY(cudaMemcpyAsync(st, plan->ws + plan->off_status, sizeof(st), cudaMemcpyDeviceToHost, s),
          "cgh_plan_status");
  CGH_TRY(cudaStreamSynchronize(s), "cgh_plan_status");
  if (pairs_needed) *pairs_needed = ((int64_t)(uint32_t)st[ST_PAIRS_HI] << 32) | (uint32_t)st[ST_PAIRS_LO];
  if (overflow) *overflow = st[ST_OVERFLOW];
  if (nonfinite) *nonfinite = st[ST_NONFINITE];
  return CGH_OK;
}

// ------------------------------------------------------------------ entry points
static cgh_status check_call(const cgh_plan* p, const cgh_params* prm) {
  if (!p) return fail(CGH_ERR_ARG, "plan is NULL");
  if (!p->ws) return fail(CGH_ERR_WORKSPACE, "no workspace attached (cgh_plan_set_workspace)");
  if (prm) {
    if (prm->N < 0) return fail(CGH_ERR_ARG, "N must be >= 0");
    if (prm->N > p->max_gaussians)
      return fail(CGH_ERR_CAPACITY, "N = %d exceeds max_gaussians = %d", prm->N, p->max_gaussians);
    if (prm->N > 0 && (!prm->xy_raw || !prm->s_raw || !prm->theta || !prm->amp || !prm->phase ||
                       !prm->alpha_raw))
      return fail(CGH_ERR_ARG, "NULL parameter array");
  }
  return CGH_OK;
}

static cgh_status check_grads(const cgh_params* prm, const cgh_grads* g) {
  if (!g) return fail(CGH_ERR_ARG, "grads is NULL");
  if (prm->N > 0 && (!g->xy_raw || !g->s_raw || !g->theta || !g->amp || !g->phase || !g->alpha_raw))
    return fail(CGH_ERR_ARG, "NULL gradient array");
  return CGH_OK;
}

#define CGH_CHECK(expr)              \
  do {                               \
    cgh_status _s = (expr);          \
    if (_s != CGH_OK) return _s;     \
  } while (0)

extern "C" cgh_status cgh_raster_fwd(cgh_plan* plan, const cgh_params* params, void* U_out,
                                     void* stream) {
  CGH_CHECK(check_call(plan, params));
  if (!params || !U_out) return fail(CGH_ERR_ARG, "NULL argument");
  CGH_TRY(launch_raster_fwd(plan, params, (float2*)U_out, (cudaStream_t)stream), "cgh_raster_fwd");
  return CGH_OK;
}

extern "C" cgh_status cgh_raster_stats(cgh_plan* plan, const cgh_params* params,
                                       int64_t* counts_out, void* stream) {
  CGH_CHECK(check_call(plan, params));
  if (!params || !counts_out) return fail(CGH_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  // the six counters live in the loss-partial slots (at least 1024 floats, 256-byte aligned)
  unsigned long long* dev = reinterpret_cast<unsigned long long*>(plan->ws + plan->off_loss);
  unsigned long long host[6];
  CGH_TRY(launch_raster_stats(plan, params, dev, s), "cgh_raster_stats");
  CGH_TRY(cudaMemcpyAsync(host, dev, sizeof(host), cudaMemcpyDeviceToHost, s), "cgh_raster_stats");
  CGH_TRY(cudaStreamSynchronize(s), "cgh_raster_stats");
  for (int k = 0; k < 6; ++k) counts_out[k] = (int64_t)host[k];
  return CGH_OK;
}

extern "C" cgh_status cgh_raster_bwd(cgh_plan* plan, const cgh_params* params, const void* dU,
                                     const cgh_grads* grads, void* stream) {
  CGH_CHECK(check_call(plan, params));
  if (!params || !dU) return fail(CGH_ERR_ARG, "NULL argument");
  CGH_CHECK(check_grads(params, grads));
  CGH_TRY(launch_raster_bwd(plan, params, (const float2*)dU, grads, (cudaStream_t)stream, true),
          "cgh_raster_bwd");
  return CGH_OK;
}

extern "C" cgh_status cgh_blasm_fwd(cgh_plan* plan, const void* U0, void* Ud_out, void* stream) {
  CGH_CHECK(check_call(plan, nullptr));
  if (!U0 || !Ud_out) return fail(CGH_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  float2* Y = (float2*)(plan->ws + plan->off_Y);
  float2* V = (float2*)(plan->ws + plan->off_V);
  CGH_TRY(launch_rows_pad_fwd(plan, (const float2*)U0, Y, plan->C, s), "cgh_blasm_fwd rows");
  CGH_TRY(launch_cols_fwd_planes(plan, Y, V, s), "cgh_blasm_fwd cols");
  CGH_TRY(launch_rows_inv_crop(plan, V, (float2*)Ud_out, plan->L * plan->C, s), "cgh_blasm_fwd crop");
  return CGH_OK;
}

extern "C" cgh_status cgh_blasm_bwd(cgh_plan* plan, const void* dUd, void* dU0_out, void* stream) {
  CGH_CHECK(check_call(plan, nullptr));
  if (!dUd || !dU0_out) return fail(CGH_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  float2* Y = (float2*)(plan->ws + plan->off_Y);
  float2* V = (float2*)(plan->ws + plan->off_V);
  CGH_TRY(launch_rows_pad_fwd(plan, (const float2*)dUd, V, plan->L * plan->C, s), "cgh_blasm_bwd rows");
  CGH_TRY(launch_cols_bwd_planes(plan, V, Y, s), "cgh_blasm_bwd cols");
  CGH_TRY(launch_rows_inv_crop(plan, Y, (float2*)dU0_out, plan->C, s), "cgh_blasm_bwd crop");
  return CGH_OK;
}

extern "C" cgh_status cgh_intensity_loss(cgh_plan* plan, const void* Ud, const float* target,
                                         float* loss_out, void* dUd_out, void* stream) {
  CGH_CHECK(check_call(plan, nullptr));
  if (!Ud || !target || !loss_out) return fail(CGH_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  float* partials = (float*)(plan->ws + plan->off_loss);
  CGH_TRY(launch_loss_pointwise(plan, (const float2*)Ud, target, partials, (float2*)dUd_out, s),
          "cgh_intensity_loss");
  CGH_TRY(launch_loss_finalize(plan, partials, pointwise_loss_blocks(plan), loss_out, s),
          "cgh_intensity_loss finalize");
  return CGH_OK;
}

extern "C" cgh_status cgh_intensity(cgh_plan* plan, const void* Ud, float* I_out, void* stream) {
  CGH_CHECK(check_call(plan, nullptr));
  if (!Ud || !I_out) return fail(CGH_ERR_ARG, "NULL argument");
  const long long total = (long long)plan->L * plan->C * plan->H * plan->W;
  CGH_TRY(launch_intensity(total, (const float2*)Ud, I_out, (cudaStream_t)stream), "cgh_intensity");
  return CGH_OK;
}

extern "C" cgh_status cgh_intensity_bwd(cgh_plan* plan, const void* Ud, const float* dI,
                                        void* dUd_out, void* stream) {
  CGH_CHECK(check_call(plan, nullptr));
  if (!Ud || !dI || !dUd_out) return fail(CGH_ERR_ARG, "NULL argument");
  const long long total = (long long)plan->L * plan->C * plan->H * plan->W;
  CGH_TRY(launch_intensity_bwd(total, (const float2*)Ud, dI, (float2*)dUd_out,
                               (cudaStream_t)stream), "cgh_intensity_bwd");
  return CGH_OK;
}

// Planes whose propagation is the identity are handled in the pixel domain when the plan
// allows it: their loss and gradient seed are taken on U(0) by the forward raster as it
// finishes each pixel (the seed into the workspace's S), and only the other planes go
// through the column and loss row passes.
static bool ident_path(const cgh_plan* p) { return p->use_ident && p->n_ident > 0; }

static cgh_status forward_chain(cgh_plan* plan, const cgh_params* params, const float* target,
                                float* loss_out, bool want_grad, cudaStream_t s,
                                bool rebin = true) {
  float2* U0 = (float2*)(plan->ws + plan->off_U0);
  float2* Y = (float2*)(plan->ws + plan->off_Y);
  float2* V = (float2*)(plan->ws + plan->off_V);
  float* partials = (float*)(plan->ws + plan->off_loss);
  if (!ident_path(plan)) {
    CGH_TRY(launch_raster_fwd(plan, params, U0, s, rebin), "raster_fwd");
    CGH_TRY(launch_rows_pad_fwd(plan, U0, Y, plan->C, s), "rows_pad_fwd");
    CGH_TRY(launch_cols_fwd_planes(plan, Y, V, s), "cols_fwd_planes");
    CGH_TRY(launch_rows_loss(plan, V, target, partials, s, want_grad, loss_out), "rows_loss");
    return CGH_OK;
  }
  const BlasmDev* prop = &plan->bl_prop;
  IdentLoss il;
  il.target = target;
  il.partials = partials + rows_loss_blocks(plan, prop);  // after the loss row pass's own
  il.seed = want_grad ? (float2*)(plan->ws + plan->off_S) : nullptr;
  il.recon_mask = plan->bl.recon_mask;
  il.gscale = 4.0f / ((float)plan->L * (float)plan->C * (float)plan->H * (float)plan->W);
  il.mask = plan->ident_mask;
  il.loss_kind = plan->bl.loss_kind;
  CGH_TRY(launch_raster_fwd(plan, params, U0, s, rebin, &il), "raster_fwd");
  if (prop->L > 0) CGH_TRY(launch_rows_pad_fwd(plan, U0, Y, plan->C, s), "rows_pad_fwd");
  CGH_TRY(launch_cols_fwd_planes(plan, Y, V, s, prop), "cols_fwd_planes");
  CGH_TRY(launch_rows_loss(plan, V, target, partials, s, want_grad, loss_out, prop,
                           ident_loss_blocks(plan)), "rows_loss");
  return CGH_OK;
}

extern "C" cgh_status cgh_forward_loss(cgh_plan* plan, const cgh_params* params,
                                       const float* target, float* loss_out, void* stream) {
  CGH_CHECK(check_call(plan, params));
  if (!params || !target || !loss_out) return fail(CGH_ERR_ARG, "NULL argument");
  return forward_chain(plan, params, target, loss_out, false, (cudaStream_t)stream);
}

static cgh_status step_impl(cgh_plan* plan, const cgh_params* params, const float* target,
                            float* loss_out, const cgh_grads* grads, const float* grad_scale,
                            bool rebin, cudaStream_t s) {
  CGH_CHECK(check_call(plan, params));
  if (!params || !target || !loss_out) return fail(CGH_ERR_ARG, "NULL argument");
  CGH_CHECK(check_grads(params, grads));
  CGH_CHECK(forward_chain(plan, params, target, loss_out, true, s, rebin));
  float2* Y = (float2*)(plan->ws + plan->off_Y);    // reused for the backward half grid
  float2* V = (float2*)(plan->ws + plan->off_V);
  float2* dU0;  // dL/dU(0)
  if (!ident_path(plan)) {
    dU0 = (float2*)(plan->ws + plan->off_U0);  // U(0) is no longer needed
    CGH_TRY(launch_cols_bwd_planes(plan, V, Y, s), "cols_bwd_planes");
    CGH_TRY(launch_rows_inv_crop(plan, Y, dU0, plan->C, s), "rows_inv_crop");
  } else {
    // identity planes' seed (in S) + adjoint of the propagated planes
    dU0 = (float2*)(plan->ws + plan->off_S);
    if (plan->bl_prop.L > 0) {
      CGH_TRY(launch_cols_bwd_planes(plan, V, Y, s, &plan->bl_prop), "cols_bwd_planes");
      CGH_TRY(launch_rows_inv_crop(plan, Y, dU0, plan->C, s, true), "rows_inv_crop");
    }
  }
  // the forward's binning is still valid for these parameters: reuse it
  CGH_TRY(launch_raster_bwd(plan, params, dU0, grads, s, false, grad_scale), "raster_bwd");
  return CGH_OK;
}

extern "C" cgh_status cgh_step(cgh_plan* plan, const cgh_params* params, const float* target,
                               float* loss_out, const cgh_grads* grads, void* stream) {
  return step_impl(plan, params, target, loss_out, grads, nullptr, true, (cudaStream_t)stream);
}

extern "C" cgh_status cgh_step_scaled(cgh_plan* plan, const cgh_params* params,
                                      const float* target, float* loss_out,
                                      const cgh_grads* grads, const float* grad_scale,
                                      int32_t reuse_binning, void* stream) {
  return step_impl(plan, params, target, loss_out, grads, grad_scale, reuse_binning == 0,
                   (cudaStream_t)stream);
}

// ------------------------------------------------------------------ Adam
namespace {
struct AdamArgs {
  float* p[8];
  const float* g[8];
  float* m[8];
  float* v[8];
  long long off[9];
  float step_size[8];
  int n;
};

__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, float b1,
                                          float b2, float eps, float inv_sqrt_bc2, float step) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  p -= step * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
  return p;
}

// Four consecutive elements per thread and 16-byte accesses (every group 16-byte aligned
// with a length divisible by 4; offsets a.off in units of 4 elements).
__global__ void k_adam4(AdamArgs a, float b1, float b2, float eps, float inv_sqrt_bc2) {
  const long long total = a.off[a.n];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int gi = 0;
    while (i >= a.off[gi + 1]) ++gi;
    const long long j = i - a.off[gi];
    float4 p = reinterpret_cast<float4*>(a.p[gi])[j];
    const float4 g = reinterpret_cast<const float4*>(a.g[gi])[j];
    float4 m = reinterpret_cast<float4*>(a.m[gi])[j];
    float4 v = reinterpret_cast<float4*>(a.v[gi])[j];
    const float st = a.step_size[gi];
    adam_one(p.x, g.x, m.x, v.x, b1, b2, eps, inv_sqrt_bc2, st);
    adam_one(p.y, g.y, m.y, v.y, b1, b2, eps, inv_sqrt_bc2, st);
    adam_one(p.z, g.z, m.z, v.z, b1, b2, eps, inv_sqrt_bc2, st);
    adam_one(p.w, g.w, m.w, v.w, b1, b2, eps, inv_sqrt_bc2, st);
    reinterpret_cast<float4*>(a.p[gi])[j] = p;
    reinterpret_cast<float4*>(a.m[gi])[j] = m;
    reinterpret_cast<float4*>(a.v[gi])[j] = v;
  }
}

__global__ void k_adam(AdamArgs a, float b1, float b2, float eps, float inv_sqrt_bc2) {
  const long long total = a.off[a.n];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int gi = 0;
    while (i >= a.off[gi + 1]) ++gi;
    const long long j = i - a.off[gi];
    const float g = a.g[gi][j];
    const float m = fmaf(b1, a.m[gi][j], (1.f - b1) * g);
    const float v = fmaf(b2, a.v[gi][j], (1.f - b2) * g * g);
    a.m[gi][j] = m;
    a.v[gi][j] = v;
    const float denom = sqrtf(v) * inv_sqrt_bc2 + eps;
    a.p[gi][j] -= a.step_size[gi] * m / denom;
  }
}
}  // namespace

cudaError_t launch_adam(const cgh_adam_group* groups, int n, int step, float b1, float b2,
                        float eps, cudaStream_t s) {
  AdamArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.off[0] = 0;
  const double bc1 = 1.0 - pow((double)b1, (double)step);
  const double bc2 = 1.0 - pow((double)b2, (double)step);
  for (int i = 0; i < n; ++i) {
    a.p[i] = groups[i].param;
    a.g[i] = groups[i].grad;
    a.m[i] = groups[i].exp_avg;
    a.v[i] = groups[i].exp_avg_sq;
    a.off[i + 1] = a.off[i] + groups[i].count;
    a.step_size[i] = (float)((double)groups[i].lr / bc1);
  }
  for (int i = n + 1; i < 9; ++i) a.off[i] = a.off[n];
  long long total = a.off[n];
  if (total == 0) return cudaSuccess;
  bool vec = true;
  for (int i = 0; i < n; ++i) {
    const uintptr_t bits = (uintptr_t)groups[i].param | (uintptr_t)groups[i].grad |
                           (uintptr_t)groups[i].exp_avg | (uintptr_t)groups[i].exp_avg_sq;
    vec = vec && (bits & 15u) == 0 && groups[i].count % 4 == 0;
  }
  if (vec) {
    for (int i = 0; i <= 8; ++i) a.off[i] /= 4;
    total /= 4;
  }
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  prof_begin(KID_ADAM, s);
  if (vec)
    k_adam4<<<(unsigned)blocks, 256, 0, s>>>(a, b1, b2, eps, (float)(1.0 / sqrt(bc2)));
  else
    k_adam<<<(unsigned)blocks, 256, 0, s>>>(a, b1, b2, eps, (float)(1.0 / sqrt(bc2)));
  prof_end(KID_ADAM, s);
  return cudaGetLastError();
}

extern "C" cgh_status cgh_adam_step(const cgh_adam_group* groups, int32_t num_groups, int32_t step,
                                    float beta1, float beta2, float eps, void* stream) {
  if (!groups || num_groups < 1 || num_groups > 8) return fail(CGH_ERR_ARG, "1..8 groups required");
  if (step < 1) return fail(CGH_ERR_ARG, "step must be >= 1");
  for (int i = 0; i < num_groups; ++i) {
    const cgh_adam_group& g = groups[i];
    if (g.count < 0) return fail(CGH_ERR_ARG, "group %d: negative count", i);
    if (g.count > 0 && (!g.param || !g.grad || !g.exp_avg || !g.exp_avg_sq))
      return fail(CGH_ERR_ARG, "group %d: NULL pointer", i);
  }
  CGH_TRY(launch_adam(groups, num_groups, step, beta1, beta2, eps, (cudaStream_t)stream),
          "cgh_adam_step");
  return CGH_OK;
}

// ------------------------------------------------------------------ Adan
namespace {
struct AdanArgs {
  float* p[8];
  const float* g[8];
  float* m[8];
  float* v[8];
  float* n[8];
  float* gp[8];
  long long off[9];
  float lr[8];
  int ngroups;
};

// d = g - g_prev (0 at step 1); m, v, n running averages; bias-corrected step (see cgh.h)
__global__ void k_adan(AdanArgs a, float b1, float b2, float b3, float eps, float wd, int first,
                       float inv_bc1, float b2_over_bc2, float inv_sqrt_bc3) {
  const long long total = a.off[a.ngroups];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int gi = 0;
    while (i >= a.off[gi + 1]) ++gi;
    const long long j = i - a.off[gi];
    const float g = a.g[gi][j];
    const float d = first ? 0.f : g - a.gp[gi][j];
    const float m = fmaf(b1, a.m[gi][j], (1.f - b1) * g);
    const float v = fmaf(b2, a.v[gi][j], (1.f - b2) * d);
    const float u = fmaf(b2, d, g);
    const float n = fmaf(b3, a.n[gi][j], (1.f - b3) * u * u);
    a.m[gi][j] = m;
    a.v[gi][j] = v;
    a.n[gi][j] = n;
    a.gp[gi][j] = g;
    const float step = fmaf(m, inv_bc1, b2_over_bc2 * v) / fmaf(sqrtf(n), inv_sqrt_bc3, eps);
    const float lr = a.lr[gi];
    a.p[gi][j] = (a.p[gi][j] - lr * step) / fmaf(lr, wd, 1.f);
  }
}
}  // namespace

extern "C" cgh_status cgh_adan_step(const cgh_adan_group* groups, int32_t num_groups, int32_t step,
                                    float beta1, float beta2, float beta3, float eps,
                                    float weight_decay, void* stream) {
  if (!groups || num_groups < 1 || num_groups > 8) return fail(CGH_ERR_ARG, "1..8 groups required");
  if (step < 1) return fail(CGH_ERR_ARG, "step must be >= 1");
  AdanArgs a;
  memset(&a, 0, sizeof(a));
  a.ngroups = num_groups;
  for (int i = 0; i < num_groups; ++i) {
    const cgh_adan_group& g = groups[i];
    if (g.count < 0) return fail(CGH_ERR_ARG, "group %d: negative count", i);
    if (g.count > 0 && (!g.param || !g.grad || !g.exp_avg || !g.exp_avg_diff || !g.exp_avg_sq ||
                        !g.prev_grad))
      return fail(CGH_ERR_ARG, "group %d: NULL pointer", i);
    a.p[i] = g.param;
    a.g[i] = g.grad;
    a.m[i] = g.exp_avg;
    a.v[i] = g.exp_avg_diff;
    a.n[i] = g.exp_avg_sq;
    a.gp[i] = g.prev_grad;
    a.lr[i] = g.lr;
    a.off[i + 1] = a.off[i] + g.count;
  }
  for (int i = num_groups + 1; i < 9; ++i) a.off[i] = a.off[num_groups];
  const long long total = a.off[num_groups];
  if (total == 0) return CGH_OK;
  const double bc1 = 1.0 - pow((double)beta1, (double)step);
  const double bc2 = 1.0 - pow((double)beta2, (double)step);
  const double bc3 = 1.0 - pow((double)beta3, (double)step);
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ADAM, s);
  k_adan<<<(unsigned)blocks, 256, 0, s>>>(a, beta1, beta2, beta3, eps, weight_decay, step == 1,
                                           (float)(1.0 / bc1), (float)((double)beta2 / bc2),
                                           (float)(1.0 / sqrt(bc3)));
  prof_end(KID_ADAM, s);
  CGH_TRY(cudaGetLastError(), "cgh_adan_step");
  return CGH_OK;
}

extern "C" int64_t cgh_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char* cgh_last_error_string(void) { return g_err; }
