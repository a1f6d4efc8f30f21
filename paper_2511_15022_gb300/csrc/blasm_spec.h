// blasm_spec.h -- registry of the compile-time specialised FFT pass kernels.
//
// Each spec translation unit instantiates the kernels of blasm_reg.cuh for a few
// transform lengths and batch shapes and answers lookups for them; a lookup that finds
// nothing makes the caller use the generic Stockham kernels of blasm.cu.
#pragma once

#include <cuda_runtime.h>

#include "cgh_internal.h"

enum SpecRowKind { SPEC_ROWS_PAD_FWD = 0, SPEC_ROWS_INV_CROP = 1, SPEC_ROWS_LOSS = 2 };
enum SpecColKind { SPEC_COLS_FWD_PLANES = 0, SPEC_COLS_BWD_PLANES = 1 };

struct SpecRowArgs {
  const BlasmDev* bl;   // plane map (rows_loss); geometry
  const float2* in;     // rows_pad_fwd / rows_inv_crop input
  float2* out;          // rows_pad_fwd / rows_inv_crop output; rows_loss: half grids (in place)
  const float* target;  // rows_loss
  float* partials;      // rows_loss
  int batches;
  int want_grad;
  float* loss_out;      // rows_loss: the finished loss (sum of partials * inv_norm)
  int* ticket;          // rows_loss: CTA counter, 0 on entry and on exit
  double inv_norm;      // rows_loss
  int extra;            // rows_loss: partials of other kernels after the pass's own
  int accumulate;       // rows_inv_crop: add into out instead of overwriting it
};

// Launch (dry = false) or only look up (dry = true) a specialised row kernel for transform
// length N with RB rows per CTA and column-block layout CB.  Returns false if there is no
// specialisation; otherwise *err receives the launch status.
bool spec_rows(int kind, int N, int RB, int CB, const cgh_plan* p, const SpecRowArgs* a,
               cudaStream_t s, cudaError_t* err, bool dry);
// Same for column kernels of length N with CB columns per CTA over the planes of `bl`.
bool spec_cols(int kind, int N, int CB, const cgh_plan* p, const BlasmDev* bl, const float2* in,
               float2* out, cudaStream_t s, cudaError_t* err, bool dry);

// per-translation-unit hooks (one file per group of padded lengths, compiled in
// parallel), tried in order by spec_rows / spec_cols
#define CGH_SPEC_HOOKS(X)                                                                      \
  bool spec_rows_##X(int kind, int N, int RB, int CB, const cgh_plan* p, const SpecRowArgs* a, \
                     cudaStream_t s, cudaError_t* err, bool dry);                             \
  bool spec_cols_##X(int kind, int N, int CB, const cgh_plan* p, const BlasmDev* bl,          \
                     const float2* in, float2* out, cudaStream_t s, cudaError_t* err, bool dry);
CGH_SPEC_HOOKS(a)
CGH_SPEC_HOOKS(b)
CGH_SPEC_HOOKS(c)
CGH_SPEC_HOOKS(d)
CGH_SPEC_HOOKS(e)
CGH_SPEC_HOOKS(f)
CGH_SPEC_HOOKS(g)
#undef CGH_SPEC_HOOKS
