// blasm_spec_e.cu -- specialised FFT passes for padded lengths 1024 and 1280 (512- and
// 640-pixel image sides of the batched workload's buckets).
#include "blasm_reg.cuh"

bool spec_rows_e(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(1024, 16, 8, 8, 2, 2, 256)
  return false;
}

bool spec_cols_e(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC(1024, 16, 8, 8, 1, 128, 3)
  CGH_COL_SPEC(1280, 16, 10, 8, 1, 160, 2)
  return false;
}
