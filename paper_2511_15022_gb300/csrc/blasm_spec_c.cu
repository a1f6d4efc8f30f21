// blasm_spec_c.cu -- specialised FFT passes for padded lengths 1536 and 2048 (768- and
// 1024-pixel image sides).
#include "blasm_reg.cuh"

bool spec_rows_c(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(1536, 16, 12, 8, 2, 2, 384)
  CGH_ROW_SPEC(2048, 16, 16, 8, 2, 2, 512)
  return false;
}

bool spec_cols_c(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC(2048, 16, 16, 8, 1, 256, 1)
  return false;
}
