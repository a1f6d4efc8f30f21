// blasm_spec_b.cu -- specialised FFT passes for padded length 512 (256 x 256 images, the
// smallest bucket of the batched workload).
#include "blasm_reg.cuh"

bool spec_rows_b(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(512, 8, 8, 8, 4, 4, 256)
  CGH_ROW_SPEC(512, 8, 8, 8, 2, 2, 128)
  return false;
}

bool spec_cols_b(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC(512, 8, 8, 8, 2, 128, 3)
  CGH_COL_SPEC(512, 8, 8, 8, 1, 64, 4)
  return false;
}
