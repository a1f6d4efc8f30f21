// blasm_spec_d.cu -- specialised FFT passes for the 2160 x 3840 hologram (padded 4320 x 7680).
#include "blasm_reg.cuh"

bool spec_rows_d(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(7680, 16, 20, 24, 1, 2, 480)
  return false;
}

bool spec_cols_d(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC_FB(4320, 24, 15, 12, 15, 24, 12, 1, 384, 1, 1)
  return false;
}
