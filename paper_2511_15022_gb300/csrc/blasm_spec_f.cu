// blasm_spec_f.cu -- specialised FFT passes for the 1440 x 2560 hologram (padded 2880 x 5120).
#include "blasm_reg.cuh"

bool spec_rows_f(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(5120, 16, 20, 16, 1, 2, 320)
  return false;
}

bool spec_cols_f(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC(2880, 20, 12, 12, 1, 240, 2)
  return false;
}
