// blasm_spec_g.cu -- specialised FFT passes for the 1800 x 3200 hologram (padded 3600 x 6400),
// the largest resolution the paper reports.
#include "blasm_reg.cuh"

bool spec_rows_g(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(6400, 20, 20, 16, 1, 2, 416)
  return false;
}

bool spec_cols_g(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC(3600, 15, 16, 15, 1, 240, 2)
  return false;
}
