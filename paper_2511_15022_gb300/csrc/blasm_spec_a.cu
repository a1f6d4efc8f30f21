// blasm_spec_a.cu -- specialised FFT passes for the 1080x1920 hologram (padded 2160 x 3840)
// and the 2160x3840 one (padded 4320 x 7680).
#include "blasm_reg.cuh"

bool spec_rows_a(int kind, int N_, int RB_, int CB_, const cgh_plan* p, const SpecRowArgs* a,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_ROW_SPEC(3840, 16, 15, 16, 2, 2, 512)
  return false;
}

bool spec_cols_a(int kind, int N_, int CB_, const cgh_plan* p, const BlasmDev* bl,
                 const float2* in, float2* out,
                 cudaStream_t s, cudaError_t* err, bool dry) {
  CGH_COL_SPEC_A(2160, 15, 12, 12, 1, 192, 2, 2)
  return false;
}
