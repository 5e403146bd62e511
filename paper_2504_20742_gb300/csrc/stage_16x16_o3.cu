// stage_16x16_o3.cu -- the plain FP32 stage kernels for tiles of 16 x 16 cells with registers
// budgeted for three CTAs per SM.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_16x16_o3() {
  static const StageSet s = make_stage_set_fp32<Tile<16, 16, 3>>();
  return &s;
}
}  // namespace ct
