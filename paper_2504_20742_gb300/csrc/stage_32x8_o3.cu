// stage_32x8_o3.cu -- the plain FP32 stage kernels for tiles of 32 x 8 cells with registers
// budgeted for three CTAs per SM.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_32x8_o3() {
  static const StageSet s = make_stage_set_fp32<Tile<32, 8, 3>>();
  return &s;
}
}  // namespace ct
