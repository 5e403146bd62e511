// stage_16x14_d2.cu -- the plain FP64 stage kernels for tiles of 16 x 14 cells with registers
// and shared memory budgeted for two CTAs per SM.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_16x14_d2() {
  static const StageSet s = make_stage_set_fp64<Tile<16, 14, 2, 2>>();
  return &s;
}
}  // namespace ct
