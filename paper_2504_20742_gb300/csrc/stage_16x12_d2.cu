// stage_16x12_d2.cu -- the plain FP64 stage kernels for tiles of 16 x 12 cells with registers
// and shared memory budgeted for two CTAs per SM.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_16x12_d2() {
  static const StageSet s = make_stage_set_fp64<Tile<16, 12, 2, 2>>();
  return &s;
}
}  // namespace ct
