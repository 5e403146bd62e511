// stage_sweep.cu -- the column-sweep FP32 stage kernels (stage_sweep.cuh): strips of 28
// columns, four warps per CTA stacked in r, 16 rows per warp, registers for four CTAs per SM.
// (Measured alternatives on the 4096 x 1024 plume, ms per step: 32 rows per warp 0.805,
// registers for three CTAs per SM 0.863 or for five 0.865, against 0.773 for this one.)
#include "stage_sweep.cuh"

namespace ct {
const StageSet* stage_set_sweep() {
  static const StageSet s = make_stage_set_sweep<SweepTile<4, 16, 4>>();
  return &s;
}
}  // namespace ct
