// stage_sweep.cu -- the column-sweep FP32 stage kernels (stage_sweep.cuh): strips of 28
// columns, four warps per CTA stacked in r, 16 rows per warp, registers for four CTAs per SM.
// (Measured alternatives on the 4096 x 1024 plume, ms per step against 0.73 for this one
// before its dry-row paths: 20 rows per warp 0.75, 32 rows 0.80; registers for five CTAs
// per SM 0.78 (16 rows) to 0.80 (12 rows), for six 0.84; two warps per CTA, eight CTAs per
// SM 0.77; the next row copied ahead into shared memory by cp.async 0.77.)
#include "stage_sweep.cuh"

namespace ct {
const StageSet* stage_set_sweep() {
  static const StageSet s = make_stage_set_sweep<SweepTile<4, 16, 4>>();
  return &s;
}
}  // namespace ct
