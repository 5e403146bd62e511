// stage_16x16.cu -- the stage kernels instantiated for tiles of 16 x 16 cells.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_16x16() {
  static const StageSet s = make_stage_set<Tile<16, 16>>();
  return &s;
}
}  // namespace ct
