// stage_32x16.cu -- the stage kernels instantiated for tiles of 32 x 16 cells.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_32x16() {
  static const StageSet s = make_stage_set<Tile<32, 16>>();
  return &s;
}
}  // namespace ct
