// stage_32x8.cu -- the stage kernels instantiated for tiles of 32 x 8 cells.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_32x8() {
  static const StageSet s = make_stage_set<Tile<32, 8>>();
  return &s;
}
}  // namespace ct
