// stage_64x8.cu -- the stage kernels instantiated for tiles of 64 x 8 cells.
#include "stage.cuh"

namespace ct {
const StageSet* stage_set_64x8() {
  static const StageSet s = make_stage_set<Tile<64, 8>>();
  return &s;
}
}  // namespace ct
