// stage_64x8.cu -- the stage kernels instantiated for tiles of 64 x 8 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_64x8(StageSet& s);   // stage_64x8_bi.cu
const StageSet* stage_set_64x8() {
  static const StageSet s = [] {
    StageSet t = make_stage_set<Tile<64, 8>>();
    add_bimodal_64x8(t);
    return t;
  }();
  return &s;
}
}  // namespace ct
