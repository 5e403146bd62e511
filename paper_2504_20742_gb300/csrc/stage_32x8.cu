// stage_32x8.cu -- the stage kernels instantiated for tiles of 32 x 8 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_32x8(StageSet& s);   // stage_32x8_bi.cu
const StageSet* stage_set_32x8() {
  static const StageSet s = [] {
    StageSet t = make_stage_set<Tile<32, 8>>();
    add_bimodal_32x8(t);
    return t;
  }();
  return &s;
}
}  // namespace ct
