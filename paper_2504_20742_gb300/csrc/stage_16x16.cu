// stage_16x16.cu -- the stage kernels instantiated for tiles of 16 x 16 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_16x16(StageSet& s);   // stage_16x16_bi.cu
const StageSet* stage_set_16x16() {
  static const StageSet s = [] {
    StageSet t = make_stage_set<Tile<16, 16>>();
    add_bimodal_16x16(t);
    return t;
  }();
  return &s;
}
}  // namespace ct
