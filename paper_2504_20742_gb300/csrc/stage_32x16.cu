// stage_32x16.cu -- the stage kernels instantiated for tiles of 32 x 16 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_32x16(StageSet& s);   // stage_32x16_bi.cu
const StageSet* stage_set_32x16() {
  static const StageSet s = [] {
    StageSet t = make_stage_set<Tile<32, 16>>();
    add_bimodal_32x16(t);
    return t;
  }();
  return &s;
}
}  // namespace ct
