// stage_16x16_bi.cu -- the bimodal-liquid stage kernels instantiated for tiles of 16 x 16 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_16x16(StageSet& s) { add_bimodal_variants<Tile<16, 16>>(s); }
}  // namespace ct
