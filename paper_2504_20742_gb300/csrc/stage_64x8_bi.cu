// stage_64x8_bi.cu -- the bimodal-liquid stage kernels instantiated for tiles of 64 x 8 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_64x8(StageSet& s) { add_bimodal_variants<Tile<64, 8>>(s); }
}  // namespace ct
