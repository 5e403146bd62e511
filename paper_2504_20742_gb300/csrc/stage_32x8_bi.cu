// stage_32x8_bi.cu -- the bimodal-liquid stage kernels instantiated for tiles of 32 x 8 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_32x8(StageSet& s) { add_bimodal_variants<Tile<32, 8>>(s); }
}  // namespace ct
