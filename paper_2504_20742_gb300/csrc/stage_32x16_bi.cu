// stage_32x16_bi.cu -- the bimodal-liquid stage kernels instantiated for tiles of 32 x 16 cells.
#include "stage.cuh"

namespace ct {
void add_bimodal_32x16(StageSet& s) { add_bimodal_variants<Tile<32, 16>>(s); }
}  // namespace ct
