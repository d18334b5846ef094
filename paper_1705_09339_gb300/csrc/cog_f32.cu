// Kernels with float model-state storage.
#define COG_T float
#define COG_SUFFIX f32
#include "cog_inst.cuh"

namespace cog {
int k1_tile_pixels() { return k1_tile_pixels_impl(); }
int k2_block_threads() { return k2_block_threads_impl(); }
}  // namespace cog
