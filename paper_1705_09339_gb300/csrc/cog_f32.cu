// Kernels with float model-state storage.
#define COG_T float
#define COG_SUFFIX f32
#include "cog_inst.cuh"

