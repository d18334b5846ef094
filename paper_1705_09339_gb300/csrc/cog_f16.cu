// Kernels with __half model-state storage.
#define COG_T __half
#define COG_SUFFIX f16
#include "cog_inst.cuh"
