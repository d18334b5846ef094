// Kernels with __nv_bfloat16 model-state storage.
#define COG_T __nv_bfloat16
#define COG_SUFFIX bf16
#include "cog_inst.cuh"
