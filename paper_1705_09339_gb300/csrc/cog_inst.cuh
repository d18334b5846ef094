// cog_inst.cuh -- instantiates the per-storage-type kernels for K = 1..8.
// Included once per storage type (COG_T, COG_SUFFIX) so the three types
// compile as separate translation units in parallel.
#include "cog_apply.cuh"
#include "cog_mixture.cuh"
#include "cog_clip.cuh"

#define COG_CAT2(a, b) a##b
#define COG_CAT(a, b) COG_CAT2(a, b)

namespace cog {

#define COG_KSWITCH(CALL)                 \
    switch (K) {                          \
    case 1: return CALL(1);               \
    case 2: return CALL(2);               \
    case 3: return CALL(3);               \
    case 4: return CALL(4);               \
    case 5: return CALL(5);               \
    case 6: return CALL(6);               \
    case 7: return CALL(7);               \
    case 8: return CALL(8);               \
    default: return cudaErrorInvalidValue; \
    }

cudaError_t COG_CAT(launch_apply_, COG_SUFFIX)(int K, const ApplyArgs &a, const LaunchCfg &lc, cudaStream_t st,
                                               const ApplyEvents *ev)
{
#define CALL_A(k) launch_apply_t<COG_T, k>(a, lc, st, ev)
    COG_KSWITCH(CALL_A)
#undef CALL_A
}

cudaError_t COG_CAT(launch_batch_, COG_SUFFIX)(int K, const BatchGroupDev &g, const LaunchCfg &lc, uint32_t k1,
                                               uint32_t k2, cudaStream_t st)
{
#define CALL_B(k) launch_batch_t<COG_T, k>(g, lc, k1, k2, st)
    COG_KSWITCH(CALL_B)
#undef CALL_B
}

int COG_CAT(k2_blocks_per_sm_, COG_SUFFIX)(int K, const LaunchCfg &lc, int mv)
{
    switch (K) {
    case 1: return k2_blocks_per_sm_t<COG_T, 1>(lc, mv);
    case 2: return k2_blocks_per_sm_t<COG_T, 2>(lc, mv);
    case 3: return k2_blocks_per_sm_t<COG_T, 3>(lc, mv);
    case 4: return k2_blocks_per_sm_t<COG_T, 4>(lc, mv);
    case 5: return k2_blocks_per_sm_t<COG_T, 5>(lc, mv);
    case 6: return k2_blocks_per_sm_t<COG_T, 6>(lc, mv);
    case 7: return k2_blocks_per_sm_t<COG_T, 7>(lc, mv);
    default: return k2_blocks_per_sm_t<COG_T, 8>(lc, mv);
    }
}

cudaError_t COG_CAT(launch_clip_, COG_SUFFIX)(int K, const ClipArgs &a, int n_sm, cudaStream_t st)
{
#define CALL_C(k) launch_clip_t<COG_T, k>(a, n_sm, st)
    COG_KSWITCH(CALL_C)
#undef CALL_C
}

int COG_CAT(k1_batch_blocks_per_sm_, COG_SUFFIX)(const LaunchCfg &lc)
{
    return k1_batch_blocks_per_sm_t<COG_T>(lc);
}

cudaError_t COG_CAT(launch_plain_, COG_SUFFIX)(int K, const DevParams &dp, const StatePtrs &s,
                                               const uint8_t *frame, uint8_t *mask, cudaStream_t st)
{
#define CALL_P(k) launch_plain_t<COG_T, k>(dp, s, frame, mask, st)
    COG_KSWITCH(CALL_P)
#undef CALL_P
}

cudaError_t COG_CAT(launch_warmup_, COG_SUFFIX)(int K, const DevParams &dp, const StatePtrs &s,
                                                const uint8_t *frames, int N, int r1, int r2,
                                                cudaStream_t st)
{
#define CALL_W(k) launch_warmup_t<COG_T, k>(dp, s, frames, N, r1, r2, st)
    COG_KSWITCH(CALL_W)
#undef CALL_W
}

}  // namespace cog
