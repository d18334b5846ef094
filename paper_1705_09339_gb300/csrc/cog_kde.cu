// cog_kde.cu -- the scene prior of Sec. 2 ("Scene Prior in Background
// Model"): per pixel and channel, a kernel density of the N training values
// with a Gaussian kernel of bandwidth bw, evaluated on the 256 grey levels in
// exact integer arithmetic and normalised to its peak:
//   h[u] = #{t : I_t = u},  k[v] = sum_{|v-u| <= 3bw} h[u] g[|v-u|],
//   q[v] = (Q k[v] + M/2) div M,  M = max_v k[v],
// with g[d] = round(2^16 exp(-d^2 / (2 bw^2))) computed on the host and
// Q = 255 for the 8-bit prior (one byte per level, 256-byte rows) or 15 for
// the 4-bit one (two levels per byte, the even grey level in the low
// nibble, 128-byte rows).
//
// Layout: warp w owns the 32 channel histograms b = 32w .. 32w + 31 (b =
// 3p + c, the prior's row order), so its lanes read 32 consecutive bytes of
// every frame.  Each lane counts its own histogram in shared memory (uint16,
// N < 65536) between KDE_PAD zero guards on each side (rows of KDE_ROW
// entries start the 32 lanes' rows in 32 different banks), loads KDE_UNROLL frames before adding
// them so that many loads are in flight, and keeps the smallest and largest
// value it saw.  The density is zero more than 3bw levels from every
// sample, so it is evaluated only on [min - 3bw, max + 3bw]: the warp then
// takes its histograms one at a time, each lane on a level of the support,
// so a histogram costs its support / 32 steps whatever its neighbours'
// supports.  For the default bandwidth (3bw = 12) the 25 taps are unrolled
// against the guarded row: one shared load and one multiply-add per tap.
#include "cog_internal.h"

namespace cog {

constexpr int KDE_WARPS = 2;
constexpr int KDE_TPB = KDE_WARPS * 32;
constexpr int KDE_PAD = 12;                       // zero guards around the 256 bins (3bw at bw = 4)
constexpr int KDE_ROW = 256 + 2 * KDE_PAD + 2;    // 141 words: lane l's row starts in bank 13 l mod 32
constexpr int KDE_UNROLL = 32;
constexpr int KDE_SMEM = KDE_WARPS * 32 * KDE_ROW * 2 + KDE_WARPS * 256;   // rows + staging lines

struct KdeW {
    uint32_t g[100];
    int R;
    uint32_t Q;   // top level: 255 (8-bit prior) or 15 (4-bit)
};

// k[v] = sum over |d| <= R of h[v + d] g[|d|], h zero outside [vmin, vmax]
__device__ __forceinline__ uint32_t kde_density(const uint16_t *h, int v, int vmin, int vmax, const KdeW &w)
{
    uint32_t acc = 0;
    for (int d = -w.R; d <= w.R; d++) {
        const int u = v + d;
        if (u >= vmin && u <= vmax) acc += (uint32_t)h[u] * w.g[d < 0 ? -d : d];
    }
    return acc;
}

// The same density with the taps unrolled (R <= KDE_PAD): h points at bin 0
// of a guarded row, so h[v + d] is zero wherever the histogram is.
template <int R>
__device__ __forceinline__ uint32_t kde_density_r(const uint16_t *h, int v, const KdeW &w)
{
    uint32_t acc = (uint32_t)h[v] * w.g[0];
#pragma unroll
    for (int d = 1; d <= R; d++) acc += ((uint32_t)h[v - d] + (uint32_t)h[v + d]) * w.g[d];
    return acc;
}

// q = floor((Q k + M/2) / M), exactly: a float estimate, then corrected
__device__ __forceinline__ uint32_t kde_quant(uint32_t k, uint64_t M, float rM, uint32_t Q)
{
    const uint64_t num = (uint64_t)Q * k + M / 2;
    uint32_t q = (uint32_t)((float)num * rM);
    while (q > 0 && (uint64_t)q * M > num) q--;
    while ((uint64_t)(q + 1) * M <= num) q++;
    return q;
}

// RF: the unrolled tap count R (12), or 0 for any R (bounds-checked taps)
template <int RF>
__global__ void __launch_bounds__(KDE_TPB) kde_kernel(int64_t P, const uint8_t *frames, int N, uint8_t *kde,
                                                      const KdeW w)
{
    extern __shared__ __align__(16) uint16_t kh[];   // [KDE_TPB][KDE_ROW]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = ((int64_t)blockIdx.x * KDE_WARPS + warp) * 32 + lane;
    const bool act = b < P * 3;
    uint16_t *row = kh + threadIdx.x * KDE_ROW;
    for (int v = 0; v < KDE_ROW; v += 2) *reinterpret_cast<uint32_t *>(row + v) = 0u;
    uint16_t *h = row + KDE_PAD;
    int vmin = 255, vmax = 0;
    const uint8_t *src = frames + b;
    const int64_t stride = P * 3;
    for (int t0 = 0; t0 < N; t0 += KDE_UNROLL) {
        uint32_t x[KDE_UNROLL];
#pragma unroll
        for (int i = 0; i < KDE_UNROLL; i++) x[i] = act && t0 + i < N ? (uint32_t)__ldcs(src + (int64_t)(t0 + i) * stride) : 256u;
#pragma unroll
        for (int i = 0; i < KDE_UNROLL; i++)
            if (x[i] < 256u) {
                h[x[i]]++;
                vmin = min(vmin, (int)x[i]);
                vmax = max(vmax, (int)x[i]);
            }
    }
    // the density: the warp takes its 32 histograms one after another, its
    // lanes on consecutive levels of the support (conflict-free reads of
    // one row), keeps the values in registers for the peak M, and writes
    // the row (256 levels, or 128 bytes of level pairs) through a per-warp
    // staging line
    uint8_t *stage = reinterpret_cast<uint8_t *>(kh + KDE_TPB * KDE_ROW) + warp * 256;
    const int lo_l = max(0, vmin - w.R), hi_l = act ? min(255, vmax + w.R) : -1;
    __syncwarp();
    for (int l = 0; l < 32; l++) {
        const int64_t bl = b - lane + l;
        if (bl >= P * 3) break;   // the same for every lane
        const int LO = __shfl_sync(0xffffffffu, lo_l, l), HI = __shfl_sync(0xffffffffu, hi_l, l);
        const int VMIN = __shfl_sync(0xffffffffu, vmin, l), VMAX = __shfl_sync(0xffffffffu, vmax, l);
        const uint16_t *hl = kh + (warp * 32 + l) * KDE_ROW + KDE_PAD;
        uint32_t kv[8], m = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int v = LO + lane + 32 * i;
            uint32_t k = 0;
            if (LO + 32 * i <= HI && v <= HI) {
                if constexpr (RF > 0) k = kde_density_r<RF>(hl, v, w);
                else k = kde_density(hl, v, VMIN, VMAX, w);
            }
            kv[i] = k;
            m = max(m, k);
        }
        const uint32_t M = __reduce_max_sync(0xffffffffu, m);
        const float rM = 1.0f / (float)M;
        *reinterpret_cast<uint2 *>(stage + 8 * lane) = make_uint2(0u, 0u);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int v = LO + lane + 32 * i;
            if (LO + 32 * i <= HI && v <= HI) stage[v] = (uint8_t)kde_quant(kv[i], M, rM, w.Q);
        }
        __syncwarp();
        const uint2 lv = *reinterpret_cast<const uint2 *>(stage + 8 * lane);   // levels 8 lane .. 8 lane + 7
        if (w.Q == 255u) {
            reinterpret_cast<uint2 *>(kde + bl * 256)[lane] = lv;
        } else {
            // levels < 16: byte j of the row is level 2j | level 2j+1 << 4
            const uint32_t lo = lv.x | (lv.x >> 4), hi = lv.y | (lv.y >> 4);
            reinterpret_cast<uint32_t *>(kde + bl * 128)[lane] = __byte_perm(lo, hi, 0x6420);
        }
        __syncwarp();   // the staging line is rewritten for the next histogram
    }
}

cudaError_t launch_kde_train(const DevParams &dp, const StatePtrs &s, const uint8_t *frames,
                             int n_frames, const uint32_t *g, int R, cudaStream_t st)
{
    if (R < 0 || R > 96) return cudaErrorInvalidValue;
    if (dp.kde_bits != 8 && dp.kde_bits != 4) return cudaErrorInvalidValue;
    KdeW w;
    for (int d = 0; d < 100; d++) w.g[d] = d <= R ? g[d] : 0u;
    w.R = R;
    w.Q = (1u << dp.kde_bits) - 1u;
    if (n_frames >= 65536) return cudaErrorInvalidValue;   // uint16 counts
    static_assert(KDE_PAD >= 12, "the unrolled taps read 12 levels past the bins");
    auto kern = R == 12 ? kde_kernel<12> : kde_kernel<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, KDE_SMEM);
    if (e != cudaSuccess) return e;
    const int64_t grid = (dp.P * 3 + KDE_TPB - 1) / KDE_TPB;
    kern<<<(unsigned)grid, KDE_TPB, KDE_SMEM, st>>>(dp.P, frames, n_frames, s.kde, w);
    return cudaGetLastError();
}

}  // namespace cog
