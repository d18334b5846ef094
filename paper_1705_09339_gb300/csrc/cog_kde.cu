// cog_kde.cu -- the scene prior of Sec. 2 ("Scene Prior in Background
// Model"): per pixel and channel, a kernel density of the N training values
// with a Gaussian kernel of bandwidth bw, evaluated on the 256 grey levels in
// exact integer arithmetic and normalised to its peak:
//   h[u] = #{t : I_t = u},  k[v] = sum_{|v-u| <= 3bw} h[u] g[|v-u|],
//   q[v] = (255 k[v] + M/2) div M,  M = max_v k[v],
// with g[d] = round(2^16 exp(-d^2 / (2 bw^2))) computed on the host.
//
// A CTA owns 16 pixels (48 channel histograms): shared-memory histograms
// filled with shared atomics, the 256-level convolution from shared memory,
// a warp max per histogram, and the quantised prior written as one
// contiguous 12 KB block (the prior is stored [P][3][256]).
#include "cog_internal.h"

namespace cog {

constexpr int KDE_PX = 16;
constexpr int KDE_TPB = 256;
constexpr int KDE_NB = KDE_PX * 3;
constexpr int KDE_SMEM = 2 * KDE_NB * 256 * 4;   // histograms + densities

struct KdeW {
    uint32_t g[100];
    int R;
};

__global__ void __launch_bounds__(KDE_TPB) kde_kernel(int64_t P, const uint8_t *frames, int N,
                                                      uint8_t *kde, const KdeW w)
{
    extern __shared__ __align__(16) uint32_t ks[];
    uint32_t *hist = ks;                    // [48][256]
    uint32_t *dens = ks + KDE_NB * 256;     // [48][256]
    __shared__ uint32_t Ms[KDE_NB];
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * KDE_PX;
    const int npx = (int)min((int64_t)KDE_PX, P - p0);
    const int nb = npx * 3;

    for (int i = tid; i < KDE_NB * 256; i += KDE_TPB) hist[i] = 0;
    __syncthreads();
    const uint8_t *base = frames + p0 * 3;
    const int64_t stride = P * 3;
    const int total = N * nb;
    for (int idx = tid; idx < total; idx += KDE_TPB) {
        const int t = idx / nb;
        const int b = idx - t * nb;
        const uint32_t v = base[(int64_t)t * stride + b];
        atomicAdd(&hist[b * 256 + v], 1u);
    }
    __syncthreads();
    const int R = w.R;
    for (int o = tid; o < nb * 256; o += KDE_TPB) {
        const int b = o >> 8, v = o & 255;
        const uint32_t *h = hist + b * 256;
        const int lo = max(0, v - R), hi = min(255, v + R);
        uint32_t acc = 0;
        for (int u = lo; u <= hi; u++) acc += h[u] * w.g[abs(v - u)];
        dens[o] = acc;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int b = warp; b < nb; b += KDE_TPB / 32) {
        uint32_t mx = 0;
        for (int v = lane; v < 256; v += 32) mx = max(mx, dens[b * 256 + v]);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) Ms[b] = mx;
    }
    __syncthreads();
    uint32_t *out = reinterpret_cast<uint32_t *>(kde + p0 * 768);
    for (int o4 = tid; o4 < nb * 64; o4 += KDE_TPB) {
        const int b = o4 >> 6;
        const uint64_t M = Ms[b];
        const float rM = 1.0f / (float)M;
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint64_t num = 255ull * dens[o4 * 4 + j] + M / 2;
            uint32_t q = (uint32_t)((float)num * rM);      // estimate, then exact fix-up
            while (q > 0 && (uint64_t)q * M > num) q--;
            while ((uint64_t)(q + 1) * M <= num) q++;
            word |= q << (8 * j);
        }
        out[o4] = word;
    }
}

cudaError_t launch_kde_train(const DevParams &dp, const StatePtrs &s, const uint8_t *frames,
                             int n_frames, const uint32_t *g, int R, cudaStream_t st)
{
    if (R < 0 || R > 96) return cudaErrorInvalidValue;
    KdeW w;
    for (int d = 0; d < 100; d++) w.g[d] = d <= R ? g[d] : 0u;
    w.R = R;
    cudaError_t e = cudaFuncSetAttribute(kde_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, KDE_SMEM);
    if (e != cudaSuccess) return e;
    const int64_t grid = (dp.P + KDE_PX - 1) / KDE_PX;
    kde_kernel<<<(unsigned)grid, KDE_TPB, KDE_SMEM, st>>>(dp.P, frames, n_frames, s.kde, w);
    return cudaGetLastError();
}

}  // namespace cog
