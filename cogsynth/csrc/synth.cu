// synth.cu -- CUDA twin of the numpy scene renderer (input generation only).
#include <cuda_runtime.h>

#include "cogsynth.h"

namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int64_t NOISE_DEN = 605395, NOISE_MEAN = 131070, NOISE_BIAS = 64;

__global__ void __launch_bounds__(256) render_kernel(const cogsynth_scene sc, const cogsynth_frame *frames,
                                                     uint8_t *out, uint8_t *gt)
{
    const int64_t P = (int64_t)sc.width * sc.height;
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= P) return;
    const cogsynth_frame &f = frames[blockIdx.y];
    const int x = (int)(p % sc.width), y = (int)(p / sc.width);
    int base[3];
    for (int c = 0; c < 3; c++) base[c] = sc.bg[p * 3 + c];
    if (sc.n_blobs > 0) {
        const int b = sc.blob_id[p];
        if (b >= 0 && ((f.modes[b >> 5] >> (b & 31)) & 1u))
            for (int c = 0; c < 3; c++) base[c] += sc.blob_delta[b * 3 + c];
        if (x >= sc.sway_x0 && x < sc.sway_x1 && y >= sc.sway_y0 && y < sc.sway_y1)
            for (int c = 0; c < 3; c++) base[c] += f.sway;
    }
    int inside_any = 0;
    for (int o = 0; o < f.n_obj; o++) {
        const int32_t *ob = f.obj[o];
        int ins;
        if (ob[0] == 0) {
            ins = x >= ob[1] && x < ob[3] && y >= ob[2] && y < ob[4];
        } else {
            const int64_t dx = x - ob[1], dy = y - ob[2], a = ob[3], b = ob[4];
            ins = (dx * b) * (dx * b) + (dy * a) * (dy * a) <= (a * b) * (a * b);
        }
        if (ins) {
            base[0] = ob[5]; base[1] = ob[6]; base[2] = ob[7];
            inside_any = 1;
        }
    }
    const int64_t sig = sc.sig16[p];
    uint8_t *dst = out + ((int64_t)blockIdx.y * P + p) * 3;
    for (int c = 0; c < 3; c++) {
        const uint64_t u = sm64(f.noise_base ^ (((uint64_t)p << 2) | (uint64_t)c));
        const int64_t s = (int64_t)(u & 0xFFFF) + (int64_t)((u >> 16) & 0xFFFF) +
                          (int64_t)((u >> 32) & 0xFFFF) + (int64_t)(u >> 48);
        const int64_t z = s - NOISE_MEAN;
        const int64_t n = (z * sig + NOISE_DEN / 2 + NOISE_BIAS * NOISE_DEN) / NOISE_DEN - NOISE_BIAS;
        int64_t v = base[c] + f.offset + n;
        v = v < 0 ? 0 : (v > 255 ? 255 : v);
        dst[c] = (uint8_t)v;
    }
    if (gt) gt[(int64_t)blockIdx.y * P + p] = inside_any ? 255 : 0;
}

}  // namespace

extern "C" int cogsynth_render(const cogsynth_scene *sc, const cogsynth_frame *frames_dev, int32_t n,
                               uint8_t *out_dev, uint8_t *gt_dev, void *stream)
{
    if (!sc || !frames_dev || !out_dev || n < 0 || n > 65535) return (int)cudaErrorInvalidValue;
    if (n == 0) return 0;
    const int64_t P = (int64_t)sc->width * sc->height;
    dim3 grid((unsigned)((P + 255) / 256), (unsigned)n);
    render_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(*sc, frames_dev, out_dev, gt_dev);
    return (int)cudaGetLastError();
}
