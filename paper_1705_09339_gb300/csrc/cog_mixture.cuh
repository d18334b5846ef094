// cog_mixture.cuh -- the plain Stauffer-Grimson mixture over a whole frame
// (the comparison baseline of the paper, Eq. 2 at rate alpha) and the
// training warm-up that runs it over the N training frames.
#pragma once

#include "cog_device.cuh"

namespace cog {

// One thread per pixel: frame bytes, record, mixture step, record, mask.
template <typename T, int K>
__global__ void __launch_bounds__(256) plain_gmm_kernel(const DevParams dp, uint8_t *gmm,
                                                        const uint8_t *frame, uint8_t *mask)
{
    const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (p >= dp.P) return;
    float I[3];
#pragma unroll
    for (int c = 0; c < 3; c++) I[c] = (float)frame[p * 3 + c];
    Mix<K> m;
    rec_load<T, K>(gmm, p, m);
    const MixOut o = mix_step<K>(m, I, dp.alpha, dp);
    rec_store<T, K>(gmm, p, m);
    mask[p] = o.fg ? 255 : 0;
}

// Training (Sec. 2): per pixel, in one pass over the N frames,
//   - residue classes: R_t = max_c |I_t - I_{t-1}| binned at r1 < r2 into
//     static / oscillating / dynamic; qa <- static fraction, qb <- dynamic
//     fraction, both of 255 with round-half-up, qb clamped to 255 - qa;
//   - mixture warm-up: component 0 = (I_0, var_init, 1), the others empty
//     (weight 0, mean 0, var_init); the mixture step at rate alpha on
//     frames 1..N-1 (every rejection stage off);
// then the running average takes the top-ranked mode, C = 0.5, and the
// previous frame and label are those of the last training frame.
template <typename T, int K>
__global__ void __launch_bounds__(128) warmup_kernel(const DevParams dp, const StatePtrs s,
                                                     const uint8_t *frames, int N, int r1, int r2)
{
    const int64_t p = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (p >= dp.P) return;
    const int64_t stride = dp.P * 3;
    uint32_t prev[3];
    Mix<K> m;
#pragma unroll
    for (int c = 0; c < 3; c++) prev[c] = frames[p * 3 + c];
#pragma unroll
    for (int k = 0; k < K; k++) {
        m.w[k] = k == 0 ? 1.f : 0.f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m.mu[k][c] = k == 0 ? (float)prev[c] : 0.f;
            m.v[k][c] = dp.var_init;
        }
    }
    uint32_t n0 = 0, n2 = 0;
    int fg = 0;
    const uint8_t *f = frames + p * 3;
    for (int t = 1; t < N; t++) {
        f += stride;
        float I[3];
        int R = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const uint32_t v = f[c];
            const int d = abs((int)v - (int)prev[c]);
            R = d > R ? d : R;
            prev[c] = v;
            I[c] = (float)v;
        }
        n0 += R <= r1;
        n2 += R > r2;
        fg = mix_step<K>(m, I, dp.alpha, dp).fg;
    }
    rec_store<T, K>(s.gmm, p, m);
    // running average <- top-ranked component (ties to the lower index)
    int best = 0;
    float rb = -1.f;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const float vbar = (m.v[k][0] + m.v[k][1] + m.v[k][2]) / 3.0f;
        const float r = m.w[k] * m.w[k] / vbar;
        if (r > rb) { rb = r; best = k; }
    }
    T *rga = reinterpret_cast<T *>(s.rga);
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (k == best) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                rga[c * s.rga_plane + p] = Store<T>::from_f(m.mu[k][c]);
                rga[(3 + c) * s.rga_plane + p] = Store<T>::from_f(m.v[k][c]);
            }
        }
    }
    reinterpret_cast<T *>(s.conf)[p] = Store<T>::from_f(0.5f);
    s.jl[p] = prev[0] | (prev[1] << 8) | (prev[2] << 16) | ((uint32_t)fg << 24);
    const uint32_t n = (uint32_t)(N - 1);
    uint32_t qa = (255u * n0 + n / 2) / n;
    uint32_t qb = (255u * n2 + n / 2) / n;
    if (qb > 255u - qa) qb = 255u - qa;
    s.qab[p] = (uint16_t)(qa | (qb << 8));
}

template <typename T, int K>
cudaError_t launch_plain_t(const DevParams &dp, const StatePtrs &s, const uint8_t *frame,
                           uint8_t *mask, cudaStream_t st)
{
    const int64_t grid = (dp.P + 255) / 256;
    plain_gmm_kernel<T, K><<<(unsigned)grid, 256, 0, st>>>(dp, s.gmm, frame, mask);
    return cudaGetLastError();
}

template <typename T, int K>
cudaError_t launch_warmup_t(const DevParams &dp, const StatePtrs &s, const uint8_t *frames, int N,
                            int r1, int r2, cudaStream_t st)
{
    const int64_t grid = (dp.P + 127) / 128;
    warmup_kernel<T, K><<<(unsigned)grid, 128, 0, st>>>(dp, s, frames, N, r1, r2);
    return cudaGetLastError();
}

}  // namespace cog
