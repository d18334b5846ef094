// cog_mixture.cuh -- the plain Stauffer-Grimson mixture over a whole frame
// (the comparison baseline of the paper, Eq. 2 at rate alpha) and the
// training warm-up that runs it over the N training frames.
#pragma once

#include "cog_device.cuh"

namespace cog {

// One thread per pixel.  The CTA's tile of mixture records (256 x 16-byte-
// multiple records, contiguous) and its frame bytes arrive by TMA bulk
// copies; each thread runs the mixture step from shared memory and writes
// its record back there; one thread stores the tile's records with a TMA
// bulk store.  Every byte moves in whole, coalesced transfers.
constexpr int PLAIN_TPB = 256;

template <typename T, int K>
__host__ __device__ constexpr int plain_smem_bytes()
{
    return PLAIN_TPB * Rec<T, K>::BYTES + PLAIN_TPB * 3 + PLAIN_TPB;
}

template <typename T, int K>
__global__ void __launch_bounds__(PLAIN_TPB) plain_gmm_kernel(const DevParams dp, uint8_t *gmm,
                                                              const uint8_t *frame, uint8_t *mask,
                                                              uint32_t frame_al16, uint32_t *err)
{
    constexpr int RB = Rec<T, K>::BYTES;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *rec_s = smem;
    uint8_t *frame_s = smem + PLAIN_TPB * RB;
    uint8_t *mask_s = frame_s + PLAIN_TPB * 3;
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * PLAIN_TPB;
    if (!in_bounds(err - CTL_ERR_WORD, (uint64_t)p0, (uint64_t)dp.P, DBG_PLAIN_TILE)) return;
    const int npx = (int)min((int64_t)PLAIN_TPB, dp.P - p0);
    const int fbytes = npx * 3, fbulk = frame_al16 ? (fbytes & ~15) : 0;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, (uint32_t)(npx * RB + fbulk));
        bulk_g2s(rec_s, gmm + p0 * RB, (uint32_t)(npx * RB), &bar);
        if (fbulk) bulk_g2s(frame_s, frame + p0 * 3, (uint32_t)fbulk, &bar);
    }
    for (int i = fbulk + tid; i < fbytes; i += PLAIN_TPB) frame_s[i] = frame[p0 * 3 + i];
    __syncthreads();
    const bool timed_out = !mbar_wait(&bar, 0);
    if (__syncthreads_or(timed_out)) {
        if (tid == 0) atomicOr(err, DERR_TMA_TIMEOUT);
        return;
    }
    if (tid < npx) {
        float I[3];
#pragma unroll
        for (int c = 0; c < 3; c++) I[c] = (float)frame_s[tid * 3 + c];
        Mix<K> m;
        rec_load<T, K>(rec_s, tid, m);
        const MixOut o = mix_step<K>(m, I, dp.alpha, dp);
        rec_store<T, K>(rec_s, tid, m);
        mask_s[tid] = o.fg ? 255 : 0;
    }
    fence_async_smem();
    __syncthreads();
    const bool mask_bulk = ((uintptr_t)(mask + p0) & 15) == 0 && (npx & 15) == 0;
    if (tid == 0) {
        bulk_s2g(gmm + p0 * RB, rec_s, (uint32_t)(npx * RB));
        if (mask_bulk) bulk_s2g(mask + p0, mask_s, (uint32_t)npx);
        bulk_commit();
        bulk_wait_read0();   // shared memory must outlive the bulk reads
    }
    if (!mask_bulk && tid < npx) mask[p0 + tid] = mask_s[tid];
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
    // running average <- top-ranked component (ties to the lower index),
    // packed with the residue weights into the stage-1 record
    const uint32_t n = (uint32_t)(N - 1);
    uint32_t qa = (255u * n0 + n / 2) / n;
    uint32_t qb = (255u * n2 + n / 2) / n;
    if (qb > 255u - qa) qb = 255u - qa;
    int pos[K];
    rank_positions<K>(m, pos);
    S1Rec<T> r;
#pragma unroll
    for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (pos[k] == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) { r.set(c, m.mu[k][c]); r.set(3 + c, m.v[k][c]); }
            r.set_top(k);
        }
    }
    r.set_qab(qa | (qb << 8));
    r.store(s.s1, p);
    reinterpret_cast<T *>(s.conf)[p] = Store<T>::from_f(0.5f);
    s.jl[p] = prev[0] | (prev[1] << 8) | (prev[2] << 16) | ((uint32_t)fg << 24);
}

template <typename T, int K>
cudaError_t launch_plain_t(const DevParams &dp, const StatePtrs &s, const uint8_t *frame,
                           uint8_t *mask, cudaStream_t st)
{
    constexpr int smem = plain_smem_bytes<T, K>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(plain_gmm_kernel<T, K>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t grid = (dp.P + PLAIN_TPB - 1) / PLAIN_TPB;
    plain_gmm_kernel<T, K><<<(unsigned)grid, PLAIN_TPB, smem, st>>>(
        dp, s.gmm, frame, mask, ((uintptr_t)frame & 15) == 0, s.ctl + CTL_ERR_WORD);
    return cudaGetLastError();
}

// The same training with per-channel mixtures (COG_PERCHAN): each channel's
// component 0 starts at (I_0c, var_init, 1), the per-channel step runs over
// frames 1..N-1, and each channel's running average takes that channel's
// top-ranked component.
template <typename T, int K>
__global__ void __launch_bounds__(128) warmup_pc_kernel(const DevParams dp, const StatePtrs s,
                                                        const uint8_t *frames, int N, int r1, int r2)
{
    const int64_t p = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (p >= dp.P) return;
    const int64_t stride = dp.P * 3;
    uint32_t prev[3];
    MixPC<K> m;
#pragma unroll
    for (int c = 0; c < 3; c++) prev[c] = frames[p * 3 + c];
#pragma unroll
    for (int c = 0; c < 3; c++) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            m.w[c][k] = k == 0 ? 1.f : 0.f;
            m.mu[c][k] = k == 0 ? (float)prev[c] : 0.f;
            m.v[c][k] = dp.var_init;
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
        fg = mix_step_pc<K>(m, I, dp.alpha, dp).fg;
    }
    uint4 u[RecPC<T, K>::NV];
    mixpc_pack<T, K>(m, u);
    uint4 *dst = reinterpret_cast<uint4 *>(s.gmm + p * RecPC<T, K>::BYTES);
#pragma unroll
    for (int i = 0; i < RecPC<T, K>::NV; i++) dst[i] = u[i];
    const uint32_t n = (uint32_t)(N - 1);
    uint32_t qa = (255u * n0 + n / 2) / n;
    uint32_t qb = (255u * n2 + n / 2) / n;
    if (qb > 255u - qa) qb = 255u - qa;
    S1Rec<T> r;
#pragma unroll
    for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float wsq[K];
#pragma unroll
        for (int k = 0; k < K; k++) wsq[k] = m.w[c][k] * m.w[c][k];
#pragma unroll
        for (int k = 0; k < K; k++) {
            int cnt = 0;
#pragma unroll
            for (int j = 0; j < K; j++) {
                if (j == k) continue;
                const float x = wsq[j] * m.v[c][k], y = wsq[k] * m.v[c][j];
                cnt += (x > y) || (x == y && j < k);
            }
            if (cnt == 0) { r.set(c, m.mu[c][k]); r.set(3 + c, m.v[c][k]); }
        }
    }
    r.set_qab(qa | (qb << 8));
    r.store(s.s1, p);
    reinterpret_cast<T *>(s.conf)[p] = Store<T>::from_f(0.5f);
    s.jl[p] = prev[0] | (prev[1] << 8) | (prev[2] << 16) | ((uint32_t)fg << 24);
}

template <typename T, int K>
cudaError_t launch_warmup_t(const DevParams &dp, const StatePtrs &s, const uint8_t *frames, int N,
                            int r1, int r2, cudaStream_t st)
{
    const int64_t grid = (dp.P + 127) / 128;
    if (dp.flags & COG_PERCHAN) warmup_pc_kernel<T, K><<<(unsigned)grid, 128, 0, st>>>(dp, s, frames, N, r1, r2);
    else warmup_kernel<T, K><<<(unsigned)grid, 128, 0, st>>>(dp, s, frames, N, r1, r2);
    return cudaGetLastError();
}

}  // namespace cog
