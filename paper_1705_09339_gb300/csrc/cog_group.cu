// cog_group.cu -- spatio-temporal grouping on the training frames (Sec. 2,
// "Clustering Similar Background - Spatio-Temporal Grouping", steps 1-6 and
// Eq. 3), for pixels that share the mixture's update behaviour:
//   features   the warm-up replayed over the N training frames; after each
//              update at frames 1..N-1 the dominant mode (rank 1 of
//              omega^2 / vbar, lower index on ties) gives vbar and omega;
//              per pixel the population standard deviations of the two
//              series over time, coded round(64 sd_v) and round(65536 sd_w)
//              (saturated at 65535);
//   K-means    K = 3 over the two codes, each scaled by its standard
//              deviation over all pixels (1 for a constant code), first
//              centroids at mean - sd, mean, mean + sd (sd = 0 for a
//              constant code), an empty cluster keeping its centroid, ties
//              to the lower cluster, until no label changes (at most
//              GROUP_MAX_IT steps, or the caller's limit); the distance is
//              evaluated in FP32, so a pixel whose two nearest centroids
//              are within FP32 rounding of a tie may go either way;
//   Eq. 3      core pixel: both codes strictly within the cluster's mean
//              +- standard deviation;
//   step 6     per cluster, the mean over its core of the trained state's
//              dominant mode (weight, means, mean variance).
// The clustering works on integer sums (exact with atomics in any order),
// and every floating-point operation is an explicitly rounded intrinsic, so
// the result does not depend on the launch shape or the atomics' order.
#include <cmath>

#include "cog_device.cuh"

namespace cog {

constexpr int GROUP_MAX_IT = 64;
constexpr int GROUP_TPB = 256;

// Grouping scratch inside the control block (zeroed by the launcher).
struct GroupBuf {
    unsigned long long n[3], s1[3][2], s2[3][2];   // per cluster: count, sums of codes and squares
    double c[3][2];                                // centroids this iteration used
    unsigned long long changed;                    // labels that changed this iteration
};
struct GroupCtl {
    unsigned long long g1[2], g2[2];               // sums over all pixels of the codes and squares
    GroupBuf buf[3];                               // iteration it uses buf[it % 3]
    unsigned long long conv_iter;                  // first iteration that changed nothing (0: none yet)
    unsigned long long n_core[3];
    double par[3][5];                              // core sums: omega, mu0, mu1, mu2, vbar
};
constexpr int CTL_GROUP_WORD = CTL_QCNT_WORD + 3 * QSEG * CTL_PAD;
static_assert(CTL_GROUP_WORD % 2 == 0, "8-byte alignment of the grouping scratch");
static_assert(CTL_GROUP_WORD * 4 + (int)sizeof(GroupCtl) <= CTL_BYTES, "grouping scratch fits the control block");

__device__ __forceinline__ GroupCtl *group_ctl(uint32_t *ctl) { return reinterpret_cast<GroupCtl *>(ctl + CTL_GROUP_WORD); }

// ---------------------------------------------------------------- features
// One thread per pixel: the warm-up of warmup_kernel (same start, same
// mixture step on frames 1..N-1) with the running mean and squared
// deviation of the dominant mode's vbar and omega (Welford's update, FP32).
template <int K>
__global__ void __launch_bounds__(128) group_features_kernel(const DevParams dp, const uint8_t *frames, int N,
                                                             uint16_t *code_v, uint16_t *code_w, GroupCtl *G)
{
    const int64_t p = (int64_t)blockIdx.x * 128 + threadIdx.x;
    uint32_t qv = 0, qw = 0;
    if (p < dp.P) {
        const int64_t stride = dp.P * 3;
        Mix<K> m;
#pragma unroll
        for (int k = 0; k < K; k++) {
            m.w[k] = k == 0 ? 1.f : 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                m.mu[k][c] = k == 0 ? (float)frames[p * 3 + c] : 0.f;
                m.v[k][c] = dp.var_init;
            }
        }
        float mv = 0.f, m2v = 0.f, mw = 0.f, m2w = 0.f;
        const uint8_t *f = frames + p * 3;
        for (int t = 1; t < N; t++) {
            f += stride;
            float I[3];
#pragma unroll
            for (int c = 0; c < 3; c++) I[c] = (float)f[c];
            mix_step<K>(m, I, dp.alpha, dp);
            // the dominant mode: largest w^2 / vbar in the division-free
            // form of rank_positions, the lower index on ties
            int top = 0;
            float wt = m.w[0] * m.w[0], vt = m.v[0][0] + m.v[0][1] + m.v[0][2];
#pragma unroll
            for (int k = 1; k < K; k++) {
                const float wk = m.w[k] * m.w[k], vk = m.v[k][0] + m.v[k][1] + m.v[k][2];
                if (wk * vt > wt * vk) {
                    top = k;
                    wt = wk;
                    vt = vk;
                }
            }
            float vb = 0.f, om = 0.f;
#pragma unroll
            for (int k = 0; k < K; k++)
                if (k == top) {
                    vb = vt / 3.f;
                    om = m.w[k];
                }
            const float rn = 1.f / (float)t;
            const float dv = vb - mv, dw = om - mw;
            mv += dv * rn;
            mw += dw * rn;
            m2v += dv * (vb - mv);
            m2w += dw * (om - mw);
        }
        const float n = (float)(N - 1);
        const float sdv = sqrtf(fmaxf(m2v / n, 0.f)), sdw = sqrtf(fmaxf(m2w / n, 0.f));
        const float cv = floorf(sdv * 64.f + 0.5f), cw = floorf(sdw * 65536.f + 0.5f);
        qv = cv > 65535.f ? 65535u : (uint32_t)cv;
        qw = cw > 65535.f ? 65535u : (uint32_t)cw;
        code_v[p] = (uint16_t)qv;
        code_w[p] = (uint16_t)qw;
    }
    // sums over all pixels: per warp, then one atomic per warp and sum
    unsigned long long a[4] = {qv, qw, (unsigned long long)qv * qv, (unsigned long long)qw * qw};
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], off);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&G->g1[0], a[0]);
        atomicAdd(&G->g1[1], a[1]);
        atomicAdd(&G->g2[0], a[2]);
        atomicAdd(&G->g2[1], a[3]);
    }
}

// Sums over all pixels of caller-given codes and their squares (the
// features kernel accumulates the same sums as it writes its codes).
__global__ void __launch_bounds__(GROUP_TPB) group_sums_kernel(int64_t P, const uint16_t *code_v, const uint16_t *code_w,
                                                               GroupCtl *G)
{
    unsigned long long a[4] = {0, 0, 0, 0};
    for (int64_t p = (int64_t)blockIdx.x * GROUP_TPB + threadIdx.x; p < P; p += (int64_t)gridDim.x * GROUP_TPB) {
        const unsigned long long qv = code_v[p], qw = code_w[p];
        a[0] += qv;
        a[1] += qw;
        a[2] += qv * qv;
        a[3] += qw * qw;
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], off);
    if ((threadIdx.x & 31) == 0) {
        if (a[0]) atomicAdd(&G->g1[0], a[0]);
        if (a[1]) atomicAdd(&G->g1[1], a[1]);
        if (a[2]) atomicAdd(&G->g2[0], a[2]);
        if (a[3]) atomicAdd(&G->g2[1], a[3]);
    }
}

// ------------------------------------------------------------------ K-means
// Feature scales from the sums over all pixels: sd0 the spread (0 for a
// constant code), sd the distance scale (1 for a constant code).
__device__ __forceinline__ void group_scales(const GroupCtl *G, double P, double mean[2], double sd0[2], double sd[2])
{
#pragma unroll
    for (int f = 0; f < 2; f++) {
        mean[f] = __ddiv_rn(__ull2double_rn(G->g1[f]), P);
        const double v = __dsub_rn(__ddiv_rn(__ull2double_rn(G->g2[f]), P), __dmul_rn(mean[f], mean[f]));
        sd0[f] = v > 0.0 ? __dsqrt_rn(v) : 0.0;
        sd[f] = v > 0.0 ? sd0[f] : 1.0;
    }
}

// Nearest of the three centroids in the scaled distance, ties to the lower,
// decided in FP32: float centroids cf and reciprocal scales iv, iw (each
// rounded once from double), every operation rounded separately.
__device__ __forceinline__ int group_nearest(uint32_t qv, uint32_t qw, const float (*cf)[2], float iv, float iw)
{
    int best = 0;
    float db = 0.f;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float tv = __fmul_rn(__fsub_rn((float)qv, cf[j][0]), iv);
        const float tw = __fmul_rn(__fsub_rn((float)qw, cf[j][1]), iw);
        const float d = __fadd_rn(__fmul_rn(tv, tv), __fmul_rn(tw, tw));
        if (j == 0 || d < db) {
            db = d;
            best = j;
        }
    }
    return best;
}

// 64-bit warp sum.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// Iteration `it` of the clustering (it = 0: first assignment from the
// initial centroids).  Iteration it >= 1 takes the centroids from the
// member sums of iteration it - 1 (an empty cluster keeps its centroid),
// reassigns every pixel in place and sums its clusters into buf[it % 3].
// Once an iteration has changed nothing, the later ones only carry its
// buffer forward.
__global__ void __launch_bounds__(GROUP_TPB) group_assign_kernel(int64_t P, const uint16_t *code_v, const uint16_t *code_w,
                                                                 uint8_t *labels, GroupCtl *G, int it)
{
    __shared__ double c_s[3][2];
    __shared__ float cf_s[3][2], is_s[2];
    __shared__ int skip_s;
    __shared__ unsigned long long acc_s[16];   // n[3], s1[3][2], s2[3][2], changed
    const int tid = threadIdx.x;
    GroupBuf &out = G->buf[it % 3];
    if (tid == 0) {
        double mean[2], sd0[2], sd[2];
        group_scales(G, (double)P, mean, sd0, sd);
        is_s[0] = __double2float_rn(__ddiv_rn(1.0, sd[0]));
        is_s[1] = __double2float_rn(__ddiv_rn(1.0, sd[1]));
        int skip = 0;
        if (it == 0) {
            for (int j = 0; j < 3; j++)
                for (int f = 0; f < 2; f++) c_s[j][f] = __dadd_rn(mean[f], __dmul_rn((double)(j - 1), sd0[f]));
        } else {
            const GroupBuf &in = G->buf[(it - 1) % 3];
            skip = it >= 2 && in.changed == 0;
            for (int j = 0; j < 3; j++)
                for (int f = 0; f < 2; f++)
                    c_s[j][f] = in.n[j] ? __ddiv_rn(__ull2double_rn(in.s1[j][f]), __ull2double_rn(in.n[j])) : in.c[j][f];
        }
        skip_s = skip;
        for (int j = 0; j < 3; j++)
            for (int f = 0; f < 2; f++) cf_s[j][f] = __double2float_rn(c_s[j][f]);
    }
    if (tid < 16) acc_s[tid] = 0;
    __syncthreads();
    if (skip_s) {
        // converged at an earlier iteration: carry its buffer forward
        if (blockIdx.x == 0 && tid == 0) {
            out = G->buf[(it - 1) % 3];
            if (G->conv_iter == 0) G->conv_iter = (unsigned long long)(it - 1);
            G->buf[(it + 1) % 3] = GroupBuf{};
        }
        return;
    }
    if (blockIdx.x == 0 && tid == 0) {
        for (int j = 0; j < 3; j++)
            for (int f = 0; f < 2; f++) out.c[j][f] = c_s[j][f];
        if (it >= 1) G->buf[(it + 1) % 3] = GroupBuf{};   // iteration it - 2's buffer, read by nobody now
    }
    unsigned long long n[3] = {0, 0, 0}, s1[3][2] = {{0, 0}, {0, 0}, {0, 0}}, s2[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    unsigned long long ch = 0;
    for (int64_t p = (int64_t)blockIdx.x * GROUP_TPB + tid; p < P; p += (int64_t)gridDim.x * GROUP_TPB) {
        const uint32_t qv = code_v[p], qw = code_w[p];
        const int l = group_nearest(qv, qw, cf_s, is_s[0], is_s[1]);
        if (it > 0) ch += labels[p] != l;
        labels[p] = (uint8_t)l;
#pragma unroll
        for (int j = 0; j < 3; j++)
            if (l == j) {
                n[j]++;
                s1[j][0] += qv;
                s1[j][1] += qw;
                s2[j][0] += (unsigned long long)qv * qv;
                s2[j][1] += (unsigned long long)qw * qw;
            }
    }
    unsigned long long v[16] = {n[0], n[1], n[2], s1[0][0], s1[0][1], s1[1][0], s1[1][1], s1[2][0], s1[2][1],
                                s2[0][0], s2[0][1], s2[1][0], s2[1][1], s2[2][0], s2[2][1], ch};
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const unsigned long long x = warp_sum_u64(v[i]);
        if ((tid & 31) == 0 && x) atomicAdd(&acc_s[i], x);
    }
    __syncthreads();
    if (tid < 16 && acc_s[tid]) {
        unsigned long long *dst = tid < 3 ? &out.n[tid]
                                : tid < 9 ? &out.s1[(tid - 3) / 2][(tid - 3) % 2]
                                : tid < 15 ? &out.s2[(tid - 9) / 2][(tid - 9) % 2] : &out.changed;
        atomicAdd(dst, acc_s[tid]);
    }
}


// -------------------------------------------------- Eq. 3 cores and step 6
// Cluster means and standard deviations of the final labels' codes; a pixel
// whose two codes both lie strictly within them is a core pixel
// (labels |= 0x80), and its trained dominant mode -- the stage-1 record's
// copy of the top-ranked component (means, variances) with that
// component's weight from the mixture record -- is summed per cluster.
template <typename T, int K>
__global__ void __launch_bounds__(GROUP_TPB) group_core_kernel(const StatePtrs s, int64_t P, const uint16_t *code_v,
                                                               const uint16_t *code_w, uint8_t *labels, GroupCtl *G,
                                                               int max_steps)
{
    __shared__ double mu_s[3][2], sg_s[3][2];
    __shared__ double par_s[3][5];
    __shared__ unsigned long long nc_s[3];
    const int tid = threadIdx.x;
    const GroupBuf &fin = G->buf[max_steps % 3];
    if (tid == 0) {
        for (int j = 0; j < 3; j++)
            for (int f = 0; f < 2; f++) {
                double m = 0.0, sg = 0.0;
                if (fin.n[j]) {
                    const double n = __ull2double_rn(fin.n[j]);
                    m = __ddiv_rn(__ull2double_rn(fin.s1[j][f]), n);
                    const double v = __dsub_rn(__ddiv_rn(__ull2double_rn(fin.s2[j][f]), n), __dmul_rn(m, m));
                    sg = v > 0.0 ? __dsqrt_rn(v) : 0.0;
                }
                mu_s[j][f] = m;
                sg_s[j][f] = sg;
            }
        if (blockIdx.x == 0 && max_steps > 0 && G->conv_iter == 0 && fin.changed == 0) G->conv_iter = max_steps;
    }
    if (tid < 15) par_s[tid / 5][tid % 5] = 0.0;
    if (tid < 3) nc_s[tid] = 0;
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * GROUP_TPB + tid; p < P; p += (int64_t)gridDim.x * GROUP_TPB) {
        const int j = labels[p];
        const double dv = fabs(__dsub_rn((double)code_v[p], mu_s[j][0]));
        const double dw = fabs(__dsub_rn((double)code_w[p], mu_s[j][1]));
        if (!(dv < sg_s[j][0] && dw < sg_s[j][1])) continue;
        labels[p] = (uint8_t)(j | 0x80);
        S1Rec<T> r;
        r.load(s.s1, p);
        const int k = r.top();
        const uint4 *src = reinterpret_cast<const uint4 *>(s.gmm + p * Rec<T, K>::BYTES);
        uint4 u[Rec<T, K>::NV];
#pragma unroll
        for (int i = 0; i < Rec<T, K>::NV; i++) u[i] = src[i];
        float om = 0.f;
#pragma unroll
        for (int kk = 0; kk < K; kk++)
            if (kk == k) om = rec_elem<T, K>(u, 7 * kk);
        atomicAdd(&nc_s[j], 1ull);
        atomicAdd(&par_s[j][0], (double)om);
        for (int c = 0; c < 3; c++) atomicAdd(&par_s[j][1 + c], (double)r.get(c));
        atomicAdd(&par_s[j][4], ((double)r.get(3) + (double)r.get(4) + (double)r.get(5)) / 3.0);
    }
    __syncthreads();
    if (tid < 3 && nc_s[tid]) atomicAdd(&G->n_core[tid], nc_s[tid]);
    if (tid < 15 && par_s[tid / 5][tid % 5] != 0.0) atomicAdd(&G->par[tid / 5][tid % 5], par_s[tid / 5][tid % 5]);
}

template <typename T, int K>
cudaError_t launch_group_t(const DevParams &dp, const StatePtrs &s, const uint8_t *frames, int N, uint16_t *codes,
                           uint8_t *labels, int max_steps, int n_sm, cudaStream_t st)
{
    GroupCtl *G = reinterpret_cast<GroupCtl *>(s.ctl + CTL_GROUP_WORD);
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(GroupCtl), st);
    if (e != cudaSuccess) return e;
    uint16_t *cv = codes, *cw = codes + dp.P;
    const int64_t need = (dp.P + GROUP_TPB - 1) / GROUP_TPB;
    const unsigned grid = (unsigned)min(need, (int64_t)n_sm * 8);
    if (frames) group_features_kernel<K><<<(unsigned)((dp.P + 127) / 128), 128, 0, st>>>(dp, frames, N, cv, cw, G);
    else group_sums_kernel<<<grid, GROUP_TPB, 0, st>>>(dp.P, cv, cw, G);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int it = 0; it <= max_steps; it++) {
        group_assign_kernel<<<grid, GROUP_TPB, 0, st>>>(dp.P, cv, cw, labels, G, it);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    group_core_kernel<T, K><<<grid, GROUP_TPB, 0, st>>>(s, dp.P, cv, cw, labels, G, max_steps);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_group_k(int K, const DevParams &dp, const StatePtrs &s, const uint8_t *frames, int N,
                           uint16_t *codes, uint8_t *labels, int max_steps, int n_sm, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_group_t<T, 1>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    case 2: return launch_group_t<T, 2>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    case 3: return launch_group_t<T, 3>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    case 4: return launch_group_t<T, 4>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    case 5: return launch_group_t<T, 5>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    case 6: return launch_group_t<T, 6>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    case 7: return launch_group_t<T, 7>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    default: return launch_group_t<T, 8>(dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    }
}

// frames == nullptr: cluster the caller's codes (no feature pass).
cudaError_t launch_group(int dtype, int K, const DevParams &dp, const StatePtrs &s, const uint8_t *frames, int N,
                         uint16_t *codes, uint8_t *labels, int max_steps, int n_sm, cudaStream_t st)
{
    if (dtype == COG_F32) return launch_group_k<float>(K, dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    if (dtype == COG_F16) return launch_group_k<__half>(K, dp, s, frames, N, codes, labels, max_steps, n_sm, st);
    return launch_group_k<__nv_bfloat16>(K, dp, s, frames, N, codes, labels, max_steps, n_sm, st);
}

int group_max_steps() { return GROUP_MAX_IT; }

// The grouping result as the host reads it back.
size_t group_ctl_offset() { return (size_t)CTL_GROUP_WORD * 4; }
size_t group_ctl_bytes() { return sizeof(GroupCtl); }
void group_ctl_decode(const void *raw, int max_steps, cog_group_stats *out)
{
    const GroupCtl *G = static_cast<const GroupCtl *>(raw);
    const GroupBuf &fin = G->buf[max_steps % 3];
    *out = cog_group_stats{};
    out->converged = G->conv_iter != 0;
    out->iterations = G->conv_iter ? (int32_t)G->conv_iter : max_steps;
    for (int j = 0; j < 3; j++) {
        out->n[j] = (int64_t)fin.n[j];
        out->n_core[j] = (int64_t)G->n_core[j];
        for (int f = 0; f < 2; f++) {
            out->code_sum[j][f] = (int64_t)fin.s1[j][f];
            out->code_sq_sum[j][f] = (int64_t)fin.s2[j][f];
        }
        if (!fin.n[j]) continue;
        const double n = (double)fin.n[j];
        for (int f = 0; f < 2; f++) {
            const double m = (double)fin.s1[j][f] / n;
            const double v = (double)fin.s2[j][f] / n - m * m;
            out->centroid[j][f] = m;
            out->sd[j][f] = v > 0.0 ? std::sqrt(v) : 0.0;
        }
        if (!G->n_core[j]) continue;
        const double nc = (double)G->n_core[j];
        out->w1[j] = G->par[j][0] / nc;
        for (int c = 0; c < 3; c++) out->mu1[j][c] = G->par[j][1 + c] / nc;
        out->v1[j] = G->par[j][4] / nc;
    }
}

}  // namespace cog
