// cog_apply.cuh -- the fused cascade kernel: one launch per frame.
//
// Sec. 2, "Cascade of Gaussians CoG": each pixel goes through
//   stage 0  frame difference / consistent-hypothesis propagation: a
//            background pixel whose value repeats the previous frame keeps
//            its label; nothing adapts;
//   stage 1  running Gaussian average with its own mean and variance
//            (adapts at the confidence-driven rate unless halted);
//   stage 2  the ordered Gaussians of Eq. 2 with the scene prior (looked up
//            only here) and the illumination counter;
// and its confidence C (Sec. 2, "Confidence Measure") sets the next frame's
// rate, threshold and halting.  Only the level that labels a pixel adapts.
//
// GB300 mapping.  A CTA owns a tile of TPB*8 consecutive pixels; a thread
// owns 8 of them.  The stage-0 inputs of the whole tile (frame bytes,
// previous frame + label, confidence) arrive by TMA bulk copies into shared
// memory.  The stage-1 planes (running average, residue weights) are read
// with 128-bit loads; when the previous frame sent enough pixels past
// stage 0 they are requested before the TMA wait, so both round trips
// overlap.  Pixels left after stage 1 are compacted through a warp scan into
// a shared queue, so the mixture stage runs densely over survivors instead of
// serialising divergent warps; each survivor's record is one aligned
// 16-byte-multiple block, fetched together with its three prior bytes.
#pragma once

#include "cog_device.cuh"

namespace cog {

constexpr int PPT = 8;   // pixels per thread

template <typename T>
__host__ __device__ constexpr int apply_smem_bytes(int TPB)
{
    // frame 3, jl 4, conf sizeof(T), queue 4, res_c 4, res_l 1 bytes per pixel
    return TPB * PPT * (3 + 4 + (int)sizeof(T) + 4 + 4 + 1);
}

template <typename T>
struct Stage1 {          // one thread's stage-1 planes: 8 pixels each
    Vec8<T> m[3], v[3];
    uint4 qab;
    __device__ __forceinline__ void load(const ApplyArgs &A, int64_t p0) {
        const T *rga = reinterpret_cast<const T *>(A.s.rga);
        qab = *reinterpret_cast<const uint4 *>(A.s.qab + p0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m[c].load(rga + c * A.s.rga_plane + p0);
            v[c].load(rga + (3 + c) * A.s.rga_plane + p0);
        }
    }
    __device__ __forceinline__ void store(const ApplyArgs &A, int64_t p0) const {
        T *rga = reinterpret_cast<T *>(A.s.rga);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m[c].store(rga + c * A.s.rga_plane + p0);
            v[c].store(rga + (3 + c) * A.s.rga_plane + p0);
        }
    }
    __device__ __forceinline__ uint32_t q(int i) const {   // qa | qb << 8 of pixel i
        return (u4get(qab, i >> 1) >> ((i & 1) * 16)) & 0xffffu;
    }
};

template <typename T, int K, int TPB>
__global__ void __launch_bounds__(TPB) apply_kernel(const ApplyArgs A)
{
    constexpr int TILE = TPB * PPT;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *frame_s = smem;
    uint32_t *jl_s = reinterpret_cast<uint32_t *>(smem + TILE * 3);
    T *c_s = reinterpret_cast<T *>(smem + TILE * 7);
    uint32_t *queue = reinterpret_cast<uint32_t *>(smem + TILE * (7 + sizeof(T)));
    float *res_c = reinterpret_cast<float *>(smem + TILE * (11 + sizeof(T)));
    uint8_t *res_l = smem + TILE * (15 + sizeof(T));
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t qcount, flag_s, pf_s, cnt_s[6];

    const DevParams &dp = A.dp;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t tile0 = (int64_t)blockIdx.x * TILE;
    const int npx = (int)min((int64_t)TILE, dp.P - tile0);
    const bool conf_on = dp.flags & COG_CONF;
    uint32_t *ctl = A.s.ctl;
    const uint32_t n = A.frame_no;

    // ---- stage the tile's stage-0 inputs (one elected thread issues TMA)
    const int fbytes = npx * 3, fbulk = A.frame_al16 ? (fbytes & ~15) : 0;
    if (tid == 0) {
        qcount = 0;
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, (uint32_t)(fbulk + TILE * 4 + TILE * sizeof(T)));
        if (fbulk) bulk_g2s(frame_s, A.frame + tile0 * 3, (uint32_t)fbulk, &bar);
        bulk_g2s(jl_s, A.s.jl + tile0, TILE * 4, &bar);
        bulk_g2s(c_s, reinterpret_cast<const T *>(A.s.conf) + tile0, TILE * sizeof(T), &bar);
    }
    if (tid < 6) cnt_s[tid] = 0;
    for (int i = fbulk + tid; i < fbytes; i += TPB) frame_s[i] = A.frame[tile0 * 3 + i];

    // ---- the previous frame's counters: illumination flag (lag one frame)
    //      and the early-fetch policy for the stage-1 planes
    if (tid < 32) {
        const uint32_t *prev = ctl + ((n + 2) % 3) * CTL_BUF_WORDS;
        const uint32_t g = __reduce_add_sync(0xffffffffu, __ldcg(prev + 5 * CTL_SLOTS + lane));
        const uint32_t s1 = __reduce_add_sync(0xffffffffu, __ldcg(prev + 1 * CTL_SLOTS + lane));
        if (lane == 0) {
            flag_s = (dp.flags & COG_ILLUM) &&
                     (uint64_t)g * 1000u > (uint64_t)dp.illum_permille * (uint64_t)dp.P;
            // past stage 0 on more than 1/16 of the pixels: nearly every
            // 8-pixel vector holds one, so fetching all of them costs little
            pf_s = A.prefetch == 1 ? 1u
                 : (A.prefetch == 2 ? 0u : (uint32_t)((uint64_t)(g + s1) * 16u > (uint64_t)dp.P));
        }
        if (blockIdx.x == 0) {
            unsigned long long *tot = reinterpret_cast<unsigned long long *>(ctl + CTL_TOT_WORD);
#pragma unroll
            for (int f = 0; f < 6; f++) {
                const uint32_t v = __reduce_add_sync(0xffffffffu, __ldcg(prev + f * CTL_SLOTS + lane));
                if (lane == 0) tot[f] += v;
            }
        }
    }
    if (blockIdx.x == 0) {
        uint32_t *nxt = ctl + ((n + 1) % 3) * CTL_BUF_WORDS;
        for (int i = tid; i < CTL_BUF_WORDS; i += TPB) nxt[i] = 0;
    }
    __syncthreads();

    const int lp0 = tid * PPT;
    const int64_t p0 = tile0 + lp0;
    const int nact = max(0, min(PPT, npx - lp0));
    Stage1<T> s1;
    const bool early = pf_s && nact > 0;
    if (early) s1.load(A, p0);

    const bool timed_out = !mbar_wait(&bar, 0);
    if (__syncthreads_or(timed_out)) {
        if (tid == 0) atomicOr(ctl + CTL_ERR_WORD, DERR_TMA_TIMEOUT);
        return;
    }

    // ---- stage 0 for the thread's 8 pixels (from shared memory)
    uint32_t need1 = 0, need2 = 0;
    {
        const uint4 a = reinterpret_cast<const uint4 *>(jl_s)[tid * 2];
        const uint4 b = reinterpret_cast<const uint4 *>(jl_s)[tid * 2 + 1];
        const uint32_t jl[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const uint2 *f2 = reinterpret_cast<const uint2 *>(frame_s + lp0 * 3);
        const uint2 x = f2[0], y = f2[1], z = f2[2];
        const uint32_t fw[6] = {x.x, x.y, y.x, y.y, z.x, z.y};
        Vec8<T> cv;
        cv.load(c_s + lp0);
        int Dv[8];
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            int D = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int b3 = i * 3 + c;
                const int v = (fw[b3 >> 2] >> ((b3 & 3) * 8)) & 0xff;
                const int d = abs(v - (int)((jl[i] >> (8 * c)) & 0xffu));
                D = d > D ? d : D;
            }
            Dv[i] = D;
            if (i < nact) {
                const float Cm = conf_on ? cv.get(i) : 0.5f;
                const bool bg_prev = (jl[i] >> 24) == 0;
                if ((dp.flags & COG_FD) && bg_prev && (float)D <= dp.tau_fd * (0.5f + Cm)) {
                    res_c[lp0 + i] = 1.f;                       // stage 0, label BG
                    res_l[lp0 + i] = (uint8_t)(COG_ST_FD << 1);
                } else {
                    need1 |= 1u << i;
                }
            }
        }

        // ---- stage 1: running Gaussian average
        if (need1) {
            if (!early) s1.load(A, p0);
            if (dp.flags & COG_RGA) {
                bool dirty = false;
#pragma unroll
                for (int i = 0; i < PPT; i++) {
                    if (!(need1 >> i & 1u)) continue;
                    float tr = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const int b3 = i * 3 + c;
                        const float I = (float)((fw[b3 >> 2] >> ((b3 & 3) * 8)) & 0xffu);
                        const float d = I - s1.m[c].get(i);
                        const float t = d * d / (dp.lam2 * s1.v[c].get(i));
                        tr = t > tr ? t : tr;
                    }
                    if (tr < 1.f) {
                        const float Cm = conf_on ? cv.get(i) : 0.5f;
                        const float ae = dp.alpha * (1.5f - Cm);
                        const bool halt = conf_on && Cm >= dp.c_halt;
                        if (!halt) {
#pragma unroll
                            for (int c = 0; c < 3; c++) {
                                const int b3 = i * 3 + c;
                                const float I = (float)((fw[b3 >> 2] >> ((b3 & 3) * 8)) & 0xffu);
                                const float m = s1.m[c].get(i) + ae * (I - s1.m[c].get(i));
                                const float d = I - m;
                                s1.m[c].set(i, m);
                                s1.v[c].set(i, clampf((1.f - ae) * s1.v[c].get(i) + ae * d * d, dp.var_min,
                                                      dp.var_max));
                            }
                            dirty = true;
                        }
                        const uint32_t q = s1.q(i);
                        const float wa = (float)(q & 0xffu) / 255.f, wb = (float)(q >> 8) / 255.f;
                        const float wg = (float)(255u - (q & 0xffu) - (q >> 8)) / 255.f;
                        res_c[lp0 + i] = wa + wb * (1.f - (float)Dv[i] / 255.f) + wg * (1.f - tr);
                        res_l[lp0 + i] = (uint8_t)(COG_ST_RGA << 1);
                    } else {
                        need2 |= 1u << i;
                    }
                }
                // stored before the mixture stage so that its reseeds land last
                if (dirty) s1.store(A, p0);
            } else {
                need2 = need1;
            }
        }
    }

    // ---- compact the survivors into the shared queue (warp scan)
    {
        const int n2 = __popc(need2);
        int incl = n2;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        const int wtot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t wbase = 0;
        if (lane == 31 && wtot) wbase = atomicAdd(&qcount, (uint32_t)wtot);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        int pos = (int)wbase + incl - n2;
#pragma unroll
        for (int i = 0; i < PPT; i++)
            if (need2 >> i & 1u) queue[pos++] = (uint32_t)(lp0 + i) | (s1.q(i) << 16);
    }
    __syncthreads();

    // ---- stage 2: ordered Gaussians + prior, dense over survivors
    {
        const uint32_t nq = qcount;
        const bool flag = flag_s;
        T *rga = reinterpret_cast<T *>(A.s.rga);
        for (uint32_t qi = tid; qi < nq; qi += TPB) {
            const uint32_t e = queue[qi];
            const int lp = e & 0xffffu;
            const uint32_t qa = (e >> 16) & 0xffu, qb = e >> 24;
            const int64_t p = tile0 + lp;
            int Iv[3];
            float I[3];
#pragma unroll
            for (int c = 0; c < 3; c++) { Iv[c] = frame_s[lp * 3 + c]; I[c] = (float)Iv[c]; }
            // the record and the three prior bytes are independent loads
            uint32_t qk[3];
#pragma unroll
            for (int c = 0; c < 3; c++) qk[c] = __ldg(A.s.kde + (p * 3 + c) * 256 + Iv[c]);
            Mix<K> m;
            rec_load<T, K>(A.s.gmm, p, m);
            int D = 0;
            const uint32_t j = jl_s[lp];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int d = abs(Iv[c] - (int)((j >> (8 * c)) & 0xffu));
                D = d > D ? d : D;
            }
            const float Cm = conf_on ? Store<T>::to_f(c_s[lp]) : 0.5f;
            const float ae = dp.alpha * (1.5f - Cm);
            const MixOut o = mix_step<K>(m, I, ae, dp);
            int label = o.fg, st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
            if (flag && o.fg) {
                illum_response<K>(m, o.tgt, dp.w_illum);
                label = 0;
                st = COG_ST_ILLUM;
            }
            rec_store<T, K>(A.s.gmm, p, m);
            if (!label) {   // transition update: the background mode seeds stage 1
#pragma unroll
                for (int k = 0; k < K; k++) {
                    if (k == o.tgt) {
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            rga[c * A.s.rga_plane + p] = Store<T>::from_f(m.mu[k][c]);
                            rga[(3 + c) * A.s.rga_plane + p] = Store<T>::from_f(m.v[k][c]);
                        }
                    }
                }
            }
            uint32_t qmin = qk[0] < qk[1] ? qk[0] : qk[1];
            qmin = qk[2] < qmin ? qk[2] : qmin;
            const float wa = (float)qa / 255.f, wb = (float)qb / 255.f;
            const float wg = (float)(255u - qa - qb) / 255.f;
            const float dhat = (float)D / 255.f;
            const float Mh = o.match >= 0 ? (o.tm < 1.f ? o.tm : 1.f) : 1.f;
            float ci;
            if ((int)qmin < dp.q_null) {
                const float den = wb + wg;
                ci = den > 0.f ? (wb * (1.f - dhat) + wg * (1.f - Mh)) / den : 0.f;
            } else {
                ci = wa * ((float)qmin / 255.f) + wb * (1.f - dhat) + wg * (1.f - Mh);
            }
            res_c[lp] = ci;
            res_l[lp] = (uint8_t)(label | (st << 1));
        }
    }
    __syncthreads();

    // ---- finalise from shared memory: confidence, previous frame + label,
    //      mask, stage map, occupancy counts
    uint32_t cnt[5] = {0, 0, 0, 0, 0};
    if (nact > 0) {
        const uint4 a = reinterpret_cast<const uint4 *>(jl_s)[tid * 2];
        const uint4 b = reinterpret_cast<const uint4 *>(jl_s)[tid * 2 + 1];
        const uint32_t jl[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const uint2 *f2 = reinterpret_cast<const uint2 *>(frame_s + lp0 * 3);
        const uint2 x = f2[0], y = f2[1], z = f2[2];
        const uint32_t fw[6] = {x.x, x.y, y.x, y.y, z.x, z.y};
        Vec8<T> cv;
        cv.load(c_s + lp0);
        Vec8<T> cn = cv;
        uint32_t jn[8];
        uint32_t mk0 = 0, mk1 = 0, sm0 = 0, sm1 = 0;
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            jn[i] = jl[i];
            if (i >= nact) continue;
            const uint32_t e = res_l[lp0 + i];
            const uint32_t label = e & 1u, st = e >> 1;
            if (conf_on) cn.set(i, (1.f - dp.eta) * cv.get(i) + dp.eta * res_c[lp0 + i]);
            const int b3 = i * 3;
            uint32_t rgb = 0;
#pragma unroll
            for (int c = 0; c < 3; c++)
                rgb |= ((fw[(b3 + c) >> 2] >> (((b3 + c) & 3) * 8)) & 0xffu) << (8 * c);
            jn[i] = rgb | (label << 24);
            const uint32_t mb = label ? 255u : 0u;
            if (i < 4) { mk0 |= mb << (8 * i); sm0 |= st << (8 * i); }
            else { mk1 |= mb << (8 * (i - 4)); sm1 |= st << (8 * (i - 4)); }
#pragma unroll
            for (int s = 0; s < 5; s++) cnt[s] += (st == (uint32_t)s);
        }
        uint4 *jg = reinterpret_cast<uint4 *>(A.s.jl + p0);
        if (jn[0] != jl[0] || jn[1] != jl[1] || jn[2] != jl[2] || jn[3] != jl[3])
            jg[0] = make_uint4(jn[0], jn[1], jn[2], jn[3]);
        if (jn[4] != jl[4] || jn[5] != jl[5] || jn[6] != jl[6] || jn[7] != jl[7])
            jg[1] = make_uint4(jn[4], jn[5], jn[6], jn[7]);
        if (conf_on) cn.store(reinterpret_cast<T *>(A.s.conf) + p0);
        if (nact == PPT && A.out_al8) {
            *reinterpret_cast<uint2 *>(A.mask + p0) = make_uint2(mk0, mk1);
            if (A.stagemap) *reinterpret_cast<uint2 *>(A.stagemap + p0) = make_uint2(sm0, sm1);
        } else {
            for (int i = 0; i < nact; i++) {
                A.mask[p0 + i] = (uint8_t)(i < 4 ? mk0 >> (8 * i) : mk1 >> (8 * (i - 4)));
                if (A.stagemap) A.stagemap[p0 + i] = (uint8_t)(i < 4 ? sm0 >> (8 * i) : sm1 >> (8 * (i - 4)));
            }
        }
    }

    // ---- stage occupancy counters (the paper's n_i, and the illumination count)
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[s]);
        if (lane == 0 && v) atomicAdd(&cnt_s[s], v);
    }
    __syncthreads();
    if (tid < 6) {
        const uint32_t v = tid < 5 ? cnt_s[tid] : cnt_s[2] + cnt_s[3] + cnt_s[4];
        if (v) atomicAdd(ctl + (n % 3) * CTL_BUF_WORDS + tid * CTL_SLOTS + (blockIdx.x & (CTL_SLOTS - 1)), v);
    }
}

template <typename T, int K>
cudaError_t launch_apply_t(const ApplyArgs &a, cudaStream_t st)
{
    constexpr int TPB = 128;
    constexpr int TILE = TPB * PPT;
    const int smem = apply_smem_bytes<T>(TPB);
    const int64_t grid = (a.dp.P + TILE - 1) / TILE;
    apply_kernel<T, K, TPB><<<(unsigned)grid, TPB, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cog
