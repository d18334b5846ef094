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
// memory.  Stage-1 planes are fetched with 128-bit loads only by threads
// that have a pixel left after stage 0.  Pixels left after stage 1 are
// compacted through a warp scan into a shared queue, so the costly mixture
// stage runs densely over survivors instead of serialising divergent warps;
// each survivor's mixture record is one aligned 16-byte-multiple block.
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

template <typename T, int K, int TPB>
__global__ void __launch_bounds__(TPB) apply_kernel(const ApplyArgs A)
{
    constexpr int TILE = TPB * PPT;
    using V8 = Vec8<T>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *frame_s = smem;
    uint32_t *jl_s = reinterpret_cast<uint32_t *>(smem + TILE * 3);
    T *c_s = reinterpret_cast<T *>(smem + TILE * 7);
    uint32_t *queue = reinterpret_cast<uint32_t *>(smem + TILE * (7 + sizeof(T)));
    float *res_c = reinterpret_cast<float *>(smem + TILE * (11 + sizeof(T)));
    uint8_t *res_l = smem + TILE * (15 + sizeof(T));
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t qcount, flag_s, cnt_s[6];

    const DevParams &dp = A.dp;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t tile0 = (int64_t)blockIdx.x * TILE;
    const int npx = (int)min((int64_t)TILE, dp.P - tile0);
    const bool conf_on = dp.flags & COG_CONF;
    uint32_t *ctl = A.s.ctl;
    const uint32_t n = A.frame_no;

    // ---- stage the tile's stage-0 inputs (one elected thread issues TMA)
    const int fbytes = npx * 3, fbulk = fbytes & ~15;
    if (tid == 0) {
        qcount = 0;
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, (uint32_t)(fbulk + TILE * 4 + TILE * sizeof(T)));
        if (fbulk) bulk_g2s(frame_s, A.frame + tile0 * 3, (uint32_t)fbulk, &bar);
        bulk_g2s(jl_s, A.s.jl + tile0, TILE * 4, &bar);
        bulk_g2s(c_s, reinterpret_cast<const T *>(A.s.conf) + tile0, TILE * sizeof(T), &bar);
    }
    if (tid < 6) cnt_s[tid] = 0;
    if (tid < fbytes - fbulk) frame_s[fbulk + tid] = A.frame[tile0 * 3 + fbulk + tid];

    // ---- illumination flag from the previous frame's counter (lag one frame)
    if (tid < 32) {
        const uint32_t *prev = ctl + ((n + 2) % 3) * CTL_BUF_WORDS;
        const uint32_t g = __reduce_add_sync(0xffffffffu, __ldcg(prev + 5 * CTL_SLOTS + lane));
        if (lane == 0)
            flag_s = (dp.flags & COG_ILLUM) &&
                     (uint64_t)g * 1000u > (uint64_t)dp.illum_permille * (uint64_t)dp.P;
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
    const bool timed_out = !mbar_wait(&bar, 0);
    if (__syncthreads_or(timed_out)) {
        if (tid == 0) atomicOr(ctl + CTL_ERR_WORD, DERR_TMA_TIMEOUT);
        return;
    }

    // ---- stage 0 for the thread's 8 pixels
    const int lp0 = tid * PPT;
    const int64_t p0 = tile0 + lp0;
    const int nact = max(0, min(PPT, npx - lp0));
    uint32_t jl[8];
    {
        const uint4 a = reinterpret_cast<const uint4 *>(jl_s)[tid * 2];
        const uint4 b = reinterpret_cast<const uint4 *>(jl_s)[tid * 2 + 1];
        jl[0] = a.x; jl[1] = a.y; jl[2] = a.z; jl[3] = a.w;
        jl[4] = b.x; jl[5] = b.y; jl[6] = b.z; jl[7] = b.w;
    }
    uint32_t fw[6];
    {
        const uint2 *f2 = reinterpret_cast<const uint2 *>(frame_s + lp0 * 3);
        const uint2 x = f2[0], y = f2[1], z = f2[2];
        fw[0] = x.x; fw[1] = x.y; fw[2] = y.x; fw[3] = y.y; fw[4] = z.x; fw[5] = z.y;
    }
    auto pix = [&](int i, int c) -> uint32_t {
        const int b = i * 3 + c;
        return (fw[b >> 2] >> ((b & 3) * 8)) & 0xffu;
    };
    V8 cv;
    cv.load(c_s + lp0);

    uint32_t need1 = 0, need2 = 0;
    uint32_t stg = 0;          // 3 bits per pixel
    float cinst[8];
    int Dv[8];
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        cinst[i] = 0.f;
        int D = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int d = abs((int)pix(i, c) - (int)((jl[i] >> (8 * c)) & 0xffu));
            D = d > D ? d : D;
        }
        Dv[i] = D;
        if (i < nact) {
            const float Cm = conf_on ? cv.get(i) : 0.5f;
            const bool bg_prev = (jl[i] >> 24) == 0;
            if ((dp.flags & COG_FD) && bg_prev && (float)D <= dp.tau_fd * (0.5f + Cm)) {
                cinst[i] = 1.f;                       // stage 0, label BG
            } else {
                need1 |= 1u << i;
            }
        }
    }

    // ---- stage 1: running Gaussian average
    uint4 qab = make_uint4(0, 0, 0, 0);
    if (need1) {
        qab = *reinterpret_cast<const uint4 *>(A.s.qab + p0);
        if (dp.flags & COG_RGA) {
            T *rga = reinterpret_cast<T *>(A.s.rga);
            V8 rm[3], rv[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                rm[c].load(rga + c * A.s.rga_plane + p0);
                rv[c].load(rga + (3 + c) * A.s.rga_plane + p0);
            }
            bool dirty = false;
#pragma unroll
            for (int i = 0; i < PPT; i++) {
                if (!(need1 >> i & 1u)) continue;
                float tr = 0.f;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float d = (float)pix(i, c) - rm[c].get(i);
                    const float t = d * d / (dp.lam2 * rv[c].get(i));
                    tr = t > tr ? t : tr;
                }
                if (tr < 1.f) {
                    const float Cm = conf_on ? cv.get(i) : 0.5f;
                    const float ae = dp.alpha * (1.5f - Cm);
                    const bool halt = conf_on && Cm >= dp.c_halt;
                    if (!halt) {
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const float I = (float)pix(i, c);
                            const float m = rm[c].get(i) + ae * (I - rm[c].get(i));
                            const float d = I - m;
                            rm[c].set(i, m);
                            rv[c].set(i, clampf((1.f - ae) * rv[c].get(i) + ae * d * d, dp.var_min, dp.var_max));
                        }
                        dirty = true;
                    }
                    const uint32_t q = u4get(qab, i >> 1) >> ((i & 1) * 16);
                    const float wa = (float)(q & 0xffu) / 255.f, wb = (float)((q >> 8) & 0xffu) / 255.f;
                    const float wg = (float)(255u - (q & 0xffu) - ((q >> 8) & 0xffu)) / 255.f;
                    cinst[i] = wa + wb * (1.f - (float)Dv[i] / 255.f) + wg * (1.f - tr);
                    stg |= (uint32_t)COG_ST_RGA << (3 * i);
                } else {
                    need2 |= 1u << i;
                }
            }
            // stored before the mixture stage so that its reseeds land last
            if (dirty) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    rm[c].store(rga + c * A.s.rga_plane + p0);
                    rv[c].store(rga + (3 + c) * A.s.rga_plane + p0);
                }
            }
        } else {
            need2 = need1;
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
        for (int i = 0; i < PPT; i++) {
            if (need2 >> i & 1u) {
                const uint32_t q = (u4get(qab, i >> 1) >> ((i & 1) * 16)) & 0xffffu;
                queue[pos++] = (uint32_t)(lp0 + i) | (q << 16);
            }
        }
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
            float I[3];
            int D = 0;
            const uint32_t j = jl_s[lp];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int v = frame_s[lp * 3 + c];
                I[c] = (float)v;
                const int d = abs(v - (int)((j >> (8 * c)) & 0xffu));
                D = d > D ? d : D;
            }
            const float Cm = conf_on ? Store<T>::to_f(c_s[lp]) : 0.5f;
            const float ae = dp.alpha * (1.5f - Cm);
            Mix<K> m;
            rec_load<T, K>(A.s.gmm, p, m);
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
            uint32_t qmin = 255;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint32_t q = A.s.kde[(p * 3 + c) * 256 + (int)I[c]];
                qmin = q < qmin ? q : qmin;
            }
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

    // ---- finalise: confidence, previous frame + label, mask, stage map
    uint32_t cnt[5] = {0, 0, 0, 0, 0};
    uint32_t jn[8];
    V8 cn = cv;
    uint32_t mk0 = 0, mk1 = 0, sm0 = 0, sm1 = 0;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        jn[i] = jl[i];
        if (i >= nact) continue;
        int label = 0, st;
        float ci;
        if (need2 >> i & 1u) {
            const uint32_t e = res_l[lp0 + i];
            label = e & 1u;
            st = e >> 1;
            ci = res_c[lp0 + i];
        } else {
            st = (stg >> (3 * i)) & 7u;
            ci = cinst[i];
        }
        if (conf_on) {
            const float Cm = cv.get(i);
            cn.set(i, (1.f - dp.eta) * Cm + dp.eta * ci);
        }
        jn[i] = pix(i, 0) | (pix(i, 1) << 8) | (pix(i, 2) << 16) | ((uint32_t)label << 24);
        const uint32_t mb = label ? 255u : 0u;
        if (i < 4) { mk0 |= mb << (8 * i); sm0 |= (uint32_t)st << (8 * i); }
        else { mk1 |= mb << (8 * (i - 4)); sm1 |= (uint32_t)st << (8 * (i - 4)); }
#pragma unroll
        for (int s = 0; s < 5; s++) cnt[s] += (st == s);
    }
    {
        uint4 *jg = reinterpret_cast<uint4 *>(A.s.jl + p0);
        if (jn[0] != jl[0] || jn[1] != jl[1] || jn[2] != jl[2] || jn[3] != jl[3])
            jg[0] = make_uint4(jn[0], jn[1], jn[2], jn[3]);
        if (jn[4] != jl[4] || jn[5] != jl[5] || jn[6] != jl[6] || jn[7] != jl[7])
            jg[1] = make_uint4(jn[4], jn[5], jn[6], jn[7]);
        if (conf_on && nact > 0) cn.store(reinterpret_cast<T *>(A.s.conf) + p0);
        if (nact == PPT) {
            *reinterpret_cast<uint2 *>(A.mask + p0) = make_uint2(mk0, mk1);
            if (A.stagemap) *reinterpret_cast<uint2 *>(A.stagemap + p0) = make_uint2(sm0, sm1);
        } else {
            for (int i = 0; i < nact; i++) {
                const uint32_t mw = i < 4 ? mk0 >> (8 * i) : mk1 >> (8 * (i - 4));
                A.mask[p0 + i] = (uint8_t)mw;
                if (A.stagemap) {
                    const uint32_t sw = i < 4 ? sm0 >> (8 * i) : sm1 >> (8 * (i - 4));
                    A.stagemap[p0 + i] = (uint8_t)sw;
                }
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
