// cog_apply.cuh -- the cascade for one frame, as two stream-ordered kernels.
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
// GB300 mapping.
//   stage01_kernel: a light streaming kernel with no shared-memory staging
//     and no barrier until its end.  A thread owns 8 consecutive pixels and
//     issues all its stage-0 loads at once as 128/64-bit vectors (previous
//     frame + label and confidence planes, frame bytes).  Pixels past stage
//     0 fetch their 16-byte stage-1 record.  Pixels past stage 1 are
//     compacted grid-wide: warp scan, CTA total, one atomic per CTA into the
//     frame's survivor queue (16 bytes per survivor carrying everything the
//     next stage needs).
//   stage2_kernel: a persistent grid walks the queue; each survivor fetches
//     its mixture record (one aligned block) and its three prior bytes in
//     one round trip, runs Eq. 2, and writes its record, label, mask and
//     confidence back.  The mixture's register footprint and divergence no
//     longer throttle the streaming stages.
#pragma once

#include "cog_device.cuh"

namespace cog {

constexpr int PPT = 4;         // pixels per thread in stage01_kernel
constexpr int K1_TPB = 256;
constexpr int K2_TPB = 128;

// Read the previous frame's counters: illumination flag (lag one frame).
__device__ __forceinline__ bool illum_flag_prev(const DevParams &dp, const uint32_t *ctl, uint32_t n, int lane)
{
    const uint32_t *prev = ctl + ((n + 2) % 3) * CTL_BUF_WORDS;
    const uint32_t g = __reduce_add_sync(0xffffffffu, __ldcg(prev + 5 * CTL_SLOTS + lane));
    return (dp.flags & COG_ILLUM) && (uint64_t)g * 1000u > (uint64_t)dp.illum_permille * (uint64_t)dp.P;
}

template <typename T, int TPB>
__global__ void __launch_bounds__(TPB) stage01_kernel(const ApplyArgs A)
{
    static_assert(PPT == 4, "frame and mask vector widths assume 4 pixels per thread");
    __shared__ uint32_t wtot_s[TPB / 32], qbase_s, cnt_s[2];
    const DevParams &dp = A.dp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = A.frame_no;
    uint32_t *ctl = A.s.ctl;
    const int64_t p0 = ((int64_t)blockIdx.x * TPB + tid) * PPT;
    const int nact = (int)max((int64_t)0, min((int64_t)PPT, dp.P - p0));
    const bool conf_on = dp.flags & COG_CONF;

    if (tid < 2) cnt_s[tid] = 0;
    if (blockIdx.x == 0) {
        // rotate the per-frame counters: clear frame n+1's, add frame n-1's
        // to the running totals
        uint32_t *nxt = ctl + ((n + 1) % 3) * CTL_BUF_WORDS;
        for (int i = tid; i < CTL_BUF_WORDS; i += TPB) nxt[i] = 0;
        if (tid == 0) ctl[CTL_QCNT_WORD + (n + 1) % 3] = 0;
        if (tid < 32) {
            const uint32_t *prev = ctl + ((n + 2) % 3) * CTL_BUF_WORDS;
            unsigned long long *tot = reinterpret_cast<unsigned long long *>(ctl + CTL_TOT_WORD);
#pragma unroll
            for (int f = 0; f < 6; f++) {
                const uint32_t v = __reduce_add_sync(0xffffffffu, __ldcg(prev + f * CTL_SLOTS + lane));
                if (lane == 0) tot[f] += v;
            }
        }
    }

    // ---- all stage-0 loads at once: previous frame + label (16 B),
    //      confidence (8 or 16 B), frame bytes (12 B)
    uint4 jl = make_uint4(0, 0, 0, 0);
    uint32_t fw[3] = {0, 0, 0};
    VecN<T, PPT> cv;
    if (nact > 0) {
        jl = *reinterpret_cast<const uint4 *>(A.s.jl + p0);
        cv.load(reinterpret_cast<const T *>(A.s.conf) + p0);
        if (A.frame_al4 && nact == PPT) {
            const uint32_t *f4 = reinterpret_cast<const uint32_t *>(A.frame + p0 * 3);
            fw[0] = f4[0]; fw[1] = f4[1]; fw[2] = f4[2];
        } else {
#pragma unroll
            for (int b3 = 0; b3 < PPT * 3; b3++)
                if (b3 < nact * 3) fw[b3 >> 2] |= (uint32_t)A.frame[p0 * 3 + b3] << ((b3 & 3) * 8);
        }
    }
    auto pix = [&](int i, int c) -> uint32_t {
        const int b3 = i * 3 + c;
        return (fw[b3 >> 2] >> ((b3 & 3) * 8)) & 0xffu;
    };
    auto Dof = [&](int i) -> int {
        const uint32_t j = u4get(jl, i);
        int D = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int d = abs((int)pix(i, c) - (int)((j >> (8 * c)) & 0xffu));
            D = d > D ? d : D;
        }
        return D;
    };

    // ---- stage 0
    uint32_t need1 = 0;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        if (i < nact) {
            const float Cm = conf_on ? cv.get(i) : 0.5f;
            const bool bg_prev = (u4get(jl, i) >> 24) == 0;
            if (!((dp.flags & COG_FD) && bg_prev && (float)Dof(i) <= dp.tau_fd * (0.5f + Cm))) need1 |= 1u << i;
        }
    }

    // ---- stage 1: running Gaussian average (records of the pixels left)
    S1Rec<T> r[PPT];
#pragma unroll
    for (int i = 0; i < PPT; i++)
        if (need1 >> i & 1u) r[i].load(A.s.s1, p0 + i);
    uint32_t need2 = 0, st1 = 0;     // st1: decided at stage 1
    VecN<T, PPT> cn = cv;            // new confidence of the pixels decided here
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        if (i >= nact) continue;
        const float Cm = conf_on ? cv.get(i) : 0.5f;
        float ci = 1.f;               // stage 0: instantaneous confidence 1
        if (need1 >> i & 1u) {
            if (!(dp.flags & COG_RGA)) { need2 |= 1u << i; continue; }
            float tr = 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float d = (float)pix(i, c) - r[i].get(c);
                const float t = __fdividef(d * d, dp.lam2 * r[i].get(3 + c));
                tr = t > tr ? t : tr;
            }
            if (!(tr < 1.f)) { need2 |= 1u << i; continue; }
            st1 |= 1u << i;
            if (!(conf_on && Cm >= dp.c_halt)) {
                const float ae = dp.alpha * (1.5f - Cm);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float I = (float)pix(i, c);
                    const float m = r[i].get(c) + ae * (I - r[i].get(c));
                    const float d = I - m;
                    r[i].set(c, m);
                    r[i].set(3 + c, clampf((1.f - ae) * r[i].get(3 + c) + ae * d * d, dp.var_min, dp.var_max));
                }
                r[i].store(A.s.s1, p0 + i);
            }
            const uint32_t q = r[i].qab();
            const float wa = (float)(q & 0xffu) / 255.f, wb = (float)(q >> 8) / 255.f;
            const float wg = (float)(255u - (q & 0xffu) - (q >> 8)) / 255.f;
            ci = wa + wb * (1.f - (float)Dof(i) / 255.f) + wg * (1.f - tr);
        }
        if (conf_on) cn.set(i, (1.f - dp.eta) * Cm + dp.eta * ci);
    }

    // ---- outputs of the pixels decided here; survivors get placeholders
    //      (previous label, old confidence, mask 0) that the mixture stage
    //      overwrites
    uint32_t n_fd = 0, n_rga = 0;
    if (nact > 0) {
        uint4 jn = jl;
        uint32_t sm = 0;
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            if (i >= nact) continue;
            const bool surv = need2 >> i & 1u;
            const uint32_t st = surv ? (uint32_t)COG_ST_GMM_BG : ((st1 >> i & 1u) ? (uint32_t)COG_ST_RGA : (uint32_t)COG_ST_FD);
            n_fd += st == COG_ST_FD;
            n_rga += st == COG_ST_RGA;
            u4set(jn, i, pix(i, 0) | (pix(i, 1) << 8) | (pix(i, 2) << 16) | (surv ? (u4get(jl, i) & 0xff000000u) : 0u));
            sm |= st << (8 * i);
        }
        if (jn.x != jl.x || jn.y != jl.y || jn.z != jl.z || jn.w != jl.w)
            *reinterpret_cast<uint4 *>(A.s.jl + p0) = jn;
        if (conf_on && need2 != ((1u << nact) - 1u)) cn.store(reinterpret_cast<T *>(A.s.conf) + p0);
        if (nact == PPT && A.out_al4) {
            *reinterpret_cast<uint32_t *>(A.mask + p0) = 0u;
            if (A.stagemap) *reinterpret_cast<uint32_t *>(A.stagemap + p0) = sm;
        } else {
            for (int i = 0; i < nact; i++) {
                A.mask[p0 + i] = 0;
                if (A.stagemap) A.stagemap[p0 + i] = (uint8_t)(sm >> (8 * i));
            }
        }
    }

    // ---- compact the survivors into the frame's queue: warp scan, one
    //      atomic per CTA
    const int n2 = __popc(need2);
    int incl = n2;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) wtot_s[warp] = (uint32_t)incl;
    const uint32_t vfd = __reduce_add_sync(0xffffffffu, n_fd);
    const uint32_t vrga = __reduce_add_sync(0xffffffffu, n_rga);
    if (lane == 0) {
        if (vfd) atomicAdd(&cnt_s[0], vfd);
        if (vrga) atomicAdd(&cnt_s[1], vrga);
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < TPB / 32; w++) tot += wtot_s[w];
        qbase_s = tot ? atomicAdd(ctl + CTL_QCNT_WORD + n % 3, tot) : 0u;
        const int slot = blockIdx.x & (CTL_SLOTS - 1);
        uint32_t *cur = ctl + (n % 3) * CTL_BUF_WORDS;
        if (cnt_s[0]) atomicAdd(cur + 0 * CTL_SLOTS + slot, cnt_s[0]);
        if (cnt_s[1]) atomicAdd(cur + 1 * CTL_SLOTS + slot, cnt_s[1]);
        if (tot) atomicAdd(cur + 5 * CTL_SLOTS + slot, tot);
    }
    __syncthreads();
    if (need2) {
        uint32_t pos = qbase_s + (uint32_t)(incl - n2);
        for (int w = 0; w < warp; w++) pos += wtot_s[w];
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            if (!(need2 >> i & 1u)) continue;
            const float Cm = conf_on ? cv.get(i) : 0.5f;
            const uint32_t rgb = pix(i, 0) | (pix(i, 1) << 8) | (pix(i, 2) << 16);
            A.s.queue[pos++] = make_uint4((uint32_t)(p0 + i), rgb | ((uint32_t)Dof(i) << 24), __float_as_uint(Cm),
                                          r[i].qab());
        }
    }
}

template <typename T, int K, int TPB>
__global__ void __launch_bounds__(TPB) stage2_kernel(const ApplyArgs A)
{
    __shared__ uint32_t flag_s, cnt_s[3];
    const DevParams &dp = A.dp;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t n = A.frame_no;
    uint32_t *ctl = A.s.ctl;
    const bool conf_on = dp.flags & COG_CONF;
    if (tid < 32) {
        const bool f = illum_flag_prev(dp, ctl, n, lane);
        if (lane == 0) flag_s = f;
    }
    if (tid < 3) cnt_s[tid] = 0;
    __syncthreads();
    const bool flag = flag_s;
    const uint32_t nq = __ldcg(ctl + CTL_QCNT_WORD + n % 3);
    uint32_t cbg = 0, cfg = 0, cil = 0;
    for (uint32_t q = blockIdx.x * TPB + tid; q < nq; q += gridDim.x * TPB) {
        const uint4 e = __ldcg(A.s.queue + q);
        const int64_t p = e.x;
        const int D = (int)(e.y >> 24);
        int Iv[3];
        float I[3];
#pragma unroll
        for (int c = 0; c < 3; c++) { Iv[c] = (e.y >> (8 * c)) & 0xff; I[c] = (float)Iv[c]; }
        const float Cm = __uint_as_float(e.z);
        const uint32_t qab = e.w & 0xffffu;
        // the record and the three prior bytes in one round trip
        uint32_t qk[3];
#pragma unroll
        for (int c = 0; c < 3; c++) qk[c] = __ldg(A.s.kde + (p * 3 + c) * 256 + Iv[c]);
        Mix<K> m;
        rec_load<T, K>(A.s.gmm, p, m);
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
            S1Rec<T> r;
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (k == o.tgt) {
#pragma unroll
                    for (int c = 0; c < 3; c++) { r.set(c, m.mu[k][c]); r.set(3 + c, m.v[k][c]); }
                }
            }
            r.set_qab(qab);
            r.store(A.s.s1, p);
        }
        if (conf_on) {
            uint32_t qmin = qk[0] < qk[1] ? qk[0] : qk[1];
            qmin = qk[2] < qmin ? qk[2] : qmin;
            const uint32_t qa = qab & 0xffu, qb = qab >> 8;
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
            reinterpret_cast<T *>(A.s.conf)[p] = Store<T>::from_f((1.f - dp.eta) * Cm + dp.eta * ci);
        }
        reinterpret_cast<uint8_t *>(A.s.jl)[p * 4 + 3] = (uint8_t)label;
        A.mask[p] = label ? 255 : 0;
        if (A.stagemap) A.stagemap[p] = (uint8_t)st;
        cbg += st == COG_ST_GMM_BG;
        cfg += st == COG_ST_FG;
        cil += st == COG_ST_ILLUM;
    }
    cbg = __reduce_add_sync(0xffffffffu, cbg);
    cfg = __reduce_add_sync(0xffffffffu, cfg);
    cil = __reduce_add_sync(0xffffffffu, cil);
    if (lane == 0) {
        if (cbg) atomicAdd(&cnt_s[0], cbg);
        if (cfg) atomicAdd(&cnt_s[1], cfg);
        if (cil) atomicAdd(&cnt_s[2], cil);
    }
    __syncthreads();
    if (tid < 3 && cnt_s[tid])
        atomicAdd(ctl + (n % 3) * CTL_BUF_WORDS + (2 + tid) * CTL_SLOTS + (blockIdx.x & (CTL_SLOTS - 1)), cnt_s[tid]);
}

template <typename T, int K>
cudaError_t launch_apply_t(const ApplyArgs &a, cudaStream_t st, const ApplyEvents *ev)
{
    const int64_t g1 = (a.dp.P + K1_TPB * PPT - 1) / (K1_TPB * PPT);
    if (ev) cudaEventRecord(ev->e0, st);
    stage01_kernel<T, K1_TPB><<<(unsigned)g1, K1_TPB, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev->e1, st);
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage2_kernel<T, K, K2_TPB>, K2_TPB, 0) !=
                cudaSuccess || per_sm < 1)
            per_sm = 4;
    }
    const int64_t need = (a.dp.P + K2_TPB - 1) / K2_TPB;
    const int64_t g2 = min((int64_t)a.k2_grid * per_sm, need);
    stage2_kernel<T, K, K2_TPB><<<(unsigned)max((int64_t)1, g2), K2_TPB, 0, st>>>(a);
    e = cudaGetLastError();
    if (ev) cudaEventRecord(ev->e2, st);
    return e;
}

}  // namespace cog
