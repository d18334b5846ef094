// cog_clip.cuh -- the cascade over a clip of consecutive frames in one
// launch, with each pixel's stage-0/1 state held on chip from the first
// frame of the clip to the last.
//
// Per pixel, frame after frame, the work is exactly that of the per-frame
// kernels (Sec. 2, "Cascade of Gaussians CoG": frame difference, running
// Gaussian average, ordered Gaussians of Eq. 2 with the scene prior, the
// confidence of "Confidence Measure"), with identical arithmetic and the
// same rounding to the storage type after every frame, so masks, stage maps,
// counts and state match frame-by-frame cog_apply bit for bit.
//
// The one coupling across pixels is the illumination counter (last
// paragraph of "Cascade of Gaussians CoG"): frame n's response depends on
// how many pixels of the whole frame n-1 reached the mixture stage.  The
// clip kernel speculates that no frame after the first is flagged, counts
// every frame's mixture-stage pixels, and after a grid-wide barrier checks
// the speculation.  If frame m's flag was wrong, every CTA restores the
// clip-start state from the undo log written during the pass and the clip
// runs again with frames 0..m fixed; each run fixes at least one more
// frame, so at most T+1 runs are needed (one in the common case).
//
// GB300 mapping.  A warp owns G x 128 consecutive pixels for the whole
// clip: their previous frame + label and confidence in registers, their
// stage-1 records in shared memory; it streams the clip's frame bytes with
// one frame of register prefetch.  Stage-1 work is compacted within the
// warp; the mixture-stage survivors of all the CTA's warps are compacted
// into one shared queue per frame and run one per thread (a warp-level
// queue would run the long mixture step for a few lanes of every warp).
// Survivors read and write their mixture records in place in HBM, the
// first touch of a record in a clip saving the original to the undo log.
// CTAs take tiles of NW x G x 128 pixels from a dynamic counter.  The grid is cooperative (all CTAs resident), so
// the barriers between the pass, the check and a rerun cannot deadlock;
// every wait is bounded by the global timer and reports a device error.
#pragma once

#include "cog_apply.cuh"

namespace cog {

constexpr int CLIP_TPB = 128;
constexpr int CLIP_G = 2;        // 128-pixel groups per warp tile
constexpr int CLIP_MINB = 3;     // CTAs per SM the register budget must allow
#define CLIP_S2_INLINE __forceinline__

// Shared memory of one warp: stage-1 records of its G x 128 pixels and the
// per-frame work lists (indices are pixel slots within the tile).
template <typename T, int G> struct alignas(16) ClipWarp {
    static constexpr int WT = G * 128;
    uint8_t s1[WT * S1Rec<T>::BYTES];
    uint2 stash[WT];       // rgb | D << 24, C- bits
    float resc[WT];        // new confidence of pixels decided at stage 1 or 2
    uint8_t list[WT];      // stage-1 work list
    uint8_t resst[WT];     // stage code of pixels past stage 0
    uint32_t touched[WT / 32];   // mixture record saved to the undo log
};

// The CTA's mixture-stage queue of one frame: survivors of all its warps,
// (warp << 8 | slot), processed densely by all its threads; counts
// double-buffered by frame parity.
template <int NW, int WT> struct ClipQueue {
    uint16_t q[NW * WT];
    uint32_t n[2];
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch: every CTA arrives once per
// barrier; `target` = (barriers so far) x gridDim.x.  Gives up after
// limit_ns (or 2^26 polls), sets DERR_GRID_TIMEOUT in the device error word
// and returns false in every thread of the CTA.
constexpr uint64_t CLIP_WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool clip_grid_sync(uint32_t *bar, uint32_t target, uint32_t *err,
                                               uint64_t limit_ns = CLIP_WAIT_NS)
{
    __syncthreads();
    int bad = 0;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0; ld_acquire_gpu(bar) < target; it++) {
            __nanosleep(128);
            if ((it & 255u) == 0 && (global_ns() - t0 > limit_ns || it > (1u << 26))) {
                atomicOr(err, DERR_GRID_TIMEOUT);
                bad = 1;
                break;
            }
        }
        __threadfence();
    }
    return !__syncthreads_or(bad);
}


// Stage 0 of one group of 4 pixels (frame words w0..w2): skip bits, the
// pixels as rgb words, and the mask of pixels that go on to stage 1.
template <typename T>
__device__ __forceinline__ void clip_stage0(const DevParams &dp, const uint4 &jl, const VecN<T, PPT> &cv,
                                            uint32_t w0, uint32_t w1, uint32_t w2, int nact, bool phase_off,
                                            uint32_t Iw[PPT], uint32_t ad[PPT], uint32_t &skip, uint32_t &need1)
{
    const bool conf_on = dp.flags & COG_CONF;
    skip = 0;
    if (phase_off) {
#pragma unroll
        for (int i = 0; i < PPT; i++)
            if (i < nact && cv.get(i) >= dp.c_skip) skip |= 1u << i;
    }
    Iw[0] = w0 & 0x00ffffffu;
    Iw[1] = __byte_perm(w0, w1, 0x0543) & 0x00ffffffu;
    Iw[2] = __byte_perm(w1, w2, 0x0432) & 0x00ffffffu;
    Iw[3] = w2 >> 8;
#pragma unroll
    for (int i = 0; i < PPT; i++) ad[i] = __vabsdiffu4(Iw[i], u4get(jl, i) & 0x00ffffffu);
    need1 = 0;
    const bool fd_on = dp.flags & COG_FD;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        if (i >= nact || (skip >> i & 1u)) continue;
        const float Cm = conf_on ? cv.get(i) : 0.5f;
        const float tau = __fmul_rn(dp.tau_fd, __fadd_rn(0.5f, Cm));
        const uint32_t t = tau >= 255.f ? 255u : (uint32_t)tau;
        const bool pass = fd_on && (u4get(jl, i) >> 24) == 0 && __vcmpgtu4(ad[i], t * 0x01010101u) == 0u;
        if (!pass) need1 |= 1u << i;
    }
}

__device__ __forceinline__ void load_frame_words(const uint8_t *f, int64_t p0, int nact, bool al4, uint32_t &w0,
                                                 uint32_t &w1, uint32_t &w2)
{
    if (nact == PPT && al4) {
        const uint32_t *f4 = reinterpret_cast<const uint32_t *>(f + p0 * 3);
        w0 = __ldcs(f4); w1 = __ldcs(f4 + 1); w2 = __ldcs(f4 + 2);
    } else {
        uint32_t fw[3] = {0, 0, 0};
#pragma unroll
        for (int b3 = 0; b3 < PPT * 3; b3++)
            if (b3 < nact * 3) fw[b3 >> 2] |= (uint32_t)f[p0 * 3 + b3] << ((b3 & 3) * 8);
        w0 = fw[0]; w1 = fw[1]; w2 = fw[2];
    }
}

// The mixture stage of one survivor (pixel p, slot `slot` of warp area V)
// in frame t: Eq. 2 on its record in place (the first touch in the clip
// saves the original to the undo log), the illumination response when the
// frame is flagged, the transition update of its stage-1 record, and its
// confidence; its stage code goes to V.resst.  (Inlined: an out-of-line
// call, meant to keep the mixture's registers apart from the per-frame
// state, measured slower.)
template <typename T, int K, int G, bool PC>
__device__ CLIP_S2_INLINE void clip_s2(const ClipArgs &A, ClipWarp<T, G> &V, int64_t p, int slot, bool flag)
{
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    constexpr int SB = S1Rec<T>::BYTES;
    constexpr int RNV = RecSel<T, K, PC>::NV, RB = RecSel<T, K, PC>::BYTES;
    const uint2 sv = V.stash[slot];
    uint4 raw[RNV];
    const uint4 *src = reinterpret_cast<const uint4 *>(A.s.gmm + p * RB);
#pragma unroll
    for (int i = 0; i < RNV; i++) raw[i] = src[i];
    uint32_t qk[3];
#pragma unroll
    for (int c = 0; c < 3; c++) qk[c] = prior_level(A.s.kde, p, c, (sv.x >> (8 * c)) & 0xffu, dp.kde_bits == 4);
    const uint32_t bit = 1u << (slot & 31);
    if (!(V.touched[slot >> 5] & bit)) {
        uint4 *u = reinterpret_cast<uint4 *>(A.undo_gmm + p * RB);
#pragma unroll
        for (int i = 0; i < RNV; i++) u[i] = raw[i];
        atomicOr(&V.touched[slot >> 5], bit);
    }
    if constexpr (PC) {
        // per-channel mixtures (COG_PERCHAN)
        const int D = (int)(sv.x >> 24);
        float I[3];
#pragma unroll
        for (int c = 0; c < 3; c++) I[c] = (float)((sv.x >> (8 * c)) & 0xffu);
        const float Cm = __uint_as_float(sv.y);
        S1Rec<T> r;
#pragma unroll
        for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = reinterpret_cast<const uint4 *>(V.s1 + slot * SB)[i];
        const uint32_t qab = r.qab();
        MixPC<K> m;
        mixpc_unpack<T, K>(raw, m);
        const MixOutPC o = mix_step_pc<K>(m, I, rate_eff(dp, Cm), dp);
        int label = o.fg, st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
        if (flag && o.fg) {
            illum_response_pc<K>(m, o, dp.w_illum);
            label = 0;
            st = COG_ST_ILLUM;
        }
        uint4 u[RecPC<T, K>::NV];
        mixpc_pack<T, K>(m, u);
        uint4 *dst = reinterpret_cast<uint4 *>(A.s.gmm + p * RB);
#pragma unroll
        for (int i = 0; i < RecPC<T, K>::NV; i++) dst[i] = u[i];
        if (!label) {
            S1Rec<T> rn;
            s1_reseed_pc<T, K>(m, o, qab, rn);
#pragma unroll
            for (int i = 0; i < S1Rec<T>::NV; i++) reinterpret_cast<uint4 *>(V.s1 + slot * SB)[i] = rn.u[i];
        }
        if (conf_on) V.resc[slot] = conf_stage2(dp, qk, qab, D, Cm, o.Mhat);
        V.resst[slot] = (uint8_t)st;
        return;
    }
    const int D = (int)(sv.x >> 24);
    float I[3];
#pragma unroll
    for (int c = 0; c < 3; c++) I[c] = (float)((sv.x >> (8 * c)) & 0xffu);
    const float Cm = __uint_as_float(sv.y);
    S1Rec<T> r;
#pragma unroll
    for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = reinterpret_cast<const uint4 *>(V.s1 + slot * SB)[i];
    const uint32_t qab = r.qab();
    Mix<K> m;
#pragma unroll
    for (int k = 0; k < K; k++) {
        m.w[k] = rec_elem<T, K>(raw, 7 * k);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m.mu[k][c] = rec_elem<T, K>(raw, 7 * k + 1 + c);
            m.v[k][c] = rec_elem<T, K>(raw, 7 * k + 4 + c);
        }
    }
    const bool mode1 = dp.flags & COG_MODE1;
    if (mode1) mode1_write_back<T, K>(m, r);
    const float ae = rate_eff(dp, Cm);
    const MixOut o = mix_step<K>(m, I, ae, dp);
    int label = o.fg, st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
    if (flag && o.fg) {
        illum_response<K>(m, o.tgt, dp.w_illum);
        label = 0;
        st = COG_ST_ILLUM;
    }
    rec_store<T, K>(A.s.gmm, p, m);
    if (mode1) {
        mode1_recache<T, K>(m, r);
#pragma unroll
        for (int i = 0; i < S1Rec<T>::NV; i++) reinterpret_cast<uint4 *>(V.s1 + slot * SB)[i] = r.u[i];
    } else if (!label) {   // transition update: the background mode seeds stage 1
        S1Rec<T> rn;
#pragma unroll
        for (int i = 0; i < S1Rec<T>::NV; i++) rn.u[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (k == o.tgt) {
#pragma unroll
                for (int c = 0; c < 3; c++) { rn.set(c, m.mu[k][c]); rn.set(3 + c, m.v[k][c]); }
            }
        }
        rn.set_qab(qab);
#pragma unroll
        for (int i = 0; i < S1Rec<T>::NV; i++) reinterpret_cast<uint4 *>(V.s1 + slot * SB)[i] = rn.u[i];
    }
    if (conf_on) {
        const float Mh = o.match >= 0 ? (o.tm < 1.f ? o.tm : 1.f) : 1.f;
        V.resc[slot] = conf_stage2(dp, qk, qab, D, Cm, Mh);
    }
    V.resst[slot] = (uint8_t)st;
}

// One CTA tile (NW warps x G x 128 pixels) through the T frames of the
// clip.  Each warp runs stages 0 and 1 of its own pixels; the survivors of
// all warps go through the mixture stage together, one per thread; then
// each warp writes its pixels' outputs.  cnt_s: the CTA's per-frame
// counters [CLIP_TMAX][CTL_FIELDS].
template <typename T, int K, int G, int NW, bool PC>
__device__ __forceinline__ void clip_tile(const ClipArgs &A, ClipWarp<T, G> *Ws, ClipQueue<NW, G * 128> &Q,
                                          uint32_t cbase, int warp, int lane, uint32_t flags, uint32_t *cnt_s)
{
    ClipWarp<T, G> &W = Ws[warp];
    const uint32_t wbase = cbase + (uint32_t)warp * (G * 128);
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    const bool sampling = (dp.flags & COG_SAMPLE) && conf_on;
    constexpr int WT = G * 128;
    constexpr int SB = S1Rec<T>::BYTES;
    const int64_t P = dp.P;

    uint4 jl[G];
    VecN<T, PPT> cv[G];
    int nact[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int64_t p0 = (int64_t)wbase + g * 128 + lane * PPT;
        nact[g] = (int)min((int64_t)PPT, max((int64_t)0, P - p0));
        jl[g] = make_uint4(0, 0, 0, 0);
        if (nact[g] > 0) {
            jl[g] = *reinterpret_cast<const uint4 *>(A.s.jl + p0);
            cv[g].load(reinterpret_cast<const T *>(A.s.conf) + p0);
            *reinterpret_cast<uint4 *>(A.undo_jl + p0) = jl[g];
            cv[g].store(reinterpret_cast<T *>(A.undo_conf) + p0);
        } else {
#pragma unroll
            for (int i = 0; i < VecN<T, PPT>::NW; i++) cv[g].w[i] = 0;
        }
    }
    // stage-1 records of the tile (planes are padded to whole 4096-pixel
    // blocks, so the tile never runs past the allocation)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(A.s.s1 + (int64_t)wbase * SB);
        uint4 *und = reinterpret_cast<uint4 *>(A.undo_s1 + (int64_t)wbase * SB);
        uint4 *dst = reinterpret_cast<uint4 *>(W.s1);
#pragma unroll
        for (int k = lane; k < WT * SB / 16; k += 32) {
            const uint4 v = src[k];
            dst[k] = v;
            und[k] = v;
        }
    }
    if (lane < WT / 32) W.touched[lane] = 0;
    if (threadIdx.x == 0) { Q.n[0] = 0; Q.n[1] = 0; }
    __syncthreads();

    uint32_t nw[G][3];
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int64_t p0 = (int64_t)wbase + g * 128 + lane * PPT;
        nw[g][0] = nw[g][1] = nw[g][2] = 0;
        if (nact[g] > 0) load_frame_words(A.frames, p0, nact[g], A.frame_al4, nw[g][0], nw[g][1], nw[g][2]);
    }
    const uint32_t lt = (1u << lane) - 1u;

    for (uint32_t t = 0; t < A.T; t++) {
        uint32_t cw[G][3];
#pragma unroll
        for (int g = 0; g < G; g++) { cw[g][0] = nw[g][0]; cw[g][1] = nw[g][1]; cw[g][2] = nw[g][2]; }
        if (t + 1 < A.T) {
            const uint8_t *fn = A.frames + (int64_t)(t + 1) * P * 3;
#pragma unroll
            for (int g = 0; g < G; g++) {
                const int64_t p0 = (int64_t)wbase + g * 128 + lane * PPT;
                if (nact[g] > 0) load_frame_words(fn, p0, nact[g], A.frame_al4, nw[g][0], nw[g][1], nw[g][2]);
            }
        }
        const uint32_t fidx = A.frame_idx0 + t;
        const bool flag = (flags >> t) & 1u;

        // ---- stage 0 and the stage-1 work list
        uint32_t Iw[G][PPT], skip[G], need1[G];
        int n1 = 0;
#pragma unroll
        for (int g = 0; g < G; g++) {
            const uint32_t p0 = wbase + g * 128 + lane * PPT;
            const bool off = sampling && (fidx + (p0 >> 6)) % (uint32_t)dp.skip_period != 0u;
            uint32_t ad[PPT];
            clip_stage0<T>(dp, jl[g], cv[g], cw[g][0], cw[g][1], cw[g][2], nact[g], off, Iw[g], ad, skip[g],
                           need1[g]);
            n1 += __popc(need1[g]);
            if (need1[g]) {
#pragma unroll
                for (int i = 0; i < PPT; i++) {
                    if (!(need1[g] >> i & 1u)) continue;
                    const int slot = g * 128 + lane * PPT + i;
                    const uint32_t m2 = __vmaxu4(ad[i], ad[i] >> 8);
                    const uint32_t D = __vmaxu4(m2, m2 >> 8) & 0xffu;
                    W.stash[slot] = make_uint2(Iw[g][i] | (D << 24), __float_as_uint(conf_on ? cv[g].get(i) : 0.5f));
                }
            }
        }
        int incl = n1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const int n1w = __shfl_sync(0xffffffffu, incl, 31);
        {
            int k = incl - n1;
#pragma unroll
            for (int g = 0; g < G; g++)
#pragma unroll
                for (int i = 0; i < PPT; i++)
                    if (need1[g] >> i & 1u) W.list[k++] = (uint8_t)(g * 128 + lane * PPT + i);
        }
        __syncwarp();

        // ---- stage 1 over the compacted list; survivors join the CTA queue
        for (int j0 = 0; j0 < n1w; j0 += 32) {
            const int j = j0 + lane;
            bool surv = false;
            int slot = 0;
            if (j < n1w) {
                slot = W.list[j];
                const uint2 sv = W.stash[slot];
                const int D = (int)(sv.x >> 24);
                const float Cm = __uint_as_float(sv.y);
                S1Rec<T> r;
#pragma unroll
                for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = reinterpret_cast<const uint4 *>(W.s1 + slot * SB)[i];
                surv = true;
                if (dp.flags & COG_RGA) {
                    bool upd;
                    const float tr = rga_step<T>(dp, r, sv.x, Cm, conf_on, upd);
                    if (tr < 1.f) {
                        surv = false;
                        if (upd) {
#pragma unroll
                            for (int i = 0; i < S1Rec<T>::NV; i++) reinterpret_cast<uint4 *>(W.s1 + slot * SB)[i] = r.u[i];
                        }
                        W.resc[slot] = conf_next(dp, Cm, conf_stage1(r.qab(), D, tr));
                        W.resst[slot] = COG_ST_RGA;
                    }
                }
            }
            const uint32_t b = __ballot_sync(0xffffffffu, surv);
            uint32_t base = 0;
            if (lane == 0 && b) base = atomicAdd(&Q.n[t & 1], (uint32_t)__popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (surv) Q.q[base + __popc(b & lt)] = (uint16_t)((warp << 8) | slot);
        }
        __syncthreads();
        if (threadIdx.x == 0) Q.n[(t + 1) & 1] = 0;   // last read in the previous frame

        // ---- stage 2: the CTA's survivors, one per thread, records in place
        {
            const uint32_t ns = Q.n[t & 1];
            for (uint32_t q = threadIdx.x; q < ns; q += NW * 32) {
                if (!in_bounds(A.s.ctl, q, (uint64_t)NW * G * 128, DBG_CLIP_ENTRY)) break;
                const uint32_t e = Q.q[q];
                const int slot = (int)(e & 0xffu);
                const int64_t pp = (int64_t)cbase + (e >> 8) * (G * 128) + slot;
                if (!in_bounds(A.s.ctl, e >> 8, (uint64_t)NW, DBG_CLIP_ENTRY) ||
                    !in_bounds(A.s.ctl, (uint64_t)pp, (uint64_t)P, DBG_CLIP_PIXEL))
                    continue;
                clip_s2<T, K, G, PC>(A, Ws[e >> 8], pp, slot, flag);
            }
        }
        __syncthreads();

        // ---- outputs of frame t; registers carry the pixels to frame t+1
        uint32_t c_fd = 0, c_rga = 0, c_bg = 0, c_fg = 0, c_il = 0, c_sk = 0;
        uint8_t *mk_out = A.masks + (int64_t)t * P;
        uint8_t *sm_out = A.stagemaps ? A.stagemaps + (int64_t)t * P : nullptr;
#pragma unroll
        for (int g = 0; g < G; g++) {
            if (nact[g] <= 0) continue;
            const int64_t p0 = (int64_t)wbase + g * 128 + lane * PPT;
            uint32_t mk = 0, sm = 0;
#pragma unroll
            for (int i = 0; i < PPT; i++) {
                if (i >= nact[g]) continue;
                const int slot = g * 128 + lane * PPT + i;
                const bool sk = skip[g] >> i & 1u;
                const uint32_t st = sk ? (uint32_t)COG_ST_SKIP
                                       : ((need1[g] >> i & 1u) ? (uint32_t)W.resst[slot] : (uint32_t)COG_ST_FD);
                c_fd += st == COG_ST_FD; c_rga += st == COG_ST_RGA; c_bg += st == COG_ST_GMM_BG;
                c_fg += st == COG_ST_FG; c_il += st == COG_ST_ILLUM; c_sk += sk;
                const uint32_t old = u4get(jl[g], i);
                uint32_t label;
                if (sk) {
                    label = old >> 24;
                } else {
                    label = st == COG_ST_FG;
                    u4set(jl[g], i, Iw[g][i] | (label << 24));
                    if (conf_on)
                        cv[g].set(i, st == COG_ST_FD ? conf_next(dp, cv[g].get(i), 1.f) : W.resc[slot]);
                }
                mk |= (label ? 255u : 0u) << (8 * i);
                sm |= st << (8 * i);
            }
            if (nact[g] == PPT && A.out_al4) {
                __stcs(reinterpret_cast<uint32_t *>(mk_out + p0), mk);
                if (sm_out) __stcs(reinterpret_cast<uint32_t *>(sm_out + p0), sm);
            } else {
                for (int i = 0; i < nact[g]; i++) {
                    mk_out[p0 + i] = (uint8_t)(mk >> (8 * i));
                    if (sm_out) sm_out[p0 + i] = (uint8_t)(sm >> (8 * i));
                }
            }
        }
        const uint32_t v[6] = {__reduce_add_sync(0xffffffffu, c_fd), __reduce_add_sync(0xffffffffu, c_rga),
                               __reduce_add_sync(0xffffffffu, c_bg), __reduce_add_sync(0xffffffffu, c_fg),
                               __reduce_add_sync(0xffffffffu, c_il), __reduce_add_sync(0xffffffffu, c_sk)};
        if (lane == 0) {
            uint32_t *cs = cnt_s + t * CTL_FIELDS;
#pragma unroll
            for (int f = 0; f < 5; f++) if (v[f]) atomicAdd(cs + f, v[f]);
            if (v[2] + v[3] + v[4]) atomicAdd(cs + 5, v[2] + v[3] + v[4]);
            if (v[5]) atomicAdd(cs + 6, v[5]);
        }
        __syncwarp();
    }

    // ---- the tile's state after the clip, in place
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (nact[g] <= 0) continue;
        const int64_t p0 = (int64_t)wbase + g * 128 + lane * PPT;
        *reinterpret_cast<uint4 *>(A.s.jl + p0) = jl[g];
        if (conf_on) cv[g].store(reinterpret_cast<T *>(A.s.conf) + p0);
    }
    {
        uint4 *dst = reinterpret_cast<uint4 *>(A.s.s1 + (int64_t)wbase * SB);
        const uint4 *src = reinterpret_cast<const uint4 *>(W.s1);
#pragma unroll
        for (int k = lane; k < WT * SB / 16; k += 32) dst[k] = src[k];
    }
    if (lane < WT / 32) A.touched[wbase / 32 + lane] = W.touched[lane];
    __syncwarp();
}

// Undo one warp tile: planes from the clip-start copies, and the mixture
// records the failed run touched.
template <typename T, int K, int G, bool PC>
__device__ __forceinline__ void clip_restore_tile(const ClipArgs &A, uint32_t wbase, int lane)
{
    constexpr int RNV = RecSel<T, K, PC>::NV, RB = RecSel<T, K, PC>::BYTES;
    constexpr int WT = G * 128;
    constexpr int SB = S1Rec<T>::BYTES;
    const int64_t P = A.dp.P;
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int64_t p0 = (int64_t)wbase + g * 128 + lane * PPT;
        if (p0 >= P) continue;
        *reinterpret_cast<uint4 *>(A.s.jl + p0) = *reinterpret_cast<const uint4 *>(A.undo_jl + p0);
        VecN<T, PPT> c;
        c.load(reinterpret_cast<const T *>(A.undo_conf) + p0);
        c.store(reinterpret_cast<T *>(A.s.conf) + p0);
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(A.undo_s1 + (int64_t)wbase * SB);
        uint4 *dst = reinterpret_cast<uint4 *>(A.s.s1 + (int64_t)wbase * SB);
        for (int k = lane; k < WT * SB / 16; k += 32) dst[k] = src[k];
    }
    for (int j = 0; j < WT; j += 32) {
        const uint32_t word = __ldcg(A.touched + wbase / 32 + j / 32);
        if (word >> lane & 1u) {
            const int64_t p = (int64_t)wbase + j + lane;
            const uint4 *src = reinterpret_cast<const uint4 *>(A.undo_gmm + p * RB);
            uint4 *dst = reinterpret_cast<uint4 *>(A.s.gmm + p * RB);
#pragma unroll
            for (int i = 0; i < RNV; i++) dst[i] = src[i];
        }
    }
}

template <typename T, int K, int G, bool PC>
__global__ void __launch_bounds__(CLIP_TPB, CLIP_MINB) clip_kernel(const __grid_constant__ ClipArgs A)
{
    constexpr int NW = CLIP_TPB / 32;
    extern __shared__ __align__(16) uint8_t clip_smem[];
    ClipWarp<T, G> *W = reinterpret_cast<ClipWarp<T, G> *>(clip_smem);
    __shared__ ClipQueue<NW, G * 128> Q;
    __shared__ uint32_t cnt_s[CLIP_TMAX * CTL_FIELDS];
    __shared__ uint32_t flags_s, tile_s, tf_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevParams &dp = A.dp;
    uint32_t *ctl = A.s.ctl;
    uint32_t *err = ctl + CTL_ERR_WORD;
    uint32_t *bar = A.sync;
    const uint32_t n0 = A.frame_mod3;

    if (warp == 0) {   // frame 0's flag comes from the frame before the clip
        const bool f = illum_flag_prev(dp, ctl, n0, lane);
        if (lane == 0) flags_s = f ? 1u : 0u;
    }
    __syncthreads();
    uint32_t flags = flags_s;
    uint32_t nsync = 0;
    uint32_t run = 0;
    for (;; run++) {
        const int bank = (int)(run % 3);
        for (int i = tid; i < CLIP_TMAX * CTL_FIELDS; i += CLIP_TPB) cnt_s[i] = 0;
        if (blockIdx.x == 0 && run >= 1) {
            // the bank and tile counter of the run after this one were last
            // read before the barrier that ended the previous run
            const int nb = (int)((run + 1) % 3);
            for (int i = tid; i < CLIP_TMAX * CTL_FIELDS * CLIP_SLOTS; i += CLIP_TPB)
                A.cnt[clip_cnt_word(nb, i / (CTL_FIELDS * CLIP_SLOTS), (i / CLIP_SLOTS) % CTL_FIELDS, i % CLIP_SLOTS)] = 0;
            if (tid == 0) A.sync[CLIP_TILE_WORD + 32 * nb] = 0;
        }
        __syncthreads();
        // ---- the pass: CTAs take tiles until none is left
        for (;;) {
            if (tid == 0) tile_s = atomicAdd(A.sync + CLIP_TILE_WORD + 32 * bank, 1u);
            __syncthreads();
            const uint32_t ct = tile_s;
            __syncthreads();
            if (ct >= A.n_tiles) break;
            clip_tile<T, K, G, NW, PC>(A, W, Q, ct * (uint32_t)(NW * G * 128), warp, lane, flags, cnt_s);
        }
        __syncthreads();
        for (int i = tid; i < (int)A.T * CTL_FIELDS; i += CLIP_TPB)
            if (cnt_s[i]) atomicAdd(A.cnt + clip_cnt_word(bank, i / CTL_FIELDS, i % CTL_FIELDS, blockIdx.x % CLIP_SLOTS), cnt_s[i]);
        if (!clip_grid_sync(bar, ++nsync * gridDim.x, err)) return;
        // ---- check the speculated flags against the counts
        if (warp == 0) {
            uint32_t ng = 0;
            if (lane < (int)A.T)
                for (int s = 0; s < CLIP_SLOTS; s++) ng += __ldcg(A.cnt + clip_cnt_word(bank, lane, 5, s));
            // frame lane + 1 is flagged when frame lane sent more than the
            // threshold share of the frame to the mixture stage
            const bool f = (dp.flags & COG_ILLUM) && lane + 1 < (int)A.T &&
                           (uint64_t)ng * 1000u > (uint64_t)dp.illum_permille * (uint64_t)dp.P;
            const uint32_t tf = (__ballot_sync(0xffffffffu, f) << 1) | (flags & 1u);
            if (lane == 0) tf_s = tf;
        }
        __syncthreads();
        const uint32_t tf = tf_s;
        const uint32_t diff = (tf ^ flags) & (A.T >= 32 ? 0xffffffffu : ((1u << A.T) - 1u));
        if (!diff) break;
        if (run >= A.T) {   // cannot happen: each run fixes one more frame
            if (blockIdx.x == 0 && tid == 0) atomicOr(err, DERR_CLIP_RUNS);
            return;
        }
        // frames before the first wrong flag were right; the flag of that
        // frame is now known; later ones take this run's counts as a guess
        flags = tf;
        for (uint32_t wt = blockIdx.x * NW + warp; wt < A.n_tiles * NW; wt += gridDim.x * NW)
            clip_restore_tile<T, K, G, PC>(A, wt * (uint32_t)(G * 128), lane);
        if (!clip_grid_sync(bar, ++nsync * gridDim.x, err)) return;
    }

    // ---- the control block as frame-by-frame application leaves it after
    //      the clip's last frame
    if (blockIdx.x == 0 && warp == 0) {
        const int bank = (int)(run % 3);
        unsigned long long *tot = reinterpret_cast<unsigned long long *>(ctl + CTL_TOT_WORD);
        const uint32_t nl = (n0 + A.T - 1) % 3;
        uint32_t last = 0;
#pragma unroll 1
        for (int f = 0; f < 7; f++) {
            uint64_t add = __reduce_add_sync(0xffffffffu, __ldcg(ctl + ctl_slot((n0 + 2) % 3, f, lane)));
            uint32_t v = 0;
            if (lane < (int)A.T)
                for (int s = 0; s < CLIP_SLOTS; s++) v += __ldcg(A.cnt + clip_cnt_word(bank, lane, f, s));
            add += __reduce_add_sync(0xffffffffu, lane + 1 < (int)A.T ? v : 0u);
            const uint32_t vl = __shfl_sync(0xffffffffu, v, (int)A.T - 1);
            if (lane == 0) tot[f] += add;
            if (lane == f) last = vl;
        }
        __syncwarp();
        for (int i = lane; i < 3 * CTL_FIELDS * CTL_SLOTS; i += 32)
            ctl[ctl_slot(i / (CTL_FIELDS * CTL_SLOTS), (i / CTL_SLOTS) % CTL_FIELDS, i % CTL_SLOTS)] = 0;
        for (int i = lane; i < 3 * QSEG; i += 32) ctl[ctl_qcnt(i / QSEG, i % QSEG)] = 0;
        __syncwarp();
        if (lane < 7) ctl[ctl_slot((int)nl, lane, 0)] = last;
        if (lane == 0) {
            A.sync[CLIP_RUNS_WORD] = run + 1;
            A.sync[CLIP_RUNS_WORD + 1] = (uint32_t)bank;
            A.sync[CLIP_RUNS_WORD + 2] = flags;
        }
    }
}

template <typename T, int G>
size_t clip_smem_bytes()
{
    return sizeof(ClipWarp<T, G>) * (CLIP_TPB / 32);
}

// CTAs of the clip kernel that fit on one SM (asked every launch: a launch
// covers up to 32 frames, and the answer must match the device current now)
template <typename T, int K, int G, bool PC>
int clip_blocks_per_sm()
{
    int b = 0;
    const size_t sm = clip_smem_bytes<T, G>();
    if (cudaFuncSetAttribute(clip_kernel<T, K, G, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, clip_kernel<T, K, G, PC>, CLIP_TPB, sm) != cudaSuccess)
        b = 0;
    return b;
}

template <typename T, int K, bool PC>
cudaError_t launch_clip_pc(const ClipArgs &a0, int n_sm, cudaStream_t st)
{
    constexpr int G = CLIP_G;
    constexpr int CT = CLIP_TPB / 32 * G * 128;   // pixels per CTA tile
    ClipArgs a = a0;
    a.n_tiles = (uint32_t)((a.dp.P + CT - 1) / CT);
    const int bps = clip_blocks_per_sm<T, K, G, PC>();
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const int grid = (int)min((int64_t)bps * n_sm, (int64_t)a.n_tiles);
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((const void *)clip_kernel<T, K, G, PC>, dim3(grid), dim3(CLIP_TPB), args,
                                       clip_smem_bytes<T, G>(), st);
}

template <typename T, int K>
cudaError_t launch_clip_t(const ClipArgs &a, int n_sm, cudaStream_t st)
{
    if (a.dp.flags & COG_PERCHAN) return launch_clip_pc<T, K, true>(a, n_sm, st);
    return launch_clip_pc<T, K, false>(a, n_sm, st);
}

}  // namespace cog
