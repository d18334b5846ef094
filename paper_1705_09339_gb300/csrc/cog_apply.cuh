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
//     and one barrier at its end (the CTA's stage counts).  A thread owns 4
//     consecutive pixels and issues all its stage-0 loads at once as
//     128/64-bit vectors (previous frame + label and confidence planes,
//     frame bytes), and writes its pixels' outputs at once.  Pixels past
//     stage 0 are compacted per CTA and fetch their 16-byte stage-1
//     record.  Pixels past stage 1 go to the frame's survivor queue, one
//     atomic per warp pass (16 bytes per survivor carrying everything the
//     next stage needs).
//   stage2_kernel: a persistent grid walks the queue; each survivor fetches
//     its mixture record (one aligned block) and its three prior bytes in
//     one round trip, runs Eq. 2 on the record in its stored form, and
//     writes its record, label, mask and confidence back.  The mixture's
//     register footprint and divergence no longer throttle the streaming
//     stages.
#pragma once

#include "cog_device.cuh"

namespace cog {

constexpr int PPT = 4;         // pixels per group (one 32-bit mask word)
constexpr int K1_G = K1_PX_PER_THREAD / PPT;   // groups per thread in stage01_kernel
constexpr int K1_TPB = 128;    // default launch shape (the autotuner may pick others)
constexpr int K2_TPB = 64;
constexpr int WPX = 32 * PPT * K1_G;   // pixels per warp in stage01_kernel
static_assert(K1_G * PPT == K1_PX_PER_THREAD && WPX <= 256, "slots of a warp's pixels are bytes");
// Queue segments: warp w of the first kernel puts up to WPX survivors into
// segment w % QSEG.  The layout sizes a segment for ceil(CTAs / QSEG) tiles
// of K1_TILE pixels, which holds every warp that maps to it.
static_assert(WPX * 32 % K1_TILE == 0, "queue segment sizing assumes whole K1 tiles per segment");
constexpr float R255 = 1.f / 255.f;
// Register budget of stage01_kernel: threads per SM it must fit
constexpr int K1_THREADS_PER_SM = 1280;

// Read the previous frame's counters: illumination flag (lag one frame).
__device__ __forceinline__ bool illum_flag_prev(const DevParams &dp, const uint32_t *ctl, uint32_t n, int lane)
{
    const uint32_t g = __reduce_add_sync(0xffffffffu, __ldcg(ctl + ctl_slot((n + 2) % 3, 5, lane)));
    return (dp.flags & COG_ILLUM) && (uint64_t)g * 1000u > (uint64_t)dp.illum_permille * (uint64_t)dp.P;
}

// Stage-1 confidence term: a + b (1 - D/255) + g (1 - t_r).
__device__ __forceinline__ float conf_stage1(uint32_t q, int D, float tr)
{
    const float wa = __fmul_rn((float)(q & 0xffu), R255), wb = __fmul_rn((float)(q >> 8), R255);
    const float wg = __fmul_rn((float)(255u - (q & 0xffu) - (q >> 8)), R255);
    const float dterm = __fsub_rn(1.f, __fmul_rn((float)D, R255));
    return __fmaf_rn(wg, __fsub_rn(1.f, tr), __fmaf_rn(wb, dterm, wa));
}

// Stage 1 of one pixel (Sec. 1, running Gaussian average; Sec. 3.2
// halting): t_r = max_c (I_c - m_c)^2 / (lambda^2 v_c) against 1.  A
// background pixel adapts (m, v) at alpha (1.5 - C-) unless halted (C- >=
// c_halt); r is updated in place and *upd says whether it changed.  ix
// holds I (r | g << 8 | b << 16).  Returns t_r (>= 1: on to stage 2).
template <typename T>
__device__ __forceinline__ float rga_step(const DevParams &dp, S1Rec<T> &r, uint32_t ix, float Cm, bool conf_on,
                                          bool &upd)
{
    float m[3], v[3], I[3];
    r.unpack(m, v);
#pragma unroll
    for (int c = 0; c < 3; c++) I[c] = (float)((ix >> (8 * c)) & 0xffu);
    float tr = 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float t = eq2_chan_stat(I[c], m[c], v[c], dp.lam2);
        tr = t > tr ? t : tr;
    }
    upd = tr < 1.f && !(conf_on && Cm >= dp.c_halt);
    if (upd) {
        const float ae = rate_eff(dp, Cm);
#pragma unroll
        for (int c = 0; c < 3; c++) eq2_chan_update(I[c], ae, __fsub_rn(1.f, ae), m[c], v[c], dp);
        r.pack(m, v);
    }
    return tr;
}

// Shared memory of one CTA of stage01_kernel: its compacted stage-1 work
// list (CPX = pixels of the CTA).  Entry j: ix = I (r | g << 8 | b << 16) |
// D << 24 and cs = the pixel's C- bits; with 16-bit state cs also carries
// the pixel's slot in the CTA (bits 16..31), with FP32 state the slot sits
// in slot[j].
template <typename T, int CPX> struct K1List {
    uint32_t ix[CPX];
    uint32_t cs[CPX];
    uint16_t slot[Store<T>::bytes == 4 ? CPX : 1];
};

// A thread's PPT consecutive pixels in stage01_kernel: loaded state, frame
// words, per-pixel D and the stage-0 outcome.
template <typename T> struct K1Px {
    uint4 jl;                 // previous frame + label
    VecN<T, PPT> cv;          // confidence C-
    uint32_t Iw[PPT];         // this frame's pixels as r | g << 8 | b << 16
    uint32_t D[PPT];          // max_c |I_c - J_c|
    uint32_t act;             // bits: pixel inside the frame
    uint32_t skip;            // bits: not sampled this frame (COG_SAMPLE)
    uint32_t need1;           // bits: past stage 0
};

// A thread's stage-0 inputs copied ahead into shared memory by the batched
// stage-0/1 kernel (previous frame + label, confidence words, frame words).
template <typename T> struct K1Slot {
    const uint4 *jl;
    const uint32_t *cv;
    const uint32_t *fr;
};
template <typename T, int TPB> struct K1Pre {
    uint4 jl[TPB];
    uint32_t cv[TPB][VecN<T, PPT>::NW];
    uint32_t fr[TPB][4];
    __device__ __forceinline__ K1Slot<T> slot(int tid) const { return {&jl[tid], cv[tid], fr[tid]}; }
};

// Loads and stage 0 of a thread's pixels p0 .. p0 + 3 (PF: a full group
// whose inputs were copied ahead, with no temporal sampling).
//   Stage 0 (Sec. 2, CHP): a background pixel whose D = max_c |I_c - J_c|
//   is at most tau_fd (0.5 + C-) keeps its label.  D is an integer, so the
//   test is D <= floor(tau).
//   Temporal sampling (Sec. 2, "Confidence based temporal sampling"): in a
//   frame off its 64-pixel block's phase, a pixel with C- >= c_skip is not
//   looked at (a group of 4 never straddles two blocks); a group whose
//   pixels are all skipped reads no frame bytes.
template <typename T, bool FULL, bool PF = false>
__device__ __forceinline__ void k1_stage0(const ApplyArgs &A, K1Px<T> &X, uint32_t p0, const K1Slot<T> *pf = nullptr)
{
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    const int nact = FULL ? PPT : (int)min((int64_t)PPT, max((int64_t)0, dp.P - (int64_t)p0));
    X.act = (1u << nact) - 1u;
    X.skip = 0;
    X.need1 = 0;
    uint32_t w0 = 0, w1 = 0, w2 = 0;
    X.jl = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int i = 0; i < VecN<T, PPT>::NW; i++) X.cv.w[i] = 0;
    if (PF) {
        X.jl = *pf->jl;
#pragma unroll
        for (int i = 0; i < VecN<T, PPT>::NW; i++) X.cv.w[i] = pf->cv[i];
        w0 = pf->fr[0]; w1 = pf->fr[1]; w2 = pf->fr[2];
    } else if (FULL || nact > 0) {
        // the planes are padded to whole 4-pixel groups: vector loads stay in bounds
        X.jl = *reinterpret_cast<const uint4 *>(A.s.jl + p0);
        X.cv.load(reinterpret_cast<const T *>(A.s.conf) + p0);
        if ((dp.flags & COG_SAMPLE) && conf_on && (A.frame_idx + (p0 >> 6)) % (uint32_t)dp.skip_period != 0u) {
#pragma unroll
            for (int i = 0; i < PPT; i++)
                if (X.cv.get(i) >= dp.c_skip) X.skip |= 1u << i;
            X.skip &= X.act;
        }
        if (X.skip == X.act) {
            // every pixel of the group keeps its label this frame
        } else if (A.frame_al4 && (FULL || nact == PPT)) {
            const uint32_t *f4 = reinterpret_cast<const uint32_t *>(A.frame + (size_t)p0 * 3);
            w0 = f4[0]; w1 = f4[1]; w2 = f4[2];
        } else {
            uint32_t fw[3] = {0, 0, 0};
#pragma unroll
            for (int b3 = 0; b3 < PPT * 3; b3++)
                if (b3 < nact * 3) fw[b3 >> 2] |= (uint32_t)A.frame[(size_t)p0 * 3 + b3] << ((b3 & 3) * 8);
            w0 = fw[0]; w1 = fw[1]; w2 = fw[2];
        }
    }
    X.Iw[0] = w0 & 0x00ffffffu;
    X.Iw[1] = __byte_perm(w0, w1, 0x0543) & 0x00ffffffu;
    X.Iw[2] = __byte_perm(w1, w2, 0x0432) & 0x00ffffffu;
    X.Iw[3] = w2 >> 8;
    const bool fd_on = dp.flags & COG_FD;
    uint32_t pass = 0;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        const uint32_t j = u4get(X.jl, i);
        // per-byte |I - J| (the top byte of both is 0), then the largest
        const uint32_t ad = __vabsdiffu4(X.Iw[i], j & 0x00ffffffu);
        X.D[i] = __vimax3_u32(ad & 0xffu, (ad >> 8) & 0xffu, ad >> 16);
        const float Cm = conf_on ? X.cv.get(i) : 0.5f;
        // floor(tau_fd (0.5 + C-)); the conversion saturates, tau >= 0
        const uint32_t t = __float2uint_rz(__fmul_rn(dp.tau_fd, __fadd_rn(0.5f, Cm)));
        pass |= (uint32_t)((j >> 24) == 0u && X.D[i] <= t) << i;
    }
    if (!fd_on) pass = 0;
    X.need1 = X.act & ~X.skip & ~pass;
}

// The thread's own outputs, written before stage 1 runs: the previous frame
// becomes this frame with label 0, the mask 0 (the mixture stage sets its
// survivors' labels and masks; a stage-1 background pixel keeps both), the
// confidence of the pixels decided at stage 0 (the others keep C- until
// stage 1 or 2 writes theirs); a skipped pixel keeps everything and shows
// its carried label.  Returns the pixels decided at stage 0.
template <typename T, bool FULL>
__device__ __forceinline__ uint32_t k1_own_out(const ApplyArgs &A, const K1Px<T> &X, uint32_t p0)
{
    const DevParams &dp = A.dp;
    const uint32_t fd = X.act & ~X.skip & ~X.need1;
    if (!(FULL || X.act)) return 0;
    uint4 jn = make_uint4(X.Iw[0], X.Iw[1], X.Iw[2], X.Iw[3]);
    uint32_t mk = 0;
    const uint32_t keep = FULL ? X.skip : (X.skip | ~X.act);
    if (keep) {
#pragma unroll
        for (int i = 0; i < PPT; i++) {
            const uint32_t j = u4get(X.jl, i);
            if (keep >> i & 1u) u4set(jn, i, j);
            if (X.skip >> i & 1u) mk |= ((j >> 24) ? 255u : 0u) << (8 * i);
        }
    }
    // a thread whose pixels are all skipped by the temporal sampling changes
    // nothing but its mask: its previous-frame and confidence words are
    // not rewritten
    const bool all_skipped = X.skip == X.act;
    if (!all_skipped) *reinterpret_cast<uint4 *>(A.s.jl + p0) = jn;
    if ((dp.flags & COG_CONF) && !all_skipped) {
        // C <- (1 - eta) C- + eta for the stage-0 pixels (c_inst = 1)
        VecN<T, PPT> cn = X.cv;
        if (Store<T>::bytes == 2) {
#pragma unroll
            for (int h = 0; h < PPT / 2; h++) {
                if (!(fd >> (2 * h) & 3u)) continue;
                const float2 c = Pair<T>::to_f2(X.cv.w[h]);
                const float lo = (fd >> (2 * h) & 1u) ? conf_next(dp, c.x, 1.f) : c.x;
                const float hi = (fd >> (2 * h + 1) & 1u) ? conf_next(dp, c.y, 1.f) : c.y;
                cn.w[h] = Pair<T>::from_f2(lo, hi);
            }
        } else {
#pragma unroll
            for (int i = 0; i < PPT; i++)
                if (fd >> i & 1u) cn.set(i, conf_next(dp, X.cv.get(i), 1.f));
        }
        cn.store(reinterpret_cast<T *>(A.s.conf) + p0);
    }
    uint32_t sm = 0;
    if (A.stagemap) {
#pragma unroll
        for (int i = 0; i < PPT; i++)
            sm |= ((X.skip >> i & 1u) ? (uint32_t)COG_ST_SKIP
                                      : ((fd >> i & 1u) ? (uint32_t)COG_ST_FD : (uint32_t)COG_ST_GMM_BG)) << (8 * i);
    }
    if ((FULL || X.act == 0xfu) && A.out_al4) {
        *reinterpret_cast<uint32_t *>(A.mask + p0) = mk;
        if (A.stagemap) *reinterpret_cast<uint32_t *>(A.stagemap + p0) = sm;
    } else {
        for (int i = 0; i < PPT; i++) {
            if (!(X.act >> i & 1u)) continue;
            A.mask[p0 + i] = (uint8_t)(mk >> (8 * i));
            if (A.stagemap) A.stagemap[p0 + i] = (uint8_t)(sm >> (8 * i));
        }
    }
    return fd;
}

// Shared memory of a stage-0/1 CTA: its stage-1 list and per-warp counts.
template <typename T, int TPB> struct K1Shared {
    K1List<T, TPB * PPT> L;
    uint32_t wcnt[TPB / 32];
    uint32_t cnt[TPB / 32][4];
};
template <typename T, int TPB> __device__ __forceinline__ K1Shared<T, TPB> &k1_shared()
{
    __shared__ K1Shared<T, TPB> sh;
    return sh;
}

// One CTA of the stage-0/1 pass over stream A: tile `cta` of its frame
// (CPX = 4 TPB consecutive pixels, each thread owning 4 of them).
//   1. every thread loads its pixels, runs stage 0 and writes its outputs;
//   2. the pixels past stage 0 of the whole CTA are compacted into one
//      shared list (warp ballots, then the warps' offsets), so stage 1 runs
//      ceil(n / 32) warp passes for the CTA's n candidates, spread over its
//      warps, instead of at least one partly idle pass per warp;
//   3. a stage-1 lane writes its pixel's results itself (the owners' stores
//      came before the barrier), and survivors go straight to the frame's
//      queue segment of the warp (one atomic per warp pass);
//   4. the stage counts are summed over the CTA and added to the frame's
//      counters once.
template <typename T, int TPB, bool PF = false>
__device__ __forceinline__ void k1_cta(const ApplyArgs &A, uint32_t cta, const K1Slot<T> *pf = nullptr)
{
    static_assert(PPT == 4 && K1_G == 1, "frame and mask vector widths assume one group of 4 pixels per thread");
    constexpr int NW = TPB / 32, CPX = TPB * PPT;
    constexpr bool WIDE = Store<T>::bytes == 4;
    static_assert(CPX <= 65536, "slots fit 16 bits");
    K1Shared<T, TPB> &sh = k1_shared<T, TPB>();   // one copy per kernel, whichever variants it inlines
    K1List<T, CPX> &L = sh.L;
    uint32_t(&wcnt_s)[NW] = sh.wcnt;
    uint32_t(&cnt_s)[NW][4] = sh.cnt;
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = A.frame_no;
    uint32_t *ctl = A.s.ctl;
    const uint32_t cbase = cta * CPX;
    const uint32_t p0 = cbase + (uint32_t)tid * PPT;

    if (cta == 0) {
        // rotate the per-frame counters: clear frame n+1's, add frame n-1's
        // to the running totals
        for (int i = tid; i < CTL_FIELDS * CTL_SLOTS; i += TPB) ctl[ctl_slot((n + 1) % 3, i / CTL_SLOTS, i % CTL_SLOTS)] = 0;
        if (tid < QSEG) ctl[ctl_qcnt((n + 1) % 3, tid)] = 0;
        if (tid < 32) {
            unsigned long long *tot = reinterpret_cast<unsigned long long *>(ctl + CTL_TOT_WORD);
#pragma unroll
            for (int f = 0; f < 7; f++) {
                const uint32_t v = __reduce_add_sync(0xffffffffu, __ldcg(ctl + ctl_slot((n + 2) % 3, f, lane)));
                if (lane == 0) tot[f] += v;
            }
        }
    }

    // ---- 1. stage 0 and the owners' outputs
    K1Px<T> X;
    uint32_t fd;
    if (PF) {
        k1_stage0<T, true, true>(A, X, p0, pf);
        fd = k1_own_out<T, true>(A, X, p0);
    } else if ((int64_t)cbase + CPX <= dp.P) {
        k1_stage0<T, true>(A, X, p0);
        fd = k1_own_out<T, true>(A, X, p0);
    } else {
        k1_stage0<T, false>(A, X, p0);
        fd = k1_own_out<T, false>(A, X, p0);
    }

    // ---- 2. the CTA's stage-1 list, candidates in pixel order
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t nw = 0, dst = 0;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        const uint32_t b = __ballot_sync(0xffffffffu, X.need1 >> i & 1u);
        nw += __popc(b);
        dst += __popc(b & lt);
    }
    if (lane == 0) wcnt_s[warp] = nw;
    __syncthreads();
    uint32_t n1 = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const uint32_t c = wcnt_s[w];
        dst += w < warp ? c : 0u;
        n1 += c;
    }
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        if (!(X.need1 >> i & 1u)) continue;
        const uint32_t slot = (uint32_t)tid * PPT + i;
        if (!in_bounds(ctl, dst, CPX, DBG_K1_LIST)) continue;
        L.ix[dst] = X.Iw[i] | (X.D[i] << 24);
        if (WIDE) {
            L.cs[dst] = X.cv.w[i];
            L.slot[dst] = (uint16_t)slot;
        } else {
            L.cs[dst] = ((X.cv.w[i >> 1] >> (16 * (i & 1))) & 0xffffu) | (slot << 16);
        }
        dst++;
    }
    __syncthreads();

    // ---- 3. stage 1 (Sec. 1, running Gaussian average), 32 candidates per
    //      warp pass; warp w's survivors go to queue segment (global warp) % QSEG
    const uint32_t seg = (cta * NW + warp) & (QSEG - 1);
    uint32_t n_rga = 0, ne = 0;
    for (uint32_t j0 = (uint32_t)warp * 32; j0 < n1; j0 += TPB) {
        const uint32_t j = j0 + (uint32_t)lane;
        bool surv = false;
        uint4 ent = make_uint4(0, 0, 0, 0);
        const uint32_t ix = j < n1 ? L.ix[j] : 0u, cs = j < n1 ? L.cs[j] : 0u;
        const uint32_t p = cbase + (WIDE ? (j < n1 ? (uint32_t)L.slot[j] : 0u) : (cs >> 16));
        if (j < n1 && in_bounds(ctl, p, (uint64_t)dp.P, DBG_K1_PIXEL)) {
            const int D = (int)(ix >> 24);
            const float Cm = conf_on ? Store<T>::unbits(WIDE ? cs : (cs & 0xffffu)) : 0.5f;
            S1Rec<T> r;
            r.load(A.s.s1, p);
            surv = true;
            if (dp.flags & COG_RGA) {
                bool upd;
                const float tr = rga_step<T>(dp, r, ix, Cm, conf_on, upd);
                if (tr < 1.f) {
                    surv = false;
                    if (upd) r.store(A.s.s1, p);
                    if (conf_on)
                        reinterpret_cast<T *>(A.s.conf)[p] =
                            Store<T>::from_f(conf_next(dp, Cm, conf_stage1(r.qab(), D, tr)));
                    if (A.stagemap) A.stagemap[p] = (uint8_t)COG_ST_RGA;
                    n_rga++;
                }
            }
            if (surv) ent = make_uint4(p, ix, __float_as_uint(Cm), r.qab());
        }
        const uint32_t b = __ballot_sync(0xffffffffu, surv);
        if (b) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(A.s.ctl + ctl_qcnt(n % 3, seg), (uint32_t)__popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            const uint32_t k = base + __popc(b & lt);
            if (surv && in_bounds(ctl, k, (uint64_t)A.s.qseg_cap, DBG_K1_QUEUE))
                A.s.queue[(int64_t)seg * A.s.qseg_cap + k] = ent;
        }
        ne += __popc(b);
    }

    // ---- 4. the CTA's counts (fields: 0 stage 0, 1 stage 1, 6 skipped,
    //      5 reached the mixture stage)
    const uint32_t c0 = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(fd));
    const uint32_t c1 = __reduce_add_sync(0xffffffffu, n_rga);
    const uint32_t c2 = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(X.skip));
    if (lane == 0) {
        cnt_s[warp][0] = c0;
        cnt_s[warp][1] = c1;
        cnt_s[warp][2] = c2;
        cnt_s[warp][3] = ne;
    }
    __syncthreads();
    if (tid < 4) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) v += cnt_s[w][tid];
        const int f = tid == 0 ? 0 : (tid == 1 ? 1 : (tid == 2 ? 6 : 5));
        if (v) atomicAdd(ctl + ctl_slot(n % 3, f, cta & (CTL_SLOTS - 1)), v);
    }
    // (a persistent caller's next tile writes wcnt_s only after its own
    // first barrier, which every thread reaches after the reads above)
}

template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, K1_THREADS_PER_SM / TPB) stage01_kernel(const ApplyArgs A)
{
    // programmatic dependent launch: let the mixture stage's CTAs be
    // scheduled as this grid drains, and wait for the previous frame's
    // kernels before touching the state they write
    grid_launch_dependents();
    grid_wait_prior();
    k1_cta<T, TPB>(A, blockIdx.x);
}

// ---- stage 2: one survivor of the queue, in two halves (its loads, then
//      the mixture step and its stores)
// Mixture record size: shared weights (K x 7 values) or per-channel
// mixtures (K x 9, COG_PERCHAN).
template <typename T, int K, bool PC> struct RecSel {
    static constexpr int NV = PC ? RecPC<T, K>::NV : Rec<T, K>::NV;
    static constexpr int BYTES = PC ? RecPC<T, K>::BYTES : Rec<T, K>::BYTES;
};

template <typename T, int K, bool PC = false> struct S2In {
    uint4 e;
    uint4 rec[RecSel<T, K, PC>::NV];
    uint32_t qk[3];
    S1Rec<T> s1;   // COG_MODE1 only: the stage-1 copy of the rank-1 mode
};

template <typename T, int K, bool PC = false, bool M1 = false>
__device__ __forceinline__ bool s2_load(const ApplyArgs &A, int64_t qi, S2In<T, K, PC> &in)
{
    in.e = __ldcg(A.s.queue + qi);
    const int64_t p = in.e.x;
    if (!in_bounds(A.s.ctl, (uint64_t)p, (uint64_t)A.dp.P, DBG_K2_PIXEL)) return false;
#pragma unroll
    for (int c = 0; c < 3; c++) in.qk[c] = prior_level(A.s.kde, p, c, (in.e.y >> (8 * c)) & 0xffu, A.dp.kde_bits == 4);
    const uint4 *src = reinterpret_cast<const uint4 *>(A.s.gmm + p * RecSel<T, K, PC>::BYTES);
#pragma unroll
    for (int i = 0; i < RecSel<T, K, PC>::NV; i++) in.rec[i] = src[i];
    if (M1) in.s1.load(A.s.s1, p);
    return true;
}

// Confidence of a pixel decided at stage 2 (Sec. 2, "Confidence Measure"):
// prior term from the smallest of the three prior levels (0..255 scale),
// unless the prior is nullified (that minimum below q_null).
__device__ __forceinline__ float conf_stage2(const DevParams &dp, const uint32_t qk[3], uint32_t qab, int D, float Cm,
                                             float Mh)
{
    uint32_t qmin = qk[0] < qk[1] ? qk[0] : qk[1];
    qmin = qk[2] < qmin ? qk[2] : qmin;
    const uint32_t qa = qab & 0xffu, qb = qab >> 8;
    const float wa = __fmul_rn((float)qa, R255), wb = __fmul_rn((float)qb, R255);
    const float wg = __fmul_rn((float)(255u - qa - qb), R255);
    const float dterm = __fsub_rn(1.f, __fmul_rn((float)D, R255)), mterm = __fsub_rn(1.f, Mh);
    float ci;
    if ((int)qmin < dp.q_null) {
        const float den = __fadd_rn(wb, wg);
        ci = den > 0.f ? __fdiv_rn(__fmaf_rn(wg, mterm, __fmul_rn(wb, dterm)), den) : 0.f;
    } else {
        ci = __fmaf_rn(wg, mterm, __fmaf_rn(wb, dterm, __fmul_rn(wa, __fmul_rn((float)qmin, R255))));
    }
    return conf_next(dp, Cm, ci);
}

// Stage 2 with per-channel mixtures (COG_PERCHAN): returns the stage code.
template <typename T, int K>
__device__ __forceinline__ int s2_finish_pc(const ApplyArgs &A, const S2In<T, K, true> &in, bool flag)
{
    const DevParams &dp = A.dp;
    const int64_t p = in.e.x;
    const int D = (int)(in.e.y >> 24);
    float I[3];
#pragma unroll
    for (int c = 0; c < 3; c++) I[c] = (float)((in.e.y >> (8 * c)) & 0xffu);
    const float Cm = __uint_as_float(in.e.z);
    const uint32_t qab = in.e.w & 0xffffu;
    MixPC<K> m;
    mixpc_unpack<T, K>(in.rec, m);
    const MixOutPC o = mix_step_pc<K>(m, I, rate_eff(dp, Cm), dp);
    int label = o.fg, st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
    if (flag && o.fg) {
        illum_response_pc<K>(m, o, dp.w_illum);
        label = 0;
        st = COG_ST_ILLUM;
    }
    uint4 u[RecPC<T, K>::NV];
    mixpc_pack<T, K>(m, u);
    uint4 *dst = reinterpret_cast<uint4 *>(A.s.gmm + p * RecPC<T, K>::BYTES);
#pragma unroll
    for (int i = 0; i < RecPC<T, K>::NV; i++) dst[i] = u[i];
    if (!label) {
        S1Rec<T> r;
        s1_reseed_pc<T, K>(m, o, qab, r);
        r.store(A.s.s1, p);
    }
    if (dp.flags & COG_CONF)
        reinterpret_cast<T *>(A.s.conf)[p] = Store<T>::from_f(conf_stage2(dp, in.qk, qab, D, Cm, o.Mhat));
    reinterpret_cast<uint8_t *>(A.s.jl)[p * 4 + 3] = (uint8_t)label;
    A.mask[p] = label ? 255 : 0;
    if (A.stagemap) A.stagemap[p] = (uint8_t)st;
    return st;
}

template <typename T, int K, bool M1>
__device__ __forceinline__ int s2_finish(const ApplyArgs &A, S2In<T, K> &in, bool flag)
{
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    const int64_t p = in.e.x;
    const int D = (int)(in.e.y >> 24);
    float I[3];
#pragma unroll
    for (int c = 0; c < 3; c++) I[c] = (float)((in.e.y >> (8 * c)) & 0xffu);
    const float Cm = __uint_as_float(in.e.z);
    const uint32_t qab = in.e.w & 0xffffu;
    const float ae = rate_eff(dp, Cm);
    MixOut o;
    int label, st;
    if constexpr (M1) {
        // stage 1 is a copy of the rank-1 mode: written back first, and
        // re-taken from the updated mixture
        Mix<K> m;
#pragma unroll
        for (int k = 0; k < K; k++) {
            m.w[k] = rec_elem<T, K>(in.rec, 7 * k);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                m.mu[k][c] = rec_elem<T, K>(in.rec, 7 * k + 1 + c);
                m.v[k][c] = rec_elem<T, K>(in.rec, 7 * k + 4 + c);
            }
        }
        mode1_write_back<T, K>(m, in.s1);
        o = mix_step<K>(m, I, ae, dp);
        label = o.fg;
        st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
        if (flag && o.fg) {
            illum_response<K>(m, o.tgt, dp.w_illum);
            label = 0;
            st = COG_ST_ILLUM;
        }
        rec_store<T, K>(A.s.gmm, p, m);
        S1Rec<T> r = in.s1;
        mode1_recache<T, K>(m, r);
        r.store(A.s.s1, p);
    } else {
        // the record stays in its stored form (fewer live registers)
        float tmv[6];
        o = mix_step_packed<T, K>(in.rec, I, ae, dp, flag, tmv);
        label = o.fg;
        st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
        if (flag && o.fg) {   // illumination response (applied inside the step)
            label = 0;
            st = COG_ST_ILLUM;
        }
        uint4 *dst = reinterpret_cast<uint4 *>(A.s.gmm + p * Rec<T, K>::BYTES);
#pragma unroll
        for (int i = 0; i < Rec<T, K>::NV; i++) dst[i] = in.rec[i];
        if (!label) {   // transition update: the background mode seeds stage 1
            S1Rec<T> r;
#pragma unroll
            for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = make_uint4(0, 0, 0, 0);
            r.pack(tmv, tmv + 3);
            r.set_qab(qab);
            r.store(A.s.s1, p);
        }
    }
    if (conf_on) {
        const float Mh = o.match >= 0 ? (o.tm < 1.f ? o.tm : 1.f) : 1.f;
        reinterpret_cast<T *>(A.s.conf)[p] = Store<T>::from_f(conf_stage2(dp, in.qk, qab, D, Cm, Mh));
    }
    reinterpret_cast<uint8_t *>(A.s.jl)[p * 4 + 3] = (uint8_t)label;
    A.mask[p] = label ? 255 : 0;
    if (A.stagemap) A.stagemap[p] = (uint8_t)st;
    return st;
}

// One of ncta CTAs walking stream A's survivor queue.  V: the mixture
// variant (mix_variant: 0 shared weights, 1 per-channel, 2 COG_MODE1).
template <typename T, int K, int TPB, int V>
__device__ __forceinline__ void k2_cta(const ApplyArgs &A, uint32_t cta, uint32_t ncta)
{
    __shared__ uint32_t flag_s, cnt_s[3], segp_s[QSEG + 1];
    const DevParams &dp = A.dp;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t n = A.frame_no;
    uint32_t *ctl = A.s.ctl;
    if (tid < 32) {
        const bool f = illum_flag_prev(dp, ctl, n, lane);
        // exclusive prefix of the queue segments' lengths
        const uint32_t len = __ldcg(ctl + ctl_qcnt(n % 3, lane));
        uint32_t incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        segp_s[lane] = incl - len;
        if (lane == 31) segp_s[QSEG] = incl;
        if (lane == 0) flag_s = f;
    }
    if (tid < 3) cnt_s[tid] = 0;
    __syncthreads();
    const bool flag = flag_s;
    const uint32_t nq = segp_s[QSEG];
    const uint32_t stride = ncta * TPB;
    auto entry = [&](uint32_t q) -> int64_t {   // flat index -> queue slot (-1: failed check)
        int lo = 0;
#pragma unroll
        for (int step = QSEG / 2; step >= 1; step >>= 1)
            if (segp_s[lo + step] <= q) lo += step;
        if (!in_bounds(ctl, q - segp_s[lo], (uint64_t)A.s.qseg_cap, DBG_K2_QUEUE)) return -1;
        return (int64_t)lo * A.s.qseg_cap + (q - segp_s[lo]);
    };
    uint32_t cbg = 0, cfg = 0, cil = 0;
    for (uint32_t q = cta * TPB + tid; q < nq; q += stride) {
        constexpr bool PC = V == 1;
        S2In<T, K, PC> a;
        const int64_t qi = entry(q);
        if (qi < 0 || !s2_load<T, K, PC, V == 2>(A, qi, a)) continue;
        int st;
        if constexpr (PC) st = s2_finish_pc<T, K>(A, a, flag);
        else st = s2_finish<T, K, V == 2>(A, a, flag);
        cbg += st == COG_ST_GMM_BG; cfg += st == COG_ST_FG; cil += st == COG_ST_ILLUM;
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
    if (tid < 3 && cnt_s[tid]) atomicAdd(ctl + ctl_slot(n % 3, 2 + tid, cta & (CTL_SLOTS - 1)), cnt_s[tid]);
}

// The same walk over stream A's survivor queue, software-pipelined for a
// CTA that takes many survivors per thread (the batched step).  While a
// thread runs the mixture step of its current survivor, cp.async copies
// into its own shared slots the queue entry two survivors ahead and, from
// the entry already there, the next survivor's record, its three prior
// words (and with COG_MODE1 its stage-1 record).  Nothing is held in
// registers across survivors, and no thread reads another's slots, so the
// per-thread copy groups need no barrier.
template <typename T, int K, int TPB, int V> struct K2Pipe {
    static constexpr bool PC = V == 1, M1 = V == 2;
    static constexpr int RNV = RecSel<T, K, PC>::NV;
    static constexpr int SNV = M1 ? S1Rec<T>::NV : 0;
    static constexpr int W = RNV + SNV + 1;   // uint4 words per slot: record, stage-1 record, prior words
    uint4 slot[2][W][TPB];                    // [buffer][word][thread]: consecutive threads, consecutive words
    uint4 ent[3][TPB];                        // queue entries of three consecutive survivors
};

template <typename T, int K, int TPB, int V>
__device__ __forceinline__ void k2_issue_copies(const ApplyArgs &A, K2Pipe<T, K, TPB, V> &S, int b, uint4 e)
{
    using PP = K2Pipe<T, K, TPB, V>;
    const int tid = threadIdx.x;
    const int64_t p = e.x;
    const uint8_t *rec = A.s.gmm + p * RecSel<T, K, PP::PC>::BYTES;
#pragma unroll
    for (int i = 0; i < PP::RNV; i++) cp_async16(&S.slot[b][i][tid], rec + 16 * i);
    if constexpr (PP::M1) {
#pragma unroll
        for (int i = 0; i < PP::SNV; i++)
            cp_async16(&S.slot[b][PP::RNV + i][tid], A.s.s1 + p * S1Rec<T>::BYTES + 16 * i);
    }
    // the aligned word holding each channel's prior level
    uint32_t *pw = reinterpret_cast<uint32_t *>(&S.slot[b][PP::W - 1][tid]);
    const bool four = A.dp.kde_bits == 4;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const uint32_t v = (e.y >> (8 * c)) & 0xffu;
        const int64_t byte = four ? (p * 3 + c) * 128 + (v >> 1) : (p * 3 + c) * 256 + v;
        cp_async4(pw + c, A.s.kde + (byte & ~(int64_t)3));
    }
}

template <typename T, int K, int TPB, int V>
__device__ __forceinline__ void k2_cta_pipe(const ApplyArgs &A, uint32_t cta, uint32_t ncta)
{
    using PP = K2Pipe<T, K, TPB, V>;
    __shared__ PP S;
    __shared__ uint32_t flag_s, cnt_s[3], segp_s[QSEG + 1];
    const DevParams &dp = A.dp;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t n = A.frame_no;
    uint32_t *ctl = A.s.ctl;
    if (tid < 32) {
        const bool f = illum_flag_prev(dp, ctl, n, lane);
        const uint32_t len = __ldcg(ctl + ctl_qcnt(n % 3, lane));
        uint32_t incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        segp_s[lane] = incl - len;
        if (lane == 31) segp_s[QSEG] = incl;
        if (lane == 0) flag_s = f;
    }
    if (tid < 3) cnt_s[tid] = 0;
    __syncthreads();
    const bool flag = flag_s;
    const uint32_t nq = segp_s[QSEG];
    const uint32_t stride = ncta * TPB;
    // copy the queue entry of flat index q into entry slot j; false if
    // there is none
    auto issue_entry = [&](uint32_t q, int j) -> bool {
        if (q >= nq) return false;
        int lo = 0;
#pragma unroll
        for (int step = QSEG / 2; step >= 1; step >>= 1)
            if (segp_s[lo + step] <= q) lo += step;
        if (!in_bounds(ctl, q - segp_s[lo], (uint64_t)A.s.qseg_cap, DBG_K2_QUEUE)) return false;
        cp_async16(&S.ent[j][tid], A.s.queue + (int64_t)lo * A.s.qseg_cap + (q - segp_s[lo]));
        return true;
    };
    // copy the data of the survivor whose entry is in slot j into buffer bb
    auto issue_rec = [&](int j, int bb) -> bool {
        const uint4 e = S.ent[j][tid];
        if (!in_bounds(ctl, (uint64_t)e.x, (uint64_t)dp.P, DBG_K2_PIXEL)) return false;
        k2_issue_copies<T, K, TPB, V>(A, S, bb, e);
        return true;
    };
    const uint32_t q0 = cta * TPB + tid;
    uint32_t ev = 0, rv = 0;   // bit j: entry slot j / record buffer j holds a survivor
    ev |= issue_entry(q0, 0) ? 1u : 0u;
    ev |= issue_entry(q0 + stride, 1) ? 2u : 0u;
    cp_async_commit();
    cp_async_wait<0>();
    if ((ev & 1u) && issue_rec(0, 0)) rv |= 1u;
    cp_async_commit();
    uint32_t cbg = 0, cfg = 0, cil = 0;
    int j = 0, b = 0;          // entry slot and record buffer of the current survivor
    for (uint32_t q = q0; q < nq; q += stride) {
        cp_async_wait<0>();    // the current survivor's data and the next one's entry
        const int j1 = j == 2 ? 0 : j + 1, j2 = j1 == 2 ? 0 : j1 + 1;
        ev &= ~(1u << j2);
        if (issue_entry(q + 2 * stride, j2)) ev |= 1u << j2;
        rv &= ~(1u << (b ^ 1));
        if ((ev >> j1 & 1u) && issue_rec(j1, b ^ 1)) rv |= 1u << (b ^ 1);
        cp_async_commit();
        if (rv >> b & 1u) {
            S2In<T, K, PP::PC> a;
            a.e = S.ent[j][tid];
#pragma unroll
            for (int i = 0; i < PP::RNV; i++) a.rec[i] = S.slot[b][i][tid];
            if constexpr (PP::M1) {
#pragma unroll
                for (int i = 0; i < PP::SNV; i++) a.s1.u[i] = S.slot[b][PP::RNV + i][tid];
            }
            const uint4 w = S.slot[b][PP::W - 1][tid];
            const uint32_t wv[3] = {w.x, w.y, w.z};
            const bool four = dp.kde_bits == 4;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint32_t v = (a.e.y >> (8 * c)) & 0xffu;
                const uint32_t byte = four ? (v >> 1) : v;   // the byte's offset within the row
                const uint32_t x = (wv[c] >> (8 * (byte & 3u))) & 0xffu;   // rows start word-aligned
                a.qk[c] = four ? 17u * ((x >> ((v & 1u) << 2)) & 15u) : x;
            }
            int st;
            if constexpr (PP::PC) st = s2_finish_pc<T, K>(A, a, flag);
            else st = s2_finish<T, K, PP::M1>(A, a, flag);
            cbg += st == COG_ST_GMM_BG; cfg += st == COG_ST_FG; cil += st == COG_ST_ILLUM;
        }
        j = j1;
        b ^= 1;
    }
    cp_async_wait<0>();
    cbg = __reduce_add_sync(0xffffffffu, cbg);
    cfg = __reduce_add_sync(0xffffffffu, cfg);
    cil = __reduce_add_sync(0xffffffffu, cil);
    if (lane == 0) {
        if (cbg) atomicAdd(&cnt_s[0], cbg);
        if (cfg) atomicAdd(&cnt_s[1], cfg);
        if (cil) atomicAdd(&cnt_s[2], cil);
    }
    __syncthreads();
    if (tid < 3 && cnt_s[tid]) atomicAdd(ctl + ctl_slot(n % 3, 2 + tid, cta & (CTL_SLOTS - 1)), cnt_s[tid]);
}

template <typename T, int K, int TPB, int V>
__global__ void __launch_bounds__(TPB) stage2_kernel(const ApplyArgs A)
{
    grid_launch_dependents();
    grid_wait_prior();     // the queue and counters come from stage01_kernel
    k2_cta<T, K, TPB, V>(A, blockIdx.x, gridDim.x);
}

// ---- batched: many streams of one storage type and K in one launch each
__device__ __forceinline__ int batch_stream(const uint32_t *pre, int n, uint32_t x)
{
    int lo = 0, hi = n;            // largest s < n with pre[s] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// A persistent grid walks the active streams' tiles (the step plan's
// prefix gives inactive streams no tiles).  Each thread copies its next
// tile's stage-0 inputs into its shared slot with cp.async while the CTA
// runs the current tile, for full tiles of streams with 4-byte aligned
// frames and no temporal sampling (the others load as they go).
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, K1_THREADS_PER_SM / TPB) stage01_batch_kernel(const BatchGroupDev G)
{
    __shared__ K1Pre<T, TPB> pre[2];
    grid_launch_dependents();
    grid_wait_prior();
    const int tid = threadIdx.x;
    const uint32_t total = __ldg(G.k1_pre + G.n);
    // stream and tile of the CTA's t-th tile; false past the end or on a
    // failed check (the same for every thread of the CTA)
    auto locate = [&](uint32_t t, int &s, uint32_t &tile) -> bool {
        if (t >= total) return false;
        s = batch_stream(G.k1_pre, G.n, t);
        if (!in_bounds(G.descs[0].s.ctl, (uint64_t)s, (uint64_t)G.n, DBG_BATCH_STREAM)) return false;
        tile = t - __ldg(G.k1_pre + s);
        return in_bounds(G.descs[s].s.ctl, (uint64_t)tile * TPB * PPT, (uint64_t)G.descs[s].dp.P, DBG_BATCH_TILE);
    };
    auto prefetch = [&](const ApplyArgs &A, uint32_t tile, int b) -> bool {
        const uint32_t cbase = tile * TPB * PPT, p0 = cbase + (uint32_t)tid * PPT;
        if ((int64_t)cbase + TPB * PPT > A.dp.P || !A.frame_al4 || (A.dp.flags & COG_SAMPLE)) return false;
        cp_async16(&pre[b].jl[tid], A.s.jl + p0);
        const T *cv = reinterpret_cast<const T *>(A.s.conf) + p0;
        if (VecN<T, PPT>::NW == 4) cp_async16(pre[b].cv[tid], cv);
        else cp_async8(pre[b].cv[tid], cv);
        const uint8_t *f = A.frame + (size_t)p0 * 3;
#pragma unroll
        for (int i = 0; i < 3; i++) cp_async4(&pre[b].fr[tid][i], f + 4 * i);
        return true;
    };
    uint32_t t = blockIdx.x, tile = 0;
    int s = 0, b = 0;
    bool ok = locate(t, s, tile);
    bool pf = ok && prefetch(G.descs[s], tile, 0);
    cp_async_commit();
    while (ok) {
        const uint32_t tn = t + gridDim.x;
        uint32_t tile_n = 0;
        int sn = 0;
        const bool ok_n = locate(tn, sn, tile_n);
        const bool pf_n = ok_n && prefetch(G.descs[sn], tile_n, b ^ 1);
        cp_async_commit();
        cp_async_wait<1>();   // this tile's copies (the group before the one just committed)
        if (pf) {
            const K1Slot<T> sl = pre[b].slot(tid);
            k1_cta<T, TPB, true>(G.descs[s], tile, &sl);
        } else {
            k1_cta<T, TPB>(G.descs[s], tile);
        }
        t = tn; s = sn; tile = tile_n; ok = ok_n; pf = pf_n; b ^= 1;
    }
    cp_async_wait<0>();
}

// The mixture-stage CTAs are split among the active streams only.
// Registers of the batched mixture stage.  Warps get registers per SM
// sub-partition (16K each), so 72 registers fit 7 warps (14 CTAs of 64
// threads per SM) and 96 fit 5 (10 CTAs), where 97-112 fit 4 (8 CTAs):
// K <= 3 at 72, K = 4, 5 at 96, larger K as the compiler chooses.
template <int K> constexpr int k2_batch_maxreg() { return K <= 3 ? 72 : (K <= 5 ? 96 : 255); }

template <typename T, int K, int TPB, int V>
__global__ void __launch_bounds__(TPB) __maxnreg__(k2_batch_maxreg<K>()) stage2_batch_kernel(const BatchGroupDev G)
{
    grid_launch_dependents();
    grid_wait_prior();
    if (blockIdx.x >= __ldg(G.k2_pre + G.n)) return;
    const int s = batch_stream(G.k2_pre, G.n, blockIdx.x);
    if (!in_bounds(G.descs[0].s.ctl, (uint64_t)s, (uint64_t)G.n, DBG_BATCH_STREAM)) return;
    // a batch gives each CTA many survivors per thread: the pipelined walk,
    // where its shared slots fit
    if constexpr (sizeof(K2Pipe<T, K, TPB, V>) <= 40 * 1024)
        k2_cta_pipe<T, K, TPB, V>(G.descs[s], blockIdx.x - G.k2_pre[s], G.k2_pre[s + 1] - G.k2_pre[s]);
    else
        k2_cta<T, K, TPB, V>(G.descs[s], blockIdx.x - G.k2_pre[s], G.k2_pre[s + 1] - G.k2_pre[s]);
}

// Launch with programmatic stream serialization: the kernel may be
// scheduled before the preceding kernel on the stream finishes; it waits in
// grid_wait_prior() for that kernel's results.
template <typename Kern>
cudaError_t launch_pdl(Kern kern, int64_t grid, int block, cudaStream_t st, const ApplyArgs &a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// ---- launch shapes: first-kernel CTA size in {64, 128, 256}, mixture-stage
//      CTA size in {64, 128}, mixture-stage CTAs per SM (0: as many as fit)
template <typename T>
void (*k1_single(int tpb))(ApplyArgs)
{
    return tpb == 64 ? stage01_kernel<T, 64> : (tpb == 256 ? stage01_kernel<T, 256> : stage01_kernel<T, 128>);
}
template <typename T, int K>
void (*k2_single(int tpb, int mv))(ApplyArgs)
{
    if (mv == 1) return tpb == 128 ? stage2_kernel<T, K, 128, 1> : stage2_kernel<T, K, 64, 1>;
    if (mv == 2) return tpb == 128 ? stage2_kernel<T, K, 128, 2> : stage2_kernel<T, K, 64, 2>;
    return tpb == 128 ? stage2_kernel<T, K, 128, 0> : stage2_kernel<T, K, 64, 0>;
}
template <typename T>
void (*k1_batch(int tpb))(BatchGroupDev)
{
    return tpb == 64 ? stage01_batch_kernel<T, 64>
                     : (tpb == 256 ? stage01_batch_kernel<T, 256> : stage01_batch_kernel<T, 128>);
}
template <typename T, int K>
void (*k2_batch(int tpb, int mv))(BatchGroupDev)
{
    if (mv == 1) return tpb == 128 ? stage2_batch_kernel<T, K, 128, 1> : stage2_batch_kernel<T, K, 64, 1>;
    if (mv == 2) return tpb == 128 ? stage2_batch_kernel<T, K, 128, 2> : stage2_batch_kernel<T, K, 64, 2>;
    return tpb == 128 ? stage2_batch_kernel<T, K, 128, 0> : stage2_batch_kernel<T, K, 64, 0>;
}

template <typename KernT>
int blocks_per_sm(KernT k, int tpb)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, tpb, 0) != cudaSuccess || b < 1) b = 1;
    return b;
}

namespace {
// Mixture-stage CTAs that fit on one SM, by CTA size (64, 128) and K; one
// table per translation unit (storage type), filled on first use.
int k2_occupancy[3][2][KMAX + 1];   // [mixture variant][CTA size][K]
}

template <typename T, int K>
cudaError_t launch_apply_t(const ApplyArgs &a, const LaunchCfg &lc, cudaStream_t st, const ApplyEvents *ev)
{
    const int64_t g1 = (a.dp.P + lc.k1_tpb * K1_PX_PER_THREAD - 1) / (lc.k1_tpb * K1_PX_PER_THREAD);
    if (ev) cudaEventRecord(ev->e0, st);
    cudaError_t e = launch_pdl(k1_single<T>(lc.k1_tpb), g1, lc.k1_tpb, st, a);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev->e1, st);
    const int mv = mix_variant(a.dp.flags);
    int &ps = k2_occupancy[mv][lc.k2_tpb == 128][K];
    if (!ps) ps = blocks_per_sm(k2_single<T, K>(lc.k2_tpb, mv), lc.k2_tpb);
    const int use = lc.k2_per_sm > 0 && lc.k2_per_sm < ps ? lc.k2_per_sm : ps;
    const int64_t need = (a.dp.P + lc.k2_tpb - 1) / lc.k2_tpb;
    const int64_t g2 = min((int64_t)a.k2_grid * use, need);
    e = launch_pdl(k2_single<T, K>(lc.k2_tpb, mv), max((int64_t)1, g2), lc.k2_tpb, st, a);
    if (ev) cudaEventRecord(ev->e2, st);
    return e;
}

template <typename T, int K>
cudaError_t launch_batch_t(const BatchGroupDev &g, const LaunchCfg &lc, uint32_t k1_ctas, uint32_t k2_ctas,
                           cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.stream = st;
    cfg.gridDim = dim3(k1_ctas);
    cfg.blockDim = dim3(lc.k1_tpb);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k1_batch<T>(lc.k1_tpb), g);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(k2_ctas);
    cfg.blockDim = dim3(lc.k2_tpb);
    return cudaLaunchKernelEx(&cfg, k2_batch<T, K>(lc.k2_tpb, g.mv), g);
}

template <typename T, int K>
int k2_blocks_per_sm_t(const LaunchCfg &lc, int mv)
{
    const int ps = blocks_per_sm(k2_batch<T, K>(lc.k2_tpb, mv), lc.k2_tpb);
    return lc.k2_per_sm > 0 && lc.k2_per_sm < ps ? lc.k2_per_sm : ps;
}

template <typename T>
int k1_batch_blocks_per_sm_t(const LaunchCfg &lc)
{
    return blocks_per_sm(k1_batch<T>(lc.k1_tpb), lc.k1_tpb);
}

}  // namespace cog
