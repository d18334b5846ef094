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
    const float wa = (float)(q & 0xffu) * R255, wb = (float)(q >> 8) * R255;
    const float wg = (float)(255u - (q & 0xffu) - (q >> 8)) * R255;
    return wa + wb * (1.f - (float)D * R255) + wg * (1.f - tr);
}

// Shared memory of one warp of stage01_kernel: the stage-1 work list and
// what its pixels need, and the results the owners collect.
struct K1Warp {
    uint2 stash[WPX];      // rgb | D << 24, C- bits
    uint8_t list[WPX];     // pixel slot (lane * 4 + i)
    uint8_t resst[WPX];    // 1: decided at stage 1, 2: survivor
    float resc[WPX];       // new C of pixels decided at stage 1
};

// One group of PPT consecutive pixels of a thread in stage01_kernel: its
// loaded state, its frame words and its stage-0 outcome.
template <typename T> struct K1Group {
    uint4 jl;                 // previous frame + label of the 4 pixels
    VecN<T, PPT> cv;          // confidence
    uint32_t Iw[PPT];         // this frame's pixels as r | g << 8 | b << 16
    uint32_t ad[PPT];         // per-channel |I - J|, byte-wise
    uint32_t skip, need1;     // bits: skipped by sampling, past stage 0
    int nact;                 // pixels of the group inside the frame
};

// Stage-0 loads of one group: previous frame + label (16 B), confidence (8
// or 16 B), frame bytes (12 B).  With temporal sampling, a 64-pixel block
// off its phase reads its frame bytes only if some pixel in the group has
// not saturated (Sec. 2, "Confidence based temporal sampling"; a group of 4
// never straddles two blocks).
template <typename T, bool FULL>
__device__ __forceinline__ void k1_group_load(const ApplyArgs &A, K1Group<T> &G, uint32_t p0)
{
    const DevParams &dp = A.dp;
    G.nact = FULL ? PPT : (int)min((int64_t)PPT, max((int64_t)0, dp.P - (int64_t)p0));
    G.jl = make_uint4(0, 0, 0, 0);
    G.skip = 0;
    uint32_t w0 = 0, w1 = 0, w2 = 0;
#pragma unroll
    for (int i = 0; i < VecN<T, PPT>::NW; i++) G.cv.w[i] = 0;
    if (FULL || G.nact > 0) {
        G.jl = *reinterpret_cast<const uint4 *>(A.s.jl + p0);
        G.cv.load(reinterpret_cast<const T *>(A.s.conf) + p0);
        const bool sampling = (dp.flags & COG_SAMPLE) && (dp.flags & COG_CONF);
        if (sampling && (A.frame_idx + (p0 >> 6)) % (uint32_t)dp.skip_period != 0u) {
#pragma unroll
            for (int i = 0; i < PPT; i++)
                if ((FULL || i < G.nact) && G.cv.get(i) >= dp.c_skip) G.skip |= 1u << i;
        }
        if (G.skip == (1u << G.nact) - 1u) {
            // every pixel of the group keeps its label this frame
        } else if (A.frame_al4 && (FULL || G.nact == PPT)) {
            const uint32_t *f4 = reinterpret_cast<const uint32_t *>(A.frame + (size_t)p0 * 3);
            w0 = f4[0]; w1 = f4[1]; w2 = f4[2];
        } else {
            uint32_t fw[3] = {0, 0, 0};
#pragma unroll
            for (int b3 = 0; b3 < PPT * 3; b3++)
                if (b3 < G.nact * 3) fw[b3 >> 2] |= (uint32_t)A.frame[(size_t)p0 * 3 + b3] << ((b3 & 3) * 8);
            w0 = fw[0]; w1 = fw[1]; w2 = fw[2];
        }
    }
    G.Iw[0] = w0 & 0x00ffffffu;
    G.Iw[1] = __byte_perm(w0, w1, 0x0543) & 0x00ffffffu;
    G.Iw[2] = __byte_perm(w1, w2, 0x0432) & 0x00ffffffu;
    G.Iw[3] = w2 >> 8;
}

// Stage 0 of one group: D = max_c |I_c - J_c| <= tau_fd (0.5 + C-) on a
// background pixel.  D is an integer, so the test is D <= floor(tau)
// applied to every channel at once.
template <typename T, bool FULL>
__device__ __forceinline__ void k1_group_stage0(const DevParams &dp, K1Group<T> &G)
{
    const bool conf_on = dp.flags & COG_CONF;
    const bool fd_on = dp.flags & COG_FD;
#pragma unroll
    for (int i = 0; i < PPT; i++) G.ad[i] = __vabsdiffu4(G.Iw[i], u4get(G.jl, i) & 0x00ffffffu);
    G.need1 = 0;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        if ((!FULL && i >= G.nact) || (G.skip >> i & 1u)) continue;
        const float Cm = conf_on ? G.cv.get(i) : 0.5f;
        const float tau = dp.tau_fd * (0.5f + Cm);
        const uint32_t t = tau >= 255.f ? 255u : (uint32_t)tau;      // floor, tau >= 0
        const bool pass = fd_on && (u4get(G.jl, i) >> 24) == 0 && __vcmpgtu4(G.ad[i], t * 0x01010101u) == 0u;
        if (!pass) G.need1 |= 1u << i;
    }
}

// Outputs of one group: the previous frame becomes this frame with label 0
// (the mixture stage sets its survivors' labels), the mask 0 (likewise),
// the confidence of the pixels decided here; a pixel skipped by the
// temporal sampling keeps everything and shows its carried label.
template <typename T, bool FULL>
__device__ __forceinline__ void k1_group_out(const ApplyArgs &A, const K1Warp &W, const K1Group<T> &G, uint32_t p0,
                                             int slot0, uint32_t &n_fd, uint32_t &n_skip)
{
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    if (!(FULL || G.nact > 0)) return;
    uint4 jn;
    uint32_t sm = 0, mk = 0;
    VecN<T, PPT> cn = G.cv;
    bool any_c = false;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        const bool act = FULL || i < G.nact;
        const bool sk = G.skip >> i & 1u;
        const uint32_t r1 = (G.need1 >> i & 1u) ? W.resst[slot0 + i] : 0u;
        n_fd += act && !sk && r1 == 0;
        n_skip += sk;
        if (conf_on && act && !sk && r1 != 2) {
            cn.set(i, r1 == 0 ? (1.f - dp.eta) * G.cv.get(i) + dp.eta : W.resc[slot0 + i]);
            any_c = true;
        }
        u4set(jn, i, act && !sk ? G.Iw[i] : u4get(G.jl, i));
        if (sk) mk |= ((u4get(G.jl, i) >> 24) ? 255u : 0u) << (8 * i);
        sm |= (sk ? (uint32_t)COG_ST_SKIP
                  : (r1 == 0 ? (uint32_t)COG_ST_FD : (r1 == 1 ? (uint32_t)COG_ST_RGA : (uint32_t)COG_ST_GMM_BG)))
              << (8 * i);
    }
    if (jn.x != G.jl.x || jn.y != G.jl.y || jn.z != G.jl.z || jn.w != G.jl.w)
        *reinterpret_cast<uint4 *>(A.s.jl + p0) = jn;
    if (any_c) cn.store(reinterpret_cast<T *>(A.s.conf) + p0);
    if ((FULL || G.nact == PPT) && A.out_al4) {
        *reinterpret_cast<uint32_t *>(A.mask + p0) = mk;
        if (A.stagemap) *reinterpret_cast<uint32_t *>(A.stagemap + p0) = sm;
    } else {
        for (int i = 0; i < G.nact; i++) {
            A.mask[p0 + i] = (uint8_t)(mk >> (8 * i));
            if (A.stagemap) A.stagemap[p0 + i] = (uint8_t)(sm >> (8 * i));
        }
    }
}

// One warp's WPX pixels (K1_G groups of 128: each lane owns 4 consecutive
// pixels of every group) through stages 0 and 1.  FULL: every pixel of the
// warp lies inside the frame (all warps but the last one's).  Returns the
// warp's survivor count; counts of the pixels decided here are added to
// n_fd / n_rga / n_skip (per lane).
template <typename T, bool FULL>
__device__ __forceinline__ int k1_warp(const ApplyArgs &A, K1Warp &W, uint32_t wbase, int lane, uint32_t seg,
                                       uint32_t &n_fd, uint32_t &n_rga, uint32_t &n_skip)
{
    const DevParams &dp = A.dp;
    const bool conf_on = dp.flags & COG_CONF;
    K1Group<T> grp[K1_G];
#pragma unroll
    for (int g = 0; g < K1_G; g++) k1_group_load<T, FULL>(A, grp[g], wbase + g * 128 + (uint32_t)lane * PPT);
#pragma unroll
    for (int g = 0; g < K1_G; g++) k1_group_stage0<T, FULL>(dp, grp[g]);

    // ---- the stage-1 work list of the warp
    int n1 = 0;
#pragma unroll
    for (int g = 0; g < K1_G; g++) n1 += __popc(grp[g].need1);
    int incl = n1;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    const int n1w = __shfl_sync(0xffffffffu, incl, 31);
    {
        int k = incl - n1;
#pragma unroll
        for (int g = 0; g < K1_G; g++) {
            if (!grp[g].need1) continue;
#pragma unroll
            for (int i = 0; i < PPT; i++) {
                if (!(grp[g].need1 >> i & 1u)) continue;
                const int slot = g * 128 + lane * PPT + i;
                W.list[k++] = (uint8_t)slot;
                const uint32_t m2 = __vmaxu4(grp[g].ad[i], grp[g].ad[i] >> 8);
                const uint32_t D = __vmaxu4(m2, m2 >> 8) & 0xffu;
                W.stash[slot] = make_uint2(grp[g].Iw[i] | (D << 24),
                                           __float_as_uint(conf_on ? grp[g].cv.get(i) : 0.5f));
            }
        }
    }
    __syncwarp();

    // ---- stage 1 over the compacted list: one pass per 32 pixels left
    int ne = 0;
    const uint32_t lt = (1u << lane) - 1u;
    for (int j0 = 0; j0 < n1w; j0 += 32) {
        const int j = j0 + lane;
        bool surv = false;
        uint4 ent = make_uint4(0, 0, 0, 0);
        if (j < n1w) {
            const int slot = W.list[j];
            const uint32_t p = wbase + slot;
            const uint2 sv = W.stash[slot];
            const int D = (int)(sv.x >> 24);
            const float Cm = __uint_as_float(sv.y);
            S1Rec<T> r;
            r.load(A.s.s1, p);
            if (dp.flags & COG_RGA) {
                float tr = 0.f;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float d = (float)((sv.x >> (8 * c)) & 0xffu) - r.get(c);
                    const float t = __fdividef(d * d, dp.lam2 * r.get(3 + c));
                    tr = t > tr ? t : tr;
                }
                if (tr < 1.f) {
                    if (!(conf_on && Cm >= dp.c_halt)) {
                        const float ae = dp.alpha * (1.5f - Cm);
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const float I = (float)((sv.x >> (8 * c)) & 0xffu);
                            const float m = r.get(c) + ae * (I - r.get(c));
                            const float d = I - m;
                            r.set(c, m);
                            r.set(3 + c, clampf((1.f - ae) * r.get(3 + c) + ae * d * d, dp.var_min, dp.var_max));
                        }
                        r.store(A.s.s1, p);
                    }
                    W.resc[slot] = (1.f - dp.eta) * Cm + dp.eta * conf_stage1(r.qab(), D, tr);
                    W.resst[slot] = 1;
                    n_rga++;
                } else {
                    surv = true;
                }
            } else {
                surv = true;
            }
            if (surv) {
                W.resst[slot] = 2;
                ent = make_uint4(p, sv.x, sv.y, r.qab());
            }
        }
        // survivors of this pass go straight to the frame's queue segment
        const uint32_t b = __ballot_sync(0xffffffffu, surv);
        if (b) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(A.s.ctl + ctl_qcnt(A.frame_no % 3, seg), (uint32_t)__popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (surv) A.s.queue[(int64_t)seg * A.s.qseg_cap + base + __popc(b & lt)] = ent;
        }
        ne += __popc(b);
    }
    __syncwarp();

#pragma unroll
    for (int g = 0; g < K1_G; g++)
        k1_group_out<T, FULL>(A, W, grp[g], wbase + g * 128 + (uint32_t)lane * PPT, g * 128 + lane * PPT, n_fd, n_skip);
    return ne;
}

// One CTA of the stage-0/1 pass over stream A: tile `cta` of its frame.
template <typename T, int TPB>
__device__ __forceinline__ void k1_cta(const ApplyArgs &A, uint32_t cta)
{
    static_assert(PPT == 4, "frame and mask vector widths assume groups of 4 pixels");
    constexpr int NW = TPB / 32;
    __shared__ K1Warp W_s[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = A.frame_no;
    uint32_t *ctl = A.s.ctl;
    const uint32_t wbase = (cta * NW + warp) * WPX;

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

    // warp w puts its survivors into queue segment w % QSEG
    const uint32_t gwarp = cta * NW + warp;
    const uint32_t seg = gwarp & (QSEG - 1);
    uint32_t n_fd = 0, n_rga = 0, n_skip = 0;
    int ne;
    if ((int64_t)wbase + WPX <= A.dp.P) ne = k1_warp<T, true>(A, W_s[warp], wbase, lane, seg, n_fd, n_rga, n_skip);
    else ne = k1_warp<T, false>(A, W_s[warp], wbase, lane, seg, n_fd, n_rga, n_skip);

    // per-warp counts (padded counters)
    const uint32_t vfd = __reduce_add_sync(0xffffffffu, n_fd);
    const uint32_t vrga = __reduce_add_sync(0xffffffffu, n_rga);
    const uint32_t vskip = __reduce_add_sync(0xffffffffu, n_skip);
    if (lane == 0) {
        const uint32_t slot = gwarp & (CTL_SLOTS - 1);
        if (vfd) atomicAdd(ctl + ctl_slot(n % 3, 0, slot), vfd);
        if (vrga) atomicAdd(ctl + ctl_slot(n % 3, 1, slot), vrga);
        if (vskip) atomicAdd(ctl + ctl_slot(n % 3, 6, slot), vskip);
        if (ne) atomicAdd(ctl + ctl_slot(n % 3, 5, slot), (uint32_t)ne);
    }
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

template <typename T, int K, bool PC = false>
__device__ __forceinline__ void s2_load(const ApplyArgs &A, int64_t qi, S2In<T, K, PC> &in)
{
    in.e = __ldcg(A.s.queue + qi);
    const int64_t p = in.e.x;
#pragma unroll
    for (int c = 0; c < 3; c++) in.qk[c] = __ldg(A.s.kde + (p * 3 + c) * 256 + ((in.e.y >> (8 * c)) & 0xffu));
    const uint4 *src = reinterpret_cast<const uint4 *>(A.s.gmm + p * RecSel<T, K, PC>::BYTES);
#pragma unroll
    for (int i = 0; i < RecSel<T, K, PC>::NV; i++) in.rec[i] = src[i];
    if (!PC && (A.dp.flags & COG_MODE1)) in.s1.load(A.s.s1, p);
}

// Confidence of a pixel decided at stage 2 (Sec. 2, "Confidence Measure"):
// prior term from the three prior bytes unless the prior is nullified.
__device__ __forceinline__ float conf_stage2(const DevParams &dp, const uint32_t qk[3], uint32_t qab, int D, float Cm,
                                             float Mh)
{
    uint32_t qmin = qk[0] < qk[1] ? qk[0] : qk[1];
    qmin = qk[2] < qmin ? qk[2] : qmin;
    const uint32_t qa = qab & 0xffu, qb = qab >> 8;
    const float wa = (float)qa * R255, wb = (float)qb * R255;
    const float wg = (float)(255u - qa - qb) * R255;
    const float dhat = (float)D * R255;
    float ci;
    if ((int)qmin < dp.q_null) {
        const float den = wb + wg;
        ci = den > 0.f ? (wb * (1.f - dhat) + wg * (1.f - Mh)) / den : 0.f;
    } else {
        ci = wa * ((float)qmin * R255) + wb * (1.f - dhat) + wg * (1.f - Mh);
    }
    return (1.f - dp.eta) * Cm + dp.eta * ci;
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
    const MixOutPC o = mix_step_pc<K>(m, I, dp.alpha * (1.5f - Cm), dp);
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

template <typename T, int K>
__device__ __forceinline__ int s2_finish(const ApplyArgs &A, const S2In<T, K> &in, bool flag)
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
    const bool mode1 = dp.flags & COG_MODE1;
    if (mode1) mode1_write_back<T, K>(m, in.s1);
    const float ae = dp.alpha * (1.5f - Cm);
    const MixOut o = mix_step<K>(m, I, ae, dp);
    int label = o.fg, st = o.fg ? COG_ST_FG : COG_ST_GMM_BG;
    if (flag && o.fg) {
        illum_response<K>(m, o.tgt, dp.w_illum);
        label = 0;
        st = COG_ST_ILLUM;
    }
    rec_store<T, K>(A.s.gmm, p, m);
    if (mode1) {
        S1Rec<T> r = in.s1;
        mode1_recache<T, K>(m, r);
        r.store(A.s.s1, p);
    } else if (!label) {   // transition update: the background mode seeds stage 1
        S1Rec<T> r;
#pragma unroll
        for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = make_uint4(0, 0, 0, 0);
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
        const float Mh = o.match >= 0 ? (o.tm < 1.f ? o.tm : 1.f) : 1.f;
        reinterpret_cast<T *>(A.s.conf)[p] = Store<T>::from_f(conf_stage2(dp, in.qk, qab, D, Cm, Mh));
    }
    reinterpret_cast<uint8_t *>(A.s.jl)[p * 4 + 3] = (uint8_t)label;
    A.mask[p] = label ? 255 : 0;
    if (A.stagemap) A.stagemap[p] = (uint8_t)st;
    return st;
}

// One of ncta CTAs walking stream A's survivor queue.
template <typename T, int K, int TPB, bool PC = false>
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
    auto entry = [&](uint32_t q) -> int64_t {   // flat index -> queue slot
        int lo = 0;
#pragma unroll
        for (int step = QSEG / 2; step >= 1; step >>= 1)
            if (segp_s[lo + step] <= q) lo += step;
        return (int64_t)lo * A.s.qseg_cap + (q - segp_s[lo]);
    };
    uint32_t cbg = 0, cfg = 0, cil = 0;
    for (uint32_t q = cta * TPB + tid; q < nq; q += stride) {
        S2In<T, K, PC> a;
        s2_load<T, K, PC>(A, entry(q), a);
        int st;
        if constexpr (PC) st = s2_finish_pc<T, K>(A, a, flag);
        else st = s2_finish<T, K>(A, a, flag);
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

template <typename T, int K, int TPB, bool PC = false>
__global__ void __launch_bounds__(TPB) stage2_kernel(const ApplyArgs A)
{
    grid_launch_dependents();
    grid_wait_prior();     // the queue and counters come from stage01_kernel
    k2_cta<T, K, TPB, PC>(A, blockIdx.x, gridDim.x);
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
// prefix gives inactive streams no tiles).
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, K1_THREADS_PER_SM / TPB) stage01_batch_kernel(const BatchGroupDev G)
{
    grid_launch_dependents();
    grid_wait_prior();
    const uint32_t total = __ldg(G.k1_pre + G.n);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int s = batch_stream(G.k1_pre, G.n, t);
        k1_cta<T, TPB>(G.descs[s], t - __ldg(G.k1_pre + s));
    }
}

// The mixture-stage CTAs are split among the active streams only.
template <typename T, int K, int TPB, bool PC = false>
__global__ void __launch_bounds__(TPB) stage2_batch_kernel(const BatchGroupDev G)
{
    grid_launch_dependents();
    grid_wait_prior();
    if (blockIdx.x >= __ldg(G.k2_pre + G.n)) return;
    const int s = batch_stream(G.k2_pre, G.n, blockIdx.x);
    k2_cta<T, K, TPB, PC>(G.descs[s], blockIdx.x - G.k2_pre[s], G.k2_pre[s + 1] - G.k2_pre[s]);
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
void (*k2_single(int tpb, bool pc))(ApplyArgs)
{
    if (pc) return tpb == 128 ? stage2_kernel<T, K, 128, true> : stage2_kernel<T, K, 64, true>;
    return tpb == 128 ? stage2_kernel<T, K, 128> : stage2_kernel<T, K, 64>;
}
template <typename T>
void (*k1_batch(int tpb))(BatchGroupDev)
{
    return tpb == 64 ? stage01_batch_kernel<T, 64>
                     : (tpb == 256 ? stage01_batch_kernel<T, 256> : stage01_batch_kernel<T, 128>);
}
template <typename T, int K>
void (*k2_batch(int tpb, bool pc))(BatchGroupDev)
{
    if (pc) return tpb == 128 ? stage2_batch_kernel<T, K, 128, true> : stage2_batch_kernel<T, K, 64, true>;
    return tpb == 128 ? stage2_batch_kernel<T, K, 128> : stage2_batch_kernel<T, K, 64>;
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
int k2_occupancy[2][2][KMAX + 1];   // [per-channel][CTA size][K]
}

template <typename T, int K>
cudaError_t launch_apply_t(const ApplyArgs &a, const LaunchCfg &lc, cudaStream_t st, const ApplyEvents *ev)
{
    const int64_t g1 = (a.dp.P + lc.k1_tpb * K1_PX_PER_THREAD - 1) / (lc.k1_tpb * K1_PX_PER_THREAD);
    if (ev) cudaEventRecord(ev->e0, st);
    cudaError_t e = launch_pdl(k1_single<T>(lc.k1_tpb), g1, lc.k1_tpb, st, a);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev->e1, st);
    const bool pc = a.dp.flags & COG_PERCHAN;
    int &ps = k2_occupancy[pc][lc.k2_tpb == 128][K];
    if (!ps) ps = blocks_per_sm(k2_single<T, K>(lc.k2_tpb, pc), lc.k2_tpb);
    const int use = lc.k2_per_sm > 0 && lc.k2_per_sm < ps ? lc.k2_per_sm : ps;
    const int64_t need = (a.dp.P + lc.k2_tpb - 1) / lc.k2_tpb;
    const int64_t g2 = min((int64_t)a.k2_grid * use, need);
    e = launch_pdl(k2_single<T, K>(lc.k2_tpb, pc), max((int64_t)1, g2), lc.k2_tpb, st, a);
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
    return cudaLaunchKernelEx(&cfg, k2_batch<T, K>(lc.k2_tpb, g.pc != 0), g);
}

template <typename T, int K>
int k2_blocks_per_sm_t(const LaunchCfg &lc, bool pc)
{
    const int ps = blocks_per_sm(k2_batch<T, K>(lc.k2_tpb, pc), lc.k2_tpb);
    return lc.k2_per_sm > 0 && lc.k2_per_sm < ps ? lc.k2_per_sm : ps;
}

template <typename T>
int k1_batch_blocks_per_sm_t(const LaunchCfg &lc)
{
    return blocks_per_sm(k1_batch<T>(lc.k1_tpb), lc.k1_tpb);
}

}  // namespace cog
