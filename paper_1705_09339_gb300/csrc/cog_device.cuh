// cog_device.cuh -- device-side building blocks of the CoG kernels:
// storage-type conversion, 128-bit vector access to the state planes, the
// per-pixel mixture record, and the Stauffer-Grimson step of Eq. 2 that the
// cascade's last stage, the plain-mixture baseline and the training warm-up
// share.  All arithmetic is FP32 whatever the storage type.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "cog_internal.h"

namespace cog {

// ----------------------------------------------------------------- storage
template <typename T> struct Store;

template <> struct Store<float> {
    static constexpr int bytes = 4;
    __device__ __forceinline__ static float to_f(float x) { return x; }
    __device__ __forceinline__ static float from_f(float x) { return x; }
    __device__ __forceinline__ static uint32_t bits(float x) { return __float_as_uint(x); }
    __device__ __forceinline__ static float unbits(uint32_t b) { return __uint_as_float(b); }
};
template <> struct Store<__half> {
    static constexpr int bytes = 2;
    __device__ __forceinline__ static float to_f(__half x) { return __half2float(x); }
    __device__ __forceinline__ static __half from_f(float x) { return __float2half_rn(x); }
    __device__ __forceinline__ static uint32_t bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
    __device__ __forceinline__ static float unbits(uint32_t b) { return __half2float(__ushort_as_half((unsigned short)b)); }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr int bytes = 2;
    __device__ __forceinline__ static float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
    __device__ __forceinline__ static __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
    __device__ __forceinline__ static uint32_t bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    __device__ __forceinline__ static float unbits(uint32_t b) { return __bfloat162float(__ushort_as_bfloat16((unsigned short)b)); }
};

// Two 16-bit values in one word (low, high) to and from floats, with one
// conversion per pair.
template <typename T> struct Pair;
template <> struct Pair<float> {   // unused: FP32 state is read by word
    __device__ __forceinline__ static float2 to_f2(uint32_t) { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static uint32_t from_f2(float, float) { return 0u; }
};
template <> struct Pair<__half> {
    __device__ __forceinline__ static float2 to_f2(uint32_t w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    __device__ __forceinline__ static uint32_t from_f2(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <> struct Pair<__nv_bfloat16> {
    __device__ __forceinline__ static float2 to_f2(uint32_t w) {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
    __device__ __forceinline__ static uint32_t from_f2(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

__device__ __forceinline__ uint32_t u4get(const uint4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ void u4set(uint4 &v, int i, uint32_t x)
{
    if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
}

// Eight consecutive values of a plane (8 x T = 16 or 32 bytes, aligned).
template <typename T> struct Vec8 {
    static constexpr int NV = (8 * Store<T>::bytes) / 16;   // uint4 per 8 values
    uint4 u[NV];
    __device__ __forceinline__ void load(const T *p) {
#pragma unroll
        for (int i = 0; i < NV; i++) u[i] = reinterpret_cast<const uint4 *>(p)[i];
    }
    __device__ __forceinline__ void store(T *p) const {
#pragma unroll
        for (int i = 0; i < NV; i++) reinterpret_cast<uint4 *>(p)[i] = u[i];
    }
    __device__ __forceinline__ float get(int i) const {
        if (Store<T>::bytes == 4) return Store<T>::unbits(u4get(u[i >> 2], i & 3));
        uint32_t w = u4get(u[i >> 3], (i >> 1) & 3);
        return Store<T>::unbits((i & 1) ? (w >> 16) : (w & 0xffffu));
    }
    __device__ __forceinline__ void set(int i, float x) {
        uint32_t b = Store<T>::bits(x);
        if (Store<T>::bytes == 4) { u4set(u[i >> 2], i & 3, b); return; }
        uint32_t w = u4get(u[i >> 3], (i >> 1) & 3);
        w = (i & 1) ? ((w & 0xffffu) | (b << 16)) : ((w & 0xffff0000u) | b);
        u4set(u[i >> 3], (i >> 1) & 3, w);
    }
};

// N consecutive values of a plane held as raw 32-bit words, loaded and
// stored with the widest aligned vector (N*sizeof(T) = 8, 16 or 32 bytes).
template <typename T, int N> struct VecN {
    static constexpr int BYTES = N * Store<T>::bytes;
    static constexpr int NW = BYTES / 4;
    uint32_t w[NW];
    __device__ __forceinline__ void load(const T *p) {
        if (BYTES % 16 == 0) {
#pragma unroll
            for (int i = 0; i < BYTES / 16; i++) {
                const uint4 v = reinterpret_cast<const uint4 *>(p)[i];
                w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < BYTES / 8; i++) {
                const uint2 v = reinterpret_cast<const uint2 *>(p)[i];
                w[2 * i] = v.x; w[2 * i + 1] = v.y;
            }
        }
    }
    __device__ __forceinline__ void store(T *p) const {
        if (BYTES % 16 == 0) {
#pragma unroll
            for (int i = 0; i < BYTES / 16; i++)
                reinterpret_cast<uint4 *>(p)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < BYTES / 8; i++)
                reinterpret_cast<uint2 *>(p)[i] = make_uint2(w[2 * i], w[2 * i + 1]);
        }
    }
    __device__ __forceinline__ float get(int i) const {
        if (Store<T>::bytes == 4) return Store<T>::unbits(w[i]);
        const uint32_t x = w[i >> 1];
        return Store<T>::unbits((i & 1) ? (x >> 16) : (x & 0xffffu));
    }
    __device__ __forceinline__ void set(int i, float x) {
        const uint32_t b = Store<T>::bits(x);
        if (Store<T>::bytes == 4) { w[i] = b; return; }
        const uint32_t o = w[i >> 1];
        w[i >> 1] = (i & 1) ? ((o & 0xffffu) | (b << 16)) : ((o & 0xffff0000u) | b);
    }
};

// ------------------------------------------------------------ mixture record
// Per-pixel record: K components of (w, mu0, mu1, mu2, v0, v1, v2), stored
// contiguously and padded to a 16-byte multiple so one survivor's record is
// fetched with whole 128-bit loads.
template <typename T, int K> struct Rec {
    static constexpr int NE = 7 * K;
    static constexpr int NV = (NE * Store<T>::bytes + 15) / 16;
    static constexpr int BYTES = NV * 16;
};

template <int K> struct Mix {
    float w[K], mu[K][3], v[K][3];
};

// ----------------------------------------------------------- stage-1 record
// Per-pixel running average and residue weights, one aligned block per
// pixel: (m0, m1, m2, v0, v1, v2, qa | qb << 8), 16 bytes with 16-bit
// storage, 32 with FP32.  Only pixels past stage 0 touch it, so a 32-byte
// sector serves two pixels instead of sixteen planes' worth.
template <typename T> struct S1Rec {
    static constexpr int BYTES = Store<T>::bytes == 4 ? 32 : 16;
    static constexpr int NV = BYTES / 16;
    uint4 u[NV];
    __device__ __forceinline__ void load(const uint8_t *base, int64_t p) {
#pragma unroll
        for (int i = 0; i < NV; i++) u[i] = reinterpret_cast<const uint4 *>(base + p * BYTES)[i];
    }
    __device__ __forceinline__ void store(uint8_t *base, int64_t p) const {
#pragma unroll
        for (int i = 0; i < NV; i++) reinterpret_cast<uint4 *>(base + p * BYTES)[i] = u[i];
    }
    __device__ __forceinline__ float get(int e) const {   // e: 0..2 mean, 3..5 variance
        if (Store<T>::bytes == 4) return Store<T>::unbits(u4get(u[e >> 2], e & 3));
        const uint32_t w = u4get(u[0], e >> 1);
        return Store<T>::unbits((e & 1) ? (w >> 16) : (w & 0xffffu));
    }
    __device__ __forceinline__ void set(int e, float x) {
        const uint32_t b = Store<T>::bits(x);
        if (Store<T>::bytes == 4) { u4set(u[e >> 2], e & 3, b); return; }
        uint32_t w = u4get(u[0], e >> 1);
        w = (e & 1) ? ((w & 0xffffu) | (b << 16)) : ((w & 0xffff0000u) | b);
        u4set(u[0], e >> 1, w);
    }
    __device__ __forceinline__ uint32_t qab() const {
        return Store<T>::bytes == 4 ? u4get(u[NV - 1], 2) : (u[0].w & 0xffffu);
    }
    __device__ __forceinline__ void set_qab(uint32_t q) {
        if (Store<T>::bytes == 4) u4set(u[NV - 1], 2, q);
        else u[0].w = (u[0].w & 0xffff0000u) | q;
    }
    // all six values at once: 16-bit storage converts pairs (m0 m1 | m2 v0
    // | v1 v2), FP32 reads words
    __device__ __forceinline__ void unpack(float m[3], float v[3]) const {
        if (Store<T>::bytes == 4) {
#pragma unroll
            for (int c = 0; c < 3; c++) { m[c] = get(c); v[c] = get(3 + c); }
            return;
        }
        const float2 a = Pair<T>::to_f2(u[0].x), b = Pair<T>::to_f2(u[0].y), c = Pair<T>::to_f2(u[0].z);
        m[0] = a.x; m[1] = a.y; m[2] = b.x; v[0] = b.y; v[1] = c.x; v[2] = c.y;
    }
    __device__ __forceinline__ void pack(const float m[3], const float v[3]) {
        if (Store<T>::bytes == 4) {
#pragma unroll
            for (int c = 0; c < 3; c++) { set(c, m[c]); set(3 + c, v[c]); }
            return;
        }
        u[0].x = Pair<T>::from_f2(m[0], m[1]);
        u[0].y = Pair<T>::from_f2(m[2], v[0]);
        u[0].z = Pair<T>::from_f2(v[1], v[2]);
    }
    // COG_MODE1: the mixture component this record mirrors
    __device__ __forceinline__ int top() const {
        return Store<T>::bytes == 4 ? (int)(u4get(u[NV - 1], 3) & 0xffu) : (int)((u[0].w >> 16) & 0xffu);
    }
    __device__ __forceinline__ void set_top(int k) {
        if (Store<T>::bytes == 4) u4set(u[NV - 1], 3, (uint32_t)k);
        else u[0].w = (u[0].w & 0x0000ffffu) | ((uint32_t)k << 16);
    }
};

template <typename T, int K>
__device__ __forceinline__ float rec_elem(const uint4 *u, int e)
{
    if (Store<T>::bytes == 4) return Store<T>::unbits(u4get(u[e >> 2], e & 3));
    uint32_t w = u4get(u[e >> 3], (e >> 1) & 3);
    return Store<T>::unbits((e & 1) ? (w >> 16) : (w & 0xffffu));
}

template <typename T, int K>
__device__ __forceinline__ void rec_load(const uint8_t *gmm, int64_t p, Mix<K> &m)
{
    constexpr int NV = Rec<T, K>::NV;
    uint4 u[NV];
    const uint4 *src = reinterpret_cast<const uint4 *>(gmm + p * Rec<T, K>::BYTES);
#pragma unroll
    for (int i = 0; i < NV; i++) u[i] = src[i];
#pragma unroll
    for (int k = 0; k < K; k++) {
        m.w[k] = rec_elem<T, K>(u, 7 * k);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m.mu[k][c] = rec_elem<T, K>(u, 7 * k + 1 + c);
            m.v[k][c] = rec_elem<T, K>(u, 7 * k + 4 + c);
        }
    }
}

template <typename T, int K>
__device__ __forceinline__ void rec_store(uint8_t *gmm, int64_t p, const Mix<K> &m)
{
    constexpr int NV = Rec<T, K>::NV;
    constexpr int NE = Rec<T, K>::NE;
    uint4 u[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) u[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int e = 0; e < NE; e++) {
        const int k = e / 7, f = e % 7;
        const float x = f == 0 ? m.w[k] : (f < 4 ? m.mu[k][f - 1] : m.v[k][f - 4]);
        const uint32_t b = Store<T>::bits(x);
        if (Store<T>::bytes == 4) {
            u4set(u[e >> 2], e & 3, b);
        } else {
            uint32_t w = u4get(u[e >> 3], (e >> 1) & 3);
            w |= (e & 1) ? (b << 16) : b;
            u4set(u[e >> 3], (e >> 1) & 3, w);
        }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(gmm + p * Rec<T, K>::BYTES);
#pragma unroll
    for (int i = 0; i < NV; i++) dst[i] = u[i];
}

__device__ __forceinline__ float clampf(float x, float lo, float hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

// ----------------------------------------------------- Eq. 2 mixture step
// Ordered Gaussians (Stauffer-Grimson with diagonal covariance):
//   rank key w^2 / mean variance, descending, ties to the lower index;
//   match = first component in rank order with max_c (I-mu)^2/(lam^2 v) < 1;
//   background iff a match exists and the weight ranked before it is <= T
//   (decided on the state before the update);
//   update at rate a (rho = a): weights (1-a) w + a [k = match], the matched
//   mean and variance move toward I; with no match the lowest-ranked
//   component restarts at (I, var_init, w_init); weights renormalised.
struct MixOut {
    int match;   // matched component or -1
    int tgt;     // matched or restarted component
    int fg;      // 1 = foreground
    float tm;    // match statistic of the matched component (pre-update)
};

// Eq. 2 arithmetic with every rounding written out, so that every kernel
// that runs the mixture step (per frame, packed or not, clip, batch, plain
// mixture, warm-up) rounds identically whatever the compiler would fuse.
// A channel matches when (I - mu)^2 < lambda^2 v.
__device__ __forceinline__ bool eq2_chan_match(float I, float mu, float v, float lam2)
{
    const float d = __fsub_rn(I, mu);
    return __fmul_rn(d, d) < __fmul_rn(lam2, v);
}
// (I - mu)^2 / (lambda^2 v), the match statistic
__device__ __forceinline__ float eq2_chan_stat(float I, float mu, float v, float lam2)
{
    const float d = __fsub_rn(I, mu);
    return __fdividef(__fmul_rn(d, d), __fmul_rn(lam2, v));
}
// matched component: mu <- mu + a (I - mu), v <- (1 - a) v + a (I - mu_new)^2
__device__ __forceinline__ void eq2_chan_update(float I, float a, float b, float &mu, float &v, const DevParams &dp)
{
    mu = __fmaf_rn(a, __fsub_rn(I, mu), mu);
    const float d = __fsub_rn(I, mu);
    v = clampf(__fmaf_rn(__fmul_rn(a, d), d, __fmul_rn(b, v)), dp.var_min, dp.var_max);
}
// rank key parts: w^2 and v0 + v1 + v2
__device__ __forceinline__ float eq2_wsq(float w) { return __fmul_rn(w, w); }
__device__ __forceinline__ float eq2_vsum(float v0, float v1, float v2) { return __fadd_rn(__fadd_rn(v0, v1), v2); }
// j ranks before k
__device__ __forceinline__ bool eq2_before(float wsq_j, float vs_j, float wsq_k, float vs_k, bool j_lower)
{
    const float x = __fmul_rn(wsq_j, vs_k), y = __fmul_rn(wsq_k, vs_j);
    return x > y || (x == y && j_lower);
}

// The confidence-driven rate alpha (1.5 - C-) and the confidence update
// C <- (1 - eta) C- + eta c_inst (Sec. 2, "Confidence Measure"), rounded
// the same way everywhere.
__device__ __forceinline__ float rate_eff(const DevParams &dp, float Cm)
{
    return __fmul_rn(dp.alpha, __fsub_rn(1.5f, Cm));
}
__device__ __forceinline__ float conf_next(const DevParams &dp, float Cm, float ci)
{
    return __fmaf_rn(__fsub_rn(1.f, dp.eta), Cm, __fmul_rn(dp.eta, ci));
}

// Bounds check of the COG_DEBUG build: true when i < n.  A failure sets
// DERR_BOUNDS, the first one records its site, index and limit, and the
// caller skips the access.  Other builds compile every check to true.
#ifdef COG_DEBUG
static __device__ __noinline__ bool dbg_fail(uint32_t *ctl, uint64_t i, uint64_t n, uint32_t site)
{
    if (atomicCAS(ctl + CTL_DBG_WORD, 0u, site) == 0u) {
        ctl[CTL_DBG_WORD + 1] = (uint32_t)i;
        ctl[CTL_DBG_WORD + 2] = (uint32_t)(i >> 32);
        ctl[CTL_DBG_WORD + 3] = (uint32_t)n;
        ctl[CTL_DBG_WORD + 4] = (uint32_t)(n >> 32);
    }
    atomicOr(ctl + CTL_ERR_WORD, DERR_BOUNDS);
    return false;
}
__device__ __forceinline__ bool in_bounds(uint32_t *ctl, uint64_t i, uint64_t n, uint32_t site)
{
    return i < n || dbg_fail(ctl, i, n, site);
}
#else
__device__ __forceinline__ constexpr bool in_bounds(uint32_t *, uint64_t, uint64_t, uint32_t) { return true; }
#endif

// The scene prior's level for channel c of pixel p at grey level v, on the
// 0..255 scale the confidence and the nullification test use (Sec. 2,
// "Scene Prior in Background Model"): the stored byte of the 8-bit prior,
// or 17 times the 4-bit level (q / 15 = 17 q / 255), read from the nibble
// the level occupies (even v low, odd v high).
__device__ __forceinline__ uint32_t prior_level(const uint8_t *kde, int64_t p, int c, uint32_t v, bool four_bit)
{
    if (!four_bit) return __ldg(kde + (p * 3 + c) * 256 + v);
    const uint32_t b = __ldg(kde + (p * 3 + c) * 128 + (v >> 1));
    return 17u * ((b >> ((v & 1u) << 2)) & 15u);
}

// Decisions are taken in division-free form: the rank order compares
// w_j^2 (v_k0+v_k1+v_k2) with w_k^2 (v_j0+v_j1+v_j2) (the mean's 1/3
// cancels), and a channel matches when (I-mu)^2 < lam^2 v.  These differ
// from the quotient forms only within rounding of the threshold.
template <int K>
__device__ __forceinline__ void rank_positions_k(const float wsq[K], const float vs[K], int pos[K])
{
#pragma unroll
    for (int k = 0; k < K; k++) {
        int c = 0;
#pragma unroll
        for (int j = 0; j < K; j++) {
            if (j == k) continue;
            c += eq2_before(wsq[j], vs[j], wsq[k], vs[k], j < k);
        }
        pos[k] = c;
    }
}
template <int K>
__device__ __forceinline__ void rank_positions(const Mix<K> &m, int pos[K])
{
    float wsq[K], vs[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        wsq[k] = eq2_wsq(m.w[k]);
        vs[k] = eq2_vsum(m.v[k][0], m.v[k][1], m.v[k][2]);
    }
    rank_positions_k<K>(wsq, vs, pos);
}

template <int K>
__device__ __forceinline__ MixOut mix_step(Mix<K> &m, const float I[3], float a, const DevParams &dp)
{
    int pos[K];
    rank_positions<K>(m, pos);
    MixOut o;
    o.match = -1;
    o.tm = 0.f;
    int mpos = K;
#pragma unroll
    for (int k = 0; k < K; k++) {
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; c++) ok = ok && eq2_chan_match(I[c], m.mu[k][c], m.v[k][c], dp.lam2);
        if (ok && pos[k] < mpos) { mpos = pos[k]; o.match = k; }
    }
    if (o.match >= 0) {
        float S = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (pos[k] < mpos) S = __fadd_rn(S, m.w[k]);
            if (k == o.match) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float t = eq2_chan_stat(I[c], m.mu[k][c], m.v[k][c], dp.lam2);
                    o.tm = t > o.tm ? t : o.tm;
                }
            }
        }
        o.fg = !(S <= dp.T_bg);
    } else {
        o.fg = 1;
    }
    const float b = __fsub_rn(1.f, a);
    if (o.match >= 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            m.w[k] = __fmaf_rn(b, m.w[k], k == o.match ? a : 0.f);
            if (k == o.match) {
#pragma unroll
                for (int c = 0; c < 3; c++) eq2_chan_update(I[c], a, b, m.mu[k][c], m.v[k][c], dp);
            }
        }
        o.tgt = o.match;
    } else {
        o.tgt = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
            m.w[k] = __fmul_rn(b, m.w[k]);
            if (pos[k] == K - 1) {
                o.tgt = k;
                m.w[k] = dp.w_init;
#pragma unroll
                for (int c = 0; c < 3; c++) { m.mu[k][c] = I[c]; m.v[k][c] = dp.var_init; }
            }
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < K; k++) sum = __fadd_rn(sum, m.w[k]);
    const float inv = __frcp_rn(sum);
#pragma unroll
    for (int k = 0; k < K; k++) m.w[k] = __fmul_rn(m.w[k], inv);
    return o;
}

// The same step on a record kept in its stored form (K x 7 values of T in
// 16-byte words, as Rec<T, K>): each value is converted when it is used and
// written back when it changes, so the step needs about half the registers
// of an unpacked mixture.  The arithmetic and its order are those of
// mix_step, so both give the same record.  tgt_mv receives the updated (or
// restarted) target component's means and variances.
template <typename T, int K>
__device__ __forceinline__ void rec_put(uint4 *u, int e, float x)
{
    const uint32_t b = Store<T>::bits(x);
    if (Store<T>::bytes == 4) {
        u4set(u[e >> 2], e & 3, b);
    } else {
        uint32_t w = u4get(u[e >> 3], (e >> 1) & 3);
        w = (e & 1) ? ((w & 0xffffu) | (b << 16)) : ((w & 0xffff0000u) | b);
        u4set(u[e >> 3], (e >> 1) & 3, w);
    }
}

template <typename T, int K>
__device__ __forceinline__ MixOut mix_step_packed(uint4 *u, const float I[3], float a, const DevParams &dp,
                                                  bool illum, float tgt_mv[6])
{
    int pos[K];
    uint32_t okb = 0;
    {
        float wsq[K], vs[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            wsq[k] = eq2_wsq(rec_elem<T, K>(u, 7 * k));
            const float v0 = rec_elem<T, K>(u, 7 * k + 4), v1 = rec_elem<T, K>(u, 7 * k + 5),
                        v2 = rec_elem<T, K>(u, 7 * k + 6);
            vs[k] = eq2_vsum(v0, v1, v2);
            const bool ok = eq2_chan_match(I[0], rec_elem<T, K>(u, 7 * k + 1), v0, dp.lam2) &&
                            eq2_chan_match(I[1], rec_elem<T, K>(u, 7 * k + 2), v1, dp.lam2) &&
                            eq2_chan_match(I[2], rec_elem<T, K>(u, 7 * k + 3), v2, dp.lam2);
            okb |= (uint32_t)ok << k;
        }
        rank_positions_k<K>(wsq, vs, pos);
    }
    MixOut o;
    o.match = -1;
    o.tm = 0.f;
    int mpos = K;
#pragma unroll
    for (int k = 0; k < K; k++)
        if ((okb >> k & 1u) && pos[k] < mpos) { mpos = pos[k]; o.match = k; }
    const int tgt = o.match >= 0 ? o.match : 0;
    int tk = tgt;
    if (o.match < 0) {
#pragma unroll
        for (int k = 0; k < K; k++) if (pos[k] == K - 1) tk = k;
    }
    o.tgt = tk;
    // the target component's means and variances (before the update)
    float mu[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (k == tk) {
#pragma unroll
            for (int c = 0; c < 3; c++) { mu[c] = rec_elem<T, K>(u, 7 * k + 1 + c); v[c] = rec_elem<T, K>(u, 7 * k + 4 + c); }
        }
    }
    const float b = __fsub_rn(1.f, a);
    float w[K];
    if (o.match >= 0) {
        float S = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const float wk = rec_elem<T, K>(u, 7 * k);
            if (pos[k] < mpos) S = __fadd_rn(S, wk);
            w[k] = __fmaf_rn(b, wk, k == o.match ? a : 0.f);
        }
        o.fg = !(S <= dp.T_bg);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float t = eq2_chan_stat(I[c], mu[c], v[c], dp.lam2);
            o.tm = t > o.tm ? t : o.tm;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) eq2_chan_update(I[c], a, b, mu[c], v[c], dp);
    } else {
        // the lowest-ranked component restarts (every component at the last
        // rank position, as mix_step, should rounding ever tie two there)
        o.fg = 1;
        bool rep = false;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const bool r = pos[k] == K - 1;
            w[k] = r ? dp.w_init : __fmul_rn(b, rec_elem<T, K>(u, 7 * k));
            rep = rep || (k == tk && r);
        }
        if (rep) {
#pragma unroll
            for (int c = 0; c < 3; c++) { mu[c] = I[c]; v[c] = dp.var_init; }
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < K; k++) sum = __fadd_rn(sum, w[k]);
    const float inv = __frcp_rn(sum);
#pragma unroll
    for (int k = 0; k < K; k++) w[k] = __fmul_rn(w[k], inv);
    if (illum && o.fg) {
        // the illumination response (illum_response) on the weights before
        // they are rounded to the stored type, as the unpacked path does
        float so = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) if (k != tk) so = __fadd_rn(so, w[k]);
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (so > 0.f) w[k] = (k == tk) ? dp.w_illum : __fdiv_rn(__fmul_rn(w[k], 1.f - dp.w_illum), so);
            else if (k == tk) w[k] = 1.f;
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
        rec_put<T, K>(u, 7 * k, w[k]);
        if (k == tk || (o.match < 0 && pos[k] == K - 1)) {
#pragma unroll
            for (int c = 0; c < 3; c++) { rec_put<T, K>(u, 7 * k + 1 + c, mu[c]); rec_put<T, K>(u, 7 * k + 4 + c, v[c]); }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) { tgt_mv[c] = mu[c]; tgt_mv[3 + c] = v[c]; }
    return o;
}

// --------------------------------------- per-channel mixtures (COG_PERCHAN)
// Each channel has its own K one-dimensional components with their own
// weights.  Record: per component (w0 w1 w2 mu0 mu1 mu2 v0 v1 v2), padded to
// a 16-byte multiple.
template <typename T, int K> struct RecPC {
    static constexpr int NE = 9 * K;
    static constexpr int NV = (NE * Store<T>::bytes + 15) / 16;
    static constexpr int BYTES = NV * 16;
};

template <int K> struct MixPC {
    float w[3][K], mu[3][K], v[3][K];
};

struct MixOutPC {
    int fg;          // 1 = some channel is foreground (the pixel label)
    int fg_c[3];     // per channel
    int tgt[3];      // per channel: matched or restarted component
    float Mhat;      // largest per-channel match statistic (1 if unmatched)
};

template <typename T, int K>
__device__ __forceinline__ void mixpc_unpack(const uint4 *u, MixPC<K> &m)
{
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m.w[c][k] = rec_elem<T, K>(u, 9 * k + c);
            m.mu[c][k] = rec_elem<T, K>(u, 9 * k + 3 + c);
            m.v[c][k] = rec_elem<T, K>(u, 9 * k + 6 + c);
        }
    }
}

template <typename T, int K>
__device__ __forceinline__ void mixpc_pack(const MixPC<K> &m, uint4 *u)
{
    constexpr int NV = RecPC<T, K>::NV;
    constexpr int NE = RecPC<T, K>::NE;
#pragma unroll
    for (int i = 0; i < NV; i++) u[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int e = 0; e < NE; e++) {
        const int k = e / 9, f = e % 9, c = f % 3;
        const float x = f < 3 ? m.w[c][k] : (f < 6 ? m.mu[c][k] : m.v[c][k]);
        const uint32_t b = Store<T>::bits(x);
        if (Store<T>::bytes == 4) {
            u4set(u[e >> 2], e & 3, b);
        } else {
            uint32_t w = u4get(u[e >> 3], (e >> 1) & 3);
            w |= (e & 1) ? (b << 16) : b;
            u4set(u[e >> 3], (e >> 1) & 3, w);
        }
    }
}

// One channel's step of Eq. 2 on its own 1-D mixture, with the same
// decisions and arithmetic as mix_step: rank by w^2 / v (cross-multiplied,
// ties to the lower index), first match in rank order, background iff the
// weight ranked before it is <= T, update at rate a, restart the
// lowest-ranked component on no match, renormalise.
template <int K>
__device__ __forceinline__ void mix_step_channel(float (&w)[K], float (&mu)[K], float (&v)[K], float I, float a,
                                                 const DevParams &dp, int &fg, int &tgt, float &M)
{
    int pos[K];
    float wsq[K];
#pragma unroll
    for (int k = 0; k < K; k++) wsq[k] = eq2_wsq(w[k]);
#pragma unroll
    for (int k = 0; k < K; k++) {
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < K; j++) {
            if (j == k) continue;
            cnt += eq2_before(wsq[j], v[j], wsq[k], v[k], j < k);
        }
        pos[k] = cnt;
    }
    int match = -1, mpos = K;
#pragma unroll
    for (int k = 0; k < K; k++)
        if (eq2_chan_match(I, mu[k], v[k], dp.lam2) && pos[k] < mpos) { mpos = pos[k]; match = k; }
    float tm = 0.f;
    fg = 1;
    if (match >= 0) {
        float S = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (pos[k] < mpos) S = __fadd_rn(S, w[k]);
            if (k == match) tm = eq2_chan_stat(I, mu[k], v[k], dp.lam2);
        }
        fg = !(S <= dp.T_bg);
    }
    M = match >= 0 ? (tm < 1.f ? tm : 1.f) : 1.f;
    const float b = __fsub_rn(1.f, a);
    if (match >= 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            w[k] = __fmaf_rn(b, w[k], k == match ? a : 0.f);
            if (k == match) eq2_chan_update(I, a, b, mu[k], v[k], dp);
        }
        tgt = match;
    } else {
        tgt = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
            w[k] = __fmul_rn(b, w[k]);
            if (pos[k] == K - 1) {
                tgt = k;
                w[k] = dp.w_init;
                mu[k] = I;
                v[k] = dp.var_init;
            }
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < K; k++) sum = __fadd_rn(sum, w[k]);
    const float inv = __frcp_rn(sum);
#pragma unroll
    for (int k = 0; k < K; k++) w[k] = __fmul_rn(w[k], inv);
}

template <int K>
__device__ __forceinline__ MixOutPC mix_step_pc(MixPC<K> &m, const float I[3], float a, const DevParams &dp)
{
    MixOutPC o;
    o.fg = 0;
    o.Mhat = 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float M;
        mix_step_channel<K>(m.w[c], m.mu[c], m.v[c], I[c], a, dp, o.fg_c[c], o.tgt[c], M);
        o.fg |= o.fg_c[c];
        o.Mhat = M > o.Mhat ? M : o.Mhat;
    }
    return o;
}

// Abrupt illumination change with per-channel mixtures: every channel that
// decided foreground gives its matched or new component the weight w_illum.
template <int K>
__device__ __forceinline__ void illum_response_pc(MixPC<K> &m, const MixOutPC &o, float w_illum)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (!o.fg_c[c]) continue;
        float so = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) if (k != o.tgt[c]) so = __fadd_rn(so, m.w[c][k]);
        if (so > 0.f) {
#pragma unroll
            for (int k = 0; k < K; k++)
                m.w[c][k] = (k == o.tgt[c]) ? w_illum : __fdiv_rn(__fmul_rn(m.w[c][k], 1.f - w_illum), so);
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) if (k == o.tgt[c]) m.w[c][k] = 1.f;
        }
    }
}

// Transition update with per-channel mixtures: each channel's stage-1
// values take that channel's target component.
template <typename T, int K>
__device__ __forceinline__ void s1_reseed_pc(const MixPC<K> &m, const MixOutPC &o, uint32_t qab, S1Rec<T> &r)
{
#pragma unroll
    for (int i = 0; i < S1Rec<T>::NV; i++) r.u[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            if (k == o.tgt[c]) { r.set(c, m.mu[c][k]); r.set(3 + c, m.v[c][k]); }
        }
    }
    r.set_qab(qab);
}

// COG_MODE1 (the Fig. 1 reading: stage 1 is the mixture's rank-1 mode).
// On the transition to stage 2 the stage-1 copy is written back into the
// component it mirrors; after the update the copy follows the component
// that now ranks first (ties to the lower index), whatever the label.
template <typename T, int K>
__device__ __forceinline__ void mode1_write_back(Mix<K> &m, const S1Rec<T> &r)
{
    const int k1 = r.top();
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (k == k1) {
#pragma unroll
            for (int c = 0; c < 3; c++) { m.mu[k][c] = r.get(c); m.v[k][c] = r.get(3 + c); }
        }
    }
}
template <typename T, int K>
__device__ __forceinline__ void mode1_recache(const Mix<K> &m, S1Rec<T> &r)
{
    int pos[K];
    rank_positions<K>(m, pos);
#pragma unroll
    for (int k = 0; k < K; k++) {
        if (pos[k] == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) { r.set(c, m.mu[k][c]); r.set(3 + c, m.v[k][c]); }
            r.set_top(k);
        }
    }
}

// Abrupt illumination change (Sec. 2, end of "Cascade of Gaussians"): the
// foreground decision becomes background, the matched or new mode takes
// weight w_illum and the others share the rest in proportion.
template <int K>
__device__ __forceinline__ void illum_response(Mix<K> &m, int tgt, float w_illum)
{
    float so = 0.f;
#pragma unroll
    for (int k = 0; k < K; k++) if (k != tgt) so = __fadd_rn(so, m.w[k]);
    if (so > 0.f) {
#pragma unroll
        for (int k = 0; k < K; k++)
            m.w[k] = (k == tgt) ? w_illum : __fdiv_rn(__fmul_rn(m.w[k], 1.f - w_illum), so);
    } else {
#pragma unroll
        for (int k = 0; k < K; k++) if (k == tgt) m.w[k] = 1.f;
    }
}

// ------------------------------------------------------------ bulk copies
// One-shot TMA bulk copy global -> shared completing on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Programmatic dependent launch controls (no-ops for a normally launched
// grid): allow the next grid on the stream to be scheduled, and wait until
// the preceding grid has completed and its memory is visible.
__device__ __forceinline__ void grid_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_wait_prior()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// shared -> global bulk copy (bulk-group completion)
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Asynchronous copies global -> shared (cp.async), completed per thread by
// commit groups: 16 bytes through L2 only, or 4 bytes.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's commit groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bounded wait on phase `parity`; returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok = 0;
    for (uint32_t it = 0; it < (1u << 22) && !ok; it++) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return ok != 0;
}

}  // namespace cog
