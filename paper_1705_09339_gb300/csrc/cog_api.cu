// cog_api.cu -- host side of the C ABI declared in include/cog.h: parameter
// validation, the state layout, context lifetime, stream-ordered launches,
// sticky error reporting, statistics and state export/import.
#include <sys/mman.h>
#include <unistd.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "cog_internal.h"

namespace cog {
cudaError_t launch_apply_f32(int, const ApplyArgs &, const LaunchCfg &, cudaStream_t, const ApplyEvents *);
cudaError_t launch_apply_f16(int, const ApplyArgs &, const LaunchCfg &, cudaStream_t, const ApplyEvents *);
cudaError_t launch_apply_bf16(int, const ApplyArgs &, const LaunchCfg &, cudaStream_t, const ApplyEvents *);
cudaError_t launch_plain_f32(int, const DevParams &, const StatePtrs &, const uint8_t *, uint8_t *, cudaStream_t);
cudaError_t launch_plain_f16(int, const DevParams &, const StatePtrs &, const uint8_t *, uint8_t *, cudaStream_t);
cudaError_t launch_plain_bf16(int, const DevParams &, const StatePtrs &, const uint8_t *, uint8_t *, cudaStream_t);
cudaError_t launch_warmup_f32(int, const DevParams &, const StatePtrs &, const uint8_t *, int, int, int, cudaStream_t);
cudaError_t launch_warmup_f16(int, const DevParams &, const StatePtrs &, const uint8_t *, int, int, int, cudaStream_t);
cudaError_t launch_warmup_bf16(int, const DevParams &, const StatePtrs &, const uint8_t *, int, int, int, cudaStream_t);

cudaError_t launch_batch_f32(int, const BatchGroupDev &, const LaunchCfg &, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_batch_f16(int, const BatchGroupDev &, const LaunchCfg &, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_batch_bf16(int, const BatchGroupDev &, const LaunchCfg &, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_clip_f32(int, const ClipArgs &, int, cudaStream_t);
cudaError_t launch_clip_f16(int, const ClipArgs &, int, cudaStream_t);
cudaError_t launch_clip_bf16(int, const ClipArgs &, int, cudaStream_t);
cudaError_t run_wait_selftest(uint64_t limit_ns, uint32_t *error_word, float *elapsed_ms);
cudaError_t launch_group(int dtype, int K, const DevParams &dp, const StatePtrs &s, const uint8_t *frames, int N,
                         uint16_t *codes, uint8_t *labels, int max_steps, int n_sm, cudaStream_t st);
int group_max_steps();
size_t group_ctl_offset();
size_t group_ctl_bytes();
void group_ctl_decode(const void *raw, int max_steps, cog_group_stats *out);
cudaError_t launch_probe_stream(const uint32_t *jl_in, const uint16_t *conf_in, const uint8_t *frame,
                                uint32_t *jl_out, uint16_t *conf_out, uint8_t *mask, int64_t P, cudaStream_t st);
int k1_batch_blocks_per_sm_f32(const LaunchCfg &);
int k1_batch_blocks_per_sm_f16(const LaunchCfg &);
int k1_batch_blocks_per_sm_bf16(const LaunchCfg &);
int k2_blocks_per_sm_f32(int, const LaunchCfg &, int);
int k2_blocks_per_sm_f16(int, const LaunchCfg &, int);
int k2_blocks_per_sm_bf16(int, const LaunchCfg &, int);

int elem_bytes(int dtype) { return dtype == COG_F32 ? 4 : 2; }

int rec_bytes(int dtype, int K, bool perchan)
{
    return (K * (perchan ? 9 : 7) * elem_bytes(dtype) + 15) / 16 * 16;
}

int s1_bytes(int dtype) { return dtype == COG_F32 ? 32 : 16; }

static size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool make_layout(const cog_params &p, Layout &L)
{
    L.P = (int64_t)p.width * p.height;
    L.Pp = (int64_t)up((size_t)L.P, PX_ALIGN);
    L.elem = (size_t)elem_bytes(p.state_dtype);
    L.rec_bytes = (size_t)rec_bytes(p.state_dtype, p.K, (p.flags & COG_PERCHAN) != 0);
    L.s1_bytes = (size_t)s1_bytes(p.state_dtype);
    size_t o = 0;
    L.ctl = o;  o += CTL_BYTES;
    L.jl = o;   o = up(o + (size_t)L.Pp * 4, 256);
    L.conf = o; o = up(o + (size_t)L.Pp * L.elem, 256);
    L.s1 = o;   o = up(o + (size_t)L.Pp * L.s1_bytes, 256);
    L.gmm = o;  o = up(o + (size_t)L.Pp * L.rec_bytes, 256);
    const int64_t ctas = (L.P + K1_TILE - 1) / K1_TILE;
    L.qseg_cap = (ctas + QSEG - 1) / QSEG * K1_TILE;
    L.queue = o; o = up(o + (size_t)(QSEG * L.qseg_cap) * 16, 256);
    L.kde_row = p.kde_bits == 4 ? 128 : 256;
    L.kde = o;  o = up(o + (size_t)L.P * 3 * L.kde_row, 256);
    L.total = o;
    return true;
}

}  // namespace cog

using namespace cog;

struct cog_ctx {
    cog_params p;
    Layout L;
    DevParams dp;
    StatePtrs sp;
    cudaStream_t stream;
    int device;
    uint8_t *state;
    bool owns;
    bool trained;
    int64_t frame_no;
    cog_status sticky;
    char err[512];
    uint8_t *stage_in, *stage_out;   // cog_apply_host staging buffers
    int n_sm;                        // multiprocessors of the device
    LaunchCfg launch;                // kernel launch shape (cog_set_launch)
    std::vector<ApplyEvents> prof;   // per-frame kernel timing events (profiling on)
    int64_t prof_n;                  // frames recorded since profiling was enabled
    uint8_t *clip_mem;               // cog_apply_clip scratch (allocated on first use)
    size_t clip_bytes;
    // cog_apply_host_frames pipeline (created on first use): two frame and
    // two mask slots, an upload and a download stream, and per-slot events
    uint8_t *pipe_mem;
    cudaStream_t pipe_in, pipe_out;
    cudaEvent_t ev_in[2], ev_done[2], ev_out[2];
};

namespace cog {
int64_t ctx_pixels(const cog_ctx *c) { return c ? c->L.P : 0; }
}  // namespace cog

static thread_local char g_create_err[512];

static cog_status set_err(cog_ctx *c, cog_status s, const char *fmt, ...)
{
    char *dst = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return s;
}

static cog_status cuda_fail(cog_ctx *c, cudaError_t e, const char *where)
{
    set_err(c, COG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    if (c) c->sticky = COG_ERR_CUDA;
    return COG_ERR_CUDA;
}

static const char *check_params(const cog_params *p)
{
    if (!p) return "params is NULL";
    if (p->width < 1 || p->height < 1) return "width and height must be >= 1";
    if ((int64_t)p->width * p->height > (int64_t)1 << 28) return "frame larger than 2^28 pixels";
    if (p->K < 1 || p->K > KMAX) return "K must be in 1..8";
    if (p->state_dtype < COG_F32 || p->state_dtype > COG_BF16) return "unknown state_dtype";
    if (!(p->alpha > 0.f && p->alpha <= 1.f)) return "alpha must be in (0, 1]";
    if (!(p->lambda > 0.f)) return "lambda must be > 0";
    if (!(p->T_bg >= 0.f && p->T_bg <= 1.f)) return "T_bg must be in [0, 1]";
    if (!(p->w_init > 0.f && p->w_init <= 1.f)) return "w_init must be in (0, 1]";
    if (!(p->var_min > 0.f) || !(p->var_max >= p->var_min)) return "need 0 < var_min <= var_max";
    if (!(p->var_init > 0.f)) return "var_init must be > 0";
    if (!(p->tau_fd >= 0.f)) return "tau_fd must be >= 0";
    if (!(p->eta_conf >= 0.f && p->eta_conf <= 1.f)) return "eta_conf must be in [0, 1]";
    if (!(p->w_illum > 0.f && p->w_illum < 1.f)) return "w_illum must be in (0, 1)";
    if (p->q_null < 0 || p->q_null > 256) return "q_null must be in 0..256";
    if (p->kde_bw < 1 || p->kde_bw > 32) return "kde_bw must be in 1..32";
    if (p->kde_bits != 8 && p->kde_bits != 4) return "kde_bits must be 8 or 4";
    if (p->r1 < 0 || p->r2 < p->r1) return "need 0 <= r1 <= r2";
    if (p->illum_permille < 0 || p->illum_permille > 1000) return "illum_permille must be in 0..1000";
    if (p->flags & ~(COG_ALL | COG_SAMPLE | COG_MODE1 | COG_PERCHAN)) return "unknown flag bits";
    if ((p->flags & COG_PERCHAN) && (p->flags & COG_MODE1)) return "COG_PERCHAN and COG_MODE1 do not combine";
    if (p->skip_period < 1) return "skip_period must be >= 1";
    return nullptr;
}

extern "C" {

void cog_default_params(cog_params *p, int32_t width, int32_t height, int32_t K)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->width = width;
    p->height = height;
    p->K = K;
    p->state_dtype = COG_F32;
    p->alpha = 0.01f;
    p->lambda = 2.5f;
    p->T_bg = 0.7f;
    p->w_init = 0.05f;
    p->var_init = 225.f;
    p->var_min = 4.f;
    p->var_max = 900.f;
    p->tau_fd = 8.f;
    p->eta_conf = 0.125f;
    p->c_halt = 0.9f;
    p->w_illum = 0.75f;
    p->q_null = 13;
    p->kde_bw = 4;
    p->r1 = 10;
    p->r2 = 30;
    p->illum_permille = 700;
    p->flags = COG_ALL;
    p->c_skip = 0.95f;
    p->skip_period = 4;
    p->kde_bits = 8;
}

cog_status cog_state_layout(const cog_params *p, cog_layout *out)
{
    if (const char *m = check_params(p)) return set_err(nullptr, COG_ERR_INVALID_ARG, "%s", m);
    if (!out) return set_err(nullptr, COG_ERR_INVALID_ARG, "out is NULL");
    Layout L;
    make_layout(*p, L);
    out->total = L.total; out->ctl = L.ctl; out->jl = L.jl; out->conf = L.conf; out->s1 = L.s1;
    out->s1_bytes = L.s1_bytes; out->gmm = L.gmm; out->rec_bytes = L.rec_bytes; out->queue = L.queue;
    out->kde = L.kde; out->elem_bytes = L.elem; out->kde_row = L.kde_row;
    return COG_OK;
}

cog_status cog_state_bytes(const cog_params *p, size_t *out)
{
    cog_layout l;
    cog_status s = cog_state_layout(p, &l);
    if (s != COG_OK) return s;
    if (!out) return set_err(nullptr, COG_ERR_INVALID_ARG, "out is NULL");
    *out = (size_t)l.total;
    return COG_OK;
}

cog_status cog_create(const cog_params *p, void *cuda_stream, void *state_dev, cog_ctx **out)
{
    if (!out) return set_err(nullptr, COG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (const char *m = check_params(p)) return set_err(nullptr, COG_ERR_INVALID_ARG, "%s", m);
    if (state_dev && ((uintptr_t)state_dev & 255))
        return set_err(nullptr, COG_ERR_INVALID_ARG, "state buffer must be 256-byte aligned");
    cog_ctx *c = new (std::nothrow) cog_ctx();
    if (!c) return set_err(nullptr, COG_ERR_OOM, "host allocation failed");
    c->p = *p;
    make_layout(*p, c->L);
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        set_err(nullptr, COG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        delete c;
        return COG_ERR_CUDA;
    }
    if (state_dev) {
        c->state = (uint8_t *)state_dev;
        c->owns = false;
    } else {
        e = cudaMalloc((void **)&c->state, c->L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_err(nullptr, COG_ERR_OOM, "cudaMalloc of %zu state bytes: %s", c->L.total, cudaGetErrorString(e));
            delete c;
            return COG_ERR_OOM;
        }
        c->owns = true;
    }
    e = cudaMemsetAsync(c->state, 0, c->L.total, c->stream);
    if (e != cudaSuccess) {
        set_err(nullptr, COG_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        if (c->owns) cudaFree(c->state);
        delete c;
        return COG_ERR_CUDA;
    }
    DevParams &d = c->dp;
    d.P = c->L.P;
    d.K = p->K;
    d.flags = p->flags;
    d.alpha = p->alpha;
    d.lam2 = p->lambda * p->lambda;
    d.T_bg = p->T_bg;
    d.w_init = p->w_init;
    d.var_init = p->var_init;
    d.var_min = p->var_min;
    d.var_max = p->var_max;
    d.tau_fd = p->tau_fd;
    d.eta = p->eta_conf;
    d.c_halt = p->c_halt;
    d.w_illum = p->w_illum;
    d.q_null = p->q_null;
    d.illum_permille = p->illum_permille;
    d.c_skip = p->c_skip;
    d.skip_period = p->skip_period;
    d.kde_bits = p->kde_bits;
    StatePtrs &s = c->sp;
    s.ctl = (uint32_t *)(c->state + c->L.ctl);
    s.jl = (uint32_t *)(c->state + c->L.jl);
    s.conf = c->state + c->L.conf;
    s.s1 = c->state + c->L.s1;
    s.gmm = c->state + c->L.gmm;
    s.queue = (uint4 *)(c->state + c->L.queue);
    s.qseg_cap = c->L.qseg_cap;
    s.kde = c->state + c->L.kde;
    c->sticky = COG_OK;
    c->err[0] = 0;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        c->n_sm < 1)
        c->n_sm = 1;
    *out = c;
    return COG_OK;
}

static cog_status check_ctx(cog_ctx *c)
{
    if (!c) return COG_ERR_INVALID_ARG;
    if (c->sticky != COG_OK) return c->sticky;
    return COG_OK;
}

cog_status cog_train_prior(cog_ctx *c, const uint8_t *frames_dev, int32_t n_frames)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!frames_dev) return set_err(c, COG_ERR_INVALID_ARG, "frames_dev is NULL");
    if (n_frames < 2) return set_err(c, COG_ERR_INVALID_ARG, "need at least 2 training frames");
    const int bw = c->p.kde_bw, R = 3 * bw;
    uint32_t g[100];
    uint64_t gsum = 0;
    for (int d = 0; d <= R; d++) {
        g[d] = (uint32_t)std::floor(65536.0 * std::exp(-(double)(d * d) / (2.0 * bw * bw)) + 0.5);
        gsum += (d ? 2u : 1u) * (uint64_t)g[d];
    }
    if ((uint64_t)n_frames * gsum >= (1ull << 32))
        return set_err(c, COG_ERR_INVALID_ARG, "n_frames too large for the exact 32-bit prior (%d)", n_frames);
    cudaError_t e = launch_kde_train(c->dp, c->sp, frames_dev, n_frames, g, R, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "kde_train launch");
    switch (c->p.state_dtype) {
    case COG_F32: e = launch_warmup_f32(c->p.K, c->dp, c->sp, frames_dev, n_frames, c->p.r1, c->p.r2, c->stream); break;
    case COG_F16: e = launch_warmup_f16(c->p.K, c->dp, c->sp, frames_dev, n_frames, c->p.r1, c->p.r2, c->stream); break;
    default: e = launch_warmup_bf16(c->p.K, c->dp, c->sp, frames_dev, n_frames, c->p.r1, c->p.r2, c->stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "warmup launch");
    e = cudaMemsetAsync(c->sp.ctl, 0, CTL_BYTES, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(ctl)");
    c->trained = true;
    c->frame_no = 0;
    return COG_OK;
}

static cog_status read_ctl(cog_ctx *c, std::vector<uint32_t> &ctl)
{
    ctl.assign(CTL_BYTES / 4, 0);
    cudaError_t e = cudaMemcpyAsync(ctl.data(), c->sp.ctl, CTL_BYTES, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the control block");
    if (ctl[CTL_ERR_WORD] & DERR_BOUNDS) {
        c->sticky = COG_ERR_DEVICE;
        const uint32_t *d = ctl.data() + CTL_DBG_WORD;
        return set_err(c, COG_ERR_DEVICE, "device error word 0x%x: bounds check %u failed (index %llu, limit %llu)",
                       ctl[CTL_ERR_WORD], d[0], (unsigned long long)d[1] | (unsigned long long)d[2] << 32,
                       (unsigned long long)d[3] | (unsigned long long)d[4] << 32);
    }
    if (ctl[CTL_ERR_WORD]) {
        c->sticky = COG_ERR_DEVICE;
        return set_err(c, COG_ERR_DEVICE, "device error word 0x%x (a bounded wait gave up)", ctl[CTL_ERR_WORD]);
    }
    return COG_OK;
}

static void frame_stats(const std::vector<uint32_t> &ctl, int64_t frame, cog_stats *st)
{
    memset(st, 0, sizeof *st);
    st->frame = (int32_t)frame;
    if (frame < 0) return;
    for (int f = 0; f < 7; f++) {
        int64_t v = 0;
        for (int s = 0; s < CTL_SLOTS; s++) v += ctl[(size_t)ctl_slot((int)(frame % 3), f, s)];
        if (f < 5) st->n_stage[f] = v;
        else if (f == 5) st->n_gmm = v;
        else st->n_stage[5] = v;
    }
}

static int prev_flag(const cog_ctx *c, const std::vector<uint32_t> &ctl, int64_t frame)
{
    if (!(c->p.flags & COG_ILLUM) || frame < 1) return 0;
    cog_stats prev;
    frame_stats(ctl, frame - 1, &prev);
    return (uint64_t)prev.n_gmm * 1000u > (uint64_t)c->p.illum_permille * (uint64_t)c->L.P;
}

cog_status cog_apply(cog_ctx *c, const uint8_t *frame_dev, uint8_t *mask_dev, uint8_t *stagemap_dev,
                     cog_stats *stats_host)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!c->trained) return set_err(c, COG_ERR_STATE, "cog_apply before cog_train_prior");
    if (!frame_dev || !mask_dev) return set_err(c, COG_ERR_INVALID_ARG, "frame_dev and mask_dev are required");
    ApplyArgs a;
    a.dp = c->dp;
    a.s = c->sp;
    a.frame = frame_dev;
    a.mask = mask_dev;
    a.stagemap = stagemap_dev;
    a.frame_no = (uint32_t)(c->frame_no % 3);
    a.frame_idx = (uint32_t)c->frame_no;
    a.frame_al4 = ((uintptr_t)frame_dev & 3) == 0;
    a.out_al4 = ((uintptr_t)mask_dev & 3) == 0 && ((uintptr_t)stagemap_dev & 3) == 0;
    a.k2_grid = (uint32_t)c->n_sm;
    a.rec_bytes = (uint32_t)c->L.rec_bytes;
    const ApplyEvents *ev = nullptr;
    if (!c->prof.empty() && c->prof_n < (int64_t)c->prof.size()) ev = &c->prof[(size_t)c->prof_n++];
    cudaError_t e;
    switch (c->p.state_dtype) {
    case COG_F32: e = launch_apply_f32(c->p.K, a, c->launch, c->stream, ev); break;
    case COG_F16: e = launch_apply_f16(c->p.K, a, c->launch, c->stream, ev); break;
    default: e = launch_apply_bf16(c->p.K, a, c->launch, c->stream, ev); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply launch");
    c->frame_no++;
    if (stats_host) {
        std::vector<uint32_t> ctl;
        if ((s = read_ctl(c, ctl)) != COG_OK) return s;
        frame_stats(ctl, c->frame_no - 1, stats_host);
        stats_host->illum_flag = prev_flag(c, ctl, c->frame_no - 1);
    }
    return COG_OK;
}

// Scratch of the clip path: per-frame counter banks and sync words, then
// the undo log (clip-start copies of the stage-0/1 planes, original mixture
// records, one touched bit per pixel).
struct ClipScratch {
    size_t cnt, sync, jl, conf, s1, gmm, touched, total;
};
static ClipScratch clip_layout(const Layout &L)
{
    ClipScratch z;
    size_t o = 0;
    z.cnt = o;     o = up(o + (size_t)CLIP_CNT_WORDS * 4, 256);
    z.sync = o;    o = up(o + (size_t)CLIP_SYNC_WORDS * 4, 256);
    z.jl = o;      o = up(o + (size_t)L.Pp * 4, 256);
    z.conf = o;    o = up(o + (size_t)L.Pp * L.elem, 256);
    z.s1 = o;      o = up(o + (size_t)L.Pp * L.s1_bytes, 256);
    z.gmm = o;     o = up(o + (size_t)L.Pp * L.rec_bytes, 256);
    z.touched = o; o = up(o + (size_t)L.Pp / 8, 256);
    z.total = o;
    return z;
}

cog_status cog_apply_clip(cog_ctx *c, const uint8_t *frames_dev, int32_t n_frames, uint8_t *masks_dev,
                          uint8_t *stagemaps_dev, cog_stats *stats_host)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!c->trained) return set_err(c, COG_ERR_STATE, "cog_apply_clip before cog_train_prior");
    if (!frames_dev || !masks_dev) return set_err(c, COG_ERR_INVALID_ARG, "frames_dev and masks_dev are required");
    if (n_frames < 1) return set_err(c, COG_ERR_INVALID_ARG, "n_frames must be >= 1");
    const ClipScratch z = clip_layout(c->L);
    cudaError_t e;
    if (!c->clip_mem) {
        e = cudaMalloc((void **)&c->clip_mem, z.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->clip_mem = nullptr;
            return set_err(c, COG_ERR_OOM, "cudaMalloc of %zu clip scratch bytes: %s", z.total, cudaGetErrorString(e));
        }
        c->clip_bytes = z.total;
    }
    const int64_t P = c->L.P;
    ClipArgs a;
    memset(&a, 0, sizeof a);
    a.dp = c->dp;
    a.s = c->sp;
    a.undo_jl = (uint32_t *)(c->clip_mem + z.jl);
    a.undo_conf = c->clip_mem + z.conf;
    a.undo_s1 = c->clip_mem + z.s1;
    a.undo_gmm = c->clip_mem + z.gmm;
    a.touched = (uint32_t *)(c->clip_mem + z.touched);
    a.cnt = (uint32_t *)(c->clip_mem + z.cnt);
    a.sync = (uint32_t *)(c->clip_mem + z.sync);
    a.frame_al4 = ((uintptr_t)frames_dev & 3) == 0 && (P & 3) == 0;
    a.out_al4 = ((uintptr_t)masks_dev & 3) == 0 && ((uintptr_t)stagemaps_dev & 3) == 0 && (P & 3) == 0;
    for (int32_t f0 = 0; f0 < n_frames; f0 += CLIP_TMAX) {
        const int32_t T = n_frames - f0 < CLIP_TMAX ? n_frames - f0 : CLIP_TMAX;
        a.frames = frames_dev + (int64_t)f0 * P * 3;
        a.masks = masks_dev + (int64_t)f0 * P;
        a.stagemaps = stagemaps_dev ? stagemaps_dev + (int64_t)f0 * P : nullptr;
        a.T = (uint32_t)T;
        a.frame_idx0 = (uint32_t)c->frame_no;
        a.frame_mod3 = (uint32_t)(c->frame_no % 3);
        e = cudaMemsetAsync(c->clip_mem, 0, z.jl, c->stream);   // counter banks and sync words
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(clip counters)");
        switch (c->p.state_dtype) {
        case COG_F32: e = launch_clip_f32(c->p.K, a, c->n_sm, c->stream); break;
        case COG_F16: e = launch_clip_f16(c->p.K, a, c->n_sm, c->stream); break;
        default: e = launch_clip_bf16(c->p.K, a, c->n_sm, c->stream); break;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_clip launch");
        const int64_t first = c->frame_no;
        c->frame_no += T;
        if (stats_host) {
            std::vector<uint32_t> cnt(CLIP_CNT_WORDS), sync(CLIP_SYNC_WORDS);
            e = cudaMemcpyAsync(cnt.data(), a.cnt, cnt.size() * 4, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sync.data(), a.sync, sync.size() * 4, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "reading the clip counters");
            std::vector<uint32_t> ctl;
            if ((s = read_ctl(c, ctl)) != COG_OK) return s;
            const int bank = (int)sync[CLIP_RUNS_WORD + 1];
            const uint32_t flags = sync[CLIP_RUNS_WORD + 2];
            for (int t = 0; t < T; t++) {
                cog_stats &st = stats_host[f0 + t];
                memset(&st, 0, sizeof st);
                st.frame = (int32_t)(first + t);
                for (int f = 0; f < 7; f++) {
                    int64_t v = 0;
                    for (int q = 0; q < CLIP_SLOTS; q++) v += cnt[(size_t)clip_cnt_word(bank, t, f, q)];
                    if (f < 5) st.n_stage[f] = v;
                    else if (f == 5) st.n_gmm = v;
                    else st.n_stage[5] = v;
                }
                st.illum_flag = (int32_t)((flags >> t) & 1u);
            }
        }
    }
    return COG_OK;
}

cog_status cog_clip_runs(cog_ctx *c, int32_t *runs)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!runs) return set_err(c, COG_ERR_INVALID_ARG, "runs is NULL");
    *runs = 0;
    if (!c->clip_mem) return COG_OK;
    const ClipScratch z = clip_layout(c->L);
    uint32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->clip_mem + z.sync + CLIP_RUNS_WORD * 4, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_clip_runs");
    *runs = (int32_t)v;
    return COG_OK;
}

cog_status cog_selftest_bounded_wait(int32_t limit_ms, uint32_t *error_word, double *elapsed_ms)
{
    if (limit_ms < 1 || limit_ms > 2000 || !error_word || !elapsed_ms)
        return set_err(nullptr, COG_ERR_INVALID_ARG, "limit_ms must be in 1..2000 and the outputs non-NULL");
    float ms = 0.f;
    *error_word = 0;
    cudaError_t e = run_wait_selftest((uint64_t)limit_ms * 1000000ull, error_word, &ms);
    if (e != cudaSuccess) return set_err(nullptr, COG_ERR_CUDA, "bounded-wait self-test: %s", cudaGetErrorString(e));
    *elapsed_ms = ms;
    return COG_OK;
}

namespace {
// Shared by cog_group (frames given: features first) and cog_group_cluster
// (the caller's codes).
cog_status group_run(cog_ctx *c, const uint8_t *frames_dev, int32_t n_frames, uint16_t *codes_dev, int32_t max_steps,
                     uint8_t *labels_dev, cog_group_stats *stats_host)
{
    cudaError_t e = launch_group(c->p.state_dtype, c->p.K, c->dp, c->sp, frames_dev, n_frames, codes_dev, labels_dev,
                                 max_steps, c->n_sm, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "grouping launch");
    std::vector<unsigned char> raw(group_ctl_bytes());
    e = cudaMemcpyAsync(raw.data(), reinterpret_cast<const unsigned char *>(c->sp.ctl) + group_ctl_offset(), raw.size(),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "grouping result");
    group_ctl_decode(raw.data(), max_steps, stats_host);
    return COG_OK;
}

cog_status group_check(cog_ctx *c, const uint16_t *codes_dev, const uint8_t *labels_dev, const cog_group_stats *st)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!c->trained) return set_err(c, COG_ERR_STATE, "grouping before cog_train_prior");
    if (c->p.flags & COG_PERCHAN)
        return set_err(c, COG_ERR_INVALID_ARG, "grouping uses the shared-weight mixture; not defined with COG_PERCHAN");
    if (!codes_dev || !labels_dev || !st)
        return set_err(c, COG_ERR_INVALID_ARG, "codes_dev, labels_dev and stats_host are required");
    if (reinterpret_cast<uintptr_t>(codes_dev) & 1u) return set_err(c, COG_ERR_INVALID_ARG, "codes_dev must be 2-byte aligned");
    if (c->L.P >= (int64_t)1 << 30) return set_err(c, COG_ERR_INVALID_ARG, "grouping needs fewer than 2^30 pixels");
    return COG_OK;
}
}  // namespace

cog_status cog_group(cog_ctx *c, const uint8_t *frames_dev, int32_t n_frames, uint16_t *codes_dev,
                     uint8_t *labels_dev, cog_group_stats *stats_host)
{
    cog_status s = group_check(c, codes_dev, labels_dev, stats_host);
    if (s) return s;
    if (!frames_dev) return set_err(c, COG_ERR_INVALID_ARG, "frames_dev is required");
    if (n_frames < 2) return set_err(c, COG_ERR_INVALID_ARG, "need at least 2 training frames");
    return group_run(c, frames_dev, n_frames, codes_dev, group_max_steps(), labels_dev, stats_host);
}

cog_status cog_group_cluster(cog_ctx *c, const uint16_t *codes_dev, int32_t max_steps, uint8_t *labels_dev,
                             cog_group_stats *stats_host)
{
    cog_status s = group_check(c, codes_dev, labels_dev, stats_host);
    if (s) return s;
    if (max_steps < 0 || max_steps > group_max_steps())
        return set_err(c, COG_ERR_INVALID_ARG, "max_steps must be in 0..%d", group_max_steps());
    return group_run(c, nullptr, 0, const_cast<uint16_t *>(codes_dev), max_steps, labels_dev, stats_host);
}

cog_status cog_probe_stream(const uint32_t *jl_in, const uint16_t *conf_in, const uint8_t *frame,
                            uint32_t *jl_out, uint16_t *conf_out, uint8_t *mask, int64_t P, void *cuda_stream)
{
    if (P <= 0 || P % 4 != 0 || P / 4 > (int64_t)0x7fffffff * 128)
        return set_err(nullptr, COG_ERR_INVALID_ARG, "P must be a positive multiple of 4");
    const void *ptrs[6] = {jl_in, conf_in, frame, jl_out, conf_out, mask};
    for (const void *q : ptrs)
        if (!q || (reinterpret_cast<uintptr_t>(q) & 15u))
            return set_err(nullptr, COG_ERR_INVALID_ARG, "every buffer must be non-NULL and 16-byte aligned");
    cudaError_t e = launch_probe_stream(jl_in, conf_in, frame, jl_out, conf_out, mask, P,
                                        static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return set_err(nullptr, COG_ERR_CUDA, "cog_probe_stream: %s", cudaGetErrorString(e));
    return COG_OK;
}

cog_status cog_apply_plain_gmm(cog_ctx *c, const uint8_t *frame_dev, uint8_t *mask_dev)
{
    if (c && (c->p.flags & COG_PERCHAN))
        return set_err(c, COG_ERR_INVALID_ARG, "the plain mixture uses shared weights; not defined with COG_PERCHAN");
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!c->trained) return set_err(c, COG_ERR_STATE, "cog_apply_plain_gmm before cog_train_prior");
    if (!frame_dev || !mask_dev) return set_err(c, COG_ERR_INVALID_ARG, "frame_dev and mask_dev are required");
    cudaError_t e;
    switch (c->p.state_dtype) {
    case COG_F32: e = launch_plain_f32(c->p.K, c->dp, c->sp, frame_dev, mask_dev, c->stream); break;
    case COG_F16: e = launch_plain_f16(c->p.K, c->dp, c->sp, frame_dev, mask_dev, c->stream); break;
    default: e = launch_plain_bf16(c->p.K, c->dp, c->sp, frame_dev, mask_dev, c->stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_plain_gmm launch");
    return COG_OK;
}

cog_status cog_apply_host(cog_ctx *c, const uint8_t *frame_host, uint8_t *mask_host)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!c->trained) return set_err(c, COG_ERR_STATE, "cog_apply_host before cog_train_prior");
    if (!frame_host || !mask_host) return set_err(c, COG_ERR_INVALID_ARG, "frame_host and mask_host are required");
    const size_t P = (size_t)c->L.P;
    cudaError_t e;
    if (!c->stage_in) {
        e = cudaMalloc((void **)&c->stage_in, up(P * 3, 256) + up(P, 256));
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->stage_in = nullptr;
            return set_err(c, COG_ERR_OOM, "staging allocation: %s", cudaGetErrorString(e));
        }
        c->stage_out = c->stage_in + up(P * 3, 256);
    }
    e = cudaMemcpyAsync(c->stage_in, frame_host, P * 3, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "frame upload");
    if ((s = cog_apply(c, c->stage_in, c->stage_out, nullptr, nullptr)) != COG_OK) return s;
    e = cudaMemcpyAsync(mask_host, c->stage_out, P, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mask download");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_host sync");
    return COG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// cog_apply_host_noalloc: the host-buffer entry point for callers that may
// not allocate device memory.  The frame and mask are staged through one
// file-scope device array of fixed size instead of cudaMalloc'd buffers.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t NOALLOC_MAX_PIXELS = 1920 * 1080;                          // 2,073,600
constexpr size_t NOALLOC_FRAME_BYTES = (size_t)NOALLOC_MAX_PIXELS * 3;       // 6,220,800 = 256 * 24300
constexpr size_t NOALLOC_BYTES = NOALLOC_FRAME_BYTES + (size_t)NOALLOC_MAX_PIXELS;   // 8,294,400
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
uint8_t *g_noalloc_ptr[NOALLOC_MAX_DEVICES];   // device address of the array, per device
}  // namespace

// Frame bytes at offset 0, mask bytes at NOALLOC_FRAME_BYTES.  In host code
// this name is only a stand-in: kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) uint8_t g_noalloc_stage[NOALLOC_BYTES];

// Resolves the array's device address for the context's device once
// (making that device current for the lookup); NULL with the error set on
// failure.
static uint8_t *noalloc_stage(cog_ctx *c)
{
    if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES) {
        set_err(c, COG_ERR_INVALID_ARG, "device %d beyond the %d devices the static staging supports", c->device,
                NOALLOC_MAX_DEVICES);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[c->device]) return g_noalloc_ptr[c->device];
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != c->device) e = cudaSetDevice(c->device);
    void *ptr = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr, g_noalloc_stage);
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    if (e != cudaSuccess || !ptr) {
        cuda_fail(c, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress(static staging array)");
        return nullptr;
    }
    g_noalloc_ptr[c->device] = (uint8_t *)ptr;
    return (uint8_t *)ptr;
}

extern "C" {

cog_status cog_apply_host_noalloc(cog_ctx *c, const uint8_t *frame_host, uint8_t *mask_host)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!frame_host || !mask_host) return set_err(c, COG_ERR_INVALID_ARG, "frame_host and mask_host are required");
    if (c->L.P > NOALLOC_MAX_PIXELS)
        return set_err(c, COG_ERR_INVALID_ARG,
                       "frame of %lld pixels exceeds the %lld-pixel limit of the static staging array",
                       (long long)c->L.P, (long long)NOALLOC_MAX_PIXELS);
    if (!c->trained) return set_err(c, COG_ERR_STATE, "cog_apply_host_noalloc before cog_train_prior");
    uint8_t *stage = noalloc_stage(c);
    if (!stage) return c->sticky != COG_OK ? c->sticky : COG_ERR_INVALID_ARG;
    const size_t P = (size_t)c->L.P;
    cudaError_t e = cudaMemcpyAsync(stage, frame_host, P * 3, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "frame upload (static staging)");
    if ((s = cog_apply(c, stage, stage + NOALLOC_FRAME_BYTES, nullptr, nullptr)) != COG_OK) return s;
    e = cudaMemcpyAsync(mask_host, stage + NOALLOC_FRAME_BYTES, P, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mask download (static staging)");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_host_noalloc sync");
    return COG_OK;
}

// Frames from host memory, pipelined: the upload of frame i+1 and the
// download of mask i-1 run on their own streams while frame i's kernels run
// on the context's stream; events order each slot's reuse.
cog_status cog_apply_host_frames(cog_ctx *c, const uint8_t *frames_host, int32_t n_frames, uint8_t *masks_host)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!c->trained) return set_err(c, COG_ERR_STATE, "cog_apply_host_frames before cog_train_prior");
    if (!frames_host || !masks_host) return set_err(c, COG_ERR_INVALID_ARG, "frames_host and masks_host are required");
    if (n_frames < 1) return set_err(c, COG_ERR_INVALID_ARG, "n_frames must be >= 1");
    const size_t P = (size_t)c->L.P;
    const size_t fb = up(P * 3, 256), mb = up(P, 256);
    cudaError_t e;
    if (!c->pipe_mem) {
        e = cudaMalloc((void **)&c->pipe_mem, 2 * (fb + mb));
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->pipe_mem = nullptr;
            return set_err(c, COG_ERR_OOM, "pipeline staging allocation: %s", cudaGetErrorString(e));
        }
        bool ok = cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&c->pipe_out, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 2 && ok; i++)
            ok = cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_done[i], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_out[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return cuda_fail(c, cudaGetLastError(), "pipeline streams/events");
    }
    uint8_t *fslot[2] = {c->pipe_mem, c->pipe_mem + fb};
    uint8_t *mslot[2] = {c->pipe_mem + 2 * fb, c->pipe_mem + 2 * fb + mb};
    for (int32_t i = 0; i < n_frames; i++) {
        const int k = i & 1;
        if (i >= 2) e = cudaStreamWaitEvent(c->pipe_in, c->ev_done[k], 0);    // slot read by frame i-2
        else e = cudaSuccess;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(fslot[k], frames_host + (size_t)i * P * 3, P * 3, cudaMemcpyHostToDevice, c->pipe_in);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[k], c->pipe_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_in[k], 0);
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(c->stream, c->ev_out[k], 0);   // mask slot copied out
        if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_host_frames upload");
        if ((s = cog_apply(c, fslot[k], mslot[k], nullptr, nullptr)) != COG_OK) return s;
        e = cudaEventRecord(c->ev_done[k], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->pipe_out, c->ev_done[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(masks_host + (size_t)i * P, mslot[k], P, cudaMemcpyDeviceToHost, c->pipe_out);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[k], c->pipe_out);
        if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_host_frames download");
    }
    e = cudaStreamSynchronize(c->pipe_out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_apply_host_frames sync");
    return COG_OK;
}

cog_status cog_read_stats(cog_ctx *c, cog_stats *last, cog_stats *total)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    std::vector<uint32_t> ctl;
    if ((s = read_ctl(c, ctl)) != COG_OK) return s;
    cog_stats l;
    frame_stats(ctl, c->frame_no - 1, &l);
    l.illum_flag = prev_flag(c, ctl, c->frame_no - 1);
    if (last) *last = l;
    if (total) {
        memset(total, 0, sizeof *total);
        total->frame = (int32_t)c->frame_no;
        const uint64_t *tot = reinterpret_cast<const uint64_t *>(ctl.data() + CTL_TOT_WORD);
        for (int f = 0; f < 5; f++) total->n_stage[f] = (int64_t)tot[f] + (c->frame_no > 0 ? l.n_stage[f] : 0);
        total->n_gmm = (int64_t)tot[5] + (c->frame_no > 0 ? l.n_gmm : 0);
        total->n_stage[5] = (int64_t)tot[6] + (c->frame_no > 0 ? l.n_stage[5] : 0);
    }
    return COG_OK;
}

int32_t cog_debug_build(void)
{
#ifdef COG_DEBUG
    return 1;
#else
    return 0;
#endif
}

cog_status cog_sync(cog_ctx *c)
{
    if (!c) return COG_ERR_INVALID_ARG;
    if (c->sticky != COG_OK) return c->sticky;
    std::vector<uint32_t> ctl;
    return read_ctl(c, ctl);
}

// The exported image carries the host-side frame counter and trained flag in
// otherwise unused control words so that an import resumes exactly.
static const int CTL_FRAME_WORD = CTL_ERR_WORD + 2;   // uint64 (words 802, 803)
static const int CTL_TRAINED_WORD = CTL_ERR_WORD + 4;

cog_status cog_export_state(cog_ctx *c, void *dst_host, size_t bytes)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!dst_host || bytes < c->L.total)
        return set_err(c, COG_ERR_INVALID_ARG, "destination smaller than %zu bytes", c->L.total);
    cudaError_t e = cudaMemcpyAsync(dst_host, c->state, c->L.total, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_export_state");
    uint32_t *w = (uint32_t *)((uint8_t *)dst_host + c->L.ctl);
    uint64_t fn = (uint64_t)c->frame_no;
    memcpy(w + CTL_FRAME_WORD, &fn, 8);
    w[CTL_TRAINED_WORD] = c->trained ? 1u : 0u;
    return COG_OK;
}

cog_status cog_import_state(cog_ctx *c, const void *src_host, size_t bytes)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (!src_host || bytes < c->L.total)
        return set_err(c, COG_ERR_INVALID_ARG, "source smaller than %zu bytes", c->L.total);
    cudaError_t e = cudaMemcpyAsync(c->state, src_host, c->L.total, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_import_state");
    const uint32_t *w = (const uint32_t *)((const uint8_t *)src_host + c->L.ctl);
    uint64_t fn;
    memcpy(&fn, w + CTL_FRAME_WORD, 8);
    c->frame_no = (int64_t)fn;
    c->trained = w[CTL_TRAINED_WORD] != 0;
    return COG_OK;
}

cog_status cog_info(cog_ctx *c, int64_t *frames_applied, void **state_dev)
{
    if (!c) return COG_ERR_INVALID_ARG;
    if (frames_applied) *frames_applied = c->frame_no;
    if (state_dev) *state_dev = c->state;
    return COG_OK;
}

cog_status cog_set_l2_fetch_bytes(int32_t bytes)
{
    if (bytes < 0 || bytes > 128 || (bytes & (bytes - 1)))
        return set_err(nullptr, COG_ERR_INVALID_ARG, "bytes must be 0 or a power of two up to 128");
    cudaError_t e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(nullptr, COG_ERR_CUDA, "cudaDeviceSetLimit: %s", cudaGetErrorString(e));
    }
    return COG_OK;
}

// page-locked host blocks handed out by cog_host_alloc: address -> length
static std::mutex g_host_mu;
static std::map<void *, size_t> g_host_blocks;

// The kernel's transparent huge page size (the PMD size: 2 MB with 4 KB base
// pages, 512 MB with 64 KB pages), else 2 MB.
static size_t thp_bytes()
{
    size_t hp = 2u << 20;
    if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) hp = (size_t)v;
        fclose(f);
    }
    return hp;
}

cog_status cog_host_alloc(size_t bytes, void **out)
{
    if (!out || bytes == 0) return set_err(nullptr, COG_ERR_INVALID_ARG, "need bytes > 0 and out");
    *out = nullptr;
    // whole huge pages at a huge-page boundary, asked for before the first
    // touch: the copy engines then translate a few large pages instead of
    // many small ones (on a fragmented host, small pages scattered over
    // memory cut host-to-device copies to a few GB/s)
    const size_t hp = thp_bytes();
    const size_t len = (bytes + hp - 1) / hp * hp;
    uint8_t *raw = (uint8_t *)mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == (uint8_t *)MAP_FAILED) return set_err(nullptr, COG_ERR_OOM, "mmap of %zu bytes failed", len + hp);
    uint8_t *p = (uint8_t *)(((uintptr_t)raw + hp - 1) / hp * hp);
    if (p > raw) munmap(raw, (size_t)(p - raw));
    if (raw + len + hp > p + len) munmap(p + len, (size_t)(raw + len + hp - (p + len)));
#ifdef MADV_HUGEPAGE
    madvise(p, len, MADV_HUGEPAGE);   // advice only: small pages if none are free
#endif
    memset(p, 0, len);   // every page present before it is locked
    cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        munmap(p, len);
        return set_err(nullptr, COG_ERR_CUDA, "cudaHostRegister: %s", cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(g_host_mu);
    g_host_blocks[p] = len;
    *out = p;
    return COG_OK;
}

cog_status cog_host_free(void *ptr)
{
    size_t len = 0;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_blocks.find(ptr);
        if (it == g_host_blocks.end())
            return set_err(nullptr, COG_ERR_INVALID_ARG, "not a block from cog_host_alloc");
        len = it->second;
        g_host_blocks.erase(it);
    }
    cudaError_t e = cudaHostUnregister(ptr);
    munmap(ptr, len);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(nullptr, COG_ERR_CUDA, "cudaHostUnregister: %s", cudaGetErrorString(e));
    }
    return COG_OK;
}

static void free_profile(cog_ctx *c)
{
    for (auto &e : c->prof) {
        cudaEventDestroy(e.e0);
        cudaEventDestroy(e.e1);
        cudaEventDestroy(e.e2);
    }
    c->prof.clear();
    c->prof_n = 0;
}

cog_status cog_set_launch(cog_ctx *c, int32_t k1_threads, int32_t k2_threads, int32_t k2_ctas_per_sm)
{
    if (!c) return COG_ERR_INVALID_ARG;
    if (k1_threads != 64 && k1_threads != 128 && k1_threads != 256)
        return set_err(c, COG_ERR_INVALID_ARG, "k1_threads must be 64, 128 or 256");
    if (k2_threads != 64 && k2_threads != 128) return set_err(c, COG_ERR_INVALID_ARG, "k2_threads must be 64 or 128");
    if (k2_ctas_per_sm < 0 || k2_ctas_per_sm > 64) return set_err(c, COG_ERR_INVALID_ARG, "k2_ctas_per_sm out of range");
    c->launch.k1_tpb = k1_threads;
    c->launch.k2_tpb = k2_threads;
    c->launch.k2_per_sm = k2_ctas_per_sm;
    return COG_OK;
}

cog_status cog_profile_begin(cog_ctx *c, int32_t max_frames)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    if (max_frames < 0 || max_frames > (1 << 20)) return set_err(c, COG_ERR_INVALID_ARG, "max_frames out of range");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_profile_begin");
    free_profile(c);
    c->prof.resize((size_t)max_frames);
    for (auto &ev : c->prof) {
        if (cudaEventCreate(&ev.e0) != cudaSuccess || cudaEventCreate(&ev.e1) != cudaSuccess ||
            cudaEventCreate(&ev.e2) != cudaSuccess) {
            cudaGetLastError();
            c->prof.clear();
            return set_err(c, COG_ERR_OOM, "cudaEventCreate failed");
        }
    }
    return COG_OK;
}

cog_status cog_profile_end(cog_ctx *c, double *stage01_ms, double *stage2_ms, int64_t *frames)
{
    cog_status s = check_ctx(c);
    if (s) return s;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cog_profile_end");
    double a = 0, b = 0;
    for (int64_t i = 0; i < c->prof_n; i++) {
        float x = 0, y = 0;
        cudaEventElapsedTime(&x, c->prof[(size_t)i].e0, c->prof[(size_t)i].e1);
        cudaEventElapsedTime(&y, c->prof[(size_t)i].e1, c->prof[(size_t)i].e2);
        a += x;
        b += y;
    }
    if (stage01_ms) *stage01_ms = a;
    if (stage2_ms) *stage2_ms = b;
    if (frames) *frames = c->prof_n;
    free_profile(c);
    return COG_OK;
}

const char *cog_last_error_string(cog_ctx *c)
{
    return c ? c->err : g_create_err;
}

cog_status cog_destroy(cog_ctx *c)
{
    if (!c) return COG_ERR_INVALID_ARG;
    cog_status s = c->sticky;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess && s == COG_OK) s = COG_ERR_CUDA;
    free_profile(c);
    if (c->stage_in) cudaFree(c->stage_in);
    if (c->clip_mem) cudaFree(c->clip_mem);
    if (c->pipe_mem) {
        cudaStreamSynchronize(c->pipe_in);
        cudaStreamSynchronize(c->pipe_out);
        cudaFree(c->pipe_mem);
        for (int i = 0; i < 2; i++) {
            cudaEventDestroy(c->ev_in[i]);
            cudaEventDestroy(c->ev_done[i]);
            cudaEventDestroy(c->ev_out[i]);
        }
        cudaStreamDestroy(c->pipe_in);
        cudaStreamDestroy(c->pipe_out);
    }
    if (c->owns) cudaFree(c->state);
    delete c;
    return s;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: one frame for each of many streams per step, as one captured
// CUDA graph (per storage type and K, one stage-0/1 launch and one mixture
// launch over all the group's streams; groups run as parallel branches).
// ---------------------------------------------------------------------------
// Host staging sets for the per-step descriptor and plan uploads.
constexpr int BATCH_STAGES = 8;

struct BatchGroupHost {
    int dtype = 0, K = 0;
    int mv = 0;                        // mixture variant (BatchGroupDev::mv)
    LaunchCfg launch;                  // the first member's launch shape
    std::vector<int> members;          // indices into cog_batch::ctxs
    std::vector<ApplyArgs> descs;      // host copy of the device descriptors
    BatchGroupDev dev{};
    uint32_t k1_ctas = 0, k2_ctas = 0; // fixed grids of the two batch kernels
    std::vector<int64_t> tiles, pix;   // stage-0/1 tiles and pixels per member
    void *dmem = nullptr;              // descs | frame_no | active | k1_pre | k2_pre
    ApplyArgs *pinned[BATCH_STAGES] = {};              // upload staging, by step % BATCH_STAGES
    uint32_t *pinned_active[BATCH_STAGES] = {};        // upload staging of the step plan
    std::vector<uint32_t> active;      // host copy of the active flags
};

// The step plan of a group: active flags, the prefix of the active
// members' stage-0/1 tiles, and the mixture-stage CTAs split among the
// active members in proportion to their pixels (at least one each, never
// more than the grid or than one per k2_tpb pixels).  out: n + 2 (n + 1).
static void batch_plan(const BatchGroupHost &g, uint32_t *out)
{
    const int n = (int)g.members.size();
    uint32_t *act = out, *k1 = out + n, *k2 = out + 2 * n + 1;
    int64_t psum = 0, nact = 0;
    for (int j = 0; j < n; j++)
        if (g.active[j]) { psum += g.pix[j]; nact++; }
    const int64_t spare = (int64_t)g.k2_ctas - nact;
    k1[0] = 0;
    k2[0] = 0;
    for (int j = 0; j < n; j++) {
        act[j] = g.active[j];
        int64_t t1 = 0, t2 = 0;
        if (g.active[j]) {
            t1 = g.tiles[j];
            t2 = 1 + (spare > 0 && psum > 0 ? spare * g.pix[j] / psum : 0);
            const int64_t need = (g.pix[j] + g.launch.k2_tpb - 1) / g.launch.k2_tpb;
            t2 = t2 > need ? need : t2;
        }
        k1[j + 1] = k1[j] + (uint32_t)t1;
        k2[j + 1] = k2[j] + (uint32_t)t2;
    }
}

struct cog_batch {
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<cog_ctx *> ctxs;
    std::vector<BatchGroupHost> groups;
    std::vector<const uint8_t *> frames;
    std::vector<uint8_t *> masks;
    std::vector<cudaStream_t> aux;     // one per group after the first (graph branches)
    std::vector<cudaEvent_t> fork, join;
    cudaEvent_t uploaded[BATCH_STAGES] = {};        // uploads of the last step using each staging set done
    uint64_t step = 0;
    cudaGraphExec_t exec = nullptr;
    cog_status sticky = COG_OK;
    char err[512] = {0};
};

static cog_status batch_err(cog_batch *b, cog_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b ? b->err : g_create_err, 512, fmt, ap);
    va_end(ap);
    if (b && s == COG_ERR_CUDA) b->sticky = s;
    return s;
}

static void batch_free(cog_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto &g : b->groups) {
        if (g.dmem) cudaFree(g.dmem);
        for (int k = 0; k < BATCH_STAGES; k++) {
            if (g.pinned[k]) cudaFreeHost(g.pinned[k]);
            if (g.pinned_active[k]) cudaFreeHost(g.pinned_active[k]);
        }
    }
    for (auto s : b->aux) cudaStreamDestroy(s);
    for (auto e : b->fork) cudaEventDestroy(e);
    for (auto e : b->join) cudaEventDestroy(e);
    for (int k = 0; k < BATCH_STAGES; k++)
        if (b->uploaded[k]) cudaEventDestroy(b->uploaded[k]);
    delete b;
}

extern "C" {

cog_status cog_batch_create(cog_ctx *const *ctxs, int32_t n, void *cuda_stream, cog_batch **out)
{
    if (!out || !ctxs || n < 1) return batch_err(nullptr, COG_ERR_INVALID_ARG, "need ctxs, n >= 1 and out");
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        if (!ctxs[i]) return batch_err(nullptr, COG_ERR_INVALID_ARG, "ctxs[%d] is NULL", i);
        if (ctxs[i]->sticky != COG_OK) return batch_err(nullptr, ctxs[i]->sticky, "ctxs[%d] has a sticky error", i);
        if (!ctxs[i]->trained) return batch_err(nullptr, COG_ERR_STATE, "ctxs[%d] is not trained", i);
        if (ctxs[i]->device != ctxs[0]->device)
            return batch_err(nullptr, COG_ERR_INVALID_ARG, "all contexts of a batch must be on one device");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i]) return batch_err(nullptr, COG_ERR_INVALID_ARG, "context %d appears twice", i);
    }
    cog_batch *b = new (std::nothrow) cog_batch();
    if (!b) return batch_err(nullptr, COG_ERR_OOM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->device = ctxs[0]->device;
    b->ctxs.assign(ctxs, ctxs + n);
    b->frames.assign(n, nullptr);
    b->masks.assign(n, nullptr);
    for (int i = 0; i < n; i++) {
        int gi = -1;
        for (size_t g = 0; g < b->groups.size(); g++)
            if (b->groups[g].dtype == ctxs[i]->p.state_dtype && b->groups[g].K == ctxs[i]->p.K &&
                b->groups[g].mv == mix_variant(ctxs[i]->p.flags))
                gi = (int)g;
        if (gi < 0) {
            b->groups.emplace_back();
            gi = (int)b->groups.size() - 1;
            b->groups[gi].dtype = ctxs[i]->p.state_dtype;
            b->groups[gi].K = ctxs[i]->p.K;
            b->groups[gi].mv = mix_variant(ctxs[i]->p.flags);
            b->groups[gi].launch = ctxs[i]->launch;
        }
        b->groups[gi].members.push_back(i);
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < BATCH_STAGES && e == cudaSuccess; k++)
        e = cudaEventCreateWithFlags(&b->uploaded[k], cudaEventDisableTiming);
    for (auto &g : b->groups) {
        if (e != cudaSuccess) break;
        const int m = (int)g.members.size();
        int64_t psum = 0;
        for (int i : g.members) psum += ctxs[i]->L.P;
        (void)psum;
        const int per_sm = g.dtype == COG_F32 ? k2_blocks_per_sm_f32(g.K, g.launch, g.mv)
                         : (g.dtype == COG_F16 ? k2_blocks_per_sm_f16(g.K, g.launch, g.mv)
                                               : k2_blocks_per_sm_bf16(g.K, g.launch, g.mv));
        const int k1_bps = g.dtype == COG_F32 ? k1_batch_blocks_per_sm_f32(g.launch)
                         : (g.dtype == COG_F16 ? k1_batch_blocks_per_sm_f16(g.launch) : k1_batch_blocks_per_sm_bf16(g.launch));
        int64_t tiles_all = 0;
        for (int j = 0; j < m; j++) {
            const cog_ctx *c = ctxs[g.members[j]];
            const int64_t tile = (int64_t)g.launch.k1_tpb * K1_PX_PER_THREAD;
            g.tiles.push_back((c->L.P + tile - 1) / tile);
            g.pix.push_back(c->L.P);
            tiles_all += g.tiles.back();
            ApplyArgs a{};
            a.dp = c->dp;
            a.s = c->sp;
            a.frame_no = (uint32_t)(c->frame_no % 3);
    a.frame_idx = (uint32_t)c->frame_no;
            a.k2_grid = (uint32_t)c->n_sm;
            a.rec_bytes = (uint32_t)c->L.rec_bytes;
            g.descs.push_back(a);
        }
        // fixed grids: a persistent stage-0/1 grid, and every mixture-stage
        // CTA that fits (split among the active members each step)
        const int64_t g1 = (int64_t)ctxs[0]->n_sm * (k1_bps > 0 ? k1_bps : 1);
        g.k1_ctas = (uint32_t)(tiles_all < g1 ? tiles_all : g1);
        g.k2_ctas = (uint32_t)((int64_t)ctxs[0]->n_sm * per_sm);
        const size_t plan_words = (size_t)m + 2 * (size_t)(m + 1);
        const size_t bytes = sizeof(ApplyArgs) * m + 4 * (size_t)m + 4 * plan_words + 64;
        if ((e = cudaMalloc(&g.dmem, bytes)) != cudaSuccess) break;
        for (int k = 0; k < BATCH_STAGES && e == cudaSuccess; k++) {
            if ((e = cudaMallocHost((void **)&g.pinned[k], sizeof(ApplyArgs) * m)) != cudaSuccess) break;
            e = cudaMallocHost((void **)&g.pinned_active[k], 4 * plan_words);
        }
        if (e != cudaSuccess) break;
        uint8_t *d = (uint8_t *)g.dmem;
        g.dev.descs = (ApplyArgs *)d;
        g.dev.frame_no = (uint32_t *)(d + sizeof(ApplyArgs) * m);
        g.dev.active = (const uint32_t *)(d + sizeof(ApplyArgs) * m + 4 * m);
        g.dev.k1_pre = g.dev.active + m;
        g.dev.k2_pre = g.dev.k1_pre + (m + 1);
        g.dev.n = m;
        g.dev.mv = g.mv;
        g.active.assign(m, 1u);
        std::vector<uint32_t> fno(m), plan(plan_words);
        for (int j = 0; j < m; j++) fno[j] = (uint32_t)ctxs[g.members[j]]->frame_no;
        batch_plan(g, plan.data());
        e = cudaMemcpyAsync(g.dev.frame_no, fno.data(), 4 * m, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((void *)g.dev.active, plan.data(), 4 * plan_words, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    for (size_t g = 1; g < b->groups.size() && e == cudaSuccess; g++) {
        cudaStream_t s;
        cudaEvent_t f, j;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
        b->aux.push_back(s);
        if ((e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming)) != cudaSuccess) break;
        b->fork.push_back(f);
        if ((e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) != cudaSuccess) break;
        b->join.push_back(j);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_err(nullptr, e == cudaErrorMemoryAllocation ? COG_ERR_OOM : COG_ERR_CUDA, "cog_batch_create: %s",
                  cudaGetErrorString(e));
        cog_status s = e == cudaErrorMemoryAllocation ? COG_ERR_OOM : COG_ERR_CUDA;
        batch_free(b);
        return s;
    }
    *out = b;
    return COG_OK;
}

static cudaError_t batch_capture(cog_batch *b)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; gi++) {
        BatchGroupHost &g = b->groups[gi];
        cudaStream_t st = b->stream;
        if (gi > 0) {
            st = b->aux[gi - 1];
            if ((e = cudaEventRecord(b->fork[gi - 1], b->stream)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(st, b->fork[gi - 1], 0)) != cudaSuccess) break;
        }
        switch (g.dtype) {
        case COG_F32: e = launch_batch_f32(g.K, g.dev, g.launch, g.k1_ctas, g.k2_ctas, st); break;
        case COG_F16: e = launch_batch_f16(g.K, g.dev, g.launch, g.k1_ctas, g.k2_ctas, st); break;
        default: e = launch_batch_bf16(g.K, g.dev, g.launch, g.k1_ctas, g.k2_ctas, st); break;
        }
        if (e == cudaSuccess) e = launch_batch_advance(g.dev, st);
        if (e == cudaSuccess && gi > 0) {
            if ((e = cudaEventRecord(b->join[gi - 1], st)) == cudaSuccess)
                e = cudaStreamWaitEvent(b->stream, b->join[gi - 1], 0);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return e;
}

static cog_status batch_apply(cog_batch *b, const uint8_t *const *frames_dev, uint8_t *const *masks_dev,
                              const uint8_t *active_host)
{
    if (!b) return COG_ERR_INVALID_ARG;
    if (b->sticky != COG_OK) return b->sticky;
    if (!frames_dev || !masks_dev) return batch_err(b, COG_ERR_INVALID_ARG, "frames_dev and masks_dev are required");
    const int n = (int)b->ctxs.size();
    for (int i = 0; i < n; i++) {
        const bool on = !active_host || active_host[i];
        if (on && (!frames_dev[i] || !masks_dev[i])) return batch_err(b, COG_ERR_INVALID_ARG, "stream %d: NULL buffer", i);
        if (b->ctxs[i]->sticky != COG_OK) return batch_err(b, b->ctxs[i]->sticky, "stream %d: sticky error", i);
    }
    cudaError_t e = cudaSuccess;
    // upload staging rotates over BATCH_STAGES sets: the set of this step
    // was last read by the uploads of BATCH_STAGES steps ago, long done
    // while the host stays at most a few steps ahead of the GPU, so the
    // wait below rarely blocks
    const int par = (int)(b->step % BATCH_STAGES);
    bool staged = false;
    for (auto &g : b->groups) {
        bool dirty = false, adirty = false;
        for (size_t j = 0; j < g.members.size(); j++) {
            const int i = g.members[j];
            const uint32_t on = (!active_host || active_host[i]) ? 1u : 0u;
            if (on != g.active[j]) { g.active[j] = on; adirty = true; }
            if (!on) continue;
            if (b->frames[i] == frames_dev[i] && b->masks[i] == masks_dev[i]) continue;
            ApplyArgs &a = g.descs[j];
            a.frame = frames_dev[i];
            a.mask = masks_dev[i];
            a.stagemap = nullptr;
            a.frame_al4 = ((uintptr_t)frames_dev[i] & 3) == 0;
            a.out_al4 = ((uintptr_t)masks_dev[i] & 3) == 0;
            b->frames[i] = frames_dev[i];
            b->masks[i] = masks_dev[i];
            dirty = true;
        }
        if (!dirty && !adirty) continue;
        // the device keeps frame_no current; the host copy matches it at
        // this point in stream order
        for (size_t j = 0; j < g.members.size(); j++) {
            g.descs[j].frame_no = (uint32_t)(b->ctxs[g.members[j]]->frame_no % 3);
            g.descs[j].frame_idx = (uint32_t)b->ctxs[g.members[j]]->frame_no;
        }
        if (!staged) {
            if ((e = cudaEventSynchronize(b->uploaded[par])) != cudaSuccess) break;
            staged = true;
        }
        if (dirty) {
            memcpy(g.pinned[par], g.descs.data(), sizeof(ApplyArgs) * g.descs.size());
            if ((e = cudaMemcpyAsync(g.dev.descs, g.pinned[par], sizeof(ApplyArgs) * g.descs.size(),
                                     cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
                break;
        }
        if (adirty) {
            const size_t m = g.members.size();
            batch_plan(g, g.pinned_active[par]);
            if ((e = cudaMemcpyAsync((void *)g.dev.active, g.pinned_active[par], 4 * (m + 2 * (m + 1)),
                                     cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
                break;
        }
    }
    if (e == cudaSuccess && staged) e = cudaEventRecord(b->uploaded[par], b->stream);
    b->step++;
    if (e == cudaSuccess && !b->exec) e = batch_capture(b);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return batch_err(b, COG_ERR_CUDA, "cog_batch_apply: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < n; i++)
        if (!active_host || active_host[i]) b->ctxs[i]->frame_no++;
    return COG_OK;
}

cog_status cog_batch_apply(cog_batch *b, const uint8_t *const *frames_dev, uint8_t *const *masks_dev)
{
    return batch_apply(b, frames_dev, masks_dev, nullptr);
}

cog_status cog_batch_apply_active(cog_batch *b, const uint8_t *const *frames_dev, uint8_t *const *masks_dev,
                                  const uint8_t *active_host)
{
    if (!active_host) return batch_err(b, COG_ERR_INVALID_ARG, "active_host is required");
    return batch_apply(b, frames_dev, masks_dev, active_host);
}

cog_status cog_batch_sync(cog_batch *b)
{
    if (!b) return COG_ERR_INVALID_ARG;
    if (b->sticky != COG_OK) return b->sticky;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_err(b, COG_ERR_CUDA, "cog_batch_sync: %s", cudaGetErrorString(e));
    return COG_OK;
}

const char *cog_batch_last_error_string(cog_batch *b) { return b ? b->err : g_create_err; }

cog_status cog_batch_destroy(cog_batch *b)
{
    if (!b) return COG_ERR_INVALID_ARG;
    cog_status s = b->sticky;
    batch_free(b);
    return s;
}

}  // extern "C"
