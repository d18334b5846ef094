/*
 * cog.h -- C ABI of the GB300 Cascade-of-Gaussians (CoG) background
 * subtraction library (libcog.so).
 *
 * The method is that of Kiran, Das and Yogamani, "Rejection-Cascade of
 * Gaussians: real-time adaptive background subtraction framework"
 * (arXiv 1705.09339).  The problem it states: learn a per-pixel scene prior
 * over N training frames (Sec. 2, "Scene Prior in Background Model"), then
 * classify every incoming frame pixel by pixel through a rejection cascade of
 * increasingly complex background models, adapting only the level that
 * classified the pixel (Sec. 2, "Cascade of Gaussians CoG").
 *
 * Conventions for every call
 *   - Pointers named *_dev are CUDA device pointers (for example torch
 *     tensors' data_ptr()); pointers named *_host are host pointers.  The
 *     caller owns every buffer it passes; the library never frees them.
 *   - Frames are 8-bit RGB, row-major, channels interleaved: byte
 *     (y*width + x)*3 + c.  Masks and stage maps are one byte per pixel.
 *   - Device calls are asynchronous and ordered on the CUDA stream given to
 *     cog_create.  Argument errors are reported synchronously.  CUDA launch
 *     errors and the device error word are sticky per context: the failing
 *     call, or the next call, or cog_sync, returns them.
 *   - A context is not thread-safe; different contexts are independent.
 *   - No call allocates device memory except cog_create (when it is not
 *     given a state buffer) and the first cog_apply_host (its staging
 *     buffers).
 */
#ifndef COG_H
#define COG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    COG_OK = 0,
    COG_ERR_INVALID_ARG = 1, /* null pointer, bad size, misaligned buffer, bad parameter */
    COG_ERR_OOM = 2,         /* device allocation failed                                 */
    COG_ERR_CUDA = 3,        /* a CUDA runtime call or a launch failed                   */
    COG_ERR_STATE = 4,       /* call out of order (apply before train, ...)              */
    COG_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                            */
    COG_ERR_DEVICE = 6       /* the device error word was set                            */
} cog_status;

/* Storage type of the model state; all arithmetic is FP32. */
typedef enum { COG_F32 = 0, COG_F16 = 1, COG_BF16 = 2 } cog_dtype;

/* Cascade switches (cog_params.flags). */
#define COG_FD    1u  /* stage 0: frame difference / consistent-hypothesis propagation */
#define COG_RGA   2u  /* stage 1: running Gaussian average                              */
#define COG_CONF  4u  /* confidence-driven learning rate, thresholds and halting        */
#define COG_ILLUM 8u  /* abrupt-illumination counter and response                       */
#define COG_SAMPLE 16u /* confidence-based temporal sampling (needs COG_CONF)            */
#define COG_MODE1 32u  /* stage 1 is a copy of the mixture's rank-1 mode (Fig. 1 reading:
                          CHP -> mode 1 -> the other modes); on a pixel's transition to
                          stage 2 the copy is written back into that mode (Sec. 2: the
                          parameters are updated during a transition), Eq. 2 runs, and
                          the copy then follows the mode that ranks first            */
#define COG_PERCHAN 64u /* per-channel independent mixtures (Sec. 2 assumes independent
                           R, G, B channels for the prior; here also for the mixture):
                           each channel ranks, matches and updates its own K 1-D
                           components with its own weights; a pixel is background iff
                           every channel is.  Records hold K x 9 values.  Not with
                           COG_MODE1; cog_apply_plain_gmm is not defined with it    */
#define COG_ALL   15u /* the cascade: every stage and modulation, no sampling            */

/* Stage codes written to a stage map (the cascade level that labelled the
 * pixel; the paper's per-level occupancy figure). */
#define COG_ST_FD     0
#define COG_ST_RGA    1
#define COG_ST_GMM_BG 2
#define COG_ST_FG     3
#define COG_ST_ILLUM  4
#define COG_ST_SKIP   5   /* not sampled this frame: label carried (COG_SAMPLE) */

typedef struct cog_params {
    int32_t width, height;   /* frame size in pixels, each >= 1                           */
    int32_t K;               /* Gaussians per pixel, 1..8 (Eq. 2)                         */
    int32_t state_dtype;     /* cog_dtype                                                 */
    float alpha;             /* base learning rate of Eq. 2                               */
    float lambda;            /* match threshold in standard deviations, per channel       */
    float T_bg;              /* background weight fraction T of the ordered Gaussians     */
    float w_init;            /* weight of a newly created component                       */
    float var_init;          /* variance of a newly created component                     */
    float var_min, var_max;  /* variance clamp                                            */
    float tau_fd;            /* stage-0 threshold on max_c |I - I_prev| at C = 0.5        */
    float eta_conf;          /* smoothing rate of the confidence C                        */
    float c_halt;            /* confidence at which stage-1 updates halt                  */
    float w_illum;           /* weight of the new mode after an illumination change       */
    int32_t q_null;          /* prior nullified below this peak-normalised level (/255)   */
    int32_t kde_bw;          /* scene-prior kernel bandwidth in grey levels, 1..32        */
    int32_t r1, r2;          /* residue class bounds (static <= r1 < oscillating <= r2)   */
    int32_t illum_permille;  /* illumination change when > this per mille of pixels       */
    uint32_t flags;          /* COG_* switches                                            */
    float c_skip;            /* COG_SAMPLE: pixels with C >= c_skip are looked at only    */
                             /* every skip_period frames (Sec. 2, "Confidence based       */
                             /* temporal sampling"), in 64-pixel blocks with staggered    */
                             /* phases: frame n processes block b when (n + b) % S == 0   */
    int32_t skip_period;     /* S >= 1                                                    */
    int32_t kde_bits;        /* scene-prior levels per channel value: 8 (q of 255, one     */
                             /* byte each) or 4 (q of 15, two per byte: the even grey     */
                             /* level in the low nibble); the prior enters as q / (2^bits */
                             /* - 1) and is nullified below q_null / 255 either way       */
} cog_params;

/* Per-frame statistics (the stage occupancy n_i of the paper's speed-up
 * model, Sec. 3.2). */
typedef struct cog_stats {
    int64_t n_stage[6];      /* pixels labelled at each COG_ST_* level   */
    int64_t n_gmm;           /* pixels that reached the mixture stage    */
    int32_t illum_flag;      /* illumination response active this frame  */
    int32_t frame;           /* index of the frame these counts describe */
} cog_stats;

/* Byte offsets of the state buffer's planes (for export/import decoding).
 * P = width*height; Pp = P rounded up to a multiple of 4096. */
typedef struct cog_layout {
    uint64_t total;          /* bytes of the whole state buffer                          */
    uint64_t ctl;            /* control block (counters), 4096 bytes                     */
    uint64_t jl;             /* uint32[Pp]: previous frame R,G,B in bytes 0..2, label 3  */
    uint64_t conf;           /* dtype[Pp]: confidence C                                  */
    uint64_t s1;             /* stage-1 records, s1_bytes each: m0 m1 m2 v0 v1 v2 as     */
                             /* dtype, then uint16 qa | qb << 8 (16-bit dtypes) or       */
                             /* uint32 (FP32), zero padding                              */
    uint64_t s1_bytes;       /* 16 (FP16/BF16) or 32 (FP32)                              */
    uint64_t gmm;            /* per-pixel records of rec_bytes: K x (w, mu0..2, v0..2)   */
    uint64_t rec_bytes;      /* K*7*sizeof(dtype) rounded up to 16                       */
    uint64_t queue;          /* scratch: survivor queue, 32 segments of whole 1024-entry */
                             /* tiles, 16 bytes per entry                                */
    uint64_t kde;            /* uint8[P][3][kde_row]: peak-normalised prior              */
    uint64_t elem_bytes;     /* sizeof(dtype)                                            */
    uint64_t kde_row;        /* bytes per pixel and channel of the prior: 256 (8-bit) or */
                             /* 128 (4-bit)                                              */
} cog_layout;

typedef struct cog_ctx cog_ctx;

/* Fills *p with the library defaults for a width x height stream with K
 * Gaussians: FP32 state, every stage on.  The paper states no constants;
 * the defaults are this library's documented readings. */
void cog_default_params(cog_params *p, int32_t width, int32_t height, int32_t K);

/* Validates *p and returns the state size and plane offsets.  Host only. */
cog_status cog_state_bytes(const cog_params *p, size_t *out_bytes);
cog_status cog_state_layout(const cog_params *p, cog_layout *out);

/* Creates a context bound to the current CUDA device and to cuda_stream
 * (a cudaStream_t; NULL = the legacy default stream).  state_dev: NULL to
 * let the library allocate the state, or a caller-owned device buffer of at
 * least cog_state_bytes bytes, 256-byte aligned, that outlives the context.
 * The state is zeroed on the stream. */
cog_status cog_create(const cog_params *p, void *cuda_stream, void *state_dev, cog_ctx **out);

/* Training phase (Sec. 2): frames_dev holds n_frames >= 2 frames back to
 * back (n_frames x height x width x 3 bytes, any alignment).  Builds the
 * per-pixel, per-channel kernel-density prior over the frames (Sec. 2,
 * "Scene Prior"), the residue-class confidence weights (Sec. 2,
 * "Determining Learning Rate Hyper-parameters"), and warms the mixture of
 * Eq. 2 up over the frames with every rejection stage off; the running
 * average starts at the top-ranked mode and C at 0.5.  Requires
 * n_frames * sum_d g[d] < 2^32 (n_frames <= 6500 at bandwidth 4). */
cog_status cog_train_prior(cog_ctx *ctx, const uint8_t *frames_dev, int32_t n_frames);

/* One frame through the cascade (Sec. 2, "Cascade of Gaussians CoG"):
 * stage 0 frame difference, stage 1 running Gaussian average, stage 2 the
 * ordered Gaussians of Eq. 2 with the scene prior and the confidence of
 * Sec. 2 "Confidence Measure"; only the level that labels a pixel adapts.
 * frame_dev: height x width x 3 bytes (any alignment).  mask_dev: one byte
 * per pixel (255 = foreground).  stagemap_dev: NULL, or one COG_ST_* byte
 * per pixel.  4-byte aligned frames, masks and stage maps take 32-bit
 * accesses.
 * stats_host: NULL, or receives this frame's counts (the call then
 * synchronises the stream).  Two kernels run per frame: stages 0 and 1 over
 * every pixel, then the mixture stage over the pixels left (compacted into
 * the state's survivor queue).
 * COG_ERR_STATE before cog_train_prior. */
cog_status cog_apply(cog_ctx *ctx, const uint8_t *frame_dev, uint8_t *mask_dev,
                     uint8_t *stagemap_dev, cog_stats *stats_host);

/* n_frames consecutive frames through the cascade, for video that is
 * already recorded (Sec. 2, "Cascade of Gaussians CoG", applied frame after
 * frame; the paper has no multi-frame form: this is a scheduling of the
 * same per-frame step).  Results -- masks, stage maps, counts, model state,
 * the illumination flags of the counter at the end of that section -- are
 * identical to n_frames calls of cog_apply with the same buffers.
 * frames_dev: n_frames x height x width x 3 bytes, back to back.
 * masks_dev: n_frames x height x width bytes; stagemaps_dev: NULL or the
 * same size.  Any alignment; 4-byte aligned buffers with height x width a
 * multiple of 4 take 32-bit accesses.  stats_host: NULL, or n_frames
 * entries, one per frame (the call then synchronises the stream).
 * Frames go in launches of up to 32 frames: one cooperative launch keeps
 * every pixel's stage-0/1 state on chip across its frames.  The launch
 * assumes no frame after its first is flagged as an illumination change,
 * checks that against the counts of the whole frame, and if it was wrong
 * undoes the launch's state changes and runs again with the flag fixed
 * (at most 33 runs; one when no frame is flagged).  The first call
 * allocates the context's clip scratch: counters plus an undo log of about
 * 30 + the mixture record's bytes per pixel.  Stream-ordered like
 * cog_apply; a grid-wide wait that gives up after 2 s sets the device
 * error word (COG_ERR_DEVICE from the next synchronising call).
 * COG_ERR_STATE before cog_train_prior; COG_ERR_OOM if the scratch cannot
 * be allocated. */
cog_status cog_apply_clip(cog_ctx *ctx, const uint8_t *frames_dev, int32_t n_frames, uint8_t *masks_dev,
                          uint8_t *stagemaps_dev, cog_stats *stats_host);

/* Runs the last launch of cog_apply_clip needed (1 = no illumination flag
 * was mispredicted; 0 before any clip).  Synchronises the stream. */
cog_status cog_clip_runs(cog_ctx *ctx, int32_t *runs);

/* Native continuous-batching frame server; the paper has no counterpart
 * (a deployment form of the batched step).  n trained contexts become the
 * server's streams: while it exists they belong to it (call nothing else
 * on them).  It allocates two device frame slots and two mask slots per
 * stream, a batch over the contexts (cog_batch_create) and three streams,
 * and starts a worker and a completion thread.
 *   cog_server_submit: queues one frame of stream `stream` from host memory
 *     (height x width x 3 bytes; page-locked for overlap) and the host
 *     buffer that receives its mask; both must stay valid until the frame
 *     is done (cog_server_drain).  Thread-safe; returns at once.
 *   The worker takes, while fewer than four steps are on the GPU, for
 *   every stream with a frame waiting and a free slot, the oldest frame;
 *   uploads them; runs one batched step over those streams only; downloads
 *   their masks.  Frames submitted meanwhile join the next step, whose
 *   uploads overlap the running one.
 *   cog_server_add: a further trained context joins the running server as
 *     stream *stream_out: the lowest index a camera has left, else the next
 *     index.  The worker takes it between steps: once no step is on the GPU
 *     (at most 30 s) it rebuilds the batch over all the contexts, so frames
 *     of the other streams wait for that rebuild.  Allocates the new
 *     stream's slots; returns when it has joined; COG_ERR_TIMEOUT after
 *     60 s, COG_ERR_STATE if the server is stopping, COG_ERR_INVALID_ARG for
 *     a context the server already has.  A failed join leaves the server
 *     and its status unchanged.
 *   cog_server_remove: camera `stream` leaves the running server.  Frames
 *     submitted for it from then on are refused (COG_ERR_INVALID_ARG); those
 *     already submitted are completed.  Once none is waiting or on the GPU,
 *     the worker rebuilds the batch without it between steps, as for a
 *     join, and frees its slots; the call then returns and hands the context
 *     back in *ctx_out (nullable): it belongs to the caller again (destroy
 *     it, use it alone, or add it again).  The other cameras keep their
 *     indices; the next join takes this one.  COG_ERR_INVALID_ARG for an
 *     index that is not a serving camera or for the last camera (destroy the
 *     server instead), COG_ERR_TIMEOUT after 60 s (the camera then stays),
 *     COG_ERR_STATE if the server is stopping.
 *   cog_server_drain: waits up to timeout_ms until every submitted frame is
 *     done; COG_ERR_TIMEOUT otherwise.
 *   cog_server_read_stats: counts and the p50/p99/max latency from submission
 *     to the mask being in host memory, and the seconds since creation; the
 *     latency split into the wait (submission until the worker takes the
 *     frame for a step) and the service (from then until the mask is in
 *     host memory: upload, step, download, completion notice); and the host
 *     time the worker spent issuing a step (copies, plan upload, graph
 *     launch), whose tail shows the worker blocked in the CUDA runtime.
 *   cog_server_destroy: stops the threads; frames not yet started are
 *     dropped (drain first to keep them).  Errors are sticky. */
typedef struct cog_server cog_server;
typedef struct {
    int64_t submitted, frames, steps, pixels;
    double p50_ms, p99_ms, max_ms, wall_s;
    double wait_p50_ms, wait_p99_ms;         /* submission -> taken for a step     */
    double service_p50_ms, service_p99_ms;   /* taken -> mask in host memory       */
    double enqueue_p99_ms, enqueue_max_ms;   /* per step: host time to issue it    */
} cog_server_stats;
cog_status cog_server_create(cog_ctx *const *ctxs, int32_t n, cog_server **out);
cog_status cog_server_submit(cog_server *s, int32_t stream, const uint8_t *frame_host, uint8_t *mask_host);
cog_status cog_server_add(cog_server *s, cog_ctx *ctx, int32_t *stream_out);
cog_status cog_server_remove(cog_server *s, int32_t stream, cog_ctx **ctx_out);
cog_status cog_server_drain(cog_server *s, int32_t timeout_ms);
cog_status cog_server_read_stats(cog_server *s, cog_server_stats *out);
/* Per-frame record in completion order: submission time since creation and
 * latency, both in ms; copies min(cap, done) entries, *n = frames done. */
cog_status cog_server_read_latencies(cog_server *s, float *submit_ms, float *latency_ms, int64_t cap, int64_t *n);
/* The same with the wait of each frame (submission until the worker took it
 * for a step) in wait_ms (nullable). */
cog_status cog_server_read_timeline(cog_server *s, float *submit_ms, float *wait_ms, float *latency_ms, int64_t cap,
                                    int64_t *n);
/* Per-step record of the completed steps: the host time the worker spent
 * issuing each step (enqueue_ms, in issue order) and, in parts_ms
 * (nullable, 10 floats per step, in completion order), that time split into
 * the frame uploads, the batched step (plan upload and graph launch) and
 * the mask downloads with the completion event, then the step's GPU times
 * from CUDA events: uploads, wait until the compute stream took the step,
 * batched step, wait until the download stream took it, downloads; then the
 * step's frame count and the megabytes of frames it uploaded.  Copies
 * min(cap, completed) entries, *n = steps completed. */
cog_status cog_server_read_steps(cog_server *s, float *enqueue_ms, float *parts_ms, int64_t cap, int64_t *n);
/* Clears the counters, latency and step records and restarts the clock of
 * cog_server_read_stats (for example after warm-up frames).  Every submitted
 * frame must be done (cog_server_drain): COG_ERR_STATE otherwise. */
cog_status cog_server_reset_stats(cog_server *s);
const char *cog_server_last_error_string(cog_server *s);
cog_status cog_server_destroy(cog_server *s);

/* Self-test of failure detection; the paper has no counterpart.  Runs the
 * bounded grid-wide wait that cog_apply_clip's barriers use on a count that
 * nothing completes, with a limit of limit_ms (1..2000) instead of 2 s, on
 * the current device.  The wait must give up: *error_word receives the
 * device error bits it set (2 = a grid-wide wait timed out) and
 * *elapsed_ms the kernel's duration.  Uses two static device words (no
 * allocation) and its own stream; returns COG_OK when the kernel ran to
 * completion, COG_ERR_CUDA otherwise, COG_ERR_INVALID_ARG for bad
 * arguments.  Calls that overlap on one device share the words: serialise
 * them. */
cog_status cog_selftest_bounded_wait(int32_t limit_ms, uint32_t *error_word, double *elapsed_ms);

/* Spatio-temporal grouping (Sec. 2, "Clustering Similar Background -
 * Spatio-Temporal Grouping", steps 1-6 and Eq. 3), a training-side
 * analysis of which pixels share the mixture's update behaviour:
 *   1-2  the warm-up of cog_train_prior is replayed over the same training
 *        frames; after each update at frames 1..N-1 the dominant mode (rank
 *        1 of omega^2 / vbar, lower index on ties) gives its mean variance
 *        vbar and weight omega; per pixel the population standard
 *        deviations of the two series are coded
 *        code_v = round(64 sd_v), code_w = round(65536 sd_w), <= 65535;
 *   3-4  K-means with K = 3 over (code_v, code_w), each scaled by its
 *        standard deviation over all pixels (1 for a constant code), first
 *        centroids at mean - sd, mean, mean + sd (sd = 0 for a constant
 *        code), an empty cluster keeping its centroid, ties to the lower
 *        cluster, until no label changes (at most 64 steps); the distance
 *        is evaluated in FP32 from centroids and reciprocal scales rounded
 *        to float once per step, so a pixel within FP32 rounding of a tie
 *        between its two nearest centroids may take either;
 *   5    Eq. 3: a core pixel has both codes strictly within its cluster's
 *        mean +- standard deviation;
 *   6    per cluster, the mean over its core of the trained dominant mode
 *        (the component cog_train_prior gave the running average).
 * frames_dev: the n_frames >= 2 training frames given to cog_train_prior
 * (n_frames x height x width x 3 bytes, device memory).  codes_dev: device
 * uint16 [2][P] (code_v then code_w), 2-byte aligned; labels_dev: device
 * uint8 [P], cluster 0..2 | 0x80 for a core pixel.  Both caller-owned.
 * Call it after cog_train_prior and before cog_apply (step 6 reads the
 * trained state).  Not defined with COG_PERCHAN (COG_ERR_INVALID_ARG);
 * P must be below 2^30.  Runs on the context's stream and returns when
 * stats_host is filled. */
typedef struct cog_group_stats {
    int32_t iterations;          /* K-means steps until no label changed (64 if none)  */
    int32_t converged;           /* 1: the labels settled within 64 steps              */
    int64_t n[3];                /* pixels per cluster                                 */
    int64_t n_core[3];           /* of them core pixels (Eq. 3)                        */
    int64_t code_sum[3][2];      /* per cluster: sums of code_v, code_w                */
    int64_t code_sq_sum[3][2];   /*              and of their squares                  */
    double centroid[3][2];       /* member means of the codes                          */
    double sd[3][2];             /* member standard deviations of the codes            */
    double w1[3];                /* core means of the dominant mode's weight,          */
    double mu1[3][3];            /* per-channel means                                  */
    double v1[3];                /* and mean variance                                  */
} cog_group_stats;
cog_status cog_group(cog_ctx *ctx, const uint8_t *frames_dev, int32_t n_frames, uint16_t *codes_dev,
                     uint8_t *labels_dev, cog_group_stats *stats_host);

/* Steps 3-6 of cog_group on the caller's codes (Sec. 2, "Clustering
 * Similar Background", steps 4-6 and Eq. 3): the first assignment, then at
 * most max_steps (0..64) Lloyd steps, stopping early once a step changes no
 * label; then the Eq. 3 cores and step 6.  With max_steps = s the labels
 * are those after step s (the core bit 0x80 added), which lets a caller
 * follow the clustering step by step.  stats_host->iterations is the step
 * that changed nothing, or max_steps if none did (converged = 0).
 * codes_dev: device uint16 [2][P] as cog_group writes them, 2-byte
 * aligned, read only; labels_dev: device uint8 [P].  Same state and
 * argument rules as cog_group; max_steps outside 0..64 is
 * COG_ERR_INVALID_ARG.  Returns when stats_host is filled. */
cog_status cog_group_cluster(cog_ctx *ctx, const uint16_t *codes_dev, int32_t max_steps, uint8_t *labels_dev,
                             cog_group_stats *stats_host);

/* Measurement aid; the paper has no counterpart.  One pass over the planes
 * that stage 0 touches when every pixel passes it, with no arithmetic, to
 * time the streaming floor of a kernel of that size: for every pixel p
 *   jl_out[p]   = frame[3p] | frame[3p+1] << 8 | frame[3p+2] << 16
 *                 | (jl_in[p] & 0xff000000)       (this frame, previous label)
 *   conf_out[p] = conf_in[p]                      (16-bit confidence)
 *   mask[p]     = jl_in[p] >> 24
 * 9 bytes per pixel in, 7 out, one thread per 4 pixels in 128-thread CTAs as
 * the stage-0/1 kernel.  P > 0 and a multiple of 4; every pointer 16-byte
 * aligned, device memory owned by the caller, outputs disjoint from inputs.
 * Launched on cuda_stream (a cudaStream_t) and not waited for.  Returns
 * COG_ERR_INVALID_ARG for bad arguments, COG_ERR_CUDA for a launch error. */
cog_status cog_probe_stream(const uint32_t *jl_in, const uint16_t *conf_in, const uint8_t *frame,
                            uint32_t *jl_out, uint16_t *conf_out, uint8_t *mask, int64_t P, void *cuda_stream);

/* The comparison baseline: one frame of the plain Stauffer-Grimson mixture
 * (Eq. 2 at rate alpha, no cascade, no prior, no confidence) on this
 * context's mixture state.  Same buffer rules as cog_apply. */
cog_status cog_apply_plain_gmm(cog_ctx *ctx, const uint8_t *frame_dev, uint8_t *mask_dev);

/* cog_apply for host buffers: copies frame_host (height x width x 3 bytes)
 * to the device, runs the cascade and copies the mask back into mask_host
 * (one byte per pixel).  Returns when mask_host is filled.  Page-locked host
 * buffers give full copy bandwidth; pageable ones work.  The first call
 * allocates two device staging buffers that the context keeps. */
cog_status cog_apply_host(cog_ctx *ctx, const uint8_t *frame_host, uint8_t *mask_host);

/* n_frames consecutive frames from host memory (frames_host: n_frames x
 * height x width x 3 bytes; masks_host: n_frames x height x width bytes),
 * each through the cascade as cog_apply, with the transfers pipelined: the
 * upload of the next frame and the download of the previous mask run on the
 * context's own copy streams while the current frame's kernels run, through
 * two device slots.  Results are those of n_frames cog_apply_host calls.
 * Page-locked host buffers let the copies overlap; pageable ones work.  The
 * first call allocates the slots (2 x (4 bytes per pixel)) and creates two
 * streams and six events that the context keeps.  Returns when every mask
 * is in masks_host. */
cog_status cog_apply_host_frames(cog_ctx *ctx, const uint8_t *frames_host, int32_t n_frames, uint8_t *masks_host);

/* cog_apply_host for callers that cannot allocate device memory: the
 * paper has no counterpart; this is a deployment form of the same call.
 * Some hosts must not call cudaMalloc or cudaFree at all: a frame server or
 * real-time pipeline that shares the GPU (those calls can synchronise the
 * whole device and stall every other stream), or an application that hands
 * out all device memory from its own fixed budget.  This call stages the
 * frame and the mask through one static device array of 8,294,400 bytes
 * compiled into the library (a 1920 x 1080 frame plus its mask), which every
 * GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   - Frames larger than 2,073,600 pixels are rejected with
 *     COG_ERR_INVALID_ARG before anything runs.
 *   - The first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress, with that device made current for the lookup);
 *     make that first call before any stream capture.
 *   - Every call on a device shares the one array and it keeps the last
 *     call's contents.  Nothing in it needs to start at zero: the frame area
 *     is fully overwritten before the kernels read it and the mask area is
 *     fully written before it is copied back.  Calls whose work overlaps on
 *     the GPU (contexts used from several host threads, or on several
 *     streams of one device) race on the array: serialise them.
 * Otherwise it behaves as cog_apply_host: returns when mask_host is
 * filled. */
cog_status cog_apply_host_noalloc(cog_ctx *ctx, const uint8_t *frame_host, uint8_t *mask_host);

/* Batches: one frame for each of many streams per step (cameras of uneven
 * resolution, K and storage type), run as one captured CUDA graph.  Streams
 * sharing a storage type and K form a group that one stage-0/1 launch and
 * one mixture-stage launch cover; groups run as parallel graph branches.
 * cog_batch_create: ctxs are n >= 1 distinct trained contexts on the
 * current device; cuda_stream must be a created stream (graphs cannot be
 * captured on the legacy default stream).  It allocates the batch's
 * descriptor tables.  While a context belongs to a batch, apply it only
 * through the batch.
 * cog_batch_apply: frames_dev[i] / masks_dev[i] are stream i's frame and
 * mask buffers (as cog_apply).  Asynchronous on the batch's stream.  The
 * graph is captured on the first call and replayed afterwards; changed
 * buffer pointers only update device-side descriptors.
 * cog_batch_sync waits for the batch's stream (then cog_read_stats works
 * per context).  cog_batch_destroy frees the batch, not its contexts. */
typedef struct cog_batch cog_batch;
cog_status cog_batch_create(cog_ctx *const *ctxs, int32_t n, void *cuda_stream, cog_batch **out);
cog_status cog_batch_apply(cog_batch *batch, const uint8_t *const *frames_dev, uint8_t *const *masks_dev);
/* As cog_batch_apply for the streams with active_host[i] != 0 only (a
 * host array of n flags); the other streams skip the step (their buffers
 * may be NULL, their state and frame count do not change).  The same
 * captured graph serves every subset: the flags live in device memory.
 * This is the step of a continuous-batching server. */
cog_status cog_batch_apply_active(cog_batch *batch, const uint8_t *const *frames_dev, uint8_t *const *masks_dev,
                                  const uint8_t *active_host);
cog_status cog_batch_sync(cog_batch *batch);
const char *cog_batch_last_error_string(cog_batch *batch);
cog_status cog_batch_destroy(cog_batch *batch);

/* Statistics of the most recent cog_apply frame and running totals of the
 * stage counts over every frame applied since the last training.
 * Synchronises the stream. */
cog_status cog_read_stats(cog_ctx *ctx, cog_stats *last, cog_stats *total);

/* Waits for the context's stream; returns any sticky error, and
 * COG_ERR_DEVICE when a kernel set the context's device error word (a
 * bounded wait gave up, or in the COG_DEBUG build a bounds check failed:
 * the message names the check, the index and its limit). */
cog_status cog_sync(cog_ctx *ctx);

/* 1 in the COG_DEBUG build of this library (libcog_debug.so: every
 * data-dependent index of the kernels -- survivor-queue slots, pixels taken
 * from queue entries and shared lists, batch streams and tiles -- is checked
 * before its access; a failure skips the access and sets the device error
 * word, reported by the next cog_sync), 0 otherwise.  A sanitizer
 * substitute; the paper has no counterpart. */
int32_t cog_debug_build(void);

/* Byte image of the state buffer (cog_layout.total bytes) to or from host
 * memory.  Synchronous. */
cog_status cog_export_state(cog_ctx *ctx, void *dst_host, size_t bytes);
cog_status cog_import_state(cog_ctx *ctx, const void *src_host, size_t bytes);

/* Number of frames applied since training, and the device state pointer. */
cog_status cog_info(cog_ctx *ctx, int64_t *frames_applied, void **state_dev);

/* Launch shape of the context's two cascade kernels (the autotuner's
 * knobs; results do not depend on them): k1_threads in {64, 128, 256}
 * threads per stage-0/1 CTA (4 pixels per thread), k2_threads in {64, 128}
 * per mixture-stage CTA, k2_ctas_per_sm mixture-stage CTAs per SM (0: as
 * many as fit).  Defaults 128, 64, 0.  A batch uses each group's first
 * member's shape, read at cog_batch_create. */
cog_status cog_set_launch(cog_ctx *ctx, int32_t k1_threads, int32_t k2_threads, int32_t k2_ctas_per_sm);

/* Per-kernel timing.  cog_profile_begin makes the next max_frames calls
 * of cog_apply record CUDA events on the context's stream around each of
 * its two kernels (stages 0-1, then the mixture stage); cog_profile_end
 * synchronises and returns the summed milliseconds of each kernel and the
 * number of frames recorded, then releases the events.  Both synchronise
 * the stream. */
cog_status cog_profile_begin(cog_ctx *ctx, int32_t max_frames);
cog_status cog_profile_end(cog_ctx *ctx, double *stage01_ms, double *stage2_ms, int64_t *frames);

/* Sets the L2 fetch granularity of the calling process's CUDA context on
 * the current device (cudaLimitMaxL2FetchGranularity; 0 or a power of two
 * up to 128 bytes).  The mixture stage gathers one 80-byte record and three
 * prior bytes per survivor at random addresses; with the driver's default
 * granularity each 32-byte miss pulls in neighbouring sectors that are never
 * used.  32 keeps DRAM traffic at the sectors the cascade touches.  The
 * limit applies to every kernel of the process on that device and ends with
 * the process. */
cog_status cog_set_l2_fetch_bytes(int32_t bytes);

/* Page-locked host memory for frames that the copy engines move to the
 * device (cog_apply_host_frames, the frame server): anonymous memory aligned
 * to the kernel's transparent huge page size, advised to use huge pages,
 * zeroed, then locked with cudaHostRegister; cog_host_free unlocks and
 * unmaps it.  On the Grace host of a GB300, host-to-device copies out of
 * such memory taken after the process's large device allocations ran at
 * 150-180 GB/s from its first use, where memory from cudaHostAlloc, or
 * locked memory taken before those allocations, ran at 2-12 GB/s on a first
 * pass over 3.6 GB of frames in some processes.  Any size (rounded up to
 * whole huge pages); COG_ERR_OOM if the mapping fails, COG_ERR_CUDA if it
 * cannot be locked; cog_host_free of a pointer not from cog_host_alloc
 * returns COG_ERR_INVALID_ARG.  Thread-safe.  Deployment plumbing; the
 * paper has no counterpart. */
cog_status cog_host_alloc(size_t bytes, void **out);
cog_status cog_host_free(void *ptr);

/* Human-readable description of the context's last error ("" if none).
 * With ctx == NULL: the last error of a failed cog_create on this thread. */
const char *cog_last_error_string(cog_ctx *ctx);

/* Waits for the stream, frees what the library allocated, and destroys the
 * context.  Returns the sticky error, if any. */
cog_status cog_destroy(cog_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* COG_H */
