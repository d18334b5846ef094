// cog_internal.h -- definitions shared by the library's translation units:
// the kernel parameter block, the state layout and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cog.h"

namespace cog {

constexpr int PX_ALIGN = 4096;   // pixel padding of every state plane
constexpr int KMAX = 8;

// Control block (first CTL_BYTES of the state), in 32-bit words.  Every
// atomic counter sits on its own 128-byte line (CTL_PAD words apart) so that
// the per-CTA atomics of a frame spread over L2 slices instead of queueing
// on one line.
//   ctl_slot(b, f, s)  per-frame counters: 3 rotating buffers b x 8 fields f
//              x 32 slots s; fields 0..4 = pixels labelled at each stage,
//              5 = pixels that reached the mixture stage, 6 = pixels skipped
//              by the temporal sampling.  Frame n
//              accumulates into buffer n % 3, reads buffer (n - 1) % 3 for its
//              illumination flag, and its first kernel's block 0 clears buffer
//              (n + 1) % 3.
//   CTL_TOT_WORD       running totals, 8 x uint64 (fields as above), lagging
//                      one frame
//   CTL_ERR_WORD       device error word; the next words hold host
//                      bookkeeping carried by export/import
//   ctl_qcnt(b, g)     survivor-queue segment lengths: 3 rotating frames x
//                      QSEG segments
constexpr int CTL_SLOTS = 32;
constexpr int CTL_FIELDS = 8;
constexpr int CTL_PAD = 32;
constexpr int QSEG = 32;                            // survivor-queue segments
constexpr int K1_TILE = 1024;                       // queue sizing unit: pixels of a 128-thread CTA
constexpr int K1_PX_PER_THREAD = 4;                 // pixels per thread of the stage-0/1 kernel
__host__ __device__ constexpr int ctl_slot(int buf, int f, int s)
{
    return ((buf * CTL_FIELDS + f) * CTL_SLOTS + s) * CTL_PAD;
}
constexpr int CTL_TOT_WORD = 3 * CTL_FIELDS * CTL_SLOTS * CTL_PAD;   // 24576
constexpr int CTL_ERR_WORD = CTL_TOT_WORD + 32;
constexpr int CTL_QCNT_WORD = CTL_ERR_WORD + 32;
__host__ __device__ constexpr int ctl_qcnt(int buf, int seg) { return CTL_QCNT_WORD + (buf * QSEG + seg) * CTL_PAD; }
constexpr int CTL_BYTES = ((CTL_QCNT_WORD + 3 * QSEG * CTL_PAD) * 4 + 4095) / 4096 * 4096;

// device error codes (bit flags in the error word)
constexpr uint32_t DERR_TMA_TIMEOUT = 1u;

// Everything a kernel needs, passed by value.
struct DevParams {
    int64_t P;          // pixels
    int K;
    unsigned flags;
    float alpha, lam2, T_bg, w_init, var_init, var_min, var_max;
    float tau_fd, eta, c_halt, w_illum;
    int q_null;
    int illum_permille;
    float c_skip;
    int skip_period;
    int kde_bits;       // 8: one prior level per byte; 4: two per byte
};

struct StatePtrs {
    uint32_t *ctl;
    uint32_t *jl;       // previous frame RGB + label byte
    void *conf;         // confidence plane
    uint8_t *s1;        // stage-1 records: m0 m1 m2 v0 v1 v2, qa | qb << 8
    uint8_t *gmm;       // mixture records
    uint4 *queue;       // survivor queue (scratch): QSEG segments of qseg_cap entries
    int64_t qseg_cap;   // entries per segment: every CTA of the first kernel
                        // puts up to K1_TILE survivors into segment
                        // blockIdx % QSEG, so a segment holds
                        // ceil(CTAs / QSEG) whole tiles
    uint8_t *kde;       // prior, [P][3][256] levels, or [P][3][128] nibble pairs (4-bit)
};

struct Layout {
    size_t total, ctl, jl, conf, s1, s1_bytes, gmm, rec_bytes, queue, kde, elem, kde_row;
    int64_t P, Pp;
    int64_t qseg_cap;   // survivor-queue entries per segment
};

int elem_bytes(int dtype);
int rec_bytes(int dtype, int K, bool perchan);
int s1_bytes(int dtype);
bool make_layout(const cog_params &p, Layout &L);

struct ApplyArgs {
    DevParams dp;
    StatePtrs s;
    const uint8_t *frame;
    uint8_t *mask;
    uint8_t *stagemap;   // may be null
    uint32_t frame_no;   // frames applied since training (mod 3)
    uint32_t frame_idx;  // frames applied since training (sampling phase)
    uint32_t frame_al4;  // frame pointer 4-byte aligned: 32-bit frame loads
    uint32_t out_al4;    // mask (and stage map) 4-byte aligned: 32-bit stores
    uint32_t k2_grid;    // CTAs of the persistent mixture-stage kernel
    uint32_t rec_bytes;  // bytes of one mixture record (for L2 prefetches)
};

// A batch group: streams sharing one storage type and K, run by one launch
// of each kernel.  Descriptors live in device memory so that a captured
// graph stays valid while frame buffers change.  The host rewrites the
// step plan (active flags and the two prefixes, one upload) whenever the
// set of streams with a frame changes: only those streams get work.
struct BatchGroupDev {
    ApplyArgs *descs;        // [n], frame_no field = frames applied % 3
    uint32_t *frame_no;      // [n] frames applied (full count)
    const uint32_t *active;  // [n] 1 = the stream has a frame this step
    const uint32_t *k1_pre;  // [n + 1] prefix of the active streams' stage-0/1 tiles
                             //         (an inactive stream has width 0)
    const uint32_t *k2_pre;  // [n + 1] prefix of the mixture-stage CTAs given to the
                             //         active streams (in proportion to their pixels)
    int n;
    int mv;                  // mixture variant of the group's streams: 0 shared
                             // weights, 1 per-channel (COG_PERCHAN), 2 stage 1 as
                             // the rank-1 mode (COG_MODE1)
};

// The mixture variant a stream's flags select (BatchGroupDev::mv).
__host__ __device__ inline int mix_variant(unsigned flags)
{
    return (flags & COG_PERCHAN) ? 1 : ((flags & COG_MODE1) ? 2 : 0);
}

// Launch shape of the two cascade kernels.
struct LaunchCfg {
    int k1_tpb = 128;   // stage-0/1 CTA size: 64, 128 or 256 (4 pixels per thread)
    int k2_tpb = 64;    // mixture-stage CTA size: 64 or 128
    int k2_per_sm = 0;  // mixture-stage CTAs per SM (0: as many as fit)
};

cudaError_t launch_batch_advance(const BatchGroupDev &g, cudaStream_t st);

// ---- clip of consecutive frames in one cooperative launch
constexpr int CLIP_TMAX = 32;          // frames per launch (their flags fit one word)
constexpr int CLIP_SLOTS = 8;          // counter slots per (frame, field)
constexpr uint32_t DERR_GRID_TIMEOUT = 2u;   // a grid-wide wait of the clip kernel gave up
constexpr uint32_t DERR_CLIP_RUNS = 4u;      // the clip kernel's reruns did not converge
constexpr uint32_t DERR_BOUNDS = 8u;         // COG_DEBUG build: an index failed its bounds check

// COG_DEBUG build (a sanitizer substitute): the data-dependent indices of
// the kernels (survivor-queue slots, pixels taken from queue entries and
// shared lists, batch streams and tiles) are checked before each access.
// The first failed check writes its site, index and limit into the words
// from CTL_DBG_WORD (site, index low/high, limit low/high); every failure
// sets DERR_BOUNDS, and the access is skipped.
constexpr int CTL_DBG_WORD = CTL_ERR_WORD + 8;
enum DbgSite : uint32_t {
    DBG_K1_LIST = 1,      // stage-1 list entry of a CTA (< pixels of the CTA)
    DBG_K1_PIXEL = 2,     // pixel of a stage-1 list entry (< P)
    DBG_K1_QUEUE = 3,     // survivor-queue write (< segment capacity)
    DBG_K2_QUEUE = 4,     // survivor-queue read (< the segment's written length)
    DBG_K2_PIXEL = 5,     // pixel of a queue entry (< P)
    DBG_BATCH_STREAM = 6, // batch stream of a tile or mixture CTA (< streams)
    DBG_BATCH_TILE = 7,   // a stream's stage-0/1 tile (first pixel < P)
    DBG_CLIP_ENTRY = 8,   // clip survivor entry: warp area and slot
    DBG_CLIP_PIXEL = 9,   // clip survivor pixel (< P)
    DBG_PLAIN_TILE = 10,  // plain mixture tile (first pixel < P)
};
// per-frame counters of a run: 3 banks (runs rotate) x CLIP_TMAX frames x
// CTL_FIELDS fields x CLIP_SLOTS slots, each slot on its own 128-byte line
__host__ __device__ constexpr int clip_cnt_word(int bank, int t, int f, int s)
{
    return (((bank * CLIP_TMAX + t) * CTL_FIELDS + f) * CLIP_SLOTS + s) * CTL_PAD;
}
constexpr int CLIP_CNT_WORDS = 3 * CLIP_TMAX * CTL_FIELDS * CLIP_SLOTS * CTL_PAD;
// sync words: [0] barrier arrivals; [CLIP_TILE_WORD + 32 b] tile counter of
// bank b; [CLIP_RUNS_WORD] runs used, [+1] bank of the final run, [+2] the
// flags the final run used
constexpr int CLIP_TILE_WORD = 32;
constexpr int CLIP_RUNS_WORD = 128;
constexpr int CLIP_SYNC_WORDS = 256;

struct ClipArgs {
    DevParams dp;
    StatePtrs s;
    const uint8_t *frames;    // [T][P][3]
    uint8_t *masks;           // [T][P]
    uint8_t *stagemaps;       // [T][P] or null
    uint32_t *undo_jl;        // clip-start copies of the planes
    void *undo_conf;
    uint8_t *undo_s1;
    uint8_t *undo_gmm;        // original mixture records of touched pixels
    uint32_t *touched;        // 1 bit per pixel: record saved in undo_gmm
    uint32_t *cnt;            // CLIP_CNT_WORDS
    uint32_t *sync;           // CLIP_SYNC_WORDS
    uint32_t T;               // frames in this clip, 1..CLIP_TMAX
    uint32_t frame_idx0;      // frames applied before the clip (sampling phase)
    uint32_t frame_mod3;      // the same count mod 3 (control-block buffers)
    uint32_t frame_al4, out_al4;
    uint32_t n_tiles;         // set by the launcher
};

// Optional per-kernel timing: events recorded before the first kernel,
// between the two kernels and after the second, on the launch stream.
struct ApplyEvents {
    cudaEvent_t e0, e1, e2;
};

// launchers (return the launch error)
cudaError_t launch_apply(int dtype, int K, const ApplyArgs &a, cudaStream_t st);
cudaError_t launch_plain_gmm(int dtype, int K, const DevParams &dp, const StatePtrs &s,
                             const uint8_t *frame, uint8_t *mask, cudaStream_t st);
cudaError_t launch_kde_train(const DevParams &dp, const StatePtrs &s, const uint8_t *frames,
                             int n_frames, const uint32_t *g, int R, cudaStream_t st);
cudaError_t launch_warmup(int dtype, int K, const DevParams &dp, const StatePtrs &s,
                          const uint8_t *frames, int n_frames, int r1, int r2, cudaStream_t st);

}  // namespace cog
