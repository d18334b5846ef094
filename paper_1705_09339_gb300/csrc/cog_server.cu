// cog_server.cu -- native continuous-batching frame server (host code).
//
// Many camera streams share one GPU.  Callers submit host frames from any
// thread; a worker thread repeatedly takes, while fewer than
// MAX_STEPS_IN_FLIGHT steps are on the GPU, for every stream that has a
// frame waiting and a free device slot (two per stream), the oldest frame,
// uploads those frames on a copy stream, runs one batched cascade step over
// exactly those streams (cog_batch_apply_active: one replay of one captured
// CUDA graph) and downloads their masks on a second copy stream.  Frames
// that arrive while a step is on the GPU join the next step, whose uploads
// overlap the running step.  A completion thread waits for each step's
// downloads and records every frame's latency from submission to its mask
// being in host memory.  Every wait is bounded by a condition-variable
// timeout or by a CUDA event of work already enqueued (polled, then waited
// for in short naps).  Cameras can join and leave a running server: between
// steps, once no step is on the GPU, the worker rebuilds the batch over the
// contexts that remain.  A leaving camera's submitted frames are completed
// first; its stream index is given to the next camera that joins, so the
// other cameras keep theirs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "cog_internal.h"

namespace cog {
int64_t ctx_pixels(const cog_ctx *c);   // pixels per frame of a context (cog_api.cu)
}

namespace {

using clk = std::chrono::steady_clock;

// Steps on the GPU at once.  Every step carries fixed costs (copies issued,
// plan upload, graph launch, completion), so a step per arriving frame
// cannot keep up with thousands of frames per second.  With a few steps in
// flight the GPU stays busy, and frames that arrive meanwhile gather into
// the next, larger step.
constexpr int MAX_STEPS_IN_FLIGHT = 4;

// The completion thread polls a step's event for up to this long before it
// blocks: a blocking wait's wake-up costs about a millisecond, which with a
// few steps in flight would bound the steps per second.  Past the spell
// (an idle server) it sleeps in short naps instead of spinning a core.
constexpr auto COMPLETION_SPIN = std::chrono::microseconds(3000);

// GPU-side timing of a step: events on the copy and compute streams
//   0 uploads start, 1 uploads done (up stream),
//   2 batched step starts, 3 batched step done (compute stream),
//   4 downloads start, 5 downloads done (down stream)
constexpr int STEP_TIMERS = 6;
// Floats per completed step in the step record: 3 host times, 5 GPU times,
// the frames of the step and the megabytes it uploaded
constexpr int STEP_RECORD = 10;

struct Pending {
    const uint8_t *frame;   // host, height x width x 3
    uint8_t *mask;          // host, height x width
    clk::time_point t;      // submission
    uint64_t seq;           // per-stream sequence number
};

struct Stream {
    cog_ctx *ctx = nullptr;                  // nullptr: the camera left (index free)
    bool leaving = false;                    // cog_server_remove called: no new frames
    int64_t P = 0;
    uint8_t *slot[2] = {nullptr, nullptr};   // device frame slots
    uint8_t *mslot[2] = {nullptr, nullptr};  // device mask slots
    std::deque<Pending> pending;
    int inflight = 0;
    uint64_t seq = 0;
};

struct Pick {
    int stream;
    Pending f;
    clk::time_point t_pick;   // when the worker took the frame for a step
};

struct Step {
    cudaEvent_t done = nullptr;              // completion (from the server's event pool)
    cudaEvent_t tm[STEP_TIMERS] = {};        // timing events (from the timing pool)
    float host_parts[3] = {0.f, 0.f, 0.f};   // host time issuing uploads, batched step, downloads
    std::vector<Pick> picks;
};

// A camera joining a running server: its context and device slots, handed
// to the worker, which rebuilds the batch between steps.
struct AddReq {
    cog_ctx *ctx = nullptr;
    Stream q;
    int index = -1;
    cog_status st = COG_OK;
    bool done = false;
    char msg[256] = {0};
};

// A camera leaving: taken by the worker once its stream has no frame waiting
// or on the GPU.
struct LeaveReq {
    int index = -1;
    cog_ctx *ctx = nullptr;   // the context handed back
    cog_status st = COG_OK;
    bool done = false;
    char msg[256] = {0};
};

}  // namespace

struct cog_server {
    int device = 0;
    cog_batch *batch = nullptr;
    cudaStream_t compute = nullptr, up = nullptr, down = nullptr;
    cudaEvent_t copied = nullptr, applied = nullptr;
    std::vector<Stream> streams;
    std::vector<cog_ctx *> ctxs;         // the batch's contexts, in stream order
    std::vector<int> bpos;               // stream index -> position in the batch (-1: left)
    std::deque<AddReq *> adds;           // cameras waiting to join (owned by their callers)
    std::deque<LeaveReq *> leaves;       // cameras waiting to leave (owned by their callers)
    std::condition_variable cv_added;    // join and leave requests handled
    std::mutex mu;                       // streams' queues, counts, statistics, adds
    std::condition_variable cv_work;     // work arrived or a slot freed
    std::condition_variable cv_idle;     // a step completed
    std::mutex dmu;
    std::condition_variable cv_done;
    std::deque<Step> done_q;
    std::vector<cudaEvent_t> ev_pool;    // step-completion events ready for reuse (under dmu)
    std::vector<cudaEvent_t> tm_pool;    // timing events ready for reuse (under dmu)
    std::vector<cudaEvent_t> ev_all;     // every event the pools ever made (freed with the server)
    bool stop = false, worker_done = false;
    std::thread worker, completer;
    std::vector<float> lat_ms;
    std::vector<float> sub_ms;           // submission time of each done frame, since creation
    std::vector<float> wait_ms;          // submission -> taken by the worker, per done frame
    std::vector<float> enq_ms;           // per step issued: host time to issue it
    std::vector<float> step_parts_ms;    // per step completed: STEP_RECORD floats
    int64_t frames = 0, pixels = 0, steps = 0, submitted = 0;
    int steps_in_flight = 0;             // issued and not yet completed (under mu)
    clk::time_point t0;
    cog_status sticky = COG_OK;
    char err[512] = {0};
};

static thread_local char g_server_err[512];

static cog_status server_err(cog_server *s, cog_status st, const char *fmt, ...)
{
    char *dst = s ? s->err : g_server_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    if (s && st != COG_OK && st != COG_ERR_INVALID_ARG) s->sticky = st;
    return st;
}

// A leave request whose stream has nothing waiting and nothing on the GPU.
static bool leave_ready(const cog_server *s, const LeaveReq *l)
{
    const Stream &q = s->streams[l->index];
    return q.pending.empty() && q.inflight == 0;
}

// Fails the waiting join requests and the leave requests in `which` (all
// of them when null).  A leave that fails leaves its camera serving.
static void fail_members(cog_server *s, cog_status st, const char *why, const std::vector<LeaveReq *> *which = nullptr)
{
    for (AddReq *a : s->adds) {
        a->st = st;
        a->done = true;
        snprintf(a->msg, sizeof a->msg, "%s", why);
    }
    s->adds.clear();
    std::deque<LeaveReq *> keep;
    for (LeaveReq *l : s->leaves) {
        if (which && std::find(which->begin(), which->end(), l) == which->end()) {
            keep.push_back(l);
            continue;
        }
        l->st = st;
        l->done = true;
        snprintf(l->msg, sizeof l->msg, "%s", why);
        s->streams[l->index].leaving = false;
    }
    s->leaves.swap(keep);
    s->cv_added.notify_all();
}

// Stream index -> position in the batch, from the streams' contexts.
static void rebuild_positions(cog_server *s)
{
    s->ctxs.clear();
    s->bpos.assign(s->streams.size(), -1);
    for (size_t i = 0; i < s->streams.size(); i++)
        if (s->streams[i].ctx) {
            s->bpos[i] = (int)s->ctxs.size();
            s->ctxs.push_back(s->streams[i].ctx);
        }
}

// Takes the waiting joins and the leaves whose streams are drained (called
// by the worker with s->mu held): waits, at most 30 s, until no step is on
// the GPU, rebuilds the batch over the cameras that stay and those that
// join, frees the leaving streams' slots and gives each joining camera the
// lowest free stream index (else the next one).  On failure the old batch
// and membership stay and the requests carry the error.
static void server_rebuild(cog_server *s, std::unique_lock<std::mutex> &lk)
{
    // the requests are read again after every wait: a caller whose own
    // time limit ran out meanwhile has withdrawn its request
    auto ready = [&] {
        std::vector<LeaveReq *> v;
        for (LeaveReq *l : s->leaves)
            if (leave_ready(s, l)) v.push_back(l);
        return v;
    };
    if (s->adds.empty() && ready().empty()) return;
    const clk::time_point until = clk::now() + std::chrono::seconds(30);
    while (s->steps_in_flight > 0 && s->sticky == COG_OK) {
        if (s->cv_idle.wait_until(lk, until) == std::cv_status::timeout && s->steps_in_flight > 0) {
            const std::vector<LeaveReq *> go = ready();
            fail_members(s, COG_ERR_TIMEOUT, "the running steps did not finish within 30 s", &go);
            return;
        }
    }
    const std::vector<LeaveReq *> go = ready();
    if (s->adds.empty() && go.empty()) return;
    if (s->sticky != COG_OK) {
        fail_members(s, s->sticky, "the server failed");
        return;
    }
    // the new membership: streams that stay, then the joining cameras in
    // the free indices, lowest first
    std::vector<cog_ctx *> keep(s->streams.size(), nullptr);
    for (size_t i = 0; i < s->streams.size(); i++) keep[i] = s->streams[i].ctx;
    for (LeaveReq *l : go) keep[l->index] = nullptr;
    std::vector<int> where;
    for (AddReq *a : s->adds) {
        int idx = -1;
        for (size_t i = 0; i < keep.size() && idx < 0; i++)
            if (!keep[i]) idx = (int)i;
        if (idx < 0) {
            idx = (int)keep.size();
            keep.push_back(nullptr);
        }
        keep[idx] = a->ctx;
        where.push_back(idx);
    }
    std::vector<cog_ctx *> all;
    for (cog_ctx *c : keep)
        if (c) all.push_back(c);
    if (all.empty()) {
        fail_members(s, COG_ERR_INVALID_ARG, "the last camera cannot leave", &go);
        return;
    }
    cog_batch *nb = nullptr;
    const cog_status st = cog_batch_create(all.data(), (int32_t)all.size(), s->compute, &nb);
    if (st != COG_OK) {
        fail_members(s, st, cog_batch_last_error_string(nullptr), &go);
        return;
    }
    cog_batch_destroy(s->batch);   // idle: every step that used it has completed
    s->batch = nb;
    for (LeaveReq *l : go) {
        Stream &q = s->streams[l->index];
        for (int k = 0; k < 2; k++) {
            if (q.slot[k]) cudaFree(q.slot[k]);
            if (q.mslot[k]) cudaFree(q.mslot[k]);
        }
        l->ctx = q.ctx;
        q = Stream();
        l->done = true;
        s->leaves.erase(std::remove(s->leaves.begin(), s->leaves.end(), l), s->leaves.end());
    }
    if (s->streams.size() < keep.size()) s->streams.resize(keep.size());
    for (size_t j = 0; j < s->adds.size(); j++) {
        AddReq *a = s->adds[j];
        s->streams[where[j]] = std::move(a->q);
        s->streams[where[j]].ctx = a->ctx;
        a->q = Stream();
        a->index = where[j];
        a->done = true;
    }
    s->adds.clear();
    rebuild_positions(s);
    s->cv_added.notify_all();
}

// A failed join is the caller's error, not the server's: the message is
// recorded without making the server's status sticky.
static cog_status add_err(cog_server *s, cog_status st, const char *fmt, ...)
{
    std::lock_guard<std::mutex> lk(s->mu);
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->err, sizeof s->err, fmt, ap);
    va_end(ap);
    return st;
}

// An event from a pool (under dmu), or a new one recorded in ev_all.
static cudaError_t pool_event(cog_server *s, std::vector<cudaEvent_t> &pool, unsigned flags, cudaEvent_t *out)
{
    {
        std::lock_guard<std::mutex> lk(s->dmu);
        if (!pool.empty()) {
            *out = pool.back();
            pool.pop_back();
            return cudaSuccess;
        }
    }
    const cudaError_t e = cudaEventCreateWithFlags(out, flags);
    if (e != cudaSuccess) {
        *out = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lk(s->dmu);
    s->ev_all.push_back(*out);
    return cudaSuccess;
}

static void server_worker(cog_server *s)
{
    cudaSetDevice(s->device);
    // per batch position
    std::vector<const uint8_t *> frames;
    std::vector<uint8_t *> masks;
    std::vector<uint8_t> active;
    for (;;) {
        std::vector<Pick> picks;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                bool member = !s->adds.empty();
                for (const LeaveReq *l : s->leaves) member = member || leave_ready(s, l);
                if (member && !s->stop) server_rebuild(s, lk);
                const int n = (int)s->streams.size();
                frames.resize(s->ctxs.size(), nullptr);
                masks.resize(s->ctxs.size(), nullptr);
                active.resize(s->ctxs.size(), 0);
                if (s->steps_in_flight < MAX_STEPS_IN_FLIGHT) {
                    for (int i = 0; i < n; i++) {
                        Stream &q = s->streams[i];
                        if (!q.pending.empty() && q.inflight < 2) {
                            picks.push_back({i, q.pending.front(), clk::time_point{}});
                            q.pending.pop_front();
                            q.inflight++;
                        }
                    }
                }
                if (!picks.empty() || s->stop || s->sticky != COG_OK) break;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
            if (picks.empty()) break;   // stopping, nothing left to start
            s->steps_in_flight++;
        }
        const clk::time_point t_pick = clk::now();
        for (Pick &k : picks) k.t_pick = t_pick;
        cudaError_t e = cudaSuccess;
        Step step;
        for (int k = 0; k < STEP_TIMERS && e == cudaSuccess; k++) e = pool_event(s, s->tm_pool, cudaEventDefault, &step.tm[k]);
        if (e == cudaSuccess) e = cudaEventRecord(step.tm[0], s->up);
        std::fill(active.begin(), active.end(), 0);
        for (const Pick &k : picks) {
            Stream &q = s->streams[k.stream];
            const int sl = (int)(k.f.seq & 1), b = s->bpos[k.stream];
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(q.slot[sl], k.f.frame, (size_t)q.P * 3, cudaMemcpyHostToDevice, s->up);
            frames[b] = q.slot[sl];
            masks[b] = q.mslot[sl];
            active[b] = 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(step.tm[1], s->up);
        if (e == cudaSuccess) e = cudaEventRecord(s->copied, s->up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->compute, s->copied, 0);
        if (e == cudaSuccess) e = cudaEventRecord(step.tm[2], s->compute);
        const clk::time_point t_up = clk::now();
        cog_status st = COG_OK;
        if (e == cudaSuccess) st = cog_batch_apply_active(s->batch, frames.data(), masks.data(), active.data());
        const clk::time_point t_app = clk::now();
        if (e == cudaSuccess && st == COG_OK) e = cudaEventRecord(step.tm[3], s->compute);
        if (e == cudaSuccess && st == COG_OK) e = cudaEventRecord(s->applied, s->compute);
        if (e == cudaSuccess && st == COG_OK) e = cudaStreamWaitEvent(s->down, s->applied, 0);
        if (e == cudaSuccess && st == COG_OK) e = cudaEventRecord(step.tm[4], s->down);
        for (const Pick &k : picks) {
            Stream &q = s->streams[k.stream];
            if (e == cudaSuccess && st == COG_OK)
                e = cudaMemcpyAsync(k.f.mask, q.mslot[k.f.seq & 1], (size_t)q.P, cudaMemcpyDeviceToHost, s->down);
        }
        if (e == cudaSuccess && st == COG_OK) e = cudaEventRecord(step.tm[5], s->down);
        step.picks = std::move(picks);
        // events come from pools that grow to the number of steps ever in
        // flight at once and are reused
        if (e == cudaSuccess && st == COG_OK) e = pool_event(s, s->ev_pool, cudaEventDisableTiming, &step.done);
        if (e == cudaSuccess && st == COG_OK) e = cudaEventRecord(step.done, s->down);
        const clk::time_point t_end = clk::now();
        step.host_parts[0] = std::chrono::duration<float, std::milli>(t_up - t_pick).count();
        step.host_parts[1] = std::chrono::duration<float, std::milli>(t_app - t_up).count();
        step.host_parts[2] = std::chrono::duration<float, std::milli>(t_end - t_app).count();
        if (e != cudaSuccess || st != COG_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            if (st != COG_OK) server_err(s, st, "batched step: %s", cog_batch_last_error_string(s->batch));
            else server_err(s, COG_ERR_CUDA, "batched step: %s", cudaGetErrorString(e));
            for (const Pick &k : step.picks) s->streams[k.stream].inflight--;
            s->steps_in_flight--;
            s->cv_idle.notify_all();
            break;
        }
        {
            std::lock_guard<std::mutex> lk(s->dmu);
            s->done_q.push_back(std::move(step));
        }
        s->cv_done.notify_one();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->steps++;
            s->enq_ms.push_back(std::chrono::duration<float, std::milli>(t_end - t_pick).count());
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_members(s, s->sticky != COG_OK ? s->sticky : COG_ERR_STATE, "the server is stopping");
    }
    {
        std::lock_guard<std::mutex> lk(s->dmu);
        s->worker_done = true;
    }
    s->cv_done.notify_one();
}

static void server_completer(cog_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        Step step;
        {
            std::unique_lock<std::mutex> lk(s->dmu);
            while (s->done_q.empty() && !s->worker_done) s->cv_done.wait_for(lk, std::chrono::milliseconds(50));
            if (s->done_q.empty()) break;
            step = std::move(s->done_q.front());
            s->done_q.pop_front();
        }
        // poll the step's event (a finished step is noticed within
        // microseconds), then nap between polls once the spell is over
        cudaError_t e;
        const clk::time_point t_wait = clk::now();
        while ((e = cudaEventQuery(step.done)) == cudaErrorNotReady) {
            if (clk::now() - t_wait < COMPLETION_SPIN) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        const clk::time_point now = clk::now();
        // GPU times of the step: uploads, wait until the compute stream took
        // it, batched step, wait until the download stream took it, downloads
        float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (e == cudaSuccess)
            for (int k = 0; k < 5; k++)
                if (cudaEventElapsedTime(&g[k], step.tm[k], step.tm[k + 1]) != cudaSuccess) g[k] = -1.f;
        {
            std::lock_guard<std::mutex> lk(s->dmu);
            s->ev_pool.push_back(step.done);
            for (int k = 0; k < STEP_TIMERS; k++) s->tm_pool.push_back(step.tm[k]);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (e != cudaSuccess) server_err(s, COG_ERR_CUDA, "step completion: %s", cudaGetErrorString(e));
            s->steps_in_flight--;
            s->step_parts_ms.insert(s->step_parts_ms.end(), step.host_parts, step.host_parts + 3);
            s->step_parts_ms.insert(s->step_parts_ms.end(), g, g + 5);
            int64_t up_bytes = 0;
            for (const Pick &k : step.picks) up_bytes += s->streams[k.stream].P * 3;
            s->step_parts_ms.push_back((float)step.picks.size());
            s->step_parts_ms.push_back((float)((double)up_bytes / 1e6));
            for (const Pick &k : step.picks) {
                Stream &q = s->streams[k.stream];
                q.inflight--;
                s->frames++;
                s->pixels += q.P;
                s->lat_ms.push_back(std::chrono::duration<float, std::milli>(now - k.f.t).count());
                s->sub_ms.push_back(std::chrono::duration<float, std::milli>(k.f.t - s->t0).count());
                s->wait_ms.push_back(std::chrono::duration<float, std::milli>(k.t_pick - k.f.t).count());
            }
        }
        s->cv_work.notify_one();
        s->cv_idle.notify_all();
    }
}

static void server_free(cog_server *s)
{
    for (Stream &q : s->streams)
        for (int k = 0; k < 2; k++) {
            if (q.slot[k]) cudaFree(q.slot[k]);
            if (q.mslot[k]) cudaFree(q.mslot[k]);
        }
    if (s->batch) cog_batch_destroy(s->batch);
    for (cudaEvent_t ev : s->ev_all) cudaEventDestroy(ev);
    if (s->copied) cudaEventDestroy(s->copied);
    if (s->applied) cudaEventDestroy(s->applied);
    for (cudaStream_t st : {s->compute, s->up, s->down})
        if (st) cudaStreamDestroy(st);
    delete s;
}

extern "C" {

cog_status cog_server_create(cog_ctx *const *ctxs, int32_t n, cog_server **out)
{
    if (!out) return server_err(nullptr, COG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return server_err(nullptr, COG_ERR_INVALID_ARG, "need n >= 1 contexts");
    cog_server *s = new (std::nothrow) cog_server();
    if (!s) return server_err(nullptr, COG_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->applied, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        server_err(nullptr, COG_ERR_CUDA, "server streams: %s", cudaGetErrorString(e));
        server_free(s);
        return COG_ERR_CUDA;
    }
    cog_status st = cog_batch_create(ctxs, n, s->compute, &s->batch);
    if (st != COG_OK) {
        server_err(nullptr, st, "batch: %s", cog_batch_last_error_string(nullptr));
        s->batch = nullptr;
        server_free(s);
        return st;
    }
    s->ctxs.assign(ctxs, ctxs + n);
    s->streams.resize((size_t)n);
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        const int64_t P = cog::ctx_pixels(ctxs[i]);
        Stream &q = s->streams[i];
        q.ctx = ctxs[i];
        q.P = P;
        for (int k = 0; k < 2 && e == cudaSuccess; k++) {
            e = cudaMalloc((void **)&q.slot[k], (size_t)P * 3);
            if (e == cudaSuccess) e = cudaMalloc((void **)&q.mslot[k], (size_t)P);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        server_err(nullptr, COG_ERR_OOM, "server slots: %s", cudaGetErrorString(e));
        server_free(s);
        return COG_ERR_OOM;
    }
    rebuild_positions(s);
    s->t0 = clk::now();
    s->worker = std::thread(server_worker, s);
    s->completer = std::thread(server_completer, s);
    *out = s;
    return COG_OK;
}

cog_status cog_server_submit(cog_server *s, int32_t stream, const uint8_t *frame_host, uint8_t *mask_host)
{
    if (!s) return COG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->sticky != COG_OK) return s->sticky;
        if (stream < 0 || stream >= (int32_t)s->streams.size() || !frame_host || !mask_host)
            return server_err(s, COG_ERR_INVALID_ARG, "stream index out of range or NULL buffer");
        if (s->stop) return server_err(s, COG_ERR_STATE, "server is stopping");
        Stream &q = s->streams[stream];
        if (!q.ctx || q.leaving)
            return server_err(s, COG_ERR_INVALID_ARG, "stream %d has left the server or is leaving", stream);
        q.pending.push_back({frame_host, mask_host, clk::now(), q.seq++});
        s->submitted++;
    }
    s->cv_work.notify_one();
    return COG_OK;
}

cog_status cog_server_add(cog_server *s, cog_ctx *ctx, int32_t *stream_out)
{
    if (!s || !ctx || !stream_out) return COG_ERR_INVALID_ARG;
    AddReq req;
    req.ctx = ctx;
    req.q.P = cog::ctx_pixels(ctx);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaMalloc((void **)&req.q.slot[k], (size_t)req.q.P * 3);
        if (e == cudaSuccess) e = cudaMalloc((void **)&req.q.mslot[k], (size_t)req.q.P);
    }
    auto free_slots = [&] {
        for (int k = 0; k < 2; k++) {
            if (req.q.slot[k]) cudaFree(req.q.slot[k]);
            if (req.q.mslot[k]) cudaFree(req.q.mslot[k]);
            req.q.slot[k] = req.q.mslot[k] = nullptr;
        }
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_slots();
        return add_err(s, COG_ERR_OOM, "slots of the joining camera: %s", cudaGetErrorString(e));
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop || s->sticky != COG_OK) {
        lk.unlock();
        free_slots();
        return add_err(s, COG_ERR_STATE, "the server is stopping or failed");
    }
    bool dup = std::find(s->ctxs.begin(), s->ctxs.end(), ctx) != s->ctxs.end();
    for (const AddReq *a : s->adds) dup = dup || a->ctx == ctx;
    if (dup) {
        lk.unlock();
        free_slots();
        return add_err(s, COG_ERR_INVALID_ARG, "the context already belongs to the server");
    }
    s->adds.push_back(&req);
    s->cv_work.notify_all();
    const clk::time_point until = clk::now() + std::chrono::seconds(60);
    while (!req.done) {
        if (s->cv_added.wait_until(lk, until) == std::cv_status::timeout && !req.done) {
            s->adds.erase(std::remove(s->adds.begin(), s->adds.end(), &req), s->adds.end());
            lk.unlock();
            free_slots();
            return add_err(s, COG_ERR_TIMEOUT, "the worker did not take the camera within 60 s");
        }
    }
    lk.unlock();
    if (req.st != COG_OK) {
        free_slots();
        return add_err(s, req.st, "camera join failed: %s", req.msg);
    }
    *stream_out = req.index;
    return COG_OK;
}

cog_status cog_server_remove(cog_server *s, int32_t stream, cog_ctx **ctx_out)
{
    if (!s) return COG_ERR_INVALID_ARG;
    if (ctx_out) *ctx_out = nullptr;
    LeaveReq req;
    req.index = stream;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop || s->sticky != COG_OK) {
        lk.unlock();
        return add_err(s, COG_ERR_STATE, "the server is stopping or failed");
    }
    if (stream < 0 || stream >= (int32_t)s->streams.size() || !s->streams[stream].ctx ||
        s->streams[stream].leaving) {
        lk.unlock();
        return add_err(s, COG_ERR_INVALID_ARG, "stream %d is not a camera of the server", stream);
    }
    s->streams[stream].leaving = true;
    s->leaves.push_back(&req);
    s->cv_work.notify_all();
    const clk::time_point until = clk::now() + std::chrono::seconds(60);
    while (!req.done) {
        if (s->cv_added.wait_until(lk, until) == std::cv_status::timeout && !req.done) {
            s->leaves.erase(std::remove(s->leaves.begin(), s->leaves.end(), &req), s->leaves.end());
            s->streams[stream].leaving = false;
            lk.unlock();
            return add_err(s, COG_ERR_TIMEOUT, "stream %d did not leave within 60 s", stream);
        }
    }
    lk.unlock();
    if (req.st != COG_OK) return add_err(s, req.st, "camera leave failed: %s", req.msg);
    if (ctx_out) *ctx_out = req.ctx;
    return COG_OK;
}

cog_status cog_server_drain(cog_server *s, int32_t timeout_ms)
{
    if (!s || timeout_ms < 0) return COG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const clk::time_point until = clk::now() + std::chrono::milliseconds(timeout_ms);
    while (s->frames < s->submitted && s->sticky == COG_OK) {
        if (s->cv_idle.wait_until(lk, until) == std::cv_status::timeout && s->frames < s->submitted)
            return server_err(s, COG_ERR_TIMEOUT, "drain: %lld of %lld frames done after %d ms",
                              (long long)s->frames, (long long)s->submitted, timeout_ms);
    }
    return s->sticky;
}

// Linear-interpolated quantile q of v (sorted in place); 0 when empty.
static double quantile(std::vector<float> &v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double r = q * (double)(v.size() - 1);
    const size_t i = (size_t)r;
    const double f = r - (double)i;
    return i + 1 < v.size() ? (1.0 - f) * v[i] + f * v[i + 1] : (double)v[i];
}

cog_status cog_server_read_stats(cog_server *s, cog_server_stats *out)
{
    if (!s || !out) return COG_ERR_INVALID_ARG;
    std::vector<float> lat, wait, svc, enq;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        memset(out, 0, sizeof *out);
        out->frames = s->frames;
        out->steps = s->steps;
        out->pixels = s->pixels;
        out->submitted = s->submitted;
        out->wall_s = std::chrono::duration<double>(clk::now() - s->t0).count();
        lat = s->lat_ms;
        wait = s->wait_ms;
        enq = s->enq_ms;
    }
    svc.resize(lat.size());
    for (size_t i = 0; i < lat.size(); i++) svc[i] = lat[i] - wait[i];
    out->p50_ms = quantile(lat, 0.50);
    out->p99_ms = quantile(lat, 0.99);
    out->max_ms = lat.empty() ? 0.0 : lat.back();
    out->wait_p50_ms = quantile(wait, 0.50);
    out->wait_p99_ms = quantile(wait, 0.99);
    out->service_p50_ms = quantile(svc, 0.50);
    out->service_p99_ms = quantile(svc, 0.99);
    out->enqueue_p99_ms = quantile(enq, 0.99);
    out->enqueue_max_ms = enq.empty() ? 0.0 : enq.back();
    return s->sticky;
}

cog_status cog_server_read_latencies(cog_server *s, float *submit_ms, float *latency_ms, int64_t cap, int64_t *n)
{
    return cog_server_read_timeline(s, submit_ms, nullptr, latency_ms, cap, n);
}

cog_status cog_server_read_timeline(cog_server *s, float *submit_ms, float *wait_ms, float *latency_ms, int64_t cap,
                                    int64_t *n)
{
    if (!s || !n || cap < 0 || (cap > 0 && (!submit_ms || !latency_ms))) return COG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t m = std::min<int64_t>(cap, (int64_t)s->lat_ms.size());
    if (m > 0) {
        memcpy(submit_ms, s->sub_ms.data(), sizeof(float) * (size_t)m);
        memcpy(latency_ms, s->lat_ms.data(), sizeof(float) * (size_t)m);
        if (wait_ms) memcpy(wait_ms, s->wait_ms.data(), sizeof(float) * (size_t)m);
    }
    *n = (int64_t)s->lat_ms.size();
    return COG_OK;
}

cog_status cog_server_read_steps(cog_server *s, float *enqueue_ms, float *parts_ms, int64_t cap, int64_t *n)
{
    if (!s || !n || cap < 0 || (cap > 0 && !enqueue_ms)) return COG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t done = (int64_t)(s->step_parts_ms.size() / STEP_RECORD);
    const int64_t m = std::min<int64_t>(cap, done);
    if (m > 0) {
        memcpy(enqueue_ms, s->enq_ms.data(), sizeof(float) * (size_t)std::min<int64_t>(m, (int64_t)s->enq_ms.size()));
        if (parts_ms) memcpy(parts_ms, s->step_parts_ms.data(), sizeof(float) * STEP_RECORD * (size_t)m);
    }
    *n = done;
    return COG_OK;
}

cog_status cog_server_reset_stats(cog_server *s)
{
    if (!s) return COG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->frames != s->submitted || s->steps_in_flight)
        return server_err(s, COG_ERR_STATE, "reset_stats: frames are still in flight (drain first)");
    s->frames = s->pixels = s->steps = s->submitted = 0;
    s->lat_ms.clear();
    s->sub_ms.clear();
    s->wait_ms.clear();
    s->enq_ms.clear();
    s->step_parts_ms.clear();
    s->t0 = clk::now();
    return s->sticky;
}

const char *cog_server_last_error_string(cog_server *s)
{
    return s ? s->err : g_server_err;
}

cog_status cog_server_destroy(cog_server *s)
{
    if (!s) return COG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->completer.joinable()) s->completer.join();
    const cog_status st = s->sticky;
    cudaStreamSynchronize(s->down);
    server_free(s);
    return st;
}

}  // extern "C"
