// cog_selftest.cu -- self-test of the bounded grid-wide wait that the clip
// kernel's barriers use (a wait on a count that nothing completes must give
// up after its time limit, report through the error word and leave the
// device usable), and the streaming probe that times the memory floor of a
// stage-0-sized pass.
#include "cog_clip.cuh"

namespace cog {

// [0] barrier arrivals, [1] error word; no allocation needed
static __device__ uint32_t g_selftest_words[2];

// One CTA waits at a barrier whose target (two arrivals) its single arrival
// can never reach.
__global__ void wait_selftest_kernel(uint32_t *words, uint64_t limit_ns)
{
    clip_grid_sync(words, 2u, words + 1, limit_ns);
}

cudaError_t run_wait_selftest(uint64_t limit_ns, uint32_t *error_word, float *elapsed_ms)
{
    uint32_t *w = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&w, g_selftest_words);
    if (e != cudaSuccess) return e;
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    e = cudaMemsetAsync(w, 0, 2 * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>(w, limit_ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(error_word, w + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaEventElapsedTime(elapsed_ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    return e;
}

// Streaming probe: the loads and stores of stage 0 for a group of 4 pixels
// whose every pixel passes (16 B previous frame + labels, 8 B confidence,
// 12 B frame in; 16 B, 8 B and 4 B out), with no arithmetic between them.
__global__ void __launch_bounds__(128) probe_stream_kernel(const uint4 *jl_in, const uint2 *conf_in,
                                                           const uint32_t *frame, uint4 *jl_out, uint2 *conf_out,
                                                           uint32_t *mask, int64_t groups)
{
    const int64_t g = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (g >= groups) return;
    const uint4 j = jl_in[g];
    const uint2 c = conf_in[g];
    const uint32_t w0 = frame[3 * g], w1 = frame[3 * g + 1], w2 = frame[3 * g + 2];
    uint4 o;
    o.x = (w0 & 0x00ffffffu) | (j.x & 0xff000000u);
    o.y = (__byte_perm(w0, w1, 0x0543) & 0x00ffffffu) | (j.y & 0xff000000u);
    o.z = (__byte_perm(w1, w2, 0x0432) & 0x00ffffffu) | (j.z & 0xff000000u);
    o.w = (w2 >> 8) | (j.w & 0xff000000u);
    jl_out[g] = o;
    conf_out[g] = c;
    mask[g] = __byte_perm(__byte_perm(j.x, j.y, 0x0073), __byte_perm(j.z, j.w, 0x0073), 0x5410);
}

cudaError_t launch_probe_stream(const uint32_t *jl_in, const uint16_t *conf_in, const uint8_t *frame,
                                uint32_t *jl_out, uint16_t *conf_out, uint8_t *mask, int64_t P, cudaStream_t st)
{
    const int64_t groups = P / 4;
    probe_stream_kernel<<<(unsigned)((groups + 127) / 128), 128, 0, st>>>(
        reinterpret_cast<const uint4 *>(jl_in), reinterpret_cast<const uint2 *>(conf_in),
        reinterpret_cast<const uint32_t *>(frame), reinterpret_cast<uint4 *>(jl_out),
        reinterpret_cast<uint2 *>(conf_out), reinterpret_cast<uint32_t *>(mask), groups);
    return cudaGetLastError();
}

}  // namespace cog
