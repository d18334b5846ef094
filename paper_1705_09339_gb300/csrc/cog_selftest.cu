// cog_selftest.cu -- self-test of the bounded grid-wide wait that the clip
// kernel's barriers use: a wait on a count that nothing completes must give
// up after its time limit, report through the error word and leave the
// device usable.
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

}  // namespace cog
