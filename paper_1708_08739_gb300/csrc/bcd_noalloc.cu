// RV(r) without any allocation: a single-root reach traversal of R(G) whose
// scratch lives in a file-scope device array.
//
// Some callers cannot call cudaMalloc: code that runs while an allocator is
// locked or being torn down, processes whose device memory is fully carved
// out by another framework's caching allocator, and plugins that are handed a
// stream and caller-owned buffers but no allocation rights. This entry point
// serves them: the caller passes the reverse graph and the output buffer as
// device pointers, and the call uses only the static array below.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "bcd.h"
#include "bcd_common.cuh"

namespace {

constexpr int32_t kMaxN = BC_NOALLOC_MAX_VERTICES;
constexpr int kThreads = 512;

struct NoallocScratch {
    uint32_t visited[kMaxN / 32];   // one bit per vertex
    int32_t queue[2][kMaxN];        // frontier of the current / next level
    int64_t block_count[1024];      // per-block counts for the ordered output
    uint32_t qlen[2];               // frontier sizes
    uint32_t bar_count;
    uint32_t bar_gen;
    int32_t err;
    int32_t pad;
    int64_t total;
};

// The scratch array. Every call shares it and leaves its contents behind.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of a cooperative launch; every wait gives up after timeout_ns.
__device__ bool grid_sync(NoallocScratch *s, uint32_t &gen) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t arrived = atomicAdd(&s->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&s->bar_count, 0u);
            __threadfence();
            atomicExch(&s->bar_gen, gen + 1);
        } else {
            const unsigned long long t0 = now_ns();
            unsigned long long spins = 0;
            while (*(volatile uint32_t *)&s->bar_gen == gen) {
                if (*(volatile int32_t *)&s->err) break;
                if ((++spins & 63) == 0 && now_ns() - t0 > 10000000000ull) {
                    atomicCAS(&s->err, 0, 1);
                    break;
                }
                if (spins > (1ull << 31)) {
                    atomicCAS(&s->err, 0, 1);
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        gen += 1;
        ok = *(volatile int32_t *)&s->err == 0;
    }
    __syncthreads();
    return ok;
}

__global__ void __launch_bounds__(kThreads) rv_noalloc_kernel(NoallocScratch *s, const int64_t *roff,
                                                               const int32_t *rcol, int32_t n, int32_t r,
                                                               int32_t *out, int64_t cap) {
    uint32_t gen = 0;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int words = (n + 31) / 32;
    for (long long i = tid; i < words; i += nthr) s->visited[i] = 0u;
    if (tid == 0) {
        s->qlen[0] = 1;
        s->qlen[1] = 0;
        s->queue[0][0] = r;
    }
    if (!grid_sync(s, gen)) return;
    if (tid == 0) atomicOr(&s->visited[r >> 5], 1u << (r & 31));
    if (!grid_sync(s, gen)) return;
    int cur = 0;
    // level-synchronous BFS over R(G); one warp per frontier vertex
    for (;;) {
        const uint32_t len = *(volatile uint32_t *)&s->qlen[cur];
        const long long gw = tid >> 5, nw = nthr >> 5;
        for (long long i = gw; i < len; i += nw) {
            const int32_t x = __ldcg(&s->queue[cur][i]);
            const long long b = roff[x], e = roff[x + 1];
            for (long long a = b + lane; a < e; a += 32) {
                const int32_t y = rcol[a];
                const uint32_t bit = 1u << (y & 31);
                if (!(s->visited[y >> 5] & bit)) {
                    const uint32_t old = atomicOr(&s->visited[y >> 5], bit);
                    if (!(old & bit)) {
                        const uint32_t pos = atomicAdd(&s->qlen[cur ^ 1], 1u);
                        s->queue[cur ^ 1][pos] = y;
                    }
                }
            }
        }
        if (!grid_sync(s, gen)) return;
        const uint32_t next = *(volatile uint32_t *)&s->qlen[cur ^ 1];
        if (next == 0) break;
        if (tid == 0) s->qlen[cur] = 0;
        if (!grid_sync(s, gen)) return;
        cur ^= 1;
    }
    // ordered output: per-block bit counts, one-block scan, per-block writes
    const long long per = (words + gridDim.x - 1) / gridDim.x;
    const long long w0 = (long long)blockIdx.x * per, w1 = min((long long)words, w0 + per);
    __shared__ long long s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (long long w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        uint32_t x = __ldcg(&s->visited[w]);
        if (w == (r >> 5)) x &= ~(1u << (r & 31));
        atomicAdd((unsigned long long *)&s_cnt, (unsigned long long)__popc(x));
    }
    __syncthreads();
    if (threadIdx.x == 0) s->block_count[blockIdx.x] = s_cnt;
    if (!grid_sync(s, gen)) return;
    if (tid == 0) {
        long long run = 0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            const long long c = __ldcg(&s->block_count[b]);
            s->block_count[b] = run;
            run += c;
        }
        s->total = run;
    }
    if (!grid_sync(s, gen)) return;
    const long long total = *(volatile long long *)&s->total;
    if (total > cap) return;
    // each block writes its words in order; one warp walks the block's range
    if (threadIdx.x < 32) {
        long long base = __ldcg(&s->block_count[blockIdx.x]);
        for (long long w0b = w0; w0b < w1; w0b += 32) {
            const long long w = w0b + lane;
            uint32_t x = w < w1 ? __ldcg(&s->visited[w]) : 0u;
            if (w == (r >> 5)) x &= ~(1u << (r & 31));
            const int c = __popc(x);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            long long pos = base + incl - c;
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1;
                out[pos++] = (int32_t)(w * 32 + b);
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
NoallocScratch *g_addr[64] = {nullptr};
int g_grid[64] = {0};

}  // namespace

extern "C" bc_status bc_rv_compute_noalloc(const int64_t *d_roffsets, const int32_t *d_rcols, int32_t n,
                                           int32_t r, int32_t *d_out, int64_t cap, int64_t *count,
                                           void *stream) {
    if (!d_roffsets || !d_rcols || !count || (cap > 0 && !d_out))
        return bcd::set_error(BC_E_INVALID_ARG, "bc_rv_compute_noalloc: NULL argument");
    if (n <= 0 || n > kMaxN)
        return bcd::set_error(BC_E_INVALID_ARG,
                              "bc_rv_compute_noalloc: n must be in [1, BC_NOALLOC_MAX_VERTICES = 4194304]");
    if (r < 0 || r >= n) return bcd::set_error(BC_E_INVALID_ARG, "bc_rv_compute_noalloc: vertex out of range");
    if (cap < 0) return bcd::set_error(BC_E_INVALID_ARG, "bc_rv_compute_noalloc: negative capacity");
    int dev = 0;
    BCD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return bcd::set_error(BC_E_INTERNAL, "bc_rv_compute_noalloc: device index above 63");
    NoallocScratch *s = nullptr;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            BCD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            int sms = 0, per_sm = 0;
            BCD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            BCD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rv_noalloc_kernel, kThreads, 0));
            if (per_sm < 1) return bcd::set_error(BC_E_INTERNAL, "bc_rv_compute_noalloc: kernel cannot be resident");
            g_grid[dev] = sms < 1024 ? sms : 1024;
            g_addr[dev] = (NoallocScratch *)p;
        }
        s = g_addr[dev];
        grid = g_grid[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    BCD_CUDA(cudaMemsetAsync(&s->qlen, 0, sizeof(uint32_t) * 4 + sizeof(int32_t) * 2, st));
    void *args[] = {(void *)&s, (void *)&d_roffsets, (void *)&d_rcols, (void *)&n, (void *)&r, (void *)&d_out,
                    (void *)&cap};
    BCD_CUDA(cudaLaunchCooperativeKernel((const void *)rv_noalloc_kernel, dim3(grid), dim3(kThreads), args, 0, st));
    int64_t total = 0;
    int32_t err = 0;
    BCD_CUDA(cudaMemcpyAsync(&total, &s->total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCD_CUDA(cudaMemcpyAsync(&err, &s->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BCD_CUDA(cudaStreamSynchronize(st));
    if (err) return bcd::set_error(BC_E_TIMEOUT, "bc_rv_compute_noalloc: a grid barrier wait timed out");
    *count = total;
    if (total > cap) return bcd::set_error(BC_E_BUFFER_TOO_SMALL, "bc_rv_compute_noalloc: output capacity below |RV(r)|");
    return BC_OK;
}
