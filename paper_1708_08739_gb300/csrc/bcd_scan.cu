// Device-wide exclusive scan and ordered compaction (three passes: per-tile
// totals, one-block scan of the totals, per-tile scan and write).
#include "bcd_common.cuh"
#include "bcd_scan.cuh"

namespace bcd {

namespace {

constexpr int kScanThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kScanThreads * kItems;

__device__ __forceinline__ bool pick(const uint64_t *m, int bit, long long v) {
    const uint64_t x = m[v];
    return bit >= 0 ? ((x >> bit) & 1ull) != 0ull : x != 0ull;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total.
__device__ long long block_exclusive(long long x, long long *total) {
    __shared__ long long s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (kScanThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kScanThreads / 32)) s_warp[lane] = w;
    }
    __syncthreads();
    const long long wbase = wid > 0 ? s_warp[wid - 1] : 0;
    *total = s_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return wbase + inc - x;
}

__global__ void __launch_bounds__(kScanThreads) tile_sum(const int64_t *in, int64_t len, int64_t *bsum) {
    const long long b0 = (long long)blockIdx.x * kTile;
    long long x = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const long long i = b0 + (long long)threadIdx.x * kItems + k;
        if (i < len) x += in[i];
    }
    long long tot;
    block_exclusive(x, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) tile_count(const uint64_t *m, int bit, int64_t n, int64_t *bsum) {
    const long long b0 = (long long)blockIdx.x * kTile;
    long long x = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const long long i = b0 + (long long)threadIdx.x + (long long)k * kScanThreads;
        if (i < n && pick(m, bit, i)) ++x;
    }
    long long tot;
    block_exclusive(x, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block: exclusive scan of nb totals in place; grand total to *total.
__global__ void __launch_bounds__(kScanThreads) scan_totals(int64_t *bsum, int64_t nb, int64_t *total) {
    long long carry = 0;
    for (long long base = 0; base < nb; base += kScanThreads) {
        const long long i = base + threadIdx.x;
        const long long x = i < nb ? bsum[i] : 0;
        long long tot;
        const long long ex = block_exclusive(x, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) tile_apply(const int64_t *in, int64_t len, const int64_t *boff,
                                                           int64_t *out) {
    const long long b0 = (long long)blockIdx.x * kTile;
    long long v[kItems];
    long long x = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const long long i = b0 + (long long)threadIdx.x * kItems + k;
        v[k] = i < len ? in[i] : 0;
        x += v[k];
    }
    long long tot;
    long long run = boff[blockIdx.x] + block_exclusive(x, &tot);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const long long i = b0 + (long long)threadIdx.x * kItems + k;
        if (i < len) out[i] = run;
        run += v[k];
    }
}

// Items are strided by the block width so warp ballots see consecutive ids;
// a rank among earlier ids in the tile is the sum over earlier rounds plus the
// rank inside the current round.
__global__ void __launch_bounds__(kScanThreads) tile_scatter(const uint64_t *m, int bit, int64_t n,
                                                             const int64_t *boff, int32_t *out, int32_t *pos) {
    const long long b0 = (long long)blockIdx.x * kTile;
    long long base = boff[blockIdx.x];
    for (int k = 0; k < kItems; ++k) {
        const long long i = b0 + (long long)threadIdx.x + (long long)k * kScanThreads;
        const bool p = i < n && pick(m, bit, i);
        long long tot;
        const long long ex = block_exclusive(p ? 1 : 0, &tot);
        if (p) {
            out[base + ex] = (int32_t)i;
            if (pos) pos[i] = (int32_t)(base + ex);
        }
        base += tot;
    }
}

}  // namespace

int64_t scan_scratch_len(int64_t len) { return (len + kTile - 1) / kTile + 2; }

bc_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t len, cudaStream_t s, int64_t *scratch,
                             int64_t scratch_cap) {
    const int64_t nb = (len + kTile - 1) / kTile;
    int64_t *tmp = scratch;
    bool own = false;
    if (!tmp || scratch_cap < scan_scratch_len(len)) {
        BCD_TRY(dev_alloc(&tmp, (size_t)scan_scratch_len(len)));
        own = true;
    }
    if (nb > 0) {
        tile_sum<<<(unsigned)nb, kScanThreads, 0, s>>>(in, len, tmp);
        scan_totals<<<1, kScanThreads, 0, s>>>(tmp, nb, out + len);
        tile_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, len, tmp, out);
    } else {
        BCD_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    }
    cudaError_t e = cudaGetLastError();
    if (own) {
        cudaStreamSynchronize(s);
        dev_free(tmp);
    }
    if (e != cudaSuccess) return cuda_error(e, "scan kernels");
    return BC_OK;
}

bc_status compact_mask(const uint64_t *masks, int bit, int64_t n, int32_t *out, int32_t *pos, int64_t *d_count,
                       cudaStream_t s, int64_t *scratch, int64_t scratch_cap) {
    const int64_t nb = (n + kTile - 1) / kTile;
    if (!scratch || scratch_cap < scan_scratch_len(n)) return set_error(BC_E_INTERNAL, "compact_mask: scratch too small");
    tile_count<<<(unsigned)nb, kScanThreads, 0, s>>>(masks, bit, n, scratch);
    scan_totals<<<1, kScanThreads, 0, s>>>(scratch, nb, d_count);
    tile_scatter<<<(unsigned)nb, kScanThreads, 0, s>>>(masks, bit, n, scratch, out, pos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "compaction kernels");
    return BC_OK;
}

}  // namespace bcd
