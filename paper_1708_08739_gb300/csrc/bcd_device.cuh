// Device helpers shared by the traversal kernels: bounded grid barrier,
// chunk descriptors and their dynamic hand-out, per-query tile sums.
#pragma once

#include "bcd_common.cuh"

namespace bcd {
namespace dev {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int32_t ld_vol(const int32_t *p) { return *(volatile const int32_t *)p; }

__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long *p) {
    return *(volatile const unsigned long long *)p;
}

__device__ __forceinline__ void set_err(Counters *c, int32_t code) { atomicCAS(&c->err, 0, code); }

// Grid-wide barrier for a cooperative launch. Every wait is bounded by
// timeout_ns of wall time (and a spin cap); on timeout or when another block
// has flagged an error, returns false and the caller leaves the kernel.
__device__ inline bool grid_barrier(Counters *c, uint32_t &gen, double timeout_ns) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t nb = gridDim.x;
        const uint32_t arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == nb - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicExch(&c->bar_gen, gen + 1);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned long long spins = 0;
            while (ld_acquire(&c->bar_gen) == gen) {
                if (ld_vol(&c->err) != 0) break;
                ++spins;
                if ((double)(global_ns() - t0) > timeout_ns) {
                    set_err(c, kDevTimeout);
                    break;
                }
                if (spins > (1ull << 31)) {
                    set_err(c, kDevTimeout);
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        gen += 1;
        s_err = ld_vol(&c->err);
    }
    __syncthreads();
    return s_err == 0;
}

// Start of a tile: thread 0 of each block reads the host's cancel request
// (bc_cancel); a request makes every block leave at the barrier that
// follows, the same way as any other error.
__device__ __forceinline__ void check_cancel(const TravParams &p) {
    if (threadIdx.x == 0 && p.cancel && *(volatile const int32_t *)p.cancel != 0) set_err(p.ctr, kDevCancelled);
}

template <int W>
__device__ __forceinline__ bool mask_bit(const uint64_t (&m)[W], int s) {
    return (m[s >> 6] >> (s & 63)) & 1ull;
}

// Dynamic hand-out of a level's chunks to warps: lane 0 grabs `grab`
// consecutive chunks with one atomic, so warps that drew cheap chunks take
// more and the level ends evenly.
struct ChunkGrabber {
    unsigned long long *ctr;
    long long ccnt, grab, cur, end;
    __device__ ChunkGrabber(unsigned long long *c, long long n, long long nwarps)
        : ctr(c), ccnt(n), grab(max(1ll, n / (nwarps * 8))), cur(0), end(0) {}
    __device__ __forceinline__ bool next(long long &c, int lane) {
        if (cur >= end) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(ctr, (unsigned long long)grab);
            b = __shfl_sync(kFull, b, 0);
            if ((long long)b >= ccnt) return false;
            cur = (long long)b;
            end = min(ccnt, (long long)b + grab);
        }
        c = cur++;
        return true;
    }
};

__device__ __forceinline__ Chunk load_chunk(const Chunk *c) {
    const int4 a = reinterpret_cast<const int4 *>(c)[0];
    const int4 b = reinterpret_cast<const int4 *>(c)[1];
    Chunk r;
    r.v = a.x;
    r.e = a.y;
    r.k = a.z;
    r.nch = a.w;
    r.a0 = (int64_t)(((unsigned long long)(unsigned)b.y << 32) | (unsigned)b.x);
    r.na = b.z;
    r.pad = b.w;
    return r;
}

__device__ __forceinline__ void store_chunk(Chunk *c, int v, int e, int k, int nch, long long a0, int na,
                                            int kind = 0) {
    int4 *d = reinterpret_cast<int4 *>(c);
    d[0] = make_int4(v, e, k, nch);
    d[1] = make_int4((int)(unsigned)(a0 & 0xffffffffll), (int)(unsigned)((unsigned long long)a0 >> 32), na, kind);
}

// Writes the chunk descriptors of a vertex with arcs [rb, re); the last
// field carries the row's length (the vertex's out-degree).
__device__ __forceinline__ void emit_chunks(const TravParams &p, long long c0, int v, int e, int nch, long long rb,
                                            long long re) {
    const int CH = p.chunk_arcs;
    for (int kk = 0; kk < nch; ++kk) {
        const long long a0 = rb + (long long)kk * CH;
        const long long a1 = min(re, a0 + CH);
        store_chunk(&p.chunks[c0 + kk], v, e, kk, nch, a0, (int)max(0ll, a1 - a0), (int)(re - rb));
    }
}

// Per-query partial sums of a tile's dependencies (one block): eight threads
// per query, each over every eighth source slot, combined by a fixed shuffle
// tree, so the order does not depend on scheduling. The multiplicity of a
// source is 1 (exact queries: the query needs it) or its draw count.
__device__ inline void tile_query_sums(const TravParams &p, long long tile, int S, const int32_t *tsrc,
                                       const uint64_t *s_need) {
    for (int t = threadIdx.x; t < 64 * 8; t += blockDim.x) {
        const int q = t >> 3, j = t & 7;
        const bool exact = (p.exact_q >> q) & 1ull;
        double sum = 0.0;
        int flagged = 0;
        for (int s = j; s < S; s += 8) {
            if (tsrc[s] < 0) continue;
            double mlt = 0.0;
            if (exact)
                mlt = ((s_need[s] >> q) & 1ull) ? 1.0 : 0.0;
            else if (p.mult)
                mlt = (double)p.mult[((size_t)tile * S + s) * 64 + q];
            if (mlt != 0.0) {
                sum += mlt * p.dep[s * 64 + q];
                if ((p.srcflag[s >> 6] >> (s & 63)) & 1ull) flagged = 1;
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            sum += __shfl_down_sync(kFull, sum, o, 8);
            flagged |= __shfl_down_sync(kFull, flagged, o, 8);
        }
        if (j == 0) {
            p.tile_partial[tile * 64 + q] = sum;
            if (flagged) p.qflags[q] |= 1u;
        }
    }
}

}  // namespace dev
}  // namespace bcd
