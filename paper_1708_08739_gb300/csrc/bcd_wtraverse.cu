// Weighted single-source work (Section 2 with positive integer weights, the
// SPD of each source) for a tile of 64 sources: exact distances by Dial's
// bucket order, sigma by a pull over tight in-arcs, and the dependencies of
// Eq. 4 by a pull over tight out-arcs.
//
// Distances are integers, so processing distance values in increasing order
// settles every (vertex, source) pair once: a relaxation lowers
// dist[w][s] with atomicMin and queues w in the ring slot of its new
// tentative distance (ring size a power of two above the largest weight, one
// queued-bit per vertex and slot); when the slot's distance comes up, the
// vertex is settled for exactly the sources whose distance equals it.
// sigma_s(v) is pulled over in-arcs (u, v) with dist_s(u) + w(u, v) =
// dist_s(v) (all such u are settled earlier), summed by warp trees and fp64
// atomic adds of integers (exact below 2^53). The backward pass walks the
// non-empty distance levels from the deepest, with arc (v, w) tight for s when
// dist_s(v) + w(v, w) = dist_s(w), summing c_s(w) = (1 + delta_s(w)) /
// sigma_s(w) in a fixed order per chunk and chunks in chunk order.
//
// Sources settle a vertex at many different distances, so a tile entry
// usually carries one or two sources: lanes map to arcs, and the sources of
// an entry are looped over.
#include "bcd_common.cuh"
#include "bcd_device.cuh"

namespace bcd {

namespace {

using namespace dev;

constexpr int WS = 64;  // sources per weighted tile

struct WStats {
    unsigned edges = 0, reached = 0, tight = 0, arcs = 0, vb = 0, eb = 0;
};

__device__ __forceinline__ void wflush(Counters *c, WStats &st, int lane) {
    unsigned long long v[6] = {st.edges, st.reached, st.tight, st.arcs, st.vb, st.eb};
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(kFull, v[i], o);
    if (lane == 0) {
        unsigned long long *dst[6] = {&c->edges, &c->reached, &c->tight, &c->arc_visits, &c->vb, &c->eb};
#pragma unroll
        for (int i = 0; i < 6; ++i)
            if (v[i]) atomicAdd(dst[i], v[i]);
    }
    st = WStats();
}

// Butterfly sum over the warp: every lane gets the same, order-fixed result.
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ void wqueue(const TravParams &p, int w, unsigned long long nd) {
    const int slot = (int)(nd & (unsigned long long)(p.ring - 1));
    uint32_t *qb = p.qbits + (size_t)w * (p.ring >> 5) + (slot >> 5);
    const uint32_t bit = 1u << (slot & 31);
    if (!(atomicOr(qb, bit) & bit)) {
        const unsigned long long pos = atomicAdd(&p.bcount[slot], 1ull);
        if ((long long)pos < p.bcap)
            p.buckets[(size_t)slot * p.bcap + pos] = w;
        else
            set_err(p.ctr, kDevHistOverflow);
    }
}

__global__ void __launch_bounds__(512, 2) wtrav_kernel(TravParams p) {
    extern __shared__ __align__(16) double s_wacc_all[];
    const int lane = threadIdx.x & 31;
    const long long wpb = blockDim.x >> 5;
    const long long gwarp = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    const long long nwarps = (long long)gridDim.x * wpb;
    double *wacc = s_wacc_all + (threadIdx.x >> 5) * WS;
    __shared__ uint64_t s_need[WS];
    __shared__ int32_t s_minql[WS];
    __shared__ uint64_t s_active;
    __shared__ int32_t s_lstop;
    __shared__ long long s_next;
    uint32_t gen = 0;
    WStats st;
    const int R = p.ring;
    const int stride = p.vs_stride;
    const int CH = p.chunk_arcs;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_mark = timer ? global_ns() : 0ull;
    unsigned long long ns_fwd = 0, ns_bwd = 0, ns_other = 0;
    for (int s = lane; s < WS; s += 32) wacc[s] = 0.0;

    for (long long tile = 0; tile < p.ntiles; ++tile) {
        const int32_t *tsrc = p.srcs + tile * WS;
        if (blockIdx.x == 0) {
            const int t = threadIdx.x;
            if (t < WS) {
                const int v = tsrc[t];
                if (v >= 0) {
                    p.dist[(size_t)v * WS + t] = 0ull;
                    p.sigma[(size_t)v * WS + t] = 1.0;
                    wqueue(p, v, 0ull);
                }
            }
            for (int i = t; i < WS * 64; i += blockDim.x) p.qlevel[i] = -1;
            if (t == 0) p.srcflag[0] = 0ull;
        }
        for (int s = threadIdx.x; s < WS; s += blockDim.x) {
            const int32_t v = tsrc[s];
            s_need[s] = v >= 0 ? p.need[v] : 0ull;
        }
        if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_other += t - t_mark;
            t_mark = t;
        }

        // ---------------- forward: settle distance levels in order ----------------
        long long d = 0, es = 0, pes = 0, pcnt = 0;
        int seg = 0;
        for (;;) {
            if (threadIdx.x == 0) {
                long long dn = -1;
                for (int k = 0; k < R; ++k)
                    if (ld_vol(&p.bcount[(d + k) & (R - 1)]) > 0ull) {
                        dn = d + k;
                        break;
                    }
                s_next = dn;
            }
            __syncthreads();
            const long long dn = s_next;
            __syncthreads();
            if (dn < 0) break;
            if (seg + 2 > p.maxlev) {
                if (threadIdx.x == 0) set_err(p.ctr, kDevLevelOverflow);
                return;
            }
            d = dn;
            const int slot = (int)(d & (R - 1));
            const long long cnt = (long long)ld_vol(&p.bcount[slot]);
            // settle the queued vertices whose distance for some source is d
            for (long long i = gwarp; i < cnt; i += nwarps) {
                const int x = p.buckets[(size_t)slot * p.bcap + i];
                if (lane == 0) atomicAnd(&p.qbits[(size_t)x * (R >> 5) + (slot >> 5)], ~(1u << (slot & 31)));
                const unsigned long long d0 = p.dist[(size_t)x * WS + lane];
                const unsigned long long d1 = p.dist[(size_t)x * WS + lane + 32];
                const unsigned b0 = __ballot_sync(kFull, d0 == (unsigned long long)d);
                const unsigned b1 = __ballot_sync(kFull, d1 == (unsigned long long)d);
                const uint64_t vis = p.vs[(size_t)x * stride];
                const uint64_t F = ((uint64_t)b0 | ((uint64_t)b1 << 32)) & ~vis;
                if (F == 0ull) continue;
                const long long rb = p.off[x], re = p.off[x + 1];
                const long long irb = p.roff[x], ire = p.roff[x + 1];
                const int nout = (int)max(1ll, (re - rb + CH - 1) / CH);
                const int nin = d > 0 ? (int)((ire - irb + CH - 1) / CH) : 0;
                if (lane == 0) {
                    p.vs[(size_t)x * stride] = vis | F;
                    const long long e = es + (long long)atomicAdd(&p.lev_cnt[seg], 1ull);
                    const long long c0 = (long long)atomicAdd(&p.lev_ccnt[seg], (unsigned long long)(nout + nin));
                    if (e >= p.hcap) {
                        set_err(p.ctr, kDevHistOverflow);
                    } else if (c0 + nout + nin > p.ccap) {
                        set_err(p.ctr, kDevChunkOverflow);
                    } else {
                        p.hv[e] = x;
                        p.hm[e] = F;
                        for (int kk = 0; kk < nout; ++kk) {
                            const long long a0 = rb + (long long)kk * CH;
                            store_chunk(&p.chunks[c0 + kk], x, (int)e, kk, nout, a0, (int)max(0ll, min(re, a0 + CH) - a0), 0);
                        }
                        for (int kk = 0; kk < nin; ++kk) {
                            const long long a0 = irb + (long long)kk * CH;
                            store_chunk(&p.chunks[c0 + nout + kk], x, (int)e, kk, nin, a0, (int)(min(ire, a0 + CH) - a0), 1);
                        }
                    }
                    const unsigned pc = (unsigned)__popcll(F);
                    st.reached += pc;
                    st.edges += pc * (unsigned)(re - rb);
                    if (vis == 0ull) {
                        st.vb += 1;
                        st.eb += (unsigned)(re - rb);
                    }
                }
                const uint64_t qm = p.qmask[x];
                if (qm) {
#pragma unroll
                    for (int ii = 0; ii < 2; ++ii) {
                        const int s = lane + 32 * ii;
                        if ((F >> s) & 1ull) {
                            uint64_t y = qm & s_need[s];
                            while (y) {
                                const int q = __ffsll((long long)y) - 1;
                                y &= y - 1;
                                p.qlevel[s * 64 + q] = seg;
                            }
                        }
                    }
                }
            }
            // sigma of the previous level is complete: check it against 2^53
            for (long long e = pes + gwarp; e < pes + pcnt; e += nwarps) {
                const int v = p.hv[e];
                const uint64_t F = p.hm[e];
#pragma unroll
                for (int ii = 0; ii < 2; ++ii) {
                    const int s = lane + 32 * ii;
                    if (((F >> s) & 1ull) && p.sigma[(size_t)v * WS + s] >= 9007199254740992.0)
                        atomicOr((unsigned long long *)&p.srcflag[0], 1ull << s);
                }
            }
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
            const long long ecnt = (long long)ld_vol(&p.lev_cnt[seg]);
            const long long ccnt = (long long)ld_vol(&p.lev_ccnt[seg]);
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                p.lev_start[seg] = es;
                p.lev_dist[seg] = d;
                p.bcount[slot] = 0ull;
            }
            // relax out-arcs (kind 0) and pull sigma over in-arcs (kind 1)
            ChunkGrabber grab(&p.lev_grab[seg], ccnt, nwarps);
            long long c;
            while (grab.next(c, lane)) {
                const Chunk ch = load_chunk(&p.chunks[c]);
                const uint64_t F = p.hm[ch.e];
                if (ch.pad == 0) {
                    for (int base = 0; base < ch.na; base += 32) {
                        const long long idx = ch.a0 + base + lane;
                        if (base + lane < ch.na) {
                            const int w = p.col[idx];
                            const unsigned long long nd = (unsigned long long)d + p.wt[idx];
                            bool improved = false;
                            uint64_t y = F;
                            while (y) {
                                const int s = __ffsll((long long)y) - 1;
                                y &= y - 1;
                                unsigned long long *dp = (unsigned long long *)&p.dist[(size_t)w * WS + s];
                                if (nd < *dp) {
                                    const unsigned long long old = atomicMin(dp, nd);
                                    if (nd < old) improved = true;
                                }
                            }
                            if (improved) wqueue(p, w, nd);
                            st.arcs += 1;
                        }
                    }
                } else {
                    for (int base = 0; base < ch.na; base += 32) {
                        const long long idx = ch.a0 + base + lane;
                        const bool valid = base + lane < ch.na;
                        const int u = valid ? p.rcol[idx] : 0;
                        const unsigned long long wgt = valid ? (unsigned long long)p.rwt[idx] : 0ull;
                        if (valid) st.arcs += 1;
                        uint64_t y = F;
                        while (y) {
                            const int s = __ffsll((long long)y) - 1;
                            y &= y - 1;
                            double val = 0.0;
                            if (valid && wgt <= (unsigned long long)d &&
                                p.dist[(size_t)u * WS + s] == (unsigned long long)d - wgt) {
                                val = p.sigma[(size_t)u * WS + s];
                                st.tight += 1;
                            }
                            const double sum = warp_sum(val);
                            if (lane == 0) wacc[s] += sum;
                        }
                    }
                    __syncwarp();
                    if (lane == 0) {
                        uint64_t y = F;
                        while (y) {
                            const int s = __ffsll((long long)y) - 1;
                            y &= y - 1;
                            atomicAdd(&p.sigma[(size_t)ch.v * WS + s], wacc[s]);
                            wacc[s] = 0.0;
                        }
                    }
                    __syncwarp();
                }
            }
            if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
            pes = es;
            pcnt = ecnt;
            es += ecnt;
            ++seg;
            d += 1;
        }
        // the last level's sigma
        for (long long e = pes + gwarp; e < pes + pcnt; e += nwarps) {
            const int v = p.hv[e];
            const uint64_t F = p.hm[e];
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
                const int s = lane + 32 * ii;
                if (((F >> s) & 1ull) && p.sigma[(size_t)v * WS + s] >= 9007199254740992.0)
                    atomicOr((unsigned long long *)&p.srcflag[0], 1ull << s);
            }
        }
        const int nseg = seg;
        const long long total = es;
        if (blockIdx.x == 0) {
            for (int l = threadIdx.x; l <= nseg; l += blockDim.x) p.lev_ccnt[l] = 0ull;
            if (threadIdx.x == 0) {
                p.ctr->pslots = 0ull;
                atomicMax(&p.ctr->levels_max, (unsigned long long)(nseg > 0 ? nseg - 1 : 0));
            }
        }
        if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_fwd += t - t_mark;
            t_mark = t;
        }

        // ---------------- backward (Eq. 4) over the non-empty levels ----------------
        if (!(p.flags & kFlagNoBackward)) {
            if (threadIdx.x == 0) s_lstop = 0x7fffffff;
            __syncthreads();
            for (int s = threadIdx.x; s < WS; s += blockDim.x) {
                int mq = 0x7fffffff;
                if (tsrc[s] >= 0) {
                    if (p.flags & kFlagFullBackward) {
                        mq = 0;
                    } else {
                        uint64_t y = s_need[s];
                        while (y) {
                            const int q = __ffsll((long long)y) - 1;
                            y &= y - 1;
                            const int lv = p.qlevel[s * 64 + q];
                            if (lv >= 0 && lv < mq) mq = lv;
                        }
                    }
                }
                s_minql[s] = mq;
                atomicMin(&s_lstop, mq);
            }
            __syncthreads();
            const int lstop = s_lstop;
            for (int sg = nseg - 1; sg >= lstop && lstop < nseg; --sg) {
                if (threadIdx.x == 0) {
                    uint64_t a = 0;
                    for (int b = 0; b < WS; ++b)
                        if (s_minql[b] <= sg) a |= 1ull << b;
                    s_active = a;
                }
                __syncthreads();
                const uint64_t act = s_active;
                const long long e0 = p.lev_start[sg];
                const long long ne = (long long)p.lev_cnt[sg];
                const unsigned long long dk = (unsigned long long)p.lev_dist[sg];
                // chunks of the level's out-arcs (entries with an active source)
                for (long long base = gwarp * 32; base < ne; base += nwarps * 32) {
                    const long long e = e0 + base + lane;
                    const bool valid = base + lane < ne;
                    int v = 0, nch = 0;
                    long long rb = 0, re = 0;
                    if (valid && (p.hm[e] & act)) {
                        v = p.hv[e];
                        rb = p.off[v];
                        re = p.off[v + 1];
                        nch = (int)max(1ll, (re - rb + CH - 1) / CH);
                    }
                    int x = nch;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(kFull, x, o);
                        if (lane >= o) x += y;
                    }
                    const int tot = __shfl_sync(kFull, x, 31);
                    unsigned long long cb = 0;
                    if (lane == 0 && tot) cb = atomicAdd(&p.lev_ccnt[sg], (unsigned long long)tot);
                    cb = __shfl_sync(kFull, cb, 0);
                    if (nch) {
                        const long long c0 = (long long)cb + (x - nch);
                        if (c0 + nch > p.ccap) {
                            set_err(p.ctr, kDevChunkOverflow);
                        } else {
                            for (int kk = 0; kk < nch; ++kk) {
                                const long long a0 = rb + (long long)kk * CH;
                                store_chunk(&p.chunks[c0 + kk], v, (int)e, kk, nch, a0, (int)max(0ll, min(re, a0 + CH) - a0), 0);
                            }
                            long long sl = -1;
                            if (nch > 1) {
                                const unsigned long long b = atomicAdd(&p.ctr->pslots, (unsigned long long)nch);
                                if ((long long)(b + nch) > p.pcap)
                                    set_err(p.ctr, kDevSlotOverflow);
                                else
                                    sl = (long long)b;
                            }
                            p.hslot[e] = sl;
                        }
                    }
                }
                if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
                const long long ccnt = (long long)ld_vol(&p.lev_ccnt[sg]);
                ChunkGrabber grab(&p.lev_grab[p.maxlev + 2 + sg], ccnt, nwarps);
                long long c;
                while (grab.next(c, lane)) {
                    const Chunk ch = load_chunk(&p.chunks[c]);
                    const uint64_t F = p.hm[ch.e] & act;
                    for (int base = 0; base < ch.na; base += 32) {
                        const long long idx = ch.a0 + base + lane;
                        const bool valid = base + lane < ch.na;
                        const int w = valid ? p.col[idx] : 0;
                        const unsigned long long nd = valid ? dk + p.wt[idx] : 0ull;
                        if (valid) st.arcs += 1;
                        uint64_t y = F;
                        while (y) {
                            const int s = __ffsll((long long)y) - 1;
                            y &= y - 1;
                            double val = 0.0;
                            if (valid && p.dist[(size_t)w * WS + s] == nd) val = p.sigma[(size_t)w * WS + s];
                            const double sum = warp_sum(val);
                            if (lane == 0) wacc[s] += sum;
                        }
                    }
                    __syncwarp();
                    const long long slot0 = ch.nch > 1 ? p.hslot[ch.e] : -1;
                    bool finalize = ch.nch == 1;
                    if (ch.nch > 1) {
                        double *prow = p.partial + (size_t)(slot0 + ch.k) * WS;
                        for (int s = lane; s < WS; s += 32) {
                            __stcg(&prow[s], wacc[s]);
                            wacc[s] = 0.0;
                        }
                        __threadfence();
                        __syncwarp();
                        int prev = 0;
                        if (lane == 0) prev = atomicAdd(&p.pdone[slot0], 1);
                        prev = __shfl_sync(kFull, prev, 0);
                        if (prev == ch.nch - 1) {
                            __threadfence();
                            for (int s = lane; s < WS; s += 32) {
                                double a = 0.0;
                                for (int kk = 0; kk < ch.nch; ++kk) a += __ldcg(&p.partial[(size_t)(slot0 + kk) * WS + s]);
                                wacc[s] = a;
                            }
                            if (lane == 0) p.pdone[slot0] = 0;
                            finalize = true;
                        }
                        __syncwarp();
                    }
                    if (finalize) {
                        const uint64_t qm = p.qmask[ch.v];
                        double *row = p.sigma + (size_t)ch.v * WS;
#pragma unroll
                        for (int ii = 0; ii < 2; ++ii) {
                            const int s = lane + 32 * ii;
                            if ((F >> s) & 1ull) {
                                const double sv = row[s];
                                const double dd = sv * wacc[s];
                                row[s] = (1.0 + dd) / sv;
                                if (qm) {
                                    uint64_t y = qm & s_need[s];
                                    while (y) {
                                        const int q = __ffsll((long long)y) - 1;
                                        y &= y - 1;
                                        p.dep[s * 64 + q] = dd;
                                    }
                                }
                            }
                        }
                        __syncwarp();
                        for (int s = lane; s < WS; s += 32) wacc[s] = 0.0;
                    }
                    __syncwarp();
                }
                if (blockIdx.x == 0 && threadIdx.x == 0) p.ctr->pslots = 0ull;
                if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
            }
        }
        if (timer) {
            const unsigned long long t = global_ns();
            ns_bwd += t - t_mark;
            t_mark = t;
        }
        wflush(p.ctr, st, lane);

        // ---------------- tile end ----------------
        if (blockIdx.x == 0 && threadIdx.x < 64) {
            const int q = threadIdx.x;
            const bool exact = (p.exact_q >> q) & 1ull;
            double sum = 0.0;
            bool flagged = false;
            for (int s = 0; s < WS; ++s) {
                if (tsrc[s] < 0) continue;
                double mlt = 0.0;
                if (exact)
                    mlt = ((s_need[s] >> q) & 1ull) ? 1.0 : 0.0;
                else if (p.mult)
                    mlt = (double)p.mult[((size_t)tile * WS + s) * 64 + q];
                if (mlt != 0.0) {
                    sum += mlt * p.dep[s * 64 + q];
                    if ((p.srcflag[0] >> s) & 1ull) flagged = true;
                }
            }
            p.tile_partial[tile * 64 + q] = sum;
            if (flagged) p.qflags[q] |= 1u;
        }
        if (!(p.flags & kFlagNoReset)) {
            for (long long e = gwarp; e < total; e += nwarps) {
                const int v = p.hv[e];
                const uint64_t F = p.hm[e];
#pragma unroll
                for (int ii = 0; ii < 2; ++ii) {
                    const int s = lane + 32 * ii;
                    if ((F >> s) & 1ull) {
                        p.sigma[(size_t)v * WS + s] = 0.0;
                        p.dist[(size_t)v * WS + s] = ~0ull;
                    }
                }
                if (lane == 0) p.vs[(size_t)v * stride] = 0ull;
            }
            if (blockIdx.x == 0) {
                for (int l = threadIdx.x; l <= nseg + 1; l += blockDim.x) {
                    p.lev_cnt[l] = 0ull;
                    p.lev_ccnt[l] = 0ull;
                    p.lev_grab[l] = 0ull;
                    p.lev_grab[p.maxlev + 2 + l] = 0ull;
                }
            }
        }
        if (!grid_barrier(p.ctr, gen, p.timeout_ns)) return;
        if (timer) {
            const unsigned long long t = global_ns();
            ns_other += t - t_mark;
            t_mark = t;
        }
    }
    if (timer) {
        p.ctr->ns_fwd += ns_fwd;
        p.ctr->ns_bwd += ns_bwd;
        p.ctr->ns_other += ns_other;
    }
}

}  // namespace

bc_status launch_weighted(bc_graph *g, TravParams &p) {
    const int threads = g->block_threads;
    const size_t smem = (size_t)(threads / 32) * WS * sizeof(double);
    BCD_CUDA(cudaFuncSetAttribute((const void *)wtrav_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BCD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wtrav_kernel, threads, smem));
    if (per_sm < 1) return set_error(BC_E_INTERNAL, "weighted traversal kernel cannot be resident");
    dim3 grid((unsigned)(g->num_sms * per_sm)), block((unsigned)threads);
    void *args[] = {(void *)&p};
    BCD_CUDA(cudaLaunchCooperativeKernel((const void *)wtrav_kernel, grid, block, args, smem, g->stream));
    g->launches += 1;
    g->last_grid = (int)grid.x;
    return BC_OK;
}

}  // namespace bcd
