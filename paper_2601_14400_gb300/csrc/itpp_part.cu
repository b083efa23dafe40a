// itpp_part.cu -- the per-gate merge with the table in shared memory.
//
// A gate's merge only pairs a string K with its partner QK (Sec. II.B: a
// commuting string keeps cosh(theta) of itself and sends -sinh(theta) s to QK).
// Take a window of consecutive gates whose strings act on at most a few
// sites S, and group the state by the key with the sites of S cleared: K, QK
// and every child under any gate of the window share that group.  The state
// is scattered once per window into hash partitions of that masked key (one
// streaming pass, one atomic per term on the partition's cursor), and then
// every gate of the window runs a persistent kernel that takes one partition
// at a time per CTA: the partition is staged in shared memory by bulk (TMA)
// copies, each commuting string joins its partner {K, QK} in a shared-memory
// table, one string of each pair computes both merged children, and the kept
// children of the partition are written as one contiguous segment of an
// output chunk the CTA holds (room claimed once their number is known, a
// global atomic every few partitions).  The segments, listed by the partition
// descriptors, are the partitions of the next gate of the window, so no
// scatter runs between the gates of a window.  A group holds at most 4^|S|
// terms; a partition above the staging capacity is merged in sub-passes,
// each taking the pairs of one hash class of the key with the gate's sites
// cleared, so no partition size forces a re-partition.  A gate acting on more
// sites than a window allows is a window of its own, partitioned by its pair
// key (the member of {K, QK} with the gate's lowest bit clear).
//
// The top-M select (Sec. II.C, term bound) is folded into the merge: every
// kept child is compared with a range around the threshold predicted for the
// gate; the merge counts the children above it, lists those inside it and
// leaves those below it unwritten (they are dropped by the select whenever at
// least cap_M children lie at or above the range; otherwise the merge runs
// again in full), and the select (itpp_select.cu) then works on that short
// list instead of passing over every coefficient.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"
#include "itpp_stage.cuh"

namespace itpp {

// Scatter the current state into the partitions of a window (force), or,
// inside a window, only when the previous gate's partitions hold for that
// gate alone; otherwise the next merge reads the previous merge's segments.
// The state is a contiguous run of terms, or (after a partitioned merge)
// the segments its descriptors list.
template <int W>
__device__ __forceinline__ void scatter_run(const PKey<W>* __restrict__ kin,
                                            const double* __restrict__ cin, uint64_t n,
                                            uint64_t first, uint64_t stride, const Pending<W>& pd,
                                            DevCtl* ctl, PKey<W>* pk, double* pc,
                                            unsigned int* cursor, const PartPlan& pl,
                                            const GateArg<W>& g, const PartFn<W>& f) {
    // whole warps iterate together (the cursor claim below is warp-wide);
    // U items per thread per round, their loads issued before any claim
    constexpr int U = 4;
    const unsigned int lt = (1u << (threadIdx.x & 31)) - 1u;
    for (uint64_t i0 = first; i0 < n; i0 += U * stride) {
        PKey<W> K[U];
        double c[U];
        bool live[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = i0 + (uint64_t)u * stride + threadIdx.x;
            live[u] = i < n;
            c[u] = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) { K[u].x[w] = 0; K[u].z[w] = 0; }
            if (live[u]) {
                K[u] = load_key_stream(kin + i);
                c[u] = __ldcs(cin + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (live[u] && pd.on && !cap_keep(K[u], c[u], pd.T, pd.all_ties, pd.tk)) {
                if (key_is_zero(K[u])) set_status(ctl, ST_TRACE_ZERO, 42);
                live[u] = false;
            }
            // one cursor claim per distinct partition in the warp: terms of
            // one group arrive together and would otherwise serialise on it
            const uint32_t p = live[u] ? part_of(K[u], g, f, pl.P) : 0xffffffffu;
            const unsigned int peers = __match_any_sync(0xffffffffu, p);
            const int leader = __ffs(peers) - 1;
            unsigned int base = 0;
            if (live[u] && (threadIdx.x & 31) == leader) base = atomicAdd(cursor + p, __popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (live[u]) {
                const unsigned int pos = base + __popc(peers & lt);
                if (pos < pl.R) {
                    const uint64_t d = (uint64_t)p * pl.R + pos;
                    store_key(pk + d, K[u]);
                    pc[d] = c[u];
                } else if (!f.pair) {
                    ctl->scatter_over = 1;   // the gate scatters again by its pair key
                } else {
                    set_status(ctl, ST_CAPACITY, 40);
                }
            }
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256, W == 1 ? 6 : 4)
k_part_scatter(Bufs<W> B, DevCtl* ctl, PKey<W>* pk, double* pc, unsigned int* cursor,
               uint64_t pbuf_cap, uint32_t p_max, GateArg<W> g, PartFn<W> f, int force,
               int n_sites, int target, const ChunkDesc* chunks0, const ChunkDesc* chunks1,
               int redo) {
    if (ctl->status) return;
    // the second launch of a gate's scatter runs only when the first one
    // found a partition's stride too small for the groups hashed to it; it
    // scatters by the gate's pair key (pairs always fit) into cleared cursors
    if (redo) {
        if (!ctl->scatter_over) return;
        f.pair = 1;
        force = 1;
    }
    const int cur = ctl->cur;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the next merge's counters
        ctl->count[cur ^ 1] = 0ULL;
        ctl->alloc[cur ^ 1] = 0ULL;
        ctl->nchunk[cur ^ 1] = 0u;
        ctl->sp_above = 0ULL;
        ctl->sp_ovf = 0;
    }
    if (!force && !ctl->need_scatter) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->part_from_scatter = 0;
        return;
    }
    const uint64_t n = live_count(ctl, cur);
    // The merges of a window stage each partition's stored children, which
    // hold the select's rejected ones until the predicate drops them: when
    // the previous gate stored g times the terms it kept, aim the kept terms
    // of a partition at target / g (at least target / 2) so that what the
    // next merges stage stays near the target instead of passing the staging
    // capacity.
    int t_eff = target;
    if (ctl->pend && n > 0 && ctl->pend_n > n) {
        const uint64_t t = (uint64_t)target * n / ctl->pend_n;
        t_eff = t < (uint64_t)(target / 2) ? target / 2 : (int)t;
    }
    const bool fallback = redo || (!f.pair && !window_fits(n_sites, f.sites, n));
    if (fallback) f.pair = 1;
    PartPlan pl = part_plan(n, pbuf_cap, p_max, t_eff);
    if (!f.pair) {
        // a partition's stride holds a whole group (up to 4^sites strings,
        // the terms with one pattern outside the window), however the terms
        // fall, where that keeps partitions near the target; larger windows
        // rely on the second scatter by pair key when a stride overflows
        const uint64_t gmax = 1ULL << (2 * f.sites);
        if (pl.R < gmax && gmax <= 2ULL * (uint64_t)target) {
            const uint64_t P = pbuf_cap / gmax;
            pl.P = (uint32_t)(P > 0 ? P : 1);
            pl.R = pbuf_cap / pl.P;
        }
    }
    // the chunks of the previous merge's output
    const bool seg = ctl->seg != 0;
    const uint32_t n_chunks = ctl->nchunk[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->part_from_scatter = 1;
        ctl->part_P = pl.P;
        ctl->stat_scatters += 1;
        if (fallback) ctl->part_over = 1;   // the partitions hold for this gate only
    }
    const Pending<W> pd = pending_of<W>(ctl);
    // one loop for both layouts (a single copy of the scatter body): each
    // output chunk of the previous merge by one CTA, or the contiguous run by
    // the whole grid (with a deferred top-M select every stored term is
    // scanned and its kept set applied)
    const ChunkDesc* __restrict__ cin = cur ? chunks1 : chunks0;
    uint64_t n_scan = n;
    if (!seg && pd.on) n_scan = ctl->pend_n < ctl->buf_cap ? ctl->pend_n : ctl->buf_cap;
    const uint32_t runs = seg ? n_chunks : 1u;
    for (uint32_t s = seg ? blockIdx.x : 0u; s < runs; s += seg ? gridDim.x : 1u) {
        const uint64_t off = seg ? cin[s].off : 0ULL;
        const uint64_t cnt = seg ? (uint64_t)cin[s].cnt : n_scan;
        const uint64_t first = seg ? 0ULL : (uint64_t)blockIdx.x * blockDim.x;
        const uint64_t stride = seg ? (uint64_t)blockDim.x : (uint64_t)gridDim.x * blockDim.x;
        scatter_run(B.key(cur) + off, B.coef(cur) + off, cnt, first, stride, pd, ctl, pk, pc,
                    cursor, pl, g, f);
    }
}


// Between a gate's two scatter launches: when the first found a stride too
// small, clear the cursors for the second.
__global__ void k_scatter_clear(const DevCtl* ctl, unsigned int* cursor, uint32_t p_max) {
    if (ctl->status || !ctl->scatter_over) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p_max; i += gridDim.x * blockDim.x)
        cursor[i] = 0u;
}

// The gate's merge, one partition at a time per CTA.  The partition comes
// from the scatter buffer (fixed stride, cursor) or is a segment the
// previous gate of the window wrote (descriptor).  It is copied into shared
// memory by two bulk (TMA) copies, keys and coefficients, completed on an
// mbarrier; a later partition of the same CTA has been prefetched into L2.
// One pass (stage_pass) then merges it, and its kept children go to one
// contiguous segment of the CTA's output chunk, recorded as the partition's
// descriptor for the next gate.  Chunks are claimed from the buffer's
// allocator a few hundred partitions at a time, so no partition waits on a
// global atomic.  A partition above the staging capacity is merged in
// sub-passes: each gathers the strings of one hash class of the key with
// the gate's sites cleared (which K and Q.K share) into the staging arrays.
// With a top-M bound the children below the select's predicted range are
// not written (retry_pass 0); k_merge_check then keeps that output when at
// least cap_M children were kept, and otherwise the second launch
// (retry_pass 1) merges the gate again in full from the same input.
template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (PartOcc<W, BLOCK>::kMin))
k_gate_part(const PKey<W>* __restrict__ pk, const double* __restrict__ pc,
            unsigned int* __restrict__ cursor, uint64_t pbuf_cap, PartDesc* desc0,
            PartDesc* desc1, Bufs<W> B, DevCtl* ctl, GateArg<W> g, double delta,
            uint64_t cap_out, uint64_t chunk, CandRegions cd, ChunkDesc* chunks0,
            ChunkDesc* chunks1, uint32_t max_chunks, int retry_pass) {
    using G = Stage<W>;
    using A = PassArgs<W>;
    constexpr uint32_t C = G::C, S = G::S;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ unsigned long long s_chunk, s_chsz, s_nout;
    __shared__ uint32_t s_long, s_n;
    __shared__ int s_stop;
    __shared__ Pending<W> s_pd;
    __shared__ double s_rnorm;
    __shared__ unsigned long long s_thr;   // kept: pattern above this
    const int cur = ctl->cur, nxt = cur ^ 1;
    const bool from_scatter = ctl->part_from_scatter != 0;
    const uint32_t P = ctl->part_P;
    const uint64_t R = P ? pbuf_cap / P : 0;
    const PartDesc* __restrict__ din = cur ? desc1 : desc0;
    PartDesc* __restrict__ dout = cur ? desc0 : desc1;
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    if (threadIdx.x == 0) {
        // one read of the status for the whole CTA (another CTA may set it
        // meanwhile, and every thread must leave at the same point); the
        // second launch of a gate runs only when the first one must be redone
        s_stop = ctl->status || (retry_pass && !ctl->retry);
        s_pd = pending_of<W>(ctl);
        s_rnorm = ctl->rnorm[cur];
        g_cn = 0u;
        g_range[0] = ctl->sp_lo;
        g_range[1] = ctl->sp_hi;
        s_nout = 0ULL;      // thread 0 counts the CTA's output and long partitions
        s_long = 0u;
        mbar_init(&s_bar, 1);
    }
    if (threadIdx.x == 0) {
        // children below the candidate range are left unwritten: when at
        // least cap_M children lie at or above it (checked after the merge),
        // the select would drop every one of them; otherwise the gate's
        // merge runs again without this (retry_pass)
        unsigned long long thr = dbits;
        if (!retry_pass && g_range[1] != 0ULL && g_range[0] > 0ULL && g_range[0] - 1ULL > thr)
            thr = g_range[0] - 1ULL;
        s_thr = thr;
        if (blockIdx.x == 0 && !ctl->status && !retry_pass) ctl->drop_on = thr != dbits;
    }
    for (uint32_t k = threadIdx.x; k < S; k += BLOCK) A::tab()[k] = 0u;
    __syncthreads();
    if (s_stop) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->cand_regions = gridDim.x;
        ctl->seg = 1;          // the output is the P segments this merge writes
        ctl->seg_P = P;
    }
    const Pending<W>& pd = s_pd;
    const double rnorm = s_rnorm;
    PKey<W>* __restrict__ kout = B.key(nxt);
    double* __restrict__ cout = B.coef(nxt);
    SelStats st{0ULL, 0u};
    // this CTA's output chunk: [ch_start, ch_pos) written, [ch_pos, ch_end)
    // free (the same on every thread)
    unsigned long long ch_start = 0, ch_pos = 0, ch_end = 0;
    uint32_t tag = 0, parity = 0;
    ChunkDesc* __restrict__ chunks_out = cur ? chunks0 : chunks1;
    // record the written run of a chunk for the readers of the whole state
    auto record_chunk = [&](unsigned long long start, unsigned long long end) {
        if (end == start) return;
        const unsigned int q = atomicAdd(&ctl->nchunk[nxt], 1u);
        if (q < max_chunks) {
            chunks_out[q].off = start;
            chunks_out[q].cnt = (unsigned int)(end - start);
        } else {
            set_status(ctl, ST_CAPACITY, 46);
        }
    };
    // claim room for at least `need` terms (every thread calls it)
    auto claim = [&](unsigned long long need) -> bool {
        if (threadIdx.x == 0) {
            record_chunk(ch_start, ch_pos);
            const unsigned long long sz = need > chunk ? need : chunk;
            const unsigned long long b = atomicAdd(&ctl->alloc[nxt], sz);
            if (b + sz > cap_out) {
                set_status(ctl, ST_CAPACITY, 2);
                s_chunk = ~0ULL;
            } else {
                s_chunk = b;
            }
            s_chsz = sz;
        }
        __syncthreads();
        const unsigned long long b = s_chunk;
        if (b == ~0ULL) return false;
        ch_start = b;
        ch_pos = b;
        ch_end = b + s_chsz;
        return true;
    };
    for (uint32_t p = blockIdx.x; p < P; p += gridDim.x) {
        const PKey<W>* kp;
        const double* cp;
        uint64_t np;
        if (from_scatter) {
            np = cursor[p];
            if (np > R) np = R;
            kp = pk + (uint64_t)p * R;
            cp = pc + (uint64_t)p * R;
        } else {
            np = din[p].cnt;
            kp = B.key(cur) + din[p].off;
            cp = B.coef(cur) + din[p].off;
        }
        // warm L2 with the partition this CTA takes next
        const uint32_t pn = p + gridDim.x;
        if (threadIdx.x == 0 && pn < P) {
            uint64_t nn;
            const PKey<W>* nk;
            const double* nc;
            if (from_scatter) {
                nn = cursor[pn];
                if (nn > R) nn = R;
                nk = pk + (uint64_t)pn * R;
                nc = pc + (uint64_t)pn * R;
            } else {
                nn = din[pn].cnt;
                nk = B.key(cur) + din[pn].off;
                nc = B.coef(cur) + din[pn].off;
            }
            if (nn) {
                l2_prefetch_bulk(nk, nn * sizeof(PKey<W>));
                l2_prefetch_bulk(nc, nn * sizeof(double));
            }
        }
        if (np <= C) {
            // stage the partition: keys, and the coefficients from the 16-byte
            // boundary at or below their start (one spare element when the
            // segment starts at an odd element)
            const uint32_t shift = (uint32_t)((reinterpret_cast<uint64_t>(cp) >> 3) & 1ULL);
            if (np) {
                if (threadIdx.x == 0) {
                    const uint32_t kb = (uint32_t)(np * sizeof(PKey<W>));
                    const uint32_t cb = (uint32_t)(((shift + np) * sizeof(double) + 15) & ~15ULL);
                    fence_async_shared();
                    mbar_expect(&s_bar, kb + cb);
                    bulk_g2s(A::keys(), kp, kb, &s_bar);
                    bulk_g2s(A::vals(), cp - shift, cb, &s_bar);
                }
                const bool ok = mbar_wait(&s_bar, parity, kWaitPolls);
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) {
                        set_status(ctl, ST_TIMEOUT, 45);
                        mbar_wait(&s_bar, parity, kWaitPolls);   // the copy in flight
                    }
                    __syncthreads();
                    return;
                }
                parity ^= 1u;
            }
            tag = next_tag<W, BLOCK>(tag, A::tab());
            // room for the pass's kept children, claimed once their number
            // is known: the rest of the current chunk, else a fresh one (the
            // rest of the old one is left as a hole)
            unsigned long long at = 0;
            bool failed = false;
            const uint32_t tot = stage_pass<W, BLOCK>(
                (uint32_t)np, shift, g, pd, rnorm, s_thr, ctl, nxt, tag, kout, cout, st, cd,
                [&](uint32_t t) -> unsigned long long {
                    if (ch_end - ch_pos < t && !claim(t)) {
                        failed = true;
                        return ~0ULL;
                    }
                    at = ch_pos;
                    return at;
                });
            if (failed) return;
            if (threadIdx.x == 0) {
                dout[p].off = at;
                dout[p].cnt = tot;
                s_nout += tot;
            }
            ch_pos += tot;
        } else {
            // a long partition: sub-passes (merge_long), its children one
            // segment; written in one round where room for 2 np of them is
            // at hand or within a fresh chunk, else counted first and given
            // exactly their number
            unsigned long long pre = ~0ULL;
            if (ch_end - ch_pos >= 2 * np) {
                pre = ch_pos;
            } else if (2 * np <= chunk) {
                if (!claim(2 * np)) return;
                pre = ch_pos;
            }
            unsigned long long at = pre;
            bool failed = false;
            const uint32_t done = merge_long<W, BLOCK>(
                kp, cp, np, g, pd, rnorm, s_thr, ctl, nxt, &tag, kout, cout, st, cd, pre,
                [&](uint32_t t) -> unsigned long long {
                    if (ch_end - ch_pos < t && !claim(t)) {
                        failed = true;
                        return ~0ULL;
                    }
                    at = ch_pos;
                    return at;
                },
                nullptr, &s_n);
            if (failed) return;
            ch_pos += done;
            if (threadIdx.x == 0) {
                dout[p].off = at;
                dout[p].cnt = done;
                s_nout += done;
                s_long += 1u;
            }
        }
    }
    // one atomic per warp for the largest pattern and the count above the
    // candidate range, one per CTA for the term count
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st.out_max = max(st.out_max, __shfl_xor_sync(0xffffffffu, st.out_max, o));
        st.above += __shfl_xor_sync(0xffffffffu, st.above, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (st.out_max) atomicMax(&ctl->out_max, st.out_max);
        if (st.above) atomicAdd(&ctl->sp_above, (unsigned long long)st.above);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        record_chunk(ch_start, ch_pos);
        if (s_nout) atomicAdd(&ctl->count[nxt], s_nout);
        if (s_long) atomicAdd(&ctl->stat_long, (unsigned long long)s_long);
        const uint32_t c = g_cn;
        cd.cnt[blockIdx.x] = c < cd.region ? c : (uint32_t)cd.region;
        if (c > cd.region) ctl->sp_ovf = 1;
    }
}

// After a merge that left the children below the candidate range unwritten:
// with at least cap_M children kept, the select keeps cap_M of them and every
// unwritten one lay below them all; with fewer, the unwritten ones are
// needed, so the merge's output is discarded and the gate's merge runs again
// in full (its input, the partitions or the previous gate's segments, is
// still in place).
__global__ void k_merge_check(DevCtl* ctl, uint64_t cap_M) {
    if (threadIdx.x != 0 || ctl->status) return;
    const int nxt = ctl->cur ^ 1;
    ctl->retry = 0;
    ctl->scatter_over = 0;   // the gate's scatters are done
    if (ctl->drop_on && ctl->count[nxt] < cap_M) {
        ctl->retry = 1;
        ctl->count[nxt] = 0ULL;
        ctl->alloc[nxt] = 0ULL;
        ctl->nchunk[nxt] = 0u;
        ctl->sp_above = 0ULL;
        ctl->sp_ovf = 0;
        ctl->out_max = 0ULL;
        ctl->stat_retry += 1ULL;
    }
    ctl->drop_on = 0;
}

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------
template <int W>
static Bufs<W> pbufs_of(const DeviceState& s) {
    Bufs<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    return b;
}

template <int W>
static GateArg<W> gate_of(const HostGate& h) {
    GateArg<W> g;
    for (int w = 0; w < W; ++w) { g.qx[w] = h.qx[w]; g.qz[w] = h.qz[w]; }
    g.ch = h.ch;
    g.msh = h.msh;
    g.qyy = h.qyy;
    g.maxw = h.maxw;
    return g;
}

template <int W>
static PartFn<W> part_fn_of(const HostGate& h) {
    PartFn<W> f;
    for (int w = 0; w < W; ++w) { f.kx[w] = h.keep_x[w]; f.kz[w] = h.keep_z[w]; }
    f.pair = h.pair_mode;
    f.sites = h.win_sites;
    bool found = false;
    for (int w = 0; w < 2 * W; ++w) {
        const uint64_t m = w < W ? h.qx[w] : h.qz[w - W];
        const uint64_t bit = (!found && m) ? (m & (~m + 1)) : 0ULL;
        if (w < W) f.px[w] = bit; else f.pz[w - W] = bit;
        found = found || m;
    }
    return f;
}

template <int W>
static cudaError_t scatter_w(const DeviceState& s, const HostGate& h, int force, cudaStream_t st) {
    // every gate: the merge leaves the cursors as they are (a gate whose
    // merge runs again reads its partitions twice), and whether this gate
    // scatters is decided on the device
    cudaError_t e = cudaMemsetAsync(s.part_cursor, 0, (size_t)s.part_max * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    uint64_t gs = (s.buf_cap + 255) / 256;
    const uint64_t lim = (uint64_t)s.num_sms * 8;
    if (gs > lim) gs = lim;
    if (gs < 1) gs = 1;
    for (int redo = 0; redo < 2; ++redo) {
        if (redo) k_scatter_clear<<<s.num_sms, 256, 0, st>>>(s.ctl, s.part_cursor, s.part_max);
        k_part_scatter<W><<<(int)gs, 256, 0, st>>>(pbufs_of<W>(s), s.ctl,
                                                   reinterpret_cast<PKey<W>*>(s.part_keys),
                                                   s.part_coef, s.part_cursor, s.part_cap,
                                                   s.part_max, gate_of<W>(h), part_fn_of<W>(h),
                                                   force, s.n, s.part_target, s.chunks[0],
                                                   s.chunks[1], redo);
    }
    return cudaGetLastError();
}

template <int W, int BLOCK>
static cudaError_t merge_wb(const DeviceState& s, const GateArg<W>& g, cudaStream_t st) {
    static int per_sm = 0;
    constexpr size_t smem = Stage<W>::kBytes;
    if (!per_sm) {
        cudaFuncSetAttribute(k_gate_part<W, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        // shared memory for every resident CTA's staging rather than L1
        cudaFuncSetAttribute(k_gate_part<W, BLOCK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gate_part<W, BLOCK>, BLOCK, smem);
        if (per_sm < 1) per_sm = 1;
    }
    int grid = s.num_sms * per_sm;
    if (grid > s.max_ctas) grid = s.max_ctas;   // one candidate region per CTA
    for (int pass = 0; pass < 2; ++pass) {
        k_gate_part<W, BLOCK><<<grid, BLOCK, smem, st>>>(
            reinterpret_cast<const PKey<W>*>(s.part_keys), s.part_coef, s.part_cursor, s.part_cap,
            s.part_desc[0], s.part_desc[1], pbufs_of<W>(s), s.ctl, g, s.delta, s.buf_cap,
            s.chunk, s.cand, s.chunks[0], s.chunks[1], s.max_chunks, pass);
        if (pass == 0) k_merge_check<<<1, 32, 0, st>>>(s.ctl, s.cap_M);
    }
    return cudaGetLastError();
}

// The partitioned merge's CTA size (threads loop over a partition's staged
// strings, so there is no items-per-thread parameter on this path).
template <int W>
static cudaError_t merge_w(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    const GateArg<W> g = gate_of<W>(h);
    switch (s.block) {
        case 128: return merge_wb<W, 128>(s, g, st);
        case 256: return merge_wb<W, 256>(s, g, st);
        case 512: return merge_wb<W, 512>(s, g, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_part_scatter(const DeviceState& s, const HostGate& h, int force,
                                cudaStream_t st) {
    return s.W == 1 ? scatter_w<1>(s, h, force, st) : scatter_w<2>(s, h, force, st);
}

cudaError_t launch_part_merge(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    return s.W == 1 ? merge_w<1>(s, h, st) : merge_w<2>(s, h, st);
}

void plan_windows(int W, std::vector<HostGate>& gates) {
    const int max_sites = W == 1 ? PartGeom<1>::kWinSites : PartGeom<2>::kWinSites;
    auto sites = [](const uint64_t* m) {
        return __builtin_popcountll(m[0]) + __builtin_popcountll(m[1]);
    };
    size_t k = 0;
    while (k < gates.size()) {
        uint64_t S[2] = {gates[k].qx[0] | gates[k].qz[0], gates[k].qx[1] | gates[k].qz[1]};
        if (sites(S) > max_sites) {
            // a wide gate: a window of its own, partitioned by its pair key
            HostGate& h = gates[k];
            h.pair_mode = 1;
            h.win_start = 1;
            for (int w = 0; w < 2; ++w) { h.keep_x[w] = ~0ULL; h.keep_z[w] = ~0ULL; }
            ++k;
            continue;
        }
        size_t e = k + 1;
        while (e < gates.size()) {
            const uint64_t T[2] = {S[0] | gates[e].qx[0] | gates[e].qz[0],
                                   S[1] | gates[e].qx[1] | gates[e].qz[1]};
            if (sites(T) > max_sites) break;
            S[0] = T[0];
            S[1] = T[1];
            ++e;
        }
        for (size_t j = k; j < e; ++j) {
            HostGate& h = gates[j];
            h.pair_mode = 0;
            h.win_sites = sites(S);
            h.win_start = j == k;
            for (int w = 0; w < 2; ++w) { h.keep_x[w] = ~S[w]; h.keep_z[w] = ~S[w]; }
        }
        k = e;
    }
}

// A merge CTA claims output room in chunks of about an eighth of its share
// of a bounded state (at most 2^16 terms), or exactly a partition's children
// when they need more.  What the chunks leave unused is the rest of each
// CTA's last chunk and, each time a partition did not fit, the rest of the
// chunk it left (less than that partition's children, at most a quarter of
// a chunk of at least four times the largest pass's children): the state
// buffers' slack covers two chunks per CTA and three quarters of the bound
// for the second, above the 2 cap_M children a merge writes at most.  A
// bound too small for such chunks (0 returned) makes every claim exact: one
// claim per partition, nothing left unused.
uint64_t merge_chunk(uint64_t cap_M, int max_ctas, int W) {
    uint64_t c = cap_M / (8ULL * (uint64_t)(max_ctas > 0 ? max_ctas : 1));
    uint64_t p = 16;
    while (p * 2 <= c && p < (1ULL << 16)) p *= 2;
    const uint64_t least = 4ULL * 2ULL * (uint64_t)(W == 1 ? Stage<1>::C : Stage<2>::C);
    return p < least ? 0ULL : p;
}

uint64_t merge_slack(uint64_t cap_M, int max_ctas, int W) {
    return 2ULL * (uint64_t)max_ctas * merge_chunk(cap_M, max_ctas, W) + cap_M / 4 * 3 + 4096;
}

int partition_target_default(int W) {
    return W == 1 ? PartGeom<1>::kTarget : PartGeom<2>::kTarget;
}

uint32_t partition_max(uint64_t cap_M, int target) {
    const uint64_t t = (uint64_t)target;
    return (uint32_t)((cap_M + t - 1) / t + 1);
}

}  // namespace itpp
