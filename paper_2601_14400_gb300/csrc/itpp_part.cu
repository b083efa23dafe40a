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
// at a time per CTA: the partition's terms stay in registers, the commuting
// ones publish (key, child for the partner) in a shared-memory table, every
// term merges with its partner's child, and the kept children of the
// partition are written as one contiguous segment of an output chunk that
// the CTA claimed beforehand (a global atomic every few hundred partitions,
// none per partition).  The segments, listed by the partition descriptors,
// are the partitions of the next gate of the window, so no scatter runs
// between the gates of a window.  A group holds at most 4^|S| terms; a
// partition that outgrows the register chunk is merged in sub-passes, each
// taking the pairs of one hash class of the key with the gate's sites
// cleared, so no partition size forces a re-partition.  A gate acting on more
// sites than a window allows is a window of its own, partitioned by its pair
// key (the member of {K, QK} with the gate's lowest bit clear).
//
// The top-M select (Sec. II.C, term bound) is folded into the merge: every
// kept child is compared with a range around the previous gate's threshold;
// the merge counts the children above it and lists those inside it, and the
// select (itpp_select.cu) then works on that short list instead of passing
// over every coefficient.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {


// Partition geometry per word count: the mean partition size the scatter
// aims for, and the largest window (sites; a group holds at most 4^sites
// terms).
template <int W> struct PartGeom;
template <> struct PartGeom<1> {
    static constexpr int kTarget = 700, kWinSites = 5;
};
template <> struct PartGeom<2> {
    static constexpr int kTarget = 300, kWinSites = 4;
};

struct PartPlan {
    uint32_t P;     // partitions
    uint64_t R;     // stride (capacity) of one partition in the scatter buffer
};

__device__ __forceinline__ PartPlan part_plan(uint64_t n, uint64_t pbuf_cap, uint32_t p_max,
                                              int target) {
    uint64_t P = (n + target - 1) / target;
    if (P < 1) P = 1;
    if (P > p_max) P = p_max;
    PartPlan pl;
    pl.P = (uint32_t)P;
    pl.R = pbuf_cap / P;
    return pl;
}

// The partition function of a window: the hash of the key with the
// window's sites cleared, or (pair mode) of the gate's pair key.
template <int W>
struct PartFn {
    uint64_t kx[W], kz[W];   // bits kept by the mask
    int pair;                // 1: pair-key mode
    int sites;               // sites of the window (mask mode)
    uint64_t px[W], pz[W];   // the pivot: the gate's lowest bit (all zero for Q = I)
};

// Mask mode needs many more possible groups than terms: a group (the terms
// with one pattern outside the window) holds up to 4^sites of them, and a
// partition that collects several large groups could outgrow its stride or
// the shared table.  So the window's mask is used only while
// 4^(n - sites) >= 64 N; a denser state (a small or saturated chain) falls
// back to the pair key of the window's first gate, valid for that gate only.
__device__ __forceinline__ bool window_fits(int n_sites, int w_sites, uint64_t n_terms) {
    const int free_bits = 2 * (n_sites - w_sites);
    const int need_bits = 6 + (n_terms > 1 ? 64 - __clzll((long long)(n_terms - 1)) : 0);
    return free_bits >= need_bits;
}

template <int W>
__device__ __forceinline__ uint32_t part_of(const PKey<W>& K, const GateArg<W>& g,
                                            const PartFn<W>& f, uint32_t P) {
    // masks and element-wise selects only: a conditional copy of the key,
    // or a selection of one of its words by index, puts the caller's key
    // arrays in local memory
    uint64_t piv = 0;
#pragma unroll
    for (int v = 0; v < W; ++v) piv |= (K.x[v] & f.px[v]) | (K.z[v] & f.pz[v]);
    const uint64_t flip = piv ? ~0ULL : 0ULL;   // pivot set: the pair key is K.Q
    PKey<W> k;
    if (f.pair) {   // the pair key K.Q when the pivot is set
#pragma unroll
        for (int v = 0; v < W; ++v) { k.x[v] = K.x[v] ^ (g.qx[v] & flip); k.z[v] = K.z[v] ^ (g.qz[v] & flip); }
    } else {        // the key with the window's sites cleared
#pragma unroll
        for (int v = 0; v < W; ++v) { k.x[v] = K.x[v] & f.kx[v]; k.z[v] = K.z[v] & f.kz[v]; }
    }
    const uint64_t h = key_hash(k);   // 32 significant bits
    return (uint32_t)((h * (uint64_t)P) >> 32);
}

// The kept set of a deferred top-M select, applied where terms are read.
template <int W>
struct Pending {
    bool on, all_ties;
    unsigned long long T;
    PKey<W> tk;
};

template <int W>
__device__ __forceinline__ Pending<W> pending_of(const DevCtl* ctl) {
    Pending<W> q;
    q.on = ctl->pend != 0;
    q.all_ties = ctl->pend_all_ties != 0;
    q.T = ctl->pend_T;
#pragma unroll
    for (int w = 0; w < W; ++w) { q.tk.x[w] = ctl->pend_tie_key[w]; q.tk.z[w] = ctl->pend_tie_key[W + w]; }
    return q;
}

// Prefetch [p, p + bytes) into L2 with one bulk (TMA) request; the range is
// widened to 16-byte boundaries, which every buffer it is used on allows
// (its byte size is a multiple of 16).
__device__ __forceinline__ void l2_prefetch_bulk(const void* p, uint64_t bytes) {
    const uint64_t a = reinterpret_cast<uint64_t>(p);
    const uint64_t lo = a & ~15ULL;
    uint64_t sz = ((a + bytes + 15ULL) & ~15ULL) - lo;
    if (sz > (1ULL << 20)) sz = 1ULL << 20;
    if (sz) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(lo), "r"((uint32_t)sz)
                         : "memory");
}

// ---------------------------------------------------------------------------
// Bulk (TMA) copies into shared memory, completed on an mbarrier.  A copy
// needs 16-byte aligned addresses and a size that is a multiple of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive on the barrier and announce `bytes` of copies that complete it.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Generic-proxy accesses to shared memory made before this fence are ordered
// before later bulk copies into it.
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Wait for the barrier's phase `parity` to complete, at most `limit` polls
// (each poll may itself suspend the thread for a while).  False: timed out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        // the thread sleeps in the wait until the phase completes or the
        // hint (nanoseconds) runs out, instead of polling
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(a), "r"(parity), "r"(1000000u) : "memory");
        if (done) return true;
    }
    return false;
}

// Sub-pass of a long partition's commuting string: a hash of the key with
// the gate's sites cleared, which K and Q.K share (they differ exactly on
// Q's bits), so a string and its partner always fall into the same one.
template <int W>
__device__ __forceinline__ uint32_t sub_pass(const PKey<W>& K, const GateArg<W>& g, uint32_t k) {
    PKey<W> m;
#pragma unroll
    for (int w = 0; w < W; ++w) { m.x[w] = K.x[w] & ~g.qx[w]; m.z[w] = K.z[w] & ~g.qz[w]; }
    return (uint32_t)((key_hash(m) * (uint64_t)k) >> 32);
}

// Append one value per lane that has one (every lane of the warp calls it)
// to this CTA's region of the candidate list: one shared-memory atomic per
// warp; entries past the region's end are dropped and counted, and the
// select then falls back to its full passes.
__device__ __forceinline__ void cand_push(bool hit, unsigned long long v, uint64_t pos,
                                          const CandRegions& cd, uint32_t* s_cn) {
    const unsigned int m = __ballot_sync(0xffffffffu, hit);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    uint32_t q = 0;
    if (lane == leader) q = atomicAdd(s_cn, (uint32_t)__popc(m));
    q = __shfl_sync(0xffffffffu, q, leader);
    if (hit) {
        const uint64_t r = (uint64_t)q + __popc(m & ((1u << lane) - 1u));
        if (r < cd.region) {
            const uint64_t e = (uint64_t)blockIdx.x * cd.region + r;
            cd.v[e] = v;
            cd.idx[e] = (uint32_t)pos;
        }
    }
}

}  // namespace

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
               int n_sites, int target, const ChunkDesc* chunks0, const ChunkDesc* chunks1) {
    if (ctl->status) return;
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
    const PartPlan pl = part_plan(n, pbuf_cap, p_max, target);
    const bool fallback = !f.pair && !window_fits(n_sites, f.sites, n);
    if (fallback) f.pair = 1;
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

// Items a CTA stages in shared memory for one pass, and the slots of its
// pair table (at most half full).
template <int W> struct StageGeom;
template <> struct StageGeom<1> { static constexpr int kItems = 1024, kSlots = 2048; };
template <> struct StageGeom<2> { static constexpr int kItems = 512, kSlots = 1024; };

// Dynamic shared memory of the merge: the staged keys, their values (raw
// coefficient in, normalised coefficient after phase A, merged child after
// phase B; two spare slots let a copy start at the 16-byte boundary below an
// odd element), the partner children b, the pair table and per-item flags.
template <int W>
struct Stage {
    static constexpr int C = StageGeom<W>::kItems, S = StageGeom<W>::kSlots;
    static constexpr size_t kKeys = 0;
    static constexpr size_t kVals = kKeys + sizeof(PKey<W>) * C;
    static constexpr size_t kB = kVals + sizeof(double) * (C + 2);
    static constexpr size_t kTab = kB + sizeof(double) * C;
    static constexpr size_t kFlags = kTab + sizeof(uint32_t) * S;
    static constexpr size_t kBytes = (kFlags + C + 15) / 16 * 16;
    static_assert(kVals % 16 == 0 && kB % 16 == 0 && kTab % 16 == 0, "alignment");
};

// Waits on a staging copy's barrier before the CTA gives up: each wait
// sleeps up to a millisecond, and a copy of a few tens of kilobytes completes
// within microseconds; this bound is seconds.
constexpr uint32_t kWaitPolls = 4096u;

// Slot of a key in a CTA's pair table: a multiply-xor of the key's 32-bit
// halves and one xorshift-multiply round.  Partitions are chosen by the full
// hash of a different key (masked or pair key), so the two are independent.
template <int W>
__device__ __forceinline__ uint32_t slot_hash(const PKey<W>& k) {
    constexpr uint32_t C[8] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu,
                               0x165667B1u, 0xD3A2646Du, 0xFD7046C5u, 0xB55A4F09u};
    uint32_t h = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h ^= (uint32_t)k.x[w] * C[4 * w] ^ (uint32_t)(k.x[w] >> 32) * C[4 * w + 1];
        h ^= (uint32_t)k.z[w] * C[4 * w + 2] ^ (uint32_t)(k.z[w] >> 32) * C[4 * w + 3];
    }
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    return h;
}

// Pair table of one pass: slot = (tag << 16) | index of a staged commuting
// string.  Tags grow with every pass of the CTA, so a slot of an earlier
// pass is free and the table needs no clearing.
template <int W>
__device__ __forceinline__ bool pair_insert(const PKey<W>& K, uint32_t i, uint32_t* tab,
                                            uint32_t tag) {
    constexpr uint32_t S = StageGeom<W>::kSlots;
    const uint32_t mine = (tag << 16) | i;
    uint32_t h = slot_hash(K) & (S - 1);
    for (uint32_t q = 0; q < S; ++q) {
        uint32_t v = tab[h];
        while ((v >> 16) != tag) {          // free: claim it
            const uint32_t o = atomicCAS(tab + h, v, mine);
            if (o == v) return true;
            v = o;
        }
        h = (h + 1) & (S - 1);
    }
    return false;
}

template <int W>
__device__ __forceinline__ bool pair_find(const PKey<W>& P, const PKey<W>* keys_s,
                                          const double* b_s, const uint32_t* tab, uint32_t tag,
                                          double* out) {
    constexpr uint32_t S = StageGeom<W>::kSlots;
    uint32_t h = slot_hash(P) & (S - 1);
    for (uint32_t q = 0; q < S; ++q) {
        const uint32_t v = tab[h];
        if ((v >> 16) != tag) return false;
        const uint32_t j = v & 0xffffu;
        if (key_eq(keys_s[j], P)) { *out = b_s[j]; return true; }
        h = (h + 1) & (S - 1);
    }
    return false;
}

// Exclusive block scan with one barrier: every warp writes its total, then
// every warp scans the warp totals with shuffles (s_warp may be rewritten
// only after the caller's next barrier).
template <int BLOCK>
__device__ __forceinline__ uint32_t block_scan_1bar(uint32_t v, uint32_t* s_warp,
                                                    uint32_t* total) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t t = lane < NW ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, t, warp > 0 ? warp - 1 : 0);
    *total = __shfl_sync(0xffffffffu, t, NW - 1);
    return (warp > 0 ? before : 0u) + x - v;
}

// Statistics of the kept children for the top-M select: the largest
// pattern, the count above the candidate range, the candidates inside it.
struct SelStats {
    const unsigned long long* range;   // shared: candidate range [lo, hi] (hi == 0: none)
    unsigned long long out_max;
    uint32_t above;
};

// Write one staged item's kept children at pos (and pos + 1) and fold them
// into the statistics.  Every lane of the warp calls it.
template <int W>
__device__ __forceinline__ void stage_emit(const PKey<W>& K, double va, double b, uint32_t o,
                                           const GateArg<W>& g, PKey<W>* kout, double* cout,
                                           uint64_t pos, SelStats& st, const CandRegions& cd,
                                           uint32_t* s_cn) {
    if (o & 1u) {
        store_key_stream(kout + pos, K);
        __stcs(cout + pos, va);
    }
    const uint64_t pb = pos + (o & 1u);
    if (o & 2u) {
        store_key_stream(kout + pb, key_xor(K, g));
        __stcs(cout + pb, b);
    }
    const unsigned long long a = (o & 1u) ? abs_pattern(va) : 0ULL;
    const unsigned long long bb = (o & 2u) ? abs_pattern(b) : 0ULL;
    st.out_max = max(st.out_max, max(a, bb));
    const unsigned long long hi = st.range[1];
    if (hi) {   // uniform
        const unsigned long long lo = st.range[0], w = hi - lo;
        st.above += (a > hi ? 1u : 0u) + (bb > hi ? 1u : 0u);
        // a - lo <= w on unsigned values: lo <= a <= hi (a kept child has a > 0)
        cand_push((o & 1u) && a - lo <= w, a - lo, pos, cd, s_cn);
        cand_push((o & 2u) && bb - lo <= w, bb - lo, pb, cd, s_cn);
    }
}

template <int W>
struct PassArgs {
    PKey<W>* keys_s;
    double* vals_s;     // item i's value at vals_s[shift + i]
    double* b_s;
    uint32_t* tab;
    uint8_t* flags_s;
    uint32_t* s_warp;
    uint32_t* s_cn;
};

// One pass of the gate over n staged strings: phase A (the deferred select's
// kept set, commutation, sign, the normalised coefficient c and the partner
// child b = c (-sinh(theta)) s, commuting strings into the pair table),
// phase B (the partner's b, the merged child, threshold and weight cutoff,
// the identity's merged coefficient as the next normaliser), a block scan of
// the kept children, and the write pass from `base` on (room the caller
// holds).  Three barriers; the staging arrays are free again when it
// returns.  Returns the kept children written (the same on every thread).
template <int W, int BLOCK>
__device__ __forceinline__ uint32_t stage_pass(const PassArgs<W>& a, uint32_t n, uint32_t shift,
                                               const GateArg<W>& g, const Pending<W>& pd,
                                               double rnorm, unsigned long long dbits,
                                               DevCtl* ctl, int nxt, uint32_t tag,
                                               PKey<W>* kout, double* cout, SelStats& st,
                                               const CandRegions& cd, unsigned long long base) {
    double* vals = a.vals_s + shift;
    // phase A
    for (uint32_t i = threadIdx.x; i < n; i += BLOCK) {
        const PKey<W> K = a.keys_s[i];
        const double raw = vals[i];
        const bool live = !pd.on || cap_keep(K, raw, pd.T, pd.all_ties, pd.tk);
        const bool id = key_is_zero(K);
        if (!live && id) set_status(ctl, ST_TRACE_ZERO, 43);
        const bool comm = live && commutes(K, g);
        const bool neg = comm && product_negative(K, g);
        // the identity's normalised value is exactly 1
        const double c = id ? 1.0 : __dmul_rn(raw, rnorm);
        const double m = __longlong_as_double(
            __double_as_longlong(g.msh) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
        vals[i] = c;
        a.b_s[i] = __dmul_rn(c, m);
        a.flags_s[i] = (uint8_t)((live ? 1u : 0u) | (comm ? 2u : 0u));
        if (comm && !pair_insert(K, i, a.tab, tag)) set_status(ctl, ST_CAPACITY, 41);
    }
    __syncthreads();                                                  // (1) table built
    // phase B
    uint32_t cnt = 0;
    for (uint32_t i = threadIdx.x; i < n; i += BLOCK) {
        const uint32_t f = a.flags_s[i];
        uint32_t o = 0;
        if (f & 1u) {
            const PKey<W> K = a.keys_s[i];
            const double c = vals[i];
            double pb = 0.0;
            bool found = false;
            if (f & 2u) found = pair_find(key_xor(K, g), a.keys_s, a.b_s, a.tab, tag, &pb);
            const double a1 = __dmul_rn(c, g.ch);                    // cosh(theta) P
            const double sum = __dadd_rn(a1, pb);                     // + the partner's child
            const double va = !(f & 2u) ? c : (found ? sum : a1);     // {P,Q} = 0: unchanged
            const bool emit_b = (f & 2u) && !found;
            // threshold and weight cutoff on the merged children (Sec. II.B)
            bool keep_a = above(va, dbits) && light(K, g.maxw);
            const bool keep_b = emit_b && above(a.b_s[i], dbits) && light(key_xor(K, g), g.maxw);
            if (key_is_zero(K)) {
                ctl->norm[nxt] = va;
                if (!keep_a) set_status(ctl, ST_TRACE_ZERO, 1);
                keep_a = true;
            }
            vals[i] = va;
            o = (keep_a ? 1u : 0u) | (keep_b ? 2u : 0u);
        }
        a.flags_s[i] = (uint8_t)o;
        cnt += __popc(o);
    }
    uint32_t tot;
    const uint32_t off = block_scan_1bar<BLOCK>(cnt, a.s_warp, &tot);   // (2)
    // the caller's room starts at base (the same on every thread)
    uint64_t pos = base + off;
    // write pass: warp-uniform rounds (the candidate list is filled warp-wide)
    for (uint32_t i0 = 0; i0 < n; i0 += BLOCK) {
        const uint32_t i = i0 + threadIdx.x;
        uint32_t o = 0;
        PKey<W> K;
#pragma unroll
        for (int w = 0; w < W; ++w) { K.x[w] = 0; K.z[w] = 0; }
        double va = 0.0, b = 0.0;
        if (i < n) {
            o = a.flags_s[i];
            if (o) {
                K = a.keys_s[i];
                va = vals[i];
                b = a.b_s[i];
            }
        }
        stage_emit(K, va, b, o, g, kout, cout, pos, st, cd, a.s_cn);
        pos += __popc(o);
    }
    __syncthreads();                                                  // (3) staging free
    return tot;
}

// The tag of the next pass (every thread calls it): slots hold 16-bit tags,
// so after 65535 passes of one CTA the table is cleared and tags restart.
template <int W, int BLOCK>
__device__ __forceinline__ uint32_t next_tag(uint32_t tag, uint32_t* tab) {
    if (tag < 0xffffu) return tag + 1u;
    for (uint32_t k = threadIdx.x; k < (uint32_t)StageGeom<W>::kSlots; k += BLOCK) tab[k] = 0u;
    __syncthreads();
    return 1u;
}

template <int W, int BLOCK>
struct PartOcc {
    // CTAs per SM the launch bound asks for: the staging and table take
    // Stage<W>::kBytes of shared memory per CTA
    static constexpr int kMin = BLOCK <= 256 ? 5 : 2;
};

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
template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (PartOcc<W, BLOCK>::kMin))
k_gate_part(const PKey<W>* __restrict__ pk, const double* __restrict__ pc,
            unsigned int* __restrict__ cursor, uint64_t pbuf_cap, PartDesc* desc0,
            PartDesc* desc1, Bufs<W> B, DevCtl* ctl, GateArg<W> g, double delta,
            uint64_t cap_out, uint64_t chunk, CandRegions cd, ChunkDesc* chunks0,
            ChunkDesc* chunks1, uint32_t max_chunks) {
    using G = Stage<W>;
    constexpr uint32_t C = G::C, S = G::S;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_warp[BLOCK / 32];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ unsigned long long s_chunk, s_chsz, s_nout, s_range[2];
    __shared__ uint32_t s_cn, s_long, s_n;
    __shared__ int s_stop;
    __shared__ Pending<W> s_pd;
    __shared__ double s_rnorm;
    const PassArgs<W> pa{reinterpret_cast<PKey<W>*>(smem + G::kKeys),
                         reinterpret_cast<double*>(smem + G::kVals),
                         reinterpret_cast<double*>(smem + G::kB),
                         reinterpret_cast<uint32_t*>(smem + G::kTab), smem + G::kFlags, s_warp,
                         &s_cn};
    const int cur = ctl->cur, nxt = cur ^ 1;
    const bool from_scatter = ctl->part_from_scatter != 0;
    const uint32_t P = ctl->part_P;
    const uint64_t R = P ? pbuf_cap / P : 0;
    const PartDesc* __restrict__ din = cur ? desc1 : desc0;
    PartDesc* __restrict__ dout = cur ? desc0 : desc1;
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    if (threadIdx.x == 0) {
        // one read of the status for the whole CTA (another CTA may set it
        // meanwhile, and every thread must leave at the same point)
        s_stop = ctl->status;
        s_pd = pending_of<W>(ctl);
        s_rnorm = ctl->rnorm[cur];
        s_cn = 0u;
        s_range[0] = ctl->sp_lo;
        s_range[1] = ctl->sp_hi;
        s_nout = 0ULL;      // thread 0 counts the CTA's output and long partitions
        s_long = 0u;
        mbar_init(&s_bar, 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !ctl->status) {
        ctl->cand_regions = gridDim.x;
        ctl->seg = 1;          // the output is the P segments this merge writes
        ctl->seg_P = P;
    }
    for (uint32_t k = threadIdx.x; k < S; k += BLOCK) pa.tab[k] = 0u;
    __syncthreads();
    if (s_stop) return;
    const Pending<W>& pd = s_pd;
    const double rnorm = s_rnorm;
    PKey<W>* __restrict__ kout = B.key(nxt);
    double* __restrict__ cout = B.coef(nxt);
    SelStats st{s_range, 0ULL, 0u};
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
                    bulk_g2s(pa.keys_s, kp, kb, &s_bar);
                    bulk_g2s(pa.vals_s, cp - shift, cb, &s_bar);
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
            // every thread has read the cursor: leave it zero for the next scatter
            if (from_scatter && threadIdx.x == 0) cursor[p] = 0u;
            tag = next_tag<W, BLOCK>(tag, pa.tab);
            // room: the partition's children (at most 2 np) fit a fresh chunk
            if (ch_end - ch_pos < 2 * np && !claim(2 * np)) return;
            const uint32_t tot = stage_pass<W, BLOCK>(pa, (uint32_t)np, shift, g, pd, rnorm, dbits,
                                                      ctl, nxt, tag, kout, cout, st, cd, ch_pos);
            if (threadIdx.x == 0) {
                dout[p].off = ch_pos;
                dout[p].cnt = tot;
                s_nout += tot;
            }
            ch_pos += tot;
        } else {
            // a long partition: k sub-passes over the hash classes of the key
            // with the gate's sites cleared (about C/2 strings each); the
            // partition's children stay one segment
            const uint32_t k = (uint32_t)((2 * np + C - 1) / C);
            if (ch_end - ch_pos < 2 * np && !claim(2 * np)) return;
            const unsigned long long start = ch_pos;
            for (uint32_t j = 0; j < k; ++j) {
                if (threadIdx.x == 0) s_n = 0u;
                __syncthreads();
                for (uint64_t i = threadIdx.x; i < np; i += BLOCK) {
                    const PKey<W> K = load_key_stream(kp + i);
                    const double raw = __ldcs(cp + i);
                    const bool live = !pd.on || cap_keep(K, raw, pd.T, pd.all_ties, pd.tk);
                    if (!live) {
                        if (key_is_zero(K)) set_status(ctl, ST_TRACE_ZERO, 43);
                        continue;
                    }
                    const uint32_t cls = commutes(K, g) ? sub_pass(K, g, k) : (uint32_t)(i % k);
                    if (cls != j) continue;
                    const uint32_t q = atomicAdd(&s_n, 1u);
                    if (q < C) {
                        pa.keys_s[q] = K;
                        pa.vals_s[q] = raw;
                    } else {
                        set_status(ctl, ST_CAPACITY, 44);
                    }
                }
                __syncthreads();
                if (j == 0 && from_scatter && threadIdx.x == 0) cursor[p] = 0u;
                const uint32_t n = s_n < C ? s_n : C;
                tag = next_tag<W, BLOCK>(tag, pa.tab);
                ch_pos += stage_pass<W, BLOCK>(pa, n, 0u, g, pd, rnorm, dbits, ctl, nxt, tag, kout,
                                               cout, st, cd, ch_pos);
            }
            if (threadIdx.x == 0) {
                dout[p].off = start;
                dout[p].cnt = (unsigned int)(ch_pos - start);
                s_nout += ch_pos - start;
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
        const uint32_t c = s_cn;
        cd.cnt[blockIdx.x] = c < cd.region ? c : (uint32_t)cd.region;
        if (c > cd.region) ctl->sp_ovf = 1;
    }
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
    if (force) {
        cudaError_t e = cudaMemsetAsync(s.part_cursor, 0, (size_t)s.part_max * sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
    }
    uint64_t gs = (s.buf_cap + 255) / 256;
    const uint64_t lim = (uint64_t)s.num_sms * 8;
    if (gs > lim) gs = lim;
    if (gs < 1) gs = 1;
    k_part_scatter<W><<<(int)gs, 256, 0, st>>>(pbufs_of<W>(s), s.ctl,
                                               reinterpret_cast<PKey<W>*>(s.part_keys),
                                               s.part_coef, s.part_cursor, s.part_cap,
                                               s.part_max, gate_of<W>(h), part_fn_of<W>(h), force,
                                               s.n, s.part_target, s.chunks[0], s.chunks[1]);
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
    k_gate_part<W, BLOCK><<<grid, BLOCK, smem, st>>>(
        reinterpret_cast<const PKey<W>*>(s.part_keys), s.part_coef, s.part_cursor, s.part_cap,
        s.part_desc[0], s.part_desc[1], pbufs_of<W>(s), s.ctl, g, s.delta, s.buf_cap, s.chunk,
        s.cand, s.chunks[0], s.chunks[1], s.max_chunks);
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
// of a bounded state (at most 2^16 terms); what the chunks leave unused is at
// most one chunk per CTA plus the tails a partition that did not fit left
// behind, which the state buffers' slack covers.
uint64_t merge_chunk(uint64_t cap_M, int max_ctas) {
    uint64_t c = cap_M / (8ULL * (uint64_t)(max_ctas > 0 ? max_ctas : 1));
    uint64_t p = 16;
    while (p * 2 <= c && p < (1ULL << 16)) p *= 2;
    return p;
}

uint64_t merge_slack(uint64_t cap_M, int max_ctas) {
    return 2ULL * (uint64_t)max_ctas * merge_chunk(cap_M, max_ctas) + cap_M / 4 + 4096;
}

int partition_target_default(int W) {
    return W == 1 ? PartGeom<1>::kTarget : PartGeom<2>::kTarget;
}

uint32_t partition_max(uint64_t cap_M, int target) {
    const uint64_t t = (uint64_t)target;
    return (uint32_t)((cap_M + t - 1) / t + 1);
}

}  // namespace itpp
