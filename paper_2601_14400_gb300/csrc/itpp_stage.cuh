// itpp_stage.cuh -- the partition merge's device building blocks, shared by
// the single propagation (itpp_part.cu) and the batched one (itpp_batch.cu):
// the partition function and plan, bulk (TMA) copies into shared memory on
// an mbarrier, the staged pass of one gate over one partition (pair table,
// merged children, threshold, write), and the sub-passes of a partition
// above the staging capacity.
#pragma once

#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"

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
// Q's bits), so a string and its partner always fall into the same one.  The
// hash is seeded apart from the partition hash: for a string with both of
// the gate's bits clear the masked key is the pair key the partition was
// chosen by, and the same hash would put all such strings of a partition in
// one class.
template <int W>
__device__ __forceinline__ uint32_t sub_pass(const PKey<W>& K, const GateArg<W>& g, uint32_t k) {
    uint32_t h = 0x3c6ef372u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint64_t mx = K.x[w] & ~g.qx[w], mz = K.z[w] & ~g.qz[w];
        h = murmur_mix(h, (uint32_t)mx);
        h = murmur_mix(h, (uint32_t)(mx >> 32));
        h = murmur_mix(h, (uint32_t)mz);
        h = murmur_mix(h, (uint32_t)(mz >> 32));
    }
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return (uint32_t)(((uint64_t)h * k) >> 32);
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

// Items a CTA stages in shared memory for one pass, and the slots of its
// pair table (at most half full).
template <int W> struct StageGeom;
template <> struct StageGeom<1> { static constexpr int kItems = 1024, kSlots = 2048; };
template <> struct StageGeom<2> { static constexpr int kItems = 512, kSlots = 1024; };

// Dynamic shared memory of the merge: the staged keys, their values (raw
// coefficient in, normalised coefficient after phase A, merged children
// after phase B; two spare slots let a copy start at the 16-byte boundary
// below an odd element), the pair table and per-item flags.
template <int W>
struct Stage {
    static constexpr int C = StageGeom<W>::kItems, S = StageGeom<W>::kSlots;
    static constexpr size_t kKeys = 0;
    static constexpr size_t kVals = kKeys + sizeof(PKey<W>) * C;
    static constexpr size_t kTab = kVals + sizeof(double) * (C + 2);
    static constexpr size_t kFlags = kTab + sizeof(uint32_t) * S;
    static constexpr size_t kBytes = (kFlags + sizeof(uint16_t) * C + 15) / 16 * 16;
    static_assert(kVals % 16 == 0 && kTab % 16 == 0, "alignment");
    static_assert(C <= 1024 && S <= 2048, "slot and index fields");
};

// The merge's dynamic shared memory (Stage<W> layout) and its small shared
// counters, at file scope so that every access is a constant offset from the
// CTA's shared window rather than a pointer held in registers.
extern __shared__ __align__(16) unsigned char g_stage[];
__shared__ uint32_t g_warp[32];  // the block scan's warp totals
__shared__ uint32_t g_cn;        // this CTA's candidates
__shared__ unsigned long long g_range[2];   // candidate range [lo, hi] (hi == 0: none)

// Waits on a staging copy's barrier before the CTA gives up: each wait
// sleeps up to a millisecond, and a copy of a few tens of kilobytes completes
// within microseconds; this bound is seconds.
constexpr uint32_t kWaitPolls = 4096u;

// Pair table of one pass.  A commuting string K and its partner Q.K agree
// outside the gate's bits, so both hash the key with those bits cleared and
// walk the same probe sequence.  A slot holds (tag << 20) | (late << 10) |
// early: the first string of a pair to arrive claims a free slot as `early`
// (late = early while it is alone); its partner, arriving later, finds it on
// the way (the first free slot of the sequence is claimed by exactly one of
// them, and the other sees the claim) and records itself as `late`.  After
// the pass's barrier a string reads its partner from its own slot, with no
// second walk.  Tags grow with every pass of the CTA, so a slot of an
// earlier pass is free and the table needs no clearing.  Returns the slot,
// or kNoSlot when the table is full.
constexpr uint32_t kNoSlot = 0xffffffffu;
constexpr uint32_t kTagMax = 0xfffu;

template <int W>
__device__ __forceinline__ uint32_t pair_join(const PKey<W>& K, const GateArg<W>& g, uint32_t i,
                                              const PKey<W>* keys_s, uint32_t* tab,
                                              uint32_t tag) {
    constexpr uint32_t S = StageGeom<W>::kSlots;
    constexpr int kBits = S == 2048 ? 11 : 10;
    static_assert(S == (1u << kBits), "slots");
    // multiplicative hash of the key with the gate's bits cleared (K and Q.K
    // agree on it)
    uint64_t hm = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        hm = (hm ^ (K.x[w] & ~g.qx[w])) * 0x9E3779B97F4A7C15ULL;
        hm = (hm ^ (K.z[w] & ~g.qz[w])) * 0xC2B2AE3D27D4EB4FULL;
    }
    uint32_t h = (uint32_t)(hm >> (64 - kBits));
    const PKey<W> P = key_xor(K, g);
    for (uint32_t q = 0; q < S; ++q) {
        uint32_t v = tab[h];
        for (;;) {
            if ((v >> 20) != tag) {                                // free: claim it
                const uint32_t o = atomicCAS(tab + h, v, (tag << 20) | (i << 10) | i);
                if (o == v) return h;
                v = o;
                continue;
            }
            const uint32_t e = v & 0x3ffu;
            if (((v >> 10) & 0x3ffu) != e || !key_eq(keys_s[e], P)) break;   // not mine
            // my partner, alone: only I write this slot now (a claimed slot is
            // changed by the partner of its string alone), no atomic needed
            tab[h] = (v & ~(0x3ffu << 10)) | (i << 10);
            return h;
        }
        h = (h + 1) & (S - 1);
    }
    return kNoSlot;
}

// Statistics of the kept children for the top-M select: the largest
// pattern, the count above the candidate range, the candidates inside it.
struct SelStats {
    unsigned long long out_max;
    uint32_t above;
};

// Write one staged item's kept children at pos (and pos + 1) and fold them
// into the statistics.  Every lane of the warp calls it.
template <int W>
__device__ __forceinline__ void stage_emit(const PKey<W>& K, double va, double b, uint32_t o,
                                           const GateArg<W>& g, PKey<W>* kout, double* cout,
                                           uint64_t pos, SelStats& st, const CandRegions& cd) {
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
    const unsigned long long hi = g_range[1];
    if (hi) {   // uniform
        const unsigned long long lo = g_range[0], w = hi - lo;
        st.above += (a > hi ? 1u : 0u) + (bb > hi ? 1u : 0u);
        // a - lo <= w on unsigned values: lo <= a <= hi (a kept child has a > 0)
        cand_push((o & 1u) && a - lo <= w, a - lo, pos, cd, &g_cn);
        cand_push((o & 2u) && bb - lo <= w, bb - lo, pb, cd, &g_cn);
    }
}

template <int W>
struct PassArgs {
    __device__ __forceinline__ static PKey<W>* keys() {
        return reinterpret_cast<PKey<W>*>(g_stage + Stage<W>::kKeys);
    }
    __device__ __forceinline__ static double* vals() {   // item i at vals()[shift + i]
        return reinterpret_cast<double*>(g_stage + Stage<W>::kVals);
    }
    __device__ __forceinline__ static uint32_t* tab() {
        return reinterpret_cast<uint32_t*>(g_stage + Stage<W>::kTab);
    }
    __device__ __forceinline__ static uint16_t* flags() {   // phase A: slot | live | comm
        return reinterpret_cast<uint16_t*>(g_stage + Stage<W>::kFlags);
    }
};

// Exclusive block scan with one barrier: every warp writes its total, then
// every warp scans the warp totals with shuffles (g_warp may be rewritten
// only after the caller's next barrier).
template <int BLOCK>
__device__ __forceinline__ uint32_t block_scan_1bar(uint32_t v, uint32_t* total) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) g_warp[warp] = x;
    __syncthreads();
    uint32_t t = lane < NW ? g_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, t, warp > 0 ? warp - 1 : 0);
    *total = __shfl_sync(0xffffffffu, t, NW - 1);
    return (warp > 0 ? before : 0u) + x - v;
}

// One pass of the gate over n staged strings.  Phase A: the deferred
// select's kept set, commutation, sign, the normalised coefficient c, and
// each commuting string joins its pair in the table.  Phase B: the later
// string of each pair present computes both merged children,
//   K:   c_K cosh(theta) + c_QK (-sinh(theta)) s,
//   QK:  c_QK cosh(theta) + c_K (-sinh(theta)) s
// (the sign s of Q.K = s QK is also that of Q.QK = s K, Sec. II.B), and
// owns both for writing; a string without its partner owns itself and its
// child QK; an anticommuting string passes through; threshold and weight
// cutoff per child, the identity's merged coefficient as the next
// normaliser.  Then a block scan of the owned children, room(total) for the
// position of the pass's segment (the same on every thread; ~0 when there is
// none: nothing is written) and the write pass.  Three barriers (and any the
// room call takes); the staging arrays are free again when it returns.
// Returns the kept children counted (the same on every thread).
template <int W, int BLOCK, class Room>
__device__ __forceinline__ uint32_t stage_pass(uint32_t n, uint32_t shift, const GateArg<W>& g,
                                               const Pending<W>& pd, double rnorm,
                                               unsigned long long dbits, DevCtl* ctl, int nxt,
                                               uint32_t tag, PKey<W>* kout, double* cout,
                                               SelStats& st, const CandRegions& cd, Room&& room) {
    using A = PassArgs<W>;
    double* vals = A::vals() + shift;
    // phase A; flags: slot (11 bits) | neg << 13 | live << 14 | comm << 15
    for (uint32_t i = threadIdx.x; i < n; i += BLOCK) {
        const PKey<W> K = A::keys()[i];
        const double raw = vals[i];
        const bool live = !pd.on || cap_keep(K, raw, pd.T, pd.all_ties, pd.tk);
        const bool id = key_is_zero(K);
        if (!live && id) set_status(ctl, ST_TRACE_ZERO, 43);
        const bool comm = live && commutes(K, g);
        const bool neg = comm && product_negative(K, g);
        // the identity's normalised value is exactly 1
        vals[i] = id ? 1.0 : __dmul_rn(raw, rnorm);
        uint32_t slot = 0;
        if (comm) {
            slot = pair_join(K, g, i, A::keys(), A::tab(), tag);
            if (slot == kNoSlot) {
                set_status(ctl, ST_CAPACITY, 41);
                slot = 0;
            }
        }
        A::flags()[i] = (uint16_t)(slot | (neg ? 0x2000u : 0u) | (live ? 0x4000u : 0u) |
                                   (comm ? 0x8000u : 0u));
    }
    __syncthreads();                                                  // (1) table built
    // phase B; flags: kept children (2 bits) | alone << 2 | neg << 3 |
    // partner << 4 (10 bits) | late << 14
    uint32_t cnt = 0;
    for (uint32_t i = threadIdx.x; i < n; i += BLOCK) {
        const uint32_t f = A::flags()[i];
        uint32_t o = 0;
        if (f & 0x4000u) {
            const PKey<W> K = A::keys()[i];
            const double c = vals[i];
            if (!(f & 0x8000u)) {            // {P,Q} = 0: unchanged
                bool keep = above(c, dbits) && light(K, g.maxw);
                if (key_is_zero(K)) {
                    ctl->norm[nxt] = c;
                    if (!keep) set_status(ctl, ST_TRACE_ZERO, 1);
                    keep = true;
                }
                o = keep ? 1u : 0u;
            } else {
                const uint32_t v = A::tab()[f & 0x7ffu];
                const uint32_t e = v & 0x3ffu, l = (v >> 10) & 0x3ffu;
                const bool neg = (f & 0x2000u) != 0;
                const double m = __longlong_as_double(
                    __double_as_longlong(g.msh) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
                const PKey<W> KQ = key_xor(K, g);
                double va, vb;
                uint32_t own = 0;
                if (l == e) {                // alone: K and its child QK
                    va = __dmul_rn(c, g.ch);
                    vb = __dmul_rn(c, m);
                    own = 0x4u;
                } else if (l == i) {         // the pair's later string: both
                    const double cq = vals[e];
                    va = __dadd_rn(__dmul_rn(c, g.ch), __dmul_rn(cq, m));
                    vb = __dadd_rn(__dmul_rn(cq, g.ch), __dmul_rn(c, m));
                    vals[i] = va;
                    vals[e] = vb;
                    own = 0x4000u | (e << 4);
                }
                if (own) {
                    bool ka = above(va, dbits) && light(K, g.maxw);
                    bool kb = above(vb, dbits) && light(KQ, g.maxw);
                    if (key_is_zero(K)) {
                        ctl->norm[nxt] = va;
                        if (!ka) set_status(ctl, ST_TRACE_ZERO, 1);
                        ka = true;
                    }
                    if (key_is_zero(KQ)) {
                        ctl->norm[nxt] = vb;
                        if (!kb) set_status(ctl, ST_TRACE_ZERO, 1);
                        kb = true;
                    }
                    o = (ka ? 1u : 0u) | (kb ? 2u : 0u) | own | (neg ? 0x8u : 0u);
                }
            }
        }
        A::flags()[i] = (uint16_t)o;
        cnt += __popc(o & 3u);
    }
    uint32_t tot;
    const uint32_t off = block_scan_1bar<BLOCK>(cnt, &tot);          // (2)
    const unsigned long long base = room(tot);
    if (base != ~0ULL) {
        uint64_t pos = base + off;
        // write pass: warp-uniform rounds (the candidate list is filled warp-wide)
        for (uint32_t i0 = 0; i0 < n; i0 += BLOCK) {
            const uint32_t i = i0 + threadIdx.x;
            uint32_t o = 0;
            PKey<W> K;
#pragma unroll
            for (int w = 0; w < W; ++w) { K.x[w] = 0; K.z[w] = 0; }
            double va = 0.0, vb = 0.0;
            if (i < n) {
                const uint32_t f = A::flags()[i];
                o = f & 3u;
                if (o) {
                    K = A::keys()[i];
                    va = vals[i];
                    if (f & 0x4u) {          // alone: both children from c
                        const double m = __longlong_as_double(
                            __double_as_longlong(g.msh) ^
                            ((f & 0x8u) ? (long long)0x8000000000000000ULL : 0LL));
                        vb = __dmul_rn(va, m);
                        va = __dmul_rn(va, g.ch);
                    } else if (f & 0x4000u) {
                        vb = vals[(f >> 4) & 0x3ffu];
                    }
                }
            }
            stage_emit(K, va, vb, o, g, kout, cout, pos, st, cd);
            pos += __popc(o);
        }
    }
    __syncthreads();                                                  // (3) staging free
    return tot;
}

// The tag of the next pass (every thread calls it): slots hold 12-bit tags,
// so after 4095 passes of one CTA the table is cleared and tags restart.
template <int W, int BLOCK>
__device__ __forceinline__ uint32_t next_tag(uint32_t tag, uint32_t* tab) {
    if (tag < kTagMax) return tag + 1u;
    for (uint32_t k = threadIdx.x; k < (uint32_t)StageGeom<W>::kSlots; k += BLOCK) tab[k] = 0u;
    __syncthreads();
    return 1u;
}

// A partition above the staging capacity, in k sub-passes over the hash
// classes of the key with the gate's sites cleared (about C/2 strings each,
// gathered into the staging arrays).  Its children stay one segment: from
// `pre` on when the caller holds room for 2 np children there (the same on
// every thread), else a first round of the sub-passes only counts them,
// room(total) gives the segment's position (~0: none, nothing is written)
// and a second round writes them.  Every thread calls it; it returns the
// children counted.
template <int W, int BLOCK, class Room>
__device__ __forceinline__ uint32_t merge_long(const PKey<W>* kp, const double* cp, uint64_t np,
                                            const GateArg<W>& g, const Pending<W>& pd,
                                            double rnorm, unsigned long long dbits, DevCtl* ctl,
                                            int nxt, uint32_t* tag,
                                            PKey<W>* kout, double* cout, SelStats& st,
                                            const CandRegions& cd, unsigned long long pre,
                                            Room&& room, unsigned int* cursor_p, uint32_t* s_n) {
    using A = PassArgs<W>;
    constexpr uint32_t C = Stage<W>::C;
    const uint32_t k = (uint32_t)((2 * np + C - 1) / C);
    uint32_t total = 0;
    for (int write = pre != ~0ULL ? 1 : 0; write < 2; ++write) {
        unsigned long long base = pre;
        if (write && pre == ~0ULL) {
            base = room(total);
            if (base == ~0ULL) break;
        }
        uint32_t done = 0;
        for (uint32_t j = 0; j < k; ++j) {
            if (threadIdx.x == 0) *s_n = 0u;
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
                const uint32_t q = atomicAdd(s_n, 1u);
                if (q < C) {
                    A::keys()[q] = K;
                    A::vals()[q] = raw;
                } else {
                    set_status(ctl, ST_CAPACITY, 44);
                }
            }
            __syncthreads();
            // every thread has read the cursor: leave it zero for the next scatter
            if (j == 0 && cursor_p && threadIdx.x == 0) *cursor_p = 0u;
            const uint32_t n = *s_n < C ? *s_n : C;
            *tag = next_tag<W, BLOCK>(*tag, A::tab());
            const unsigned long long at = write ? base + done : ~0ULL;
            done += stage_pass<W, BLOCK>(n, 0u, g, pd, rnorm, dbits, ctl, nxt, *tag, kout, cout,
                                         st, cd, [at](uint32_t) { return at; });
        }
        total = done;
    }
    return total;
}

template <int W, int BLOCK>
struct PartOcc {
    // CTAs per SM the launch bound asks for: the staging and table take
    // Stage<W>::kBytes of shared memory per CTA
    static constexpr int kMin = BLOCK <= 256 ? (W == 1 ? 6 : 5) : 2;
};

}  // namespace

}  // namespace itpp
