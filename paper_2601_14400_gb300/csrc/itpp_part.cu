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
// partition are written as one contiguous segment of the next state buffer
// (one atomic per partition).  The segments are the partitions of the next
// gate of the window, so no scatter runs between the gates of a window.  A
// group holds at most 4^|S| terms; a partition whose output outgrows the
// shared table's limit makes the next gate re-partition.  A gate acting on
// more sites than a window allows is a window of its own, partitioned by its
// pair key (the member of {K, QK} with the gate's lowest bit clear).
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {


// Shared-table geometry per word count: slots, the mean partition size the
// scatter aims for, the largest partition output a following gate of the
// window may read (its commuting terms stay under 70% of the slots), and the
// largest window (sites; a group holds at most 4^sites terms).
template <int W> struct PartGeom;
template <> struct PartGeom<1> {
    static constexpr int kSlots = 2048, kTarget = 700, kSplit = 1400, kWinSites = 5;
};
template <> struct PartGeom<2> {
    static constexpr int kSlots = 1024, kTarget = 300, kSplit = 700, kWinSites = 4;
};

template <int W>
constexpr size_t part_smem_bytes() {
    return (size_t)PartGeom<W>::kSlots * (sizeof(PKey<W>) + sizeof(double) + sizeof(uint32_t));
}

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

}  // namespace

// Scatter the current state into the partitions of a window (force), or,
// inside a window, only when the previous gate left a partition above the
// split limit; otherwise the next merge reads the previous merge's segments.
template <int W>
__global__ void __launch_bounds__(256)
k_part_scatter(Bufs<W> B, DevCtl* ctl, PKey<W>* pk, double* pc, unsigned int* cursor,
               uint64_t pbuf_cap, uint32_t p_max, GateArg<W> g, PartFn<W> f, int force,
               int n_sites, int target) {
    if (ctl->status) return;
    const int cur = ctl->cur;
    if (!force && !ctl->need_scatter) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->count[cur ^ 1] = 0ULL;
            ctl->part_from_scatter = 0;
        }
        return;
    }
    const uint64_t n = live_count(ctl, cur);
    const PartPlan pl = part_plan(n, pbuf_cap, p_max, target);
    const bool fallback = !f.pair && !window_fits(n_sites, f.sites, n);
    if (fallback) f.pair = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->count[cur ^ 1] = 0ULL;
        ctl->part_from_scatter = 1;
        ctl->part_P = pl.P;
        ctl->stat_scatters += 1;
        if (fallback) ctl->part_over = 1;   // the partitions hold for this gate only
    }
    const PKey<W>* __restrict__ kin = B.key(cur);
    const double* __restrict__ cin = B.coef(cur);
    // a deferred top-M select: scan every stored term, keep its kept set
    const Pending<W> pd = pending_of<W>(ctl);
    uint64_t n_scan = n;
    if (pd.on) n_scan = ctl->pend_n < ctl->buf_cap ? ctl->pend_n : ctl->buf_cap;
    // whole warps iterate together (the cursor claim below is warp-wide);
    // U items per thread per round, their loads issued before any claim
    constexpr int U = 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const unsigned int lt = (1u << (threadIdx.x & 31)) - 1u;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n_scan; i0 += U * stride) {
        PKey<W> K[U];
        double c[U];
        bool live[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = i0 + (uint64_t)u * stride + threadIdx.x;
            live[u] = i < n_scan;
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

// Per-item quantities of the gate on one stored term (Eq. for the commuting
// branch: cosh(theta) P and -sinh(theta) s QP).  c is the normalised input
// coefficient, b = c * (-sinh(theta) s) the child it sends to its partner QP.
// For a commuting pair {K, QK} the product sign s is the same seen from both
// members (Q K = s QK implies Q QK = s K), so the partner's incoming addend
// is exactly the b its own thread computes: each term multiplies once by
// rnorm, once by ch and once by msh, and adds its partner's b.
template <int W>
struct PartItem {
    PKey<W> K;
    double c, b;
    bool comm, live;
};

template <int W>
__device__ __forceinline__ PartItem<W> part_item(const PKey<W>* kp, const double* cp, uint64_t i,
                                                 uint64_t np, const GateArg<W>& g, double rnorm,
                                                 const Pending<W>& pd, DevCtl* ctl) {
    PartItem<W> it;
    double raw = 0.0;
    bool neg = false;
#pragma unroll
    for (int w = 0; w < W; ++w) { it.K.x[w] = 0; it.K.z[w] = 0; }
    it.live = false;
    it.comm = false;
    if (i < np) {
        it.K = load_key_stream(kp + i);
        raw = __ldcs(cp + i);
        // a deferred top-M select drops the terms outside its kept set here
        it.live = !pd.on || cap_keep(it.K, raw, pd.T, pd.all_ties, pd.tk);
        if (!it.live && key_is_zero(it.K)) set_status(ctl, ST_TRACE_ZERO, 43);
        it.comm = it.live && commutes(it.K, g);
        neg = it.comm && product_negative(it.K, g);
    }
    // the same double-precision operations on every lane; the identity's
    // normalised value is exactly 1
    it.c = key_is_zero(it.K) ? 1.0 : __dmul_rn(raw, rnorm);
    const double m = __longlong_as_double(
        __double_as_longlong(g.msh) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
    it.b = __dmul_rn(it.c, m);
    return it;
}

// Slot of a key in a partition's table (at most a few thousand slots): a
// multiply-xor of the key's 32-bit halves and one xorshift-multiply round,
// about a third of the instructions of the full key hash.  Partitions are
// chosen by the full hash of a different key (masked or pair key), so the
// two are independent.
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

// Shared-memory table of one partition: commuting keys and their b.  A slot
// belongs to the partition whose tag it holds; tags grow with the partition
// index, so a slot still tagged by an earlier partition of this CTA is free
// and the table needs no clearing between partitions.
template <int W>
__device__ __forceinline__ bool part_insert(const PartItem<W>& it, PKey<W>* t_keys, double* t_b,
                                            uint32_t* t_tag, uint32_t tag) {
    constexpr uint32_t S = PartGeom<W>::kSlots;
    uint32_t h = slot_hash(it.K) & (S - 1);
    for (uint32_t q = 0; q < S; ++q) {
        if (atomicMax(t_tag + h, tag) < tag) {
            t_keys[h] = it.K;
            t_b[h] = it.b;
            return true;
        }
        h = (h + 1) & (S - 1);
    }
    return false;
}

template <int W>
__device__ __forceinline__ bool part_find(const PKey<W>& P, const PKey<W>* t_keys,
                                          const double* t_b, const uint32_t* t_tag, uint32_t tag,
                                          double* out) {
    constexpr uint32_t S = PartGeom<W>::kSlots;
    uint32_t h = slot_hash(P) & (S - 1);
    for (uint32_t q = 0; q < S; ++q) {
        if (t_tag[h] != tag) return false;
        if (key_eq(t_keys[h], P)) { *out = t_b[h]; return true; }
        h = (h + 1) & (S - 1);
    }
    return false;
}

// Branch, merge and truncation of one item against the complete table:
// va (self child, merged) and whether the QP child is emitted.
template <int W>
__device__ __forceinline__ void part_children(const PartItem<W>& it, const GateArg<W>& g,
                                              const PKey<W>* t_keys, const double* t_b,
                                              const uint32_t* t_tag, uint32_t tag, double* va,
                                              bool* emit_b) {
    double pb = 0.0;
    bool found = false;
    if (it.comm) found = part_find(key_xor(it.K, g), t_keys, t_b, t_tag, tag, &pb);
    const double a1 = __dmul_rn(it.c, g.ch);          // cosh(theta) P
    const double sum = __dadd_rn(a1, pb);             // + the partner's child
    *va = !it.comm ? it.c : (found ? sum : a1);       // {P,Q} = 0: unchanged
    *emit_b = it.comm && !found;
}

// Flags of one item after the merge: bit 0 keeps the self child (merged
// value va), bit 1 emits the QK child (value b).  The identity is always
// kept and its merged value is the next normaliser.
template <int W>
__device__ __forceinline__ uint32_t part_flags(const PartItem<W>& it, const GateArg<W>& g,
                                               const PKey<W>* t_keys, const double* t_b,
                                               const uint32_t* t_tag, uint32_t tag,
                                               unsigned long long dbits, DevCtl* ctl, int nxt,
                                               double* va) {
    bool eb;
    part_children(it, g, t_keys, t_b, t_tag, tag, va, &eb);
    if (!it.live) return 0u;
    // threshold and weight cutoff on the merged children (Sec. II.B)
    bool keep_a = above(*va, dbits) && light(it.K, g.maxw);
    const bool keep_b = eb && above(it.b, dbits) && light(key_xor(it.K, g), g.maxw);
    if (key_is_zero(it.K)) {
        ctl->norm[nxt] = *va;
        if (!keep_a) set_status(ctl, ST_TRACE_ZERO, 1);
        keep_a = true;
    }
    return (keep_a ? 1u : 0u) | (keep_b ? 2u : 0u);
}

template <int W>
__device__ __forceinline__ void part_write(const PartItem<W>& it, const GateArg<W>& g, double va,
                                           uint32_t fl, PKey<W>* kout, double* cout,
                                           uint64_t pos) {
    if (fl & 1u) {
        store_key_stream(kout + pos, it.K);
        __stcs(cout + pos, va);
        ++pos;
    }
    if (fl & 2u) {
        store_key_stream(kout + pos, key_xor(it.K, g));
        __stcs(cout + pos, it.b);
    }
}

// Exclusive block scan with one barrier: every warp writes its total, and
// after the barrier every thread sums the totals of the warps before its own
// (s_warp may be rewritten only after the caller's next barrier).
template <int BLOCK>
__device__ __forceinline__ uint32_t scan_one_barrier(uint32_t v, uint32_t* s_warp,
                                                     uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) {
        const uint32_t t = s_warp[w];
        before += w < warp ? t : 0u;
        tot += t;
    }
    *total = tot;
    return before + x - v;
}

// One partition at a time per CTA.  The partition comes from the scatter
// buffer (fixed stride, cursor) or is a segment the previous gate of the
// window wrote (descriptor).  Its items stay in registers (BLOCK x IPT of
// them; a longer partition takes a two-pass path that reloads), the
// commuting ones publish (key, b) in a shared-memory table, then every item
// merges with its partner's b, and the kept children of the partition go to
// one contiguous segment of the next state buffer, recorded as the
// partition's descriptor for the next gate.  Three barriers per partition:
// table built; warp totals written; segment claimed.  The table is read only
// before the second, so the next partition's inserts (tagged p + 1, see
// part_insert) may start as soon as a thread has passed the third.
template <int W, int kPBlock, int kPIpt>
__global__ void __launch_bounds__(kPBlock, (W == 1 ? 1536 : 1024) / kPBlock)
k_gate_part(const PKey<W>* __restrict__ pk, const double* __restrict__ pc,
            unsigned int* __restrict__ cursor, uint64_t pbuf_cap, PartDesc* desc0,
            PartDesc* desc1, Bufs<W> B, DevCtl* ctl, GateArg<W> g, double delta,
            uint64_t cap_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int S = PartGeom<W>::kSlots;
    constexpr uint64_t CHUNK = (uint64_t)kPBlock * kPIpt;
    // a segment above this size makes the next gate re-partition: the
    // shared table's limit, or twice the register chunk for small CTAs
    constexpr uint32_t kSplitAt = (uint32_t)(2 * CHUNK) < (uint32_t)PartGeom<W>::kSplit
                                      ? (uint32_t)(2 * CHUNK) : (uint32_t)PartGeom<W>::kSplit;
    PKey<W>* t_keys = reinterpret_cast<PKey<W>*>(smem);
    double* t_b = reinterpret_cast<double*>(t_keys + S);
    uint32_t* t_tag = reinterpret_cast<uint32_t*>(t_b + S);
    __shared__ uint32_t s_warp[kPBlock / 32];
    __shared__ uint32_t s_scan[kPBlock / 32];
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_total;
    if (ctl->status) return;
    const int cur = ctl->cur, nxt = cur ^ 1;
    const bool from_scatter = ctl->part_from_scatter != 0;
    const uint32_t P = ctl->part_P;
    const uint64_t R = P ? pbuf_cap / P : 0;
    const PartDesc* __restrict__ din = cur ? desc1 : desc0;
    PartDesc* __restrict__ dout = cur ? desc0 : desc1;
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    // the normaliser and the deferred select's kept set are read from shared
    // memory where they are applied (once per item), not held in registers
    // through the merge
    __shared__ Pending<W> s_pd;
    __shared__ double s_rnorm;
    if (threadIdx.x == 0) {
        s_pd = pending_of<W>(ctl);
        s_rnorm = ctl->rnorm[cur];
    }
    const Pending<W>& pd = s_pd;
    const double& rnorm = s_rnorm;
    PKey<W>* __restrict__ kout = B.key(nxt);
    double* __restrict__ cout = B.coef(nxt);
    unsigned long long out_max = 0;   // largest |c| pattern written (top-M select range)
    for (int s2 = threadIdx.x; s2 < S; s2 += kPBlock) t_tag[s2] = 0u;
    __syncthreads();
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
        if (pn < P) {
            uint64_t nn;
            const char *nk, *nc;
            if (from_scatter) {
                nn = cursor[pn];
                if (nn > R) nn = R;
                nk = reinterpret_cast<const char*>(pk + (uint64_t)pn * R);
                nc = reinterpret_cast<const char*>(pc + (uint64_t)pn * R);
            } else {
                nn = din[pn].cnt;
                nk = reinterpret_cast<const char*>(B.key(cur) + din[pn].off);
                nc = reinterpret_cast<const char*>(B.coef(cur) + din[pn].off);
            }
            for (uint64_t b = (uint64_t)threadIdx.x * 128; b < nn * sizeof(PKey<W>); b += 128 * kPBlock)
                asm volatile("prefetch.global.L2 [%0];" :: "l"(nk + b));
            for (uint64_t b = (uint64_t)threadIdx.x * 128; b < nn * sizeof(double); b += 128 * kPBlock)
                asm volatile("prefetch.global.L2 [%0];" :: "l"(nc + b));
        }
        bool ok = true;
        if (np <= CHUNK) {
            // the whole partition in registers, items j*BLOCK + tid (coalesced)
            PartItem<W> it[kPIpt];
#pragma unroll
            for (int j = 0; j < kPIpt; ++j) {
                it[j] = part_item(kp, cp, (uint64_t)j * kPBlock + threadIdx.x, np, g, rnorm, pd, ctl);
                if (it[j].comm) ok &= part_insert(it[j], t_keys, t_b, t_tag, p + 1u);
            }
            if (!ok) set_status(ctl, ST_CAPACITY, 41);
            __syncthreads();                                   // (1) table built
            // every thread has read the cursor: leave it zero for the next scatter
            if (from_scatter && threadIdx.x == 0) cursor[p] = 0u;
            double va[kPIpt];
            uint32_t flags = 0, cnt = 0;
#pragma unroll
            for (int j = 0; j < kPIpt; ++j) {
                const uint32_t fl =
                    part_flags(it[j], g, t_keys, t_b, t_tag, p + 1u, dbits, ctl, nxt, &va[j]);
                flags |= fl << (2 * j);
                cnt += __popc(fl);
            }
            uint32_t tot;
            const uint32_t off = scan_one_barrier<kPBlock>(cnt, s_warp, &tot);   // (2)
            if (threadIdx.x == 0) {
                const unsigned long long base =
                    tot ? atomicAdd(&ctl->count[nxt], (unsigned long long)tot) : 0ULL;
                s_base = base;
                dout[p].off = base;
                dout[p].cnt = tot;
                if (tot > kSplitAt) ctl->part_over = 1;
            }
            __syncthreads();                                   // (3) segment claimed
            const unsigned long long base = s_base;
            if (base + tot > cap_out) {
                if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 2);
                return;
            }
            uint64_t pos = base + off;
#pragma unroll
            for (int j = 0; j < kPIpt; ++j) {
                const uint32_t fl = (flags >> (2 * j)) & 3u;
                part_write(it[j], g, va[j], fl, kout, cout, pos);
                pos += __popc(fl);
                out_max = max(out_max, (fl & 1u) ? abs_pattern(va[j]) : 0ULL);
                out_max = max(out_max, (fl & 2u) ? abs_pattern(it[j].b) : 0ULL);
            }
        } else {
            // a long partition: build the table, count its output, then
            // recompute and write (every item reloaded each pass)
            for (uint64_t i = threadIdx.x; i < np; i += kPBlock) {
                const PartItem<W> x = part_item(kp, cp, i, np, g, rnorm, pd, ctl);
                if (x.comm) ok &= part_insert(x, t_keys, t_b, t_tag, p + 1u);
            }
            if (!ok) set_status(ctl, ST_CAPACITY, 41);
            if (threadIdx.x == 0) s_total = 0u;
            __syncthreads();
            if (from_scatter && threadIdx.x == 0) cursor[p] = 0u;
            for (uint64_t c0 = 0; c0 < np; c0 += kPBlock) {
                const PartItem<W> x = part_item(kp, cp, c0 + threadIdx.x, np, g, rnorm, pd, ctl);
                double va;
                const uint32_t fl =
                    part_flags(x, g, t_keys, t_b, t_tag, p + 1u, dbits, ctl, nxt, &va);
                uint32_t tot;
                block_exclusive_scan<kPBlock>(__popc(fl), &tot, s_scan);
                if (threadIdx.x == 0) s_total += tot;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const uint32_t tot = s_total;
                const unsigned long long base =
                    tot ? atomicAdd(&ctl->count[nxt], (unsigned long long)tot) : 0ULL;
                s_base = base;
                dout[p].off = base;
                dout[p].cnt = tot;
                if (tot > kSplitAt) ctl->part_over = 1;
            }
            __syncthreads();
            const unsigned long long base = s_base;
            if (base + s_total > cap_out) {
                if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 2);
                return;
            }
            uint64_t run = 0;
            for (uint64_t c0 = 0; c0 < np; c0 += kPBlock) {
                const PartItem<W> x = part_item(kp, cp, c0 + threadIdx.x, np, g, rnorm, pd, ctl);
                double va;
                const uint32_t fl =
                    part_flags(x, g, t_keys, t_b, t_tag, p + 1u, dbits, ctl, nxt, &va);
                uint32_t tot;
                const uint32_t off = block_exclusive_scan<kPBlock>(__popc(fl), &tot, s_scan);
                part_write(x, g, va, fl, kout, cout, base + run + off);
                out_max = max(out_max, (fl & 1u) ? abs_pattern(va) : 0ULL);
                out_max = max(out_max, (fl & 2u) ? abs_pattern(x.b) : 0ULL);
                run += tot;
            }
            __syncthreads();   // the table is read until here
        }
    }
    // one atomic per warp for the largest pattern
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) out_max = max(out_max, __shfl_xor_sync(0xffffffffu, out_max, o));
    if ((threadIdx.x & 31) == 0 && out_max) atomicMax(&ctl->out_max, out_max);
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
                                               s.n, s.part_target);
    return cudaGetLastError();
}

template <int W, int BLOCK, int IPT>
static cudaError_t merge_wbi(const DeviceState& s, const GateArg<W>& g, cudaStream_t st) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(k_gate_part<W, BLOCK, IPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)part_smem_bytes<W>());
        // shared memory for every resident CTA's table rather than L1
        cudaFuncSetAttribute(k_gate_part<W, BLOCK, IPT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gate_part<W, BLOCK, IPT>, BLOCK,
                                                      part_smem_bytes<W>());
        if (per_sm < 1) per_sm = 1;
    }
    k_gate_part<W, BLOCK, IPT><<<s.num_sms * per_sm, BLOCK, part_smem_bytes<W>(), st>>>(
        reinterpret_cast<const PKey<W>*>(s.part_keys), s.part_coef, s.part_cursor, s.part_cap,
        s.part_desc[0], s.part_desc[1], pbufs_of<W>(s), s.ctl, g, s.delta, s.buf_cap);
    return cudaGetLastError();
}

template <int W>
static cudaError_t merge_w(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    const GateArg<W> g = gate_of<W>(h);
    switch (s.block * 16 + s.ipt) {
        case 128 * 16 + 1: return merge_wbi<W, 128, 1>(s, g, st);
        case 128 * 16 + 2: return merge_wbi<W, 128, 2>(s, g, st);
        case 128 * 16 + 4: return merge_wbi<W, 128, 4>(s, g, st);
        case 256 * 16 + 1: return merge_wbi<W, 256, 1>(s, g, st);
        case 256 * 16 + 2: return merge_wbi<W, 256, 2>(s, g, st);
        case 256 * 16 + 4: return merge_wbi<W, 256, 4>(s, g, st);
        case 512 * 16 + 1: return merge_wbi<W, 512, 1>(s, g, st);
        case 512 * 16 + 2: return merge_wbi<W, 512, 2>(s, g, st);
        case 512 * 16 + 4: return merge_wbi<W, 512, 4>(s, g, st);
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

int partition_target_default(int W) {
    return W == 1 ? PartGeom<1>::kTarget : PartGeom<2>::kTarget;
}

uint32_t partition_max(uint64_t cap_M, int target) {
    const uint64_t t = (uint64_t)target;
    return (uint32_t)((cap_M + t - 1) / t + 1);
}

}  // namespace itpp
