// itpp_part.cu -- the per-gate merge with the table in shared memory.
//
// A gate's merge only ever pairs a string K with its partner Q.K, and both
// have the same "pair key": the member of {K, Q.K} whose pivot bit (the
// lowest set bit of Q's masks) is clear.  So the state is first scattered
// into hash partitions of the pair key (one streaming pass, one atomic per
// term on the partition's cursor), and then a persistent kernel takes one
// partition at a time per CTA: it builds the partition's merge table in
// shared memory, then runs the branch-emit-merge-truncate tile body
// (itpp_gate_body.cuh) with lookups served from shared memory.  No table
// access reaches HBM; the partition's terms are read twice, the second time
// from L2.  Partitions have a fixed stride in the scatter buffer, sized 1.5x
// the mean partition, so hash-balanced states never overflow one; if one
// does (or a partition's commuting terms exceed the shared table), the
// device status reports ITPP_ERR_CAPACITY.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {


// Shared-table geometry per word count: slots, and the mean partition size
// the scatter aims for (commuting terms of a partition stay well under 70%
// of the slots even when every term commutes).
template <int W> struct PartGeom;
template <> struct PartGeom<1> { static constexpr int kSlots = 2048; static constexpr int kTarget = 700; };
template <> struct PartGeom<2> { static constexpr int kSlots = 1024; static constexpr int kTarget = 350; };

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

template <int W>
struct PivotArg {
    int word;        // 0..W-1: x[word]; W..2W-1: z[word-W]; -1: Q is the identity
    uint64_t bit;
};

template <int W>
__device__ __forceinline__ uint32_t part_of(const PKey<W>& K, const GateArg<W>& g,
                                            const PivotArg<W>& pv, uint32_t P) {
    PKey<W> k = K;
    if (pv.word >= 0) {
        const uint64_t w = pv.word < W ? K.x[pv.word] : K.z[pv.word - W];
        if (w & pv.bit) k = key_xor(K, g);
    }
    const uint64_t h = key_hash(k);   // 32 significant bits
    return (uint32_t)((h * (uint64_t)P) >> 32);
}

}  // namespace

// Scatter the current state into partitions of the gate's pair key.
template <int W>
__global__ void __launch_bounds__(256)
k_part_scatter(Bufs<W> B, DevCtl* ctl, PKey<W>* pk, double* pc, unsigned int* cursor,
               uint64_t pbuf_cap, uint32_t p_max, GateArg<W> g, PivotArg<W> pv) {
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const PartPlan pl = part_plan(n, pbuf_cap, p_max, PartGeom<W>::kTarget);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->count[cur ^ 1] = 0ULL;
    const PKey<W>* __restrict__ kin = B.k[cur];
    const double* __restrict__ cin = B.c[cur];
    // a deferred top-M select: scan every stored term, keep its kept set
    const bool pend = ctl->pend;
    uint64_t n_scan = n;
    unsigned long long T = 0;
    bool all_ties = false;
    PKey<W> tk;
    if (pend) {
        n_scan = ctl->pend_n < ctl->buf_cap ? ctl->pend_n : ctl->buf_cap;
        T = ctl->pend_T;
        all_ties = ctl->pend_all_ties;
#pragma unroll
        for (int w = 0; w < W; ++w) { tk.x[w] = ctl->pend_tie_key[w]; tk.z[w] = ctl->pend_tie_key[W + w]; }
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_scan;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = load_key_stream(kin + i);
        const double c = __ldcs(cin + i);
        if (pend && !cap_keep(K, c, T, all_ties, tk)) {
            if (key_is_zero(K)) set_status(ctl, ST_TRACE_ZERO, 42);
            continue;
        }
        const uint32_t p = part_of(K, g, pv, pl.P);
        const unsigned int pos = atomicAdd(cursor + p, 1u);
        if (pos < pl.R) {
            const uint64_t d = (uint64_t)p * pl.R + pos;
            pk[d] = K;
            pc[d] = c;
        } else {
            set_status(ctl, ST_CAPACITY, 40);
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
                                                 uint64_t np, const GateArg<W>& g, double rnorm) {
    PartItem<W> it;
    double raw = 0.0;
    bool neg = false;
#pragma unroll
    for (int w = 0; w < W; ++w) { it.K.x[w] = 0; it.K.z[w] = 0; }
    it.live = i < np;
    it.comm = false;
    if (it.live) {
        it.K = load_key_stream(kp + i);
        raw = __ldcs(cp + i);
        it.comm = commutes(it.K, g);
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

// Shared-memory table of one partition: commuting keys and their b.
template <int W>
__device__ __forceinline__ bool part_insert(const PartItem<W>& it, PKey<W>* t_keys, double* t_b,
                                            uint32_t* t_tag) {
    constexpr uint32_t S = PartGeom<W>::kSlots;
    uint32_t h = (uint32_t)key_hash(it.K) & (S - 1);
    for (uint32_t q = 0; q < S; ++q) {
        if (atomicCAS(t_tag + h, 0u, 1u) == 0u) {
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
                                          const double* t_b, const uint32_t* t_tag, double* out) {
    constexpr uint32_t S = PartGeom<W>::kSlots;
    uint32_t h = (uint32_t)key_hash(P) & (S - 1);
    for (uint32_t q = 0; q < S; ++q) {
        if (t_tag[h] == 0u) return false;
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
                                              const uint32_t* t_tag, double* va, bool* emit_b) {
    double pb = 0.0;
    bool found = false;
    if (it.comm) found = part_find(key_xor(it.K, g), t_keys, t_b, t_tag, &pb);
    const double a1 = __dmul_rn(it.c, g.ch);          // cosh(theta) P
    const double sum = __dadd_rn(a1, pb);             // + the partner's child
    *va = !it.comm ? it.c : (found ? sum : a1);       // {P,Q} = 0: unchanged
    *emit_b = it.comm && !found;
}

// One partition at a time per CTA: the partition's items stay in registers
// (BLOCK x IPT of them; a longer partition reloads the rest), the commuting
// ones publish (key, b) in a shared-memory table, then every item merges
// with its partner's b and the kept children are written out.
template <int W, int kPBlock, int kPIpt>
__global__ void __launch_bounds__(kPBlock)
k_gate_part(const PKey<W>* __restrict__ pk, const double* __restrict__ pc,
            const unsigned int* __restrict__ cursor, Bufs<W> B, DevCtl* ctl,
            uint64_t pbuf_cap, uint32_t p_max, GateArg<W> g, double delta, uint64_t cap_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int S = PartGeom<W>::kSlots;
    constexpr uint64_t CHUNK = (uint64_t)kPBlock * kPIpt;
    PKey<W>* t_keys = reinterpret_cast<PKey<W>*>(smem);
    double* t_b = reinterpret_cast<double*>(t_keys + S);
    uint32_t* t_tag = reinterpret_cast<uint32_t*>(t_b + S);
    __shared__ uint32_t s_scan[kPBlock / 32];
    __shared__ unsigned long long s_base;
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const PartPlan pl = part_plan(n, pbuf_cap, p_max, PartGeom<W>::kTarget);
    const double rnorm = ctl->rnorm[cur];
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    PKey<W>* __restrict__ kout = B.k[cur ^ 1];
    double* __restrict__ cout = B.c[cur ^ 1];
    for (uint32_t p = blockIdx.x; p < pl.P; p += gridDim.x) {
        uint64_t np = cursor[p];
        if (np > pl.R) np = pl.R;
        const PKey<W>* kp = pk + (uint64_t)p * pl.R;
        const double* cp = pc + (uint64_t)p * pl.R;
        // warm L2 with the partition this CTA takes next
        const uint32_t pn = p + gridDim.x;
        if (pn < pl.P) {
            uint64_t nn = cursor[pn];
            if (nn > pl.R) nn = pl.R;
            const char* nk = reinterpret_cast<const char*>(pk + (uint64_t)pn * pl.R);
            const char* nc = reinterpret_cast<const char*>(pc + (uint64_t)pn * pl.R);
            for (uint64_t b = (uint64_t)threadIdx.x * 128; b < nn * sizeof(PKey<W>); b += 128 * kPBlock)
                asm volatile("prefetch.global.L2 [%0];" :: "l"(nk + b));
            for (uint64_t b = (uint64_t)threadIdx.x * 128; b < nn * sizeof(double); b += 128 * kPBlock)
                asm volatile("prefetch.global.L2 [%0];" :: "l"(nc + b));
        }
        for (int s2 = threadIdx.x; s2 < S; s2 += kPBlock) t_tag[s2] = 0u;
        __syncthreads();
        // items j*BLOCK + tid (coalesced), kept in registers
        PartItem<W> it[kPIpt];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < kPIpt; ++j) {
            it[j] = part_item(kp, cp, (uint64_t)j * kPBlock + threadIdx.x, np, g, rnorm);
            if (it[j].comm) ok &= part_insert(it[j], t_keys, t_b, t_tag);
        }
        for (uint64_t i = CHUNK + threadIdx.x; i < np; i += kPBlock) {
            const PartItem<W> x = part_item(kp, cp, i, np, g, rnorm);
            if (x.comm) ok &= part_insert(x, t_keys, t_b, t_tag);
        }
        if (!ok) set_status(ctl, ST_CAPACITY, 41);
        __syncthreads();
        // the chunk held in registers, then (rarely) the rest of a long partition
        for (uint64_t c0 = 0; c0 < np; c0 += CHUNK) {
            double va[kPIpt];
            bool eb[kPIpt];
            uint32_t flags = 0;
#pragma unroll
            for (int j = 0; j < kPIpt; ++j) {
                if (c0) it[j] = part_item(kp, cp, c0 + (uint64_t)j * kPBlock + threadIdx.x, np, g, rnorm);
                part_children(it[j], g, t_keys, t_b, t_tag, &va[j], &eb[j]);
                bool keep_a = above(va[j], dbits);
                const bool keep_b = eb[j] && above(it[j].b, dbits);
                if (it[j].live) {
                    if (key_is_zero(it[j].K)) {
                        // the identity: its merged coefficient is the new trace
                        ctl->norm[cur ^ 1] = va[j];
                        if (!keep_a) set_status(ctl, ST_TRACE_ZERO, 1);
                        keep_a = true;
                    }
                    flags |= (keep_a ? 1u : 0u) << (2 * j);
                    flags |= (keep_b ? 1u : 0u) << (2 * j + 1);
                }
            }
            uint32_t tot;
            const uint32_t off = block_exclusive_scan<kPBlock>(__popc(flags), &tot, s_scan);
            if (threadIdx.x == 0)
                s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
            __syncthreads();
            const unsigned long long base = s_base;
            if (base + tot > cap_out) {
                if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 2);
                return;
            }
            uint64_t pos = base + off;
#pragma unroll
            for (int j = 0; j < kPIpt; ++j) {
                if ((flags >> (2 * j)) & 1u) {
                    store_key_stream(kout + pos, it[j].K);
                    __stcs(cout + pos, va[j]);
                    ++pos;
                }
                if ((flags >> (2 * j + 1)) & 1u) {
                    store_key_stream(kout + pos, key_xor(it[j].K, g));
                    __stcs(cout + pos, it[j].b);
                    ++pos;
                }
            }
            __syncthreads();
        }
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
static void gate_and_pivot(const HostGate& h, GateArg<W>* g, PivotArg<W>* pv) {
    for (int w = 0; w < W; ++w) { g->qx[w] = h.qx[w]; g->qz[w] = h.qz[w]; }
    g->ch = h.ch;
    g->msh = h.msh;
    g->qyy = h.qyy;
    pv->word = -1;
    pv->bit = 0;
    for (int w = 0; w < 2 * W && pv->word < 0; ++w) {
        const uint64_t m = w < W ? h.qx[w] : h.qz[w - W];
        if (m) { pv->word = w; pv->bit = m & (~m + 1); }
    }
}

template <int W>
static cudaError_t scatter_w(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    GateArg<W> g;
    PivotArg<W> pv;
    gate_and_pivot<W>(h, &g, &pv);
    cudaError_t e = cudaMemsetAsync(s.part_cursor, 0, (size_t)s.part_max * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    uint64_t gs = (s.buf_cap + 255) / 256;
    const uint64_t lim = (uint64_t)s.num_sms * 8;
    if (gs > lim) gs = lim;
    if (gs < 1) gs = 1;
    k_part_scatter<W><<<(int)gs, 256, 0, st>>>(pbufs_of<W>(s), s.ctl,
                                               reinterpret_cast<PKey<W>*>(s.part_keys),
                                               s.part_coef, s.part_cursor, s.part_cap,
                                               s.part_max, g, pv);
    return cudaGetLastError();
}

template <int W, int BLOCK, int IPT>
static cudaError_t merge_wbi(const DeviceState& s, const GateArg<W>& g, cudaStream_t st) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(k_gate_part<W, BLOCK, IPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)part_smem_bytes<W>());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gate_part<W, BLOCK, IPT>, BLOCK,
                                                      part_smem_bytes<W>());
        if (per_sm < 1) per_sm = 1;
    }
    k_gate_part<W, BLOCK, IPT><<<s.num_sms * per_sm, BLOCK, part_smem_bytes<W>(), st>>>(
        reinterpret_cast<const PKey<W>*>(s.part_keys), s.part_coef, s.part_cursor,
        pbufs_of<W>(s), s.ctl, s.part_cap, s.part_max, g, s.delta, s.buf_cap);
    return cudaGetLastError();
}

template <int W>
static cudaError_t merge_w(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    GateArg<W> g;
    PivotArg<W> pv;
    gate_and_pivot<W>(h, &g, &pv);
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

cudaError_t launch_part_scatter(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    return s.W == 1 ? scatter_w<1>(s, h, st) : scatter_w<2>(s, h, st);
}

cudaError_t launch_part_merge(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    return s.W == 1 ? merge_w<1>(s, h, st) : merge_w<2>(s, h, st);
}

uint32_t partition_max(int W, uint64_t cap_M) {
    const uint64_t t = W == 1 ? PartGeom<1>::kTarget : PartGeom<2>::kTarget;
    return (uint32_t)((cap_M + t - 1) / t + 1);
}

}  // namespace itpp
