// itpp_batch.cu -- many independent propagations advanced together.
//
// B instances (each its own Hamiltonian, gate count, state, merge table and
// control block) take their gate g of the current Trotter layer in the same
// launches: a plan kernel lays the active instances' terms and tiles out in
// one index space (exclusive prefix over instances), and the table-build,
// branch-emit and top-M kernels map each item or tile back to its instance.
// Every instance runs the device bodies of the single propagation
// (itpp_gate_body.cuh, itpp_stage.cuh), so its state is bit-identical to a
// plain run.  The merge (merge_path 0) is the partitioned one: every
// instance's terms are scattered into hash partitions of the gate's pair key
// {K, QK} (one index space of partitions over the instances), and
// persistent CTAs merge one partition at a time in shared memory, each
// partition's kept children claimed as one run of its instance's output;
// merge_path 2 builds one global table per instance instead.
// Instances with fewer gates per layer sit out the later steps.  A whole
// layer (all steps) is captured once into a CUDA graph by the C ABI and
// replayed, since every quantity that changes between layers lives on the
// device.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"
#include "itpp_stage.cuh"

namespace itpp {

namespace {

constexpr int kIpt = 2;                               // branch-emit items per thread
constexpr uint64_t kTileH = 4096;                     // histogram tile
constexpr uint64_t kTileC = 256;                      // compaction tile
constexpr unsigned long long kGatherMax = 4096;       // values resolved at once

template <int W>
struct BatchBufs {
    PKey<W>* k[2];
    double* c[2];
    Slot<W>* table;
    DevCtl* ctl;
    const GateArg<W>* gates;    // [B * max_gates]
    const int* n_gates;         // [B]
    unsigned long long* item_prefix;   // [B + 1]
    unsigned long long* tile_prefix;   // [B + 1]
    unsigned long long* cap_prefix;    // [B + 1] (histogram tiles of the select)
    unsigned long long* ccap_prefix;   // [B + 1] (compaction tiles of the select)
    uint64_t buf_cap, table_slots;
    int B, max_gates;
    // partitioned merge
    PKey<W>* pk;
    double* pc;
    unsigned int* cursor;              // [B * part_max]
    uint64_t part_cap;
    uint32_t part_max;
    int part_target, merge_path;
};

template <int W>
BatchBufs<W> batch_bufs(const BatchState& s) {
    BatchBufs<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    b.table = reinterpret_cast<Slot<W>*>(s.table);
    b.ctl = s.ctls;
    b.gates = reinterpret_cast<const GateArg<W>*>(s.gates);
    b.n_gates = s.n_gates;
    b.item_prefix = s.item_prefix;
    b.tile_prefix = s.tile_prefix;
    b.cap_prefix = s.cap_prefix;
    b.ccap_prefix = s.ccap_prefix;
    b.buf_cap = s.buf_cap;
    b.table_slots = s.table_slots;
    b.B = s.B;
    b.max_gates = s.max_gates;
    b.pk = reinterpret_cast<PKey<W>*>(s.part_keys);
    b.pc = s.part_coef;
    b.cursor = s.part_cursor;
    b.part_cap = s.part_cap;
    b.part_max = s.part_max;
    b.part_target = s.part_target;
    b.merge_path = s.merge_path;
    return b;
}

// The pair-key partition function of a gate: the member of {K, Q.K} with
// the gate's lowest bit clear, hashed (as the single propagation builds it
// for a gate partitioned by its pair key).
template <int W>
__device__ __forceinline__ PartFn<W> pair_fn(const GateArg<W>& g) {
    PartFn<W> f;
    bool found = false;
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) {
        const uint64_t m = w < W ? g.qx[w] : g.qz[w - W];
        const uint64_t bit = (!found && m) ? (m & (~m + 1)) : 0ULL;
        if (w < W) f.px[w] = bit; else f.pz[w - W] = bit;
        found = found || m;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) { f.kx[w] = ~0ULL; f.kz[w] = ~0ULL; }
    f.pair = 1;
    f.sites = 0;
    return f;
}

// Instance owning global index i: the last b with prefix[b] <= i.
__device__ __forceinline__ int owner(const unsigned long long* prefix, int B,
                                     unsigned long long i) {
    int lo = 0, hi = B;   // prefix[lo] <= i < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace

// Plan of step `step`: which instances take a gate, their items and tiles.
template <int W>
__global__ void __launch_bounds__(1024) k_b_plan(BatchBufs<W> S, int step, uint64_t kTile) {
    __shared__ unsigned long long s_part[1024];
    for (int b = threadIdx.x; b < S.B; b += blockDim.x) {
        DevCtl* ctl = S.ctl + b;
        const int active = (step < S.n_gates[b]) && !ctl->status;
        ctl->sel_pass = active;   // "takes a gate in this step"
        if (active) ctl->count[ctl->cur ^ 1] = 0ULL;
    }
    __syncthreads();
    unsigned long long carry_i = 0, carry_t = 0;
    for (int base = 0; base < S.B; base += 1024) {
        const int b = base + threadIdx.x;
        unsigned long long items = 0;
        if (b < S.B && S.ctl[b].sel_pass) items = live_count(S.ctl + b, S.ctl[b].cur);
        // merge_path 0: tiles are the instance's pair-key partitions
        unsigned long long tiles = (items + kTile - 1) / kTile;
        if (S.merge_path == 0) {
            tiles = items ? part_plan(items, S.part_cap, S.part_max, S.part_target).P : 0;
            if (b < S.B) S.ctl[b].part_P = (uint32_t)tiles;
        }
        unsigned long long incl = scan1024(items, s_part);
        const unsigned long long tot_i = s_part[1023];
        __syncthreads();
        if (b < S.B) S.item_prefix[b] = carry_i + incl - items;
        incl = scan1024(tiles, s_part);
        const unsigned long long tot_t = s_part[1023];
        __syncthreads();
        if (b < S.B) S.tile_prefix[b] = carry_t + incl - tiles;
        carry_i += tot_i;
        carry_t += tot_t;
    }
    if (threadIdx.x == 0) {
        S.item_prefix[S.B] = carry_i;
        S.tile_prefix[S.B] = carry_t;
    }
}

// merge_path 0: every active instance's terms into the pair-key partitions
// of its gate (one cursor claim per distinct partition per warp).
template <int W>
__global__ void __launch_bounds__(256) k_b_scatter(BatchBufs<W> S, int step) {
    const unsigned long long total = S.item_prefix[S.B];
    const unsigned int lt = (1u << (threadIdx.x & 31)) - 1u;
    // whole warps iterate together (the claim below is warp-wide)
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x; i0 < total;
         i0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long i = i0 + threadIdx.x;
        const bool live = i < total;
        int b = 0;
        uint32_t gp = 0xffffffffu, p = 0;
        uint64_t R = 0;
        PKey<W> K;
        double c = 0.0;
        if (live) {
            b = owner(S.item_prefix, S.B, i);
            const DevCtl* ctl = S.ctl + b;
            const int cur = ctl->cur;
            const uint64_t off = (uint64_t)b * S.buf_cap + (i - S.item_prefix[b]);
            K = load_key_stream(S.k[cur] + off);
            c = __ldcs(S.c[cur] + off);
            const GateArg<W> g = S.gates[(size_t)b * S.max_gates + step];
            const uint32_t P = ctl->part_P;
            R = S.part_cap / P;
            p = part_of(K, g, pair_fn(g), P);
            gp = (uint32_t)b * S.part_max + p;
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, gp);
        const int leader = __ffs(peers) - 1;
        unsigned int base = 0;
        if (live && (threadIdx.x & 31) == leader) base = atomicAdd(S.cursor + gp, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (live) {
            const unsigned int pos = base + __popc(peers & lt);
            if (pos < R) {
                const uint64_t d = (uint64_t)b * S.part_cap + (uint64_t)p * R + pos;
                store_key(S.pk + d, K);
                S.pc[d] = c;
            } else {
                set_status(S.ctl + b, ST_CAPACITY, 40);
            }
        }
    }
}

// merge_path 0: one partition at a time per CTA (any instance), staged in
// shared memory by two bulk copies on an mbarrier, merged by the same pass
// as the single propagation's, its kept children one run of the instance's
// output claimed by one atomic; partitions above the staging capacity in
// sub-passes.  The candidate range of the single propagation's select is
// not used (the batch's select passes over the coefficients).
template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (BLOCK <= 256 ? 4 : 2))
k_b_pmerge(BatchBufs<W> S, int step, double delta) {
    using A = PassArgs<W>;
    constexpr uint32_t C = Stage<W>::C, SL = Stage<W>::S;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_n;
    // the partition's gate, read where used (raw storage: a shared variable
    // gets no constructor, and GateArg has a default member initialiser)
    __shared__ __align__(16) unsigned char s_g_raw[sizeof(GateArg<W>)];
    GateArg<W>& s_g = *reinterpret_cast<GateArg<W>*>(s_g_raw);
    __shared__ double s_rnorm;
    if (threadIdx.x == 0) {
        g_cn = 0u;
        g_range[0] = g_range[1] = 0ULL;
        mbar_init(&s_bar, 1);
    }
    for (uint32_t k = threadIdx.x; k < SL; k += BLOCK) A::tab()[k] = 0u;
    __syncthreads();
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    const unsigned long long total = S.tile_prefix[S.B];
    const CandRegions cd{};
    Pending<W> pd;
    pd.on = false;
    pd.all_ties = false;
    pd.T = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) { pd.tk.x[w] = 0; pd.tk.z[w] = 0; }
    uint32_t tag = 0, parity = 0;
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = owner(S.tile_prefix, S.B, t);
        const uint32_t p = (uint32_t)(t - S.tile_prefix[b]);
        DevCtl* ctl = S.ctl + b;
        const int cur = ctl->cur, nxt = cur ^ 1;
        if (threadIdx.x == 0) {
            s_g = S.gates[(size_t)b * S.max_gates + step];
            s_rnorm = ctl->rnorm[cur];
        }
        // one read of the status for the whole CTA (and the gate published)
        if (__syncthreads_or(threadIdx.x == 0 ? ctl->status : 0)) continue;
        const GateArg<W>& g = s_g;
        const double rnorm = s_rnorm;
        const uint64_t R = S.part_cap / ctl->part_P;
        unsigned int* cur_p = S.cursor + (uint64_t)b * S.part_max + p;
        uint64_t np = *cur_p;
        if (np > R) np = R;
        const PKey<W>* kp = S.pk + (uint64_t)b * S.part_cap + (uint64_t)p * R;
        const double* cp = S.pc + (uint64_t)b * S.part_cap + (uint64_t)p * R;
        // selects, not a runtime index into the parameter's arrays (which
        // would copy them to local memory)
        PKey<W>* kout = (nxt ? S.k[1] : S.k[0]) + (uint64_t)b * S.buf_cap;
        double* cout = (nxt ? S.c[1] : S.c[0]) + (uint64_t)b * S.buf_cap;
        // room: one run of the instance's output, exactly the children counted
        auto room = [&](uint32_t n_out) -> unsigned long long {
            if (threadIdx.x == 0) {
                unsigned long long at = n_out ? atomicAdd(&ctl->count[nxt], (unsigned long long)n_out)
                                              : 0ULL;
                if (at + n_out > S.buf_cap) {
                    set_status(ctl, ST_CAPACITY, 47);
                    at = ~0ULL;
                }
                s_base = at;
            }
            __syncthreads();
            return s_base;
        };
        SelStats st{0ULL, 0u};
        if (np <= C) {
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
            // every thread has read the cursor: leave it zero for the next step
            if (threadIdx.x == 0) *cur_p = 0u;
            tag = next_tag<W, BLOCK>(tag, A::tab());
            stage_pass<W, BLOCK>((uint32_t)np, shift, g, pd, rnorm, dbits, ctl, nxt, tag, kout,
                                 cout, st, cd, room);
        } else {
            merge_long<W, BLOCK>(kp, cp, np, g, pd, rnorm, dbits, ctl, nxt, &tag, kout, cout, st,
                                 cd, ~0ULL, room, cur_p, &s_n);
        }
        // the largest written pattern (overflow check of post_one)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            st.out_max = max(st.out_max, __shfl_xor_sync(0xffffffffu, st.out_max, o));
        if ((threadIdx.x & 31) == 0 && st.out_max) atomicMax(&ctl->out_max, st.out_max);
    }
}

template <int W>
__global__ void __launch_bounds__(256)
k_b_insert(BatchBufs<W> S, int step, int load_pct, int probe_limit) {
    const unsigned long long total = S.item_prefix[S.B];
    int probes = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         i < total; i += (unsigned long long)gridDim.x * blockDim.x) {
        const int b = owner(S.item_prefix, S.B, i);
        DevCtl* ctl = S.ctl + b;
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const uint64_t mask = table_mask(n, S.table_slots, load_pct);
        const uint64_t off = (uint64_t)b * S.buf_cap;
        insert_one(S.k[cur] + off, S.c[cur] + off, i - S.item_prefix[b], ctl,
                   S.table + (uint64_t)b * S.table_slots, mask, ctl->gen,
                   S.gates[(size_t)b * S.max_gates + step], probe_limit, &probes);
    }
    (void)probes;
}

template <int W, int kBlock>
__global__ void __launch_bounds__(kBlock)
k_b_main(BatchBufs<W> S, int step, double delta, int load_pct, int probe_limit) {
    __shared__ uint32_t s_scan[kBlock / 32];
    __shared__ unsigned long long s_base;
    const unsigned long long total = S.tile_prefix[S.B];
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    int probes = 0;
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = owner(S.tile_prefix, S.B, t);
        DevCtl* ctl = S.ctl + b;
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const uint64_t mask = table_mask(n, S.table_slots, load_pct);
        const uint64_t off = (uint64_t)b * S.buf_cap;
        const GateArg<W> g = S.gates[(size_t)b * S.max_gates + step];
        const GlobalLookup<W> lk{S.table + (uint64_t)b * S.table_slots, mask, ctl->gen,
                                 probe_limit, ctl, &probes};
        gate_tile<W, kBlock, kIpt>(t - S.tile_prefix[b], n, S.k[cur] + off, S.c[cur] + off,
                                   S.k[cur ^ 1] + off, S.c[cur ^ 1] + off, ctl, cur, lk, g,
                                   ctl->rnorm[cur], dbits, S.buf_cap, s_scan, &s_base);
        __syncthreads();
    }
}

// Post of every instance that took a gate, then the tile plan of the top-M
// select for the instances above the bound.
template <int W>
__global__ void __launch_bounds__(1024)
k_b_post(BatchBufs<W> S, uint64_t cap_M, int cap_policy) {
    __shared__ unsigned long long s_part[1024];
    for (int b = threadIdx.x; b < S.B; b += blockDim.x) {
        DevCtl* ctl = S.ctl + b;
        ctl->sel_active = 0;
        if (!ctl->sel_pass || ctl->status) continue;
        if (post_one(ctl, cap_M, cap_policy)) {
            const int cur = ctl->cur;
            ctl->count[cur ^ 1] = 0ULL;
            ctl->norm[cur ^ 1] = ctl->norm[cur];
            ctl->rnorm[cur ^ 1] = ctl->rnorm[cur];
        }
    }
    __syncthreads();
    unsigned long long carry_h = 0, carry_c = 0;
    for (int base = 0; base < S.B; base += 1024) {
        const int b = base + threadIdx.x;
        unsigned long long items = 0;
        if (b < S.B && S.ctl[b].sel_active) items = live_count(S.ctl + b, S.ctl[b].cur);
        const unsigned long long th = (items + kTileH - 1) / kTileH;
        const unsigned long long tc = (items + kTileC - 1) / kTileC;
        unsigned long long incl = scan1024(th, s_part);
        const unsigned long long tot_h = s_part[1023];
        __syncthreads();
        if (b < S.B) S.cap_prefix[b] = carry_h + incl - th;
        incl = scan1024(tc, s_part);
        const unsigned long long tot_c = s_part[1023];
        __syncthreads();
        if (b < S.B) S.ccap_prefix[b] = carry_c + incl - tc;
        carry_h += tot_h;
        carry_c += tot_c;
    }
    if (threadIdx.x == 0) {
        S.cap_prefix[S.B] = carry_h;
        S.ccap_prefix[S.B] = carry_c;
    }
}

template <int W>
__global__ void __launch_bounds__(256) k_b_cap_hist(BatchBufs<W> S, int shift) {
    __shared__ unsigned int h[kSelBins];
    const unsigned long long total = S.cap_prefix[S.B];
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = owner(S.cap_prefix, S.B, t);
        DevCtl* ctl = S.ctl + b;
        if (ctl->sel_resolved) continue;   // resolved from its gathered values (uniform)
        for (int k = threadIdx.x; k < kSelBins; k += blockDim.x) h[k] = 0;
        __syncthreads();
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const unsigned long long prefix = ctl->sel_prefix, mask = ctl->sel_mask;
        const double* c = S.c[cur] + (uint64_t)b * S.buf_cap;
        const uint64_t lo = (t - S.cap_prefix[b]) * kTileH;
        const uint64_t hi = lo + kTileH < n ? lo + kTileH : n;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const unsigned long long v = abs_bits(__ldg(c + i));
            if ((v & mask) == prefix) atomicAdd(&h[(v >> shift) & (kSelBins - 1)], 1u);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kSelBins; k += blockDim.x)
            if (h[k]) atomicAdd(&ctl->sel_hist[k], (unsigned long long)h[k]);
        __syncthreads();
    }
}

template <int W>
__global__ void __launch_bounds__(1024) k_b_cap_pick(BatchBufs<W> S, int shift, int last) {
    DevCtl* ctl = S.ctl + blockIdx.x;
    if (!ctl->sel_active || ctl->status || ctl->sel_resolved) return;
    __shared__ unsigned long long s_part[1024];
    cap_pick_block(ctl, shift, last, s_part, kGatherMax);
}

// After a pass whose chosen digit holds at most kGatherMax values: those
// values (the |c| patterns matching the prefix so far) into a list in the
// instance's table scratch.
template <int W>
__global__ void __launch_bounds__(256) k_b_cap_gather(BatchBufs<W> S) {
    const unsigned long long total = S.cap_prefix[S.B];
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = owner(S.cap_prefix, S.B, t);
        DevCtl* ctl = S.ctl + b;
        if (!ctl->sel_small || ctl->sel_resolved || ctl->status) continue;
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const unsigned long long prefix = ctl->sel_prefix, mask = ctl->sel_mask;
        const double* c = S.c[cur] + (uint64_t)b * S.buf_cap;
        unsigned long long* list =
            reinterpret_cast<unsigned long long*>(S.table + (uint64_t)b * S.table_slots);
        const uint64_t lo = (t - S.cap_prefix[b]) * kTileH;
        const uint64_t hi = lo + kTileH < n ? lo + kTileH : n;
        // whole warps iterate together (the append below is warp-wide)
        for (uint64_t i0 = lo; i0 < hi; i0 += blockDim.x) {
            const uint64_t i = i0 + threadIdx.x;
            const unsigned long long v = i < hi ? abs_bits(__ldg(c + i)) : 0ULL;
            const bool hit = i < hi && (v & mask) == prefix;
            const unsigned int m = __ballot_sync(0xffffffffu, hit);
            if (!m) continue;
            const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
            unsigned long long q = 0;
            if (lane == leader) q = atomicAdd(&ctl->sel_cand_n, (unsigned long long)__popc(m));
            q = __shfl_sync(0xffffffffu, q, leader);
            if (hit) {
                const unsigned long long r = q + __popc(m & ((1u << lane) - 1u));
                if (r < kGatherMax) list[r] = v;
                else set_status(ctl, ST_CAPACITY, 49);
            }
        }
    }
}

// The threshold among the gathered values (one CTA per instance): sorted in
// shared memory, the sel_k-th largest is the threshold pattern T; the state
// is then what the last digit pass would leave (prefix T over every bit, the
// rank within the ties of T, their number).
template <int W>
__global__ void __launch_bounds__(1024) k_b_cap_resolve(BatchBufs<W> S) {
    DevCtl* ctl = S.ctl + blockIdx.x;
    if (!ctl->sel_active || ctl->status || !ctl->sel_small || ctl->sel_resolved) return;
    __shared__ unsigned long long v[kGatherMax];
    __shared__ unsigned int s_gt, s_eq;
    const unsigned long long n = ctl->sel_cand_n < kGatherMax ? ctl->sel_cand_n : kGatherMax;
    const unsigned long long* list =
        reinterpret_cast<const unsigned long long*>(S.table + (uint64_t)blockIdx.x * S.table_slots);
    for (unsigned int i = threadIdx.x; i < kGatherMax; i += blockDim.x) v[i] = i < n ? list[i] : 0ULL;
    if (threadIdx.x == 0) s_gt = s_eq = 0u;
    __syncthreads();
    // bitonic sort, descending
    for (unsigned int k = 2; k <= kGatherMax; k <<= 1) {
        for (unsigned int j = k >> 1; j > 0; j >>= 1) {
            for (unsigned int i = threadIdx.x; i < kGatherMax; i += blockDim.x) {
                const unsigned int l = i ^ j;
                if (l > i) {
                    const bool desc = (i & k) == 0;
                    const unsigned long long a = v[i], b = v[l];
                    if (desc ? (a < b) : (a > b)) {
                        v[i] = b;
                        v[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    const unsigned long long k = ctl->sel_k;   // 1 <= k <= n
    const unsigned long long T = v[k - 1];
    unsigned int gt = 0, eq = 0;
    for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) {
        gt += v[i] > T ? 1u : 0u;
        eq += v[i] == T ? 1u : 0u;
    }
    atomicAdd(&s_gt, gt);
    atomicAdd(&s_eq, eq);
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->sel_prefix = T;
        ctl->sel_mask = ~0ULL >> 1;
        ctl->sel_k = k - s_gt;
        ctl->sel_ties = s_eq;
        ctl->sel_tie_k = k - s_gt;
        ctl->sel_resolved = 1;
    }
}

template <int W>
__global__ void __launch_bounds__(kTileC) k_b_cap_ties(BatchBufs<W> S) {
    __shared__ uint32_t s_scan[kTileC / 32];
    __shared__ unsigned long long s_base;
    const unsigned long long total = S.ccap_prefix[S.B];
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = owner(S.ccap_prefix, S.B, t);
        DevCtl* ctl = S.ctl + b;
        if (!tie_select_needed(ctl)) continue;   // uniform over the block
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const uint64_t off = (uint64_t)b * S.buf_cap;
        const uint64_t i = (t - S.ccap_prefix[b]) * kTileC + threadIdx.x;
        const bool tie = i < n && abs_bits(__ldg(S.c[cur] + off + i)) == ctl->sel_prefix;
        uint32_t tot;
        const uint32_t o = block_exclusive_scan<kTileC>(tie ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->sel_tie_n, (unsigned long long)tot) : 0ULL;
        __syncthreads();
        PKey<W>* list = reinterpret_cast<PKey<W>*>(S.table + (uint64_t)b * S.table_slots);
        if (tie) list[s_base + o] = load_key(S.k[cur] + off + i);
        __syncthreads();
    }
}

template <int W>
__global__ void __launch_bounds__(256) k_b_tie_hist(BatchBufs<W> S, int p) {
    DevCtl* ctl = S.ctl + blockIdx.y;
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 0) return;
    const PKey<W>* list = reinterpret_cast<const PKey<W>*>(S.table + (uint64_t)blockIdx.y * S.table_slots);
    tie_hist_range<W>(ctl, list, p, (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x,
                      ctl->sel_tie_n, (unsigned long long)gridDim.x * blockDim.x);
}

template <int W>
__global__ void __launch_bounds__(1024) k_b_tie_pick(BatchBufs<W> S, int p) {
    DevCtl* ctl = S.ctl + blockIdx.x;
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 0) return;
    __shared__ unsigned long long s_part[1024];
    tie_pick_block<W>(ctl, p, s_part);
}

template <int W>
__global__ void __launch_bounds__(256) k_b_tie_find(BatchBufs<W> S) {
    DevCtl* ctl = S.ctl + blockIdx.y;
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 2) return;
    const PKey<W>* list = reinterpret_cast<const PKey<W>*>(S.table + (uint64_t)blockIdx.y * S.table_slots);
    tie_find_range<W>(ctl, list, (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x,
                      ctl->sel_tie_n, (unsigned long long)gridDim.x * blockDim.x);
}

template <int W>
__global__ void __launch_bounds__(kTileC) k_b_cap_compact(BatchBufs<W> S) {
    __shared__ uint32_t s_scan[kTileC / 32];
    __shared__ unsigned long long s_base;
    const unsigned long long total = S.ccap_prefix[S.B];
    for (unsigned long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = owner(S.ccap_prefix, S.B, t);
        DevCtl* ctl = S.ctl + b;
        if (ctl->status) continue;   // uniform over the block
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const uint64_t off = (uint64_t)b * S.buf_cap;
        const unsigned long long T = ctl->sel_prefix;
        const bool all_ties = ctl->sel_k == ctl->sel_ties;
        PKey<W> tk;
#pragma unroll
        for (int w = 0; w < W; ++w) { tk.x[w] = ctl->sel_tie_key[w]; tk.z[w] = ctl->sel_tie_key[W + w]; }
        const uint64_t i = (t - S.ccap_prefix[b]) * kTileC + threadIdx.x;
        PKey<W> K;
        double c = 0;
        bool keep = false;
        if (i < n) {
            K = load_key_stream(S.k[cur] + off + i);
            c = __ldcs(S.c[cur] + off + i);
            keep = cap_keep(K, c, T, all_ties, tk);
            if (key_is_zero(K) && !keep) set_status(ctl, ST_TRACE_ZERO, 2);
        }
        uint32_t tot;
        const uint32_t o = block_exclusive_scan<kTileC>(keep ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
        __syncthreads();
        if (keep) {
            store_key_stream(S.k[cur ^ 1] + off + s_base + o, K);
            __stcs(S.c[cur ^ 1] + off + s_base + o, c);
        }
        __syncthreads();
    }
}

template <int W>
__global__ void k_b_cap_end(BatchBufs<W> S) {
    for (int b = threadIdx.x; b < S.B; b += blockDim.x) {
        DevCtl* ctl = S.ctl + b;
        if (ctl->sel_active) {
            if (!ctl->status) ctl->cur ^= 1;
            ctl->sel_active = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// CTAs per SM of the partition merge that fit (shared memory, registers),
// with its dynamic shared memory allowed; called before any capture.
template <int W, int BLOCK>
static int pmerge_fit() {
    constexpr size_t smem = Stage<W>::kBytes;
    cudaFuncSetAttribute(k_b_pmerge<W, BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_b_pmerge<W, BLOCK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_pmerge<W, BLOCK>, BLOCK, smem);
    return per_sm > 0 ? per_sm : 1;
}

template <int W>
static int pmerge_fit_w(int block) {
    switch (block) {
        case 128: return pmerge_fit<W, 128>();
        case 512: return pmerge_fit<W, 512>();
        default: return pmerge_fit<W, 256>();
    }
}

int batch_merge_fit(int W, int block) {
    return W == 1 ? pmerge_fit_w<1>(block) : pmerge_fit_w<2>(block);
}

template <int W>
static cudaError_t batch_step_w(const BatchState& s, int step, cudaStream_t st) {
    const BatchBufs<W> S = batch_bufs<W>(s);
    const int grid = s.num_sms * 8;
    k_b_plan<W><<<1, 1024, 0, st>>>(S, step, (uint64_t)s.main_block * kIpt);
    if (s.merge_path == 0) {
        k_b_scatter<W><<<s.num_sms * s.scatter_grid, 256, 0, st>>>(S, step);
        const int gm = s.num_sms * s.merge_ctas;
        constexpr size_t smem = Stage<W>::kBytes;
        switch (s.main_block) {
            case 128: k_b_pmerge<W, 128><<<gm, 128, smem, st>>>(S, step, s.delta); break;
            case 512: k_b_pmerge<W, 512><<<gm, 512, smem, st>>>(S, step, s.delta); break;
            default:  k_b_pmerge<W, 256><<<gm, 256, smem, st>>>(S, step, s.delta); break;
        }
    } else {
        k_b_insert<W><<<s.num_sms * s.insert_grid, 256, 0, st>>>(S, step, s.load_pct, s.probe_limit);
        const int gm = s.num_sms * s.main_grid;
        switch (s.main_block) {
            case 128: k_b_main<W, 128><<<gm, 128, 0, st>>>(S, step, s.delta, s.load_pct, s.probe_limit); break;
            case 512: k_b_main<W, 512><<<gm, 512, 0, st>>>(S, step, s.delta, s.load_pct, s.probe_limit); break;
            default:  k_b_main<W, 256><<<gm, 256, 0, st>>>(S, step, s.delta, s.load_pct, s.probe_limit); break;
        }
    }
    k_b_post<W><<<1, 1024, 0, st>>>(S, s.cap_M, s.cap_policy);
    if (s.cap_policy == 1) {
        const int shifts[5] = {50, 37, 24, 11, 0};
        for (int p = 0; p < 5; ++p) {
            k_b_cap_hist<W><<<grid, 256, 0, st>>>(S, shifts[p]);
            k_b_cap_pick<W><<<s.B, 1024, 0, st>>>(S, shifts[p], p == 4 ? 1 : 0);
            if (p < 4) {   // instances whose digit held few values: resolved now
                k_b_cap_gather<W><<<grid, 256, 0, st>>>(S);
                k_b_cap_resolve<W><<<s.B, 1024, 0, st>>>(S);
            }
        }
        k_b_cap_ties<W><<<grid, kTileC, 0, st>>>(S);
        const dim3 g2(8, s.B);
        for (int p = 0; p < 8 * W; ++p) {
            k_b_tie_hist<W><<<g2, 256, 0, st>>>(S, p);
            k_b_tie_pick<W><<<s.B, 1024, 0, st>>>(S, p);
        }
        k_b_tie_find<W><<<g2, 256, 0, st>>>(S);
        k_b_cap_compact<W><<<grid, kTileC, 0, st>>>(S);
        k_b_cap_end<W><<<1, 1024, 0, st>>>(S);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchState& s, int step, cudaStream_t st) {
    return s.W == 1 ? batch_step_w<1>(s, step, st) : batch_step_w<2>(s, step, st);
}

int batch_step_launches(const BatchState& s) {
    return 4 + (s.cap_policy == 1 ? 5 * 2 + 4 * 2 + 1 + 8 * s.W * 2 + 3 : 0);
}

}  // namespace itpp
