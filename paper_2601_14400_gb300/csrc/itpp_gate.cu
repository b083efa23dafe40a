// itpp_gate.cu -- the per-gate hot path of imaginary-time Pauli propagation
// on sm_103a: one elementary step of Algorithm 1 (propagate every term with
// Eq. (ITPP_PropRules), accumulate equal strings, truncate, normalise).
//
// Merge structure used here.  For a gate Q the children of a term K are K
// itself and, when [K, Q] = 0, the string Q.K.  Both maps are bijections on
// strings, and Q.K commutes with Q exactly when K does, so a string receives
// at most two contributions: from K itself and from its partner Q.K, and an
// anticommuting string receives only its own.  The merge therefore reduces
// to a partner lookup:
//   k_gate_insert  puts every commuting term (key, raw c) into an
//                  open-addressing table keyed on (x, z);
//   k_gate_main    streams the terms once more; an anticommuting term passes
//                  through, a commuting term K finds its partner in the table
//                  and writes  c_K cosh + s c_QK (-sinh)  -- or, when the
//                  partner is absent, writes c_K cosh and emits the new string
//                  Q.K with s c_K (-sinh).  |c| <= delta is dropped in the
//                  same pass (stream compaction: block scan + one atomic per
//                  tile), and the identity's new coefficient becomes the
//                  normaliser the next read divides by.
// Two addends summed in one rounding are order-independent, so the result
// is bit-identical to any correct sequential accumulation.
#include "itpp_common.cuh"
#include "itpp_launch.h"

namespace itpp {

template <int W>
struct Bufs {
    PKey<W>* k[2];
    double* c[2];
};

template <int W>
static Bufs<W> bufs_of(const DeviceState& s) {
    Bufs<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    return b;
}

template <int W>
static GateArg<W> gate_arg(const HostGate& h) {
    GateArg<W> g;
    for (int w = 0; w < W; ++w) { g.qx[w] = h.qx[w]; g.qz[w] = h.qz[w]; }
    g.ch = h.ch;
    g.msh = h.msh;
    g.qyy = h.qyy;
    return g;
}

// ---------------------------------------------------------------------------
// Merge-table probe
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ bool table_find(const Slot<W>* __restrict__ table, uint64_t mask,
                                           unsigned gen, const PKey<W>& P, double* c,
                                           int probe_limit, DevCtl* ctl, int* probes) {
    uint64_t h = key_hash(P) & mask;
    for (int p = 0; p < probe_limit; ++p) {
        const Slot<W>* s = table + h;
        const ulonglong2* v = reinterpret_cast<const ulonglong2*>(s);
        PKey<W> k;
        double cc;
        unsigned tag;
        if constexpr (W == 1) {
            ulonglong2 a = __ldg(v), b = __ldg(v + 1);
            k.x[0] = a.x;
            k.z[0] = a.y;
            cc = __longlong_as_double((long long)b.x);
            tag = (unsigned)(b.y & 0xffffffffULL);
        } else {
            ulonglong2 a = __ldg(v), b = __ldg(v + 1), d = __ldg(v + 2);
            k.x[0] = a.x; k.x[1] = a.y;
            k.z[0] = b.x; k.z[1] = b.y;
            cc = __longlong_as_double((long long)d.x);
            tag = (unsigned)(d.y & 0xffffffffULL);
        }
        *probes += 1;
        if (tag != gen) return false;
        if (key_eq(k, P)) { *c = cc; return true; }
        h = (h + 1) & mask;
    }
    set_status(ctl, ST_HASH_PROBE, 2);
    return false;
}

// Claim a free slot for key K (keys are distinct, so no equality test is
// needed while building) and store it.
template <int W>
__device__ __forceinline__ bool table_insert(Slot<W>* table, uint64_t mask, unsigned gen,
                                             const PKey<W>& K, double c, uint32_t idx,
                                             int probe_limit, int* probes) {
    uint64_t h = key_hash(K) & mask;
    for (int p = 0; p < probe_limit; ++p) {
        Slot<W>* s = table + h;
        unsigned t = __ldcg(&s->tag);
        // A slot is free when its tag is from an older gate; a failed CAS
        // returns the tag now stored, and the loop ends as soon as that is
        // the current generation (at most one retry per competitor).
        while (t != gen) {
            unsigned old = atomicCAS(&s->tag, t, gen);
            if (old == t) {
                ulonglong2* v = reinterpret_cast<ulonglong2*>(s);
                if constexpr (W == 1) {
                    v[0] = make_ulonglong2(K.x[0], K.z[0]);
                } else {
                    v[0] = make_ulonglong2(K.x[0], K.x[1]);
                    v[1] = make_ulonglong2(K.z[0], K.z[1]);
                }
                s->c = c;
                s->idx = idx;
                *probes += p + 1;
                return true;
            }
            t = old;
        }
        h = (h + 1) & mask;
    }
    *probes += probe_limit;
    return false;
}

// ---------------------------------------------------------------------------
// k_gate_insert: table of the commuting terms of the current state.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256)
k_gate_insert(Bufs<W> B, DevCtl* ctl, Slot<W>* table, uint64_t alloc_slots, int load_pct,
              GateArg<W> g, int probe_limit) {
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const unsigned gen = ctl->gen;
    const uint64_t mask = table_mask(n, alloc_slots, load_pct);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->count[cur ^ 1] = 0ULL;
    const PKey<W>* __restrict__ kin = B.k[cur];
    const double* __restrict__ cin = B.c[cur];
    int probes = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = load_key(kin + i);
        if (!commutes(K, g)) continue;
        const double c = __ldg(cin + i);
        if (!table_insert(table, mask, gen, K, c, (uint32_t)i, probe_limit, &probes))
            set_status(ctl, ST_HASH_PROBE, 1);
    }
    // probe statistics (one atomic per warp)
    for (int o = 16; o > 0; o >>= 1) probes += __shfl_down_sync(0xffffffffu, probes, o);
    if ((threadIdx.x & 31) == 0 && probes) atomicAdd(&ctl->stat_probes, (unsigned long long)probes);
}

// ---------------------------------------------------------------------------
// k_gate_main: branch, emit, merge (partner lookup), truncate, compact.
// Each thread owns IPT consecutive input terms and up to 2*IPT outputs; a
// block scan orders the outputs of a tile and one atomic places the tile.
// ---------------------------------------------------------------------------
template <int W, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK)
k_gate_main(Bufs<W> B, DevCtl* ctl, const Slot<W>* __restrict__ table, uint64_t alloc_slots,
            int load_pct, GateArg<W> g, double delta, uint64_t cap_out, int probe_limit) {
    __shared__ uint32_t s_scan[BLOCK / 32];
    __shared__ unsigned long long s_base;
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rnorm = ctl->rnorm[cur];
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    const unsigned gen = ctl->gen;
    const uint64_t mask = table_mask(n, alloc_slots, load_pct);
    const PKey<W>* __restrict__ kin = B.k[cur];
    const double* __restrict__ cin = B.c[cur];
    PKey<W>* __restrict__ kout = B.k[cur ^ 1];
    double* __restrict__ cout = B.c[cur ^ 1];
    constexpr uint64_t TILE = (uint64_t)BLOCK * IPT;
    const uint64_t tiles = (n + TILE - 1) / TILE;
    int probes = 0;

    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        PKey<W> K[IPT];
        double va[IPT], vb[IPT];
        uint32_t flags = 0;
        const uint64_t i0 = t * TILE + (uint64_t)threadIdx.x * IPT;
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint64_t i = i0 + j;
            va[j] = 0.0;
            vb[j] = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) { K[j].x[w] = 0; K[j].z[w] = 0; }
            if (i < n) {
                K[j] = load_key_stream(kin + i);
                // normalise on load: the previous gate's trace rescaling
                const double c = normalised(__ldcs(cin + i), rnorm, key_is_zero(K[j]));
                bool keep_b = false;
                if (!commutes(K[j], g)) {
                    va[j] = c;                                   // {P,Q} = 0: unchanged
                } else {
                    const double m = product_negative(K[j], g) ? -g.msh : g.msh;
                    const PKey<W> P = key_xor(K[j], g);
                    double cp_raw;
                    if (table_find(table, mask, gen, P, &cp_raw, probe_limit, ctl, &probes)) {
                        const double cp = normalised(cp_raw, rnorm, key_is_zero(P));
                        va[j] = __dadd_rn(__dmul_rn(c, g.ch), __dmul_rn(cp, m));
                    } else {
                        va[j] = __dmul_rn(c, g.ch);              // cosh(theta) P
                        vb[j] = __dmul_rn(c, m);                 // -sinh(theta) s (Q.P)
                        keep_b = above(vb[j], dbits);
                    }
                }
                bool keep_a = above(va[j], dbits);
                if (key_is_zero(K[j])) {
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
        const uint32_t off = block_exclusive_scan<BLOCK>(__popc(flags), &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
        __syncthreads();
        const unsigned long long base = s_base;
        if (base + tot > cap_out) {
            if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 2);
            continue;
        }
        uint64_t pos = base + off;
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            if ((flags >> (2 * j)) & 1u) {
                store_key_stream(kout + pos, K[j]);
                __stcs(cout + pos, va[j]);
                ++pos;
            }
            if ((flags >> (2 * j + 1)) & 1u) {
                store_key_stream(kout + pos, key_xor(K[j], g));
                __stcs(cout + pos, vb[j]);
                ++pos;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) probes += __shfl_down_sync(0xffffffffu, probes, o);
    if ((threadIdx.x & 31) == 0 && probes) atomicAdd(&ctl->stat_probes, (unsigned long long)probes);
}

// ---------------------------------------------------------------------------
// k_gate_post: switch buffers, advance the table generation, statistics and
// the term bound.  One warp.
// ---------------------------------------------------------------------------
__global__ void k_gate_post(DevCtl* ctl, uint64_t cap_M, int cap_policy) {
    __shared__ int s_active;
    if (ctl->status) return;
    if (threadIdx.x == 0) {
        const int cur = ctl->cur, nxt = cur ^ 1;
        const unsigned long long n_in = ctl->count[cur], n_out = ctl->count[nxt];
        ctl->cur = nxt;
        ctl->rnorm[nxt] = __ddiv_rn(1.0, ctl->norm[nxt]);
        ctl->gen = ctl->gen + 1u;
        if (ctl->gen == 0u) set_status(ctl, ST_STATE, 1);   // generation counter wrapped
        ctl->stat_gates += 1;
        ctl->stat_in += n_in;
        int active = 0;
        unsigned long long kept = n_out;
        if (cap_M && n_out > cap_M) {
            if (cap_policy == 0) {
                set_status(ctl, ST_CAPACITY, 1);
            } else {
                active = 1;
                kept = cap_M;
                ctl->sel_k = cap_M;
                ctl->sel_prefix = 0;
                ctl->sel_mask = 0;
                ctl->sel_pass = 0;
                ctl->sel_tie_n = 0;
                ctl->sel_tie_k = 0;
                ctl->sel_tie_state = 0;
                ctl->sel_tie_pass = 0;
                for (int w = 0; w < 4; ++w) ctl->sel_tie_key[w] = 0;
                ctl->stat_cap += 1;
            }
        }
        ctl->sel_active = active;
        ctl->stat_out += kept;
        if (kept > ctl->stat_peak) ctl->stat_peak = kept;
        s_active = active;
    }
    __syncthreads();
    if (s_active)
        for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
}

// ---------------------------------------------------------------------------
// Top-M select (term bound with cap_policy 1): radix select of the cap_M-th
// largest |c| over its 63-bit pattern (monotone for non-negative doubles),
// 13 bits per pass from the top.  When only some of the terms at that
// threshold fit, a second radix select over their keys (16 bits per pass,
// words x[0..W-1] then z[0..W-1]) finds the largest key to keep, so that the
// kept set is "the cap_M largest |c|, ties by ascending key".  Every kernel
// of the chain returns at once when the bound holds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double c) {
    return (unsigned long long)__double_as_longlong(c) & 0x7fffffffffffffffULL;
}

template <int W>
__global__ void __launch_bounds__(256)
k_cap_hist(Bufs<W> B, DevCtl* ctl, int shift) {
    if (!ctl->sel_active || ctl->status) return;
    __shared__ unsigned int h[kSelBins];
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const unsigned long long prefix = ctl->sel_prefix, mask = ctl->sel_mask;
    const double* __restrict__ c = B.c[cur];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = abs_bits(__ldg(c + i));
        if ((b & mask) == prefix) atomicAdd(&h[(b >> shift) & (kSelBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (h[b]) atomicAdd(&ctl->sel_hist[b], (unsigned long long)h[b]);
}

// Block-wide 64-bit inclusive scan of one value per thread (1024 threads).
__device__ __forceinline__ unsigned long long scan1024(unsigned long long v,
                                                       unsigned long long* s) {
    const int t = threadIdx.x;
    s[t] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long a = (t >= o) ? s[t - o] : 0ULL;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    const unsigned long long r = s[t];
    __syncthreads();
    return r;
}

// One CTA of 1024 threads: the digit holding the k-th largest |c|.
__global__ void __launch_bounds__(1024) k_cap_pick(DevCtl* ctl, int shift, int last) {
    if (!ctl->sel_active || ctl->status) return;
    __shared__ unsigned long long s_part[1024];
    constexpr int PER = kSelBins / 1024;
    const int t = threadIdx.x;
    // thread t owns digits kSelBins-1-PER*t ... kSelBins-PER*(t+1) (descending)
    unsigned long long hv[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        hv[j] = ctl->sel_hist[kSelBins - 1 - PER * t - j];
        sum += hv[j];
    }
    const unsigned long long incl = scan1024(sum, s_part);
    unsigned long long run = incl - sum;
    const unsigned long long k = ctl->sel_k;
    __syncthreads();
    if (run < k && k <= incl) {
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            if (run < k && k <= run + hv[j]) {
                const int digit = kSelBins - 1 - PER * t - j;
                ctl->sel_k = k - run;
                ctl->sel_prefix |= (unsigned long long)digit << shift;
                ctl->sel_mask |= (unsigned long long)(kSelBins - 1) << shift;
                if (last) {
                    ctl->sel_ties = hv[j];
                    ctl->sel_tie_k = k - run;
                }
            }
            run += hv[j];
        }
    }
    __syncthreads();
    for (int b = t; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
}

// Compact the keys of the terms at the threshold into the tie list, when
// only some of them are kept.  Also prepares the output buffer.
template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_cap_ties(Bufs<W> B, DevCtl* ctl, PKey<W>* tie_list) {
    if (!ctl->sel_active || ctl->status) return;
    __shared__ uint32_t s_scan[BLOCK / 32];
    __shared__ unsigned long long s_base;
    const int cur = ctl->cur;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->count[cur ^ 1] = 0ULL;
        ctl->norm[cur ^ 1] = ctl->norm[cur];
        ctl->rnorm[cur ^ 1] = ctl->rnorm[cur];
    }
    if (ctl->sel_k == ctl->sel_ties) return;   // every tie is kept
    const uint64_t n = live_count(ctl, cur);
    const unsigned long long T = ctl->sel_prefix;
    const uint64_t tiles = (n + BLOCK - 1) / BLOCK;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t i = t * BLOCK + threadIdx.x;
        const bool tie = i < n && abs_bits(__ldg(B.c[cur] + i)) == T;
        uint32_t tot;
        const uint32_t off = block_exclusive_scan<BLOCK>(tie ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->sel_tie_n, (unsigned long long)tot) : 0ULL;
        __syncthreads();
        if (tie) tie_list[s_base + off] = load_key(B.k[cur] + i);
    }
}

template <int W>
__device__ __forceinline__ uint64_t key_word(const PKey<W>& k, int wi) {
    return wi < W ? k.x[wi] : k.z[wi - W];
}

// After p passes of 16 bits, the top 16p bits of the key (word 0 first) are
// fixed; does key k agree with the prefix there?
template <int W>
__device__ __forceinline__ bool tie_prefix_match(const PKey<W>& k, const uint64_t* pre, int p) {
    const int full = p / 4, r = 16 * (p % 4);
    for (int w = 0; w < full; ++w)
        if (key_word(k, w) != pre[w]) return false;
    if (r > 0 && (key_word(k, full) >> (64 - r)) != (pre[full] >> (64 - r))) return false;
    return true;
}

template <int W>
__global__ void __launch_bounds__(256)
k_tie_hist(DevCtl* ctl, const PKey<W>* tie_list, int p) {
    if (!ctl->sel_active || ctl->status || ctl->sel_k == ctl->sel_ties) return;
    if (ctl->sel_tie_state != 0) return;
    uint64_t pre[2 * W];
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) pre[w] = ctl->sel_tie_key[w];
    const int wi = p / 4, shift = 48 - 16 * (p % 4);
    const unsigned long long E = ctl->sel_tie_n;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         i < E + 31; i += (unsigned long long)gridDim.x * blockDim.x) {
        // whole warps iterate together so that equal digits are aggregated
        const bool in = i < E;
        unsigned int digit = 0xffffffffu;
        if (in) {
            const PKey<W> k = tie_list[i];
            if (tie_prefix_match<W>(k, pre, p))
                digit = (unsigned int)((key_word(k, wi) >> shift) & (kTieBins - 1));
        }
        const unsigned int peers = __match_any_sync(__activemask(), digit);
        const int leader = __ffs(peers) - 1;
        if (digit != 0xffffffffu && (threadIdx.x & 31) == leader)
            atomicAdd(&ctl->tie_hist[digit], (unsigned long long)__popc(peers));
    }
}

// One CTA: the digit holding the k-th smallest key.
template <int W>
__global__ void __launch_bounds__(1024) k_tie_pick(DevCtl* ctl, int p) {
    if (!ctl->sel_active || ctl->status || ctl->sel_k == ctl->sel_ties) return;
    if (ctl->sel_tie_state != 0) return;
    __shared__ unsigned long long s_part[1024];
    constexpr int PER = kTieBins / 1024;
    const int t = threadIdx.x;
    unsigned long long sum = 0;
    for (int j = 0; j < PER; ++j) sum += ctl->tie_hist[PER * t + j];
    const unsigned long long incl = scan1024(sum, s_part);
    unsigned long long run = incl - sum;
    const unsigned long long k = ctl->sel_tie_k;
    const int wi = p / 4, shift = 48 - 16 * (p % 4);
    __syncthreads();
    if (run < k && k <= incl) {
        for (int j = 0; j < PER; ++j) {
            const unsigned long long hv = ctl->tie_hist[PER * t + j];
            if (run < k && k <= run + hv) {
                const unsigned long long digit = (unsigned long long)(PER * t + j);
                ctl->sel_tie_k = k - run;
                ctl->sel_tie_key[wi] |= digit << shift;
                if (p == 8 * W - 1) ctl->sel_tie_state = 1;      // every bit fixed
                else if (hv == 1) ctl->sel_tie_state = 2;        // unique candidate
                ctl->sel_tie_pass = p + 1;
            }
            run += hv;
        }
    }
    __syncthreads();
    for (int b = t; b < kTieBins; b += blockDim.x) ctl->tie_hist[b] = 0ULL;
}

// The unique candidate of a prefix is the k-th key: copy it whole.
template <int W>
__global__ void __launch_bounds__(256) k_tie_find(DevCtl* ctl, const PKey<W>* tie_list) {
    if (!ctl->sel_active || ctl->status || ctl->sel_k == ctl->sel_ties) return;
    if (ctl->sel_tie_state != 2) return;
    uint64_t pre[2 * W];
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) pre[w] = ctl->sel_tie_key[w];
    const int p = ctl->sel_tie_pass;
    const unsigned long long E = ctl->sel_tie_n;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < E;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const PKey<W> k = tie_list[i];
        if (tie_prefix_match<W>(k, pre, p)) {
            for (int w = 0; w < 2 * W; ++w) ctl->sel_tie_key[w] = key_word(k, w);
        }
    }
}

template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_cap_compact(Bufs<W> B, DevCtl* ctl) {
    if (!ctl->sel_active || ctl->status) return;
    __shared__ uint32_t s_scan[BLOCK / 32];
    __shared__ unsigned long long s_base;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const unsigned long long T = ctl->sel_prefix;
    const bool all_ties = ctl->sel_k == ctl->sel_ties;
    PKey<W> tk;
#pragma unroll
    for (int w = 0; w < W; ++w) { tk.x[w] = ctl->sel_tie_key[w]; tk.z[w] = ctl->sel_tie_key[W + w]; }
    const uint64_t tiles = (n + BLOCK - 1) / BLOCK;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t i = t * BLOCK + threadIdx.x;
        PKey<W> K;
        double c = 0;
        bool keep = false;
        if (i < n) {
            K = load_key_stream(B.k[cur] + i);
            c = __ldcs(B.c[cur] + i);
            const unsigned long long b = abs_bits(c);
            keep = (b > T) || (b == T && (all_ties || !key_less(tk, K)));
            if (key_is_zero(K) && !keep) set_status(ctl, ST_TRACE_ZERO, 2);
        }
        uint32_t tot;
        const uint32_t off = block_exclusive_scan<BLOCK>(keep ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
        __syncthreads();
        if (keep) {
            store_key_stream(B.k[cur ^ 1] + s_base + off, K);
            __stcs(B.c[cur ^ 1] + s_base + off, c);
        }
    }
}

__global__ void k_cap_end(DevCtl* ctl) {
    if (threadIdx.x == 0 && ctl->sel_active) {
        if (!ctl->status) ctl->cur ^= 1;
        ctl->sel_active = 0;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int stream_grid(const DeviceState& s, int block, int per_sm) {
    uint64_t g = (s.buf_cap + block - 1) / block;
    uint64_t lim = (uint64_t)s.num_sms * per_sm;
    if (g > lim) g = lim;
    if (g < 1) g = 1;
    return (int)g;
}

template <int W>
static cudaError_t insert_w(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    k_gate_insert<W><<<stream_grid(s, 256, 8), 256, 0, st>>>(
        bufs_of<W>(s), s.ctl, reinterpret_cast<Slot<W>*>(s.table), s.table_slots, s.load_pct,
        gate_arg<W>(h), s.probe_limit);
    return cudaGetLastError();
}

cudaError_t launch_gate_insert(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    return s.W == 1 ? insert_w<1>(s, h, st) : insert_w<2>(s, h, st);
}

template <int W, int BLOCK, int IPT>
static cudaError_t main_wbi(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    static int per_sm = -1;
    if (per_sm < 0) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gate_main<W, BLOCK, IPT>, BLOCK, 0);
        per_sm = b > 0 ? b : 1;
    }
    uint64_t tiles = (s.buf_cap + (uint64_t)BLOCK * IPT - 1) / ((uint64_t)BLOCK * IPT);
    uint64_t g = (uint64_t)s.num_sms * per_sm;
    if (g > tiles) g = tiles;
    if (g < 1) g = 1;
    k_gate_main<W, BLOCK, IPT><<<(int)g, BLOCK, 0, st>>>(
        bufs_of<W>(s), s.ctl, reinterpret_cast<const Slot<W>*>(s.table), s.table_slots,
        s.load_pct, gate_arg<W>(h), s.delta, s.buf_cap, s.probe_limit);
    return cudaGetLastError();
}

template <int W>
static cudaError_t main_w(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    switch (s.block * 16 + s.ipt) {
        case 128 * 16 + 1: return main_wbi<W, 128, 1>(s, h, st);
        case 128 * 16 + 2: return main_wbi<W, 128, 2>(s, h, st);
        case 128 * 16 + 4: return main_wbi<W, 128, 4>(s, h, st);
        case 256 * 16 + 1: return main_wbi<W, 256, 1>(s, h, st);
        case 256 * 16 + 2: return main_wbi<W, 256, 2>(s, h, st);
        case 256 * 16 + 4: return main_wbi<W, 256, 4>(s, h, st);
        case 512 * 16 + 1: return main_wbi<W, 512, 1>(s, h, st);
        case 512 * 16 + 2: return main_wbi<W, 512, 2>(s, h, st);
        case 512 * 16 + 4: return main_wbi<W, 512, 4>(s, h, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gate_main(const DeviceState& s, const HostGate& h, cudaStream_t st) {
    return s.W == 1 ? main_w<1>(s, h, st) : main_w<2>(s, h, st);
}

cudaError_t launch_gate_post(const DeviceState& s, cudaStream_t st) {
    k_gate_post<<<1, 256, 0, st>>>(s.ctl, s.cap_M, s.cap_policy);
    return cudaGetLastError();
}

template <int W>
static cudaError_t cap_w(const DeviceState& s, cudaStream_t st) {
    const int g = stream_grid(s, 256, 8);
    const int shifts[5] = {50, 37, 24, 11, 0};
    for (int p = 0; p < 5; ++p) {
        k_cap_hist<W><<<g, 256, 0, st>>>(bufs_of<W>(s), s.ctl, shifts[p]);
        k_cap_pick<<<1, 1024, 0, st>>>(s.ctl, shifts[p], p == 4 ? 1 : 0);
    }
    PKey<W>* ties = reinterpret_cast<PKey<W>*>(s.table);   // the table is free here
    k_cap_ties<W, 256><<<g, 256, 0, st>>>(bufs_of<W>(s), s.ctl, ties);
    for (int p = 0; p < 8 * W; ++p) {
        k_tie_hist<W><<<g, 256, 0, st>>>(s.ctl, ties, p);
        k_tie_pick<W><<<1, 1024, 0, st>>>(s.ctl, p);
    }
    k_tie_find<W><<<g, 256, 0, st>>>(s.ctl, ties);
    k_cap_compact<W, 256><<<g, 256, 0, st>>>(bufs_of<W>(s), s.ctl);
    k_cap_end<<<1, 32, 0, st>>>(s.ctl);
    return cudaGetLastError();
}

int cap_launches(const DeviceState& s) { return 5 * 2 + 1 + 8 * s.W * 2 + 3; }

cudaError_t launch_cap(const DeviceState& s, cudaStream_t st) {
    return s.W == 1 ? cap_w<1>(s, st) : cap_w<2>(s, st);
}

}  // namespace itpp
