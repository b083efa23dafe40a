// itpp_gate_body.cuh -- device bodies of the per-gate kernels, shared by the
// single-propagation kernels (itpp_gate.cu) and the batched ones
// (itpp_batch.cu), so that a batched instance performs exactly the operations
// of a plain run.
//
// Merge structure.  For a gate Q the children of a term K are K itself and,
// when [K, Q] = 0, the string Q.K.  Both maps are bijections on strings, and
// Q.K commutes with Q exactly when K does, so a string receives at most two
// contributions: from K itself and from its partner Q.K; an anticommuting
// string receives only its own.  The merge is therefore a partner lookup:
// the table build puts every commuting term (key, raw c) into an
// open-addressing table keyed on (x, z); the branch-emit pass streams the
// terms once more, and a commuting term K writes c_K cosh + s c_QK (-sinh)
// when its partner is present, or c_K cosh plus the new string Q.K with
// s c_K (-sinh) when it is not.  Two addends summed in one rounding do not
// depend on their order, so the result equals any correct sequential
// accumulation bit for bit.
#pragma once

#include "itpp_common.cuh"

namespace itpp {

template <int W>
struct Bufs {
    PKey<W>* k[2];
    double* c[2];
    // by compare-select: a dynamic index into a kernel parameter array
    // makes the compiler copy the array to local memory
    __device__ __forceinline__ PKey<W>* key(int i) const { return i ? k[1] : k[0]; }
    __device__ __forceinline__ double* coef(int i) const { return i ? c[1] : c[0]; }
};

// ---------------------------------------------------------------------------
// Merge-table probe
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ bool table_find(const Slot<W>* __restrict__ table, uint64_t mask,
                                           unsigned gen, const PKey<W>& P, double* c,
                                           int probe_limit, DevCtl* ctl, int* probes,
                                           uint32_t* idx = nullptr) {
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
            if (idx) *idx = (uint32_t)(b.y >> 32);
        } else {
            ulonglong2 a = __ldg(v), b = __ldg(v + 1), d = __ldg(v + 2);
            k.x[0] = a.x; k.x[1] = a.y;
            k.z[0] = b.x; k.z[1] = b.y;
            cc = __longlong_as_double((long long)d.x);
            tag = (unsigned)(d.y & 0xffffffffULL);
            if (idx) *idx = (uint32_t)(d.y >> 32);
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

// Partner lookup in the global merge table.
template <int W>
struct GlobalLookup {
    const Slot<W>* table;
    uint64_t mask;
    unsigned gen;
    int probe_limit;
    DevCtl* ctl;
    int* probes;
    __device__ __forceinline__ bool find(const PKey<W>& P, double* c, uint32_t* idx) const {
        return table_find(table, mask, gen, P, c, probe_limit, ctl, probes, idx);
    }
};

// One input term of the table build: commuting terms are inserted.
template <int W>
__device__ __forceinline__ void insert_one(const PKey<W>* __restrict__ kin,
                                           const double* __restrict__ cin, uint64_t i,
                                           DevCtl* ctl, Slot<W>* table, uint64_t mask,
                                           unsigned gen, const GateArg<W>& g, int probe_limit,
                                           int* probes) {
    const PKey<W> K = load_key(kin + i);
    if (!commutes(K, g)) return;
    const double c = __ldg(cin + i);
    if (!table_insert(table, mask, gen, K, c, (uint32_t)i, probe_limit, probes))
        set_status(ctl, ST_HASH_PROBE, 1);
}

// One tile of the branch-emit-merge-truncate pass over a state of n terms.
// Each thread owns IPT consecutive input terms and up to 2*IPT outputs; a
// block scan orders the outputs of the tile and one atomic on the output
// count places it.  The identity's merged coefficient becomes the output's
// normaliser.  Must be called by all threads of the block.
// Output positions of one step, recorded for the adjoint (nullptr: off).
struct StepMaps {
    int* self_out;    // [n_in] output position of the term itself, -1 if dropped
    int* emit_out;    // [n_in] output position of a new partner string, -1 if none
    int* part_src;    // [n_in] input index of the partner when it was present, -1 if not
    unsigned long long* id_pos;   // output position of the identity
};

template <int W, int BLOCK, int IPT, bool REC = false, class Lookup = GlobalLookup<W>>
__device__ __forceinline__ void gate_tile(uint64_t t, uint64_t n,
                                          const PKey<W>* __restrict__ kin,
                                          const double* __restrict__ cin,
                                          PKey<W>* __restrict__ kout, double* __restrict__ cout,
                                          DevCtl* ctl, int cur, const Lookup& lk,
                                          const GateArg<W>& g, double rnorm,
                                          unsigned long long dbits, uint64_t cap_out,
                                          uint32_t* s_scan, unsigned long long* s_base,
                                          StepMaps maps = StepMaps{nullptr, nullptr, nullptr,
                                                                   nullptr}) {
    constexpr uint64_t TILE = (uint64_t)BLOCK * IPT;
    PKey<W> K[IPT];
    double va[IPT], vb[IPT];
    int psrc[IPT];
    uint32_t flags = 0;
    const uint64_t i0 = t * TILE + (uint64_t)threadIdx.x * IPT;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const uint64_t i = i0 + j;
        psrc[j] = -1;
        double raw = 0.0, cp_raw = 0.0;
        bool comm = false, found = false, neg = false;
#pragma unroll
        for (int w = 0; w < W; ++w) { K[j].x[w] = 0; K[j].z[w] = 0; }
        // integer phase: commutation, the partner's lookup, the product's sign
        if (i < n) {
            K[j] = load_key_stream(kin + i);
            raw = __ldcs(cin + i);
            comm = commutes(K[j], g);
            if (comm) {
                neg = product_negative(K[j], g);
                uint32_t pidx = 0;
                found = lk.find(key_xor(K[j], g), &cp_raw, REC ? &pidx : nullptr);
                if (REC && found) psrc[j] = (int)pidx;
            }
        }
        // floating-point phase, the same operations on every lane (no
        // divergent double-precision issue); the branch's result is selected
        // afterwards.  Normalise on load (the previous gate's trace
        // rescaling), the identity being exactly 1.
        const bool id = key_is_zero(K[j]);
        const bool pid = comm && key_is_zero_xor(K[j], g);
        const double c = id ? 1.0 : __dmul_rn(raw, rnorm);
        const double cpn = pid ? 1.0 : __dmul_rn(cp_raw, rnorm);
        // s (-sinh): the sign flip is an integer XOR of the sign bit
        const double m = __longlong_as_double(
            __double_as_longlong(g.msh) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
        const double a1 = __dmul_rn(c, g.ch);           // cosh(theta) P
        const double b1 = __dmul_rn(c, m);              // -sinh(theta) s (Q.P), no partner
        const double sum = __dadd_rn(a1, __dmul_rn(cpn, m));   // partner QP present
        va[j] = !comm ? c : (found ? sum : a1);         // {P,Q} = 0: unchanged
        vb[j] = b1;
        // threshold and weight cutoff on the merged children (Sec. II.B)
        bool keep_b = comm && !found && above(b1, dbits) && light(key_xor(K[j], g), g.maxw);
        bool keep_a = above(va[j], dbits) && light(K[j], g.maxw);
        if (i < n) {
            if (id) {
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
        *s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
    __syncthreads();
    const unsigned long long base = *s_base;
    if (base + tot > cap_out) {
        if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 2);
        return;
    }
    uint64_t pos = base + off;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const uint64_t i = i0 + j;
        if (REC && i < n) {
            maps.self_out[i] = ((flags >> (2 * j)) & 1u) ? (int)pos : -1;
            maps.emit_out[i] = ((flags >> (2 * j + 1)) & 1u)
                                   ? (int)(pos + ((flags >> (2 * j)) & 1u)) : -1;
            maps.part_src[i] = psrc[j];
            if (key_is_zero(K[j])) *maps.id_pos = pos;
        }
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

// After a gate (one thread): switch buffers, the reciprocal normaliser, the
// table generation, statistics and the term bound.  Returns 1 when the top-M
// select must run.
__device__ __forceinline__ int post_one(DevCtl* ctl, uint64_t cap_M, int cap_policy) {
    ctl->pend = 0;   // a deferred select was applied by this gate's scatter or merge
    ctl->need_scatter = ctl->part_over;
    ctl->part_over = 0;
    // a child beyond the largest double (or NaN) from finite inputs: the
    // weights overflowed the state's range; the largest written pattern
    // (partitioned merge) and the normaliser (every path) show it
    constexpr unsigned long long kInfBits = 0x7ff0000000000000ULL;
    if (ctl->out_max >= kInfBits) set_status(ctl, ST_STATE, 4);
    ctl->sel_hi = ctl->out_max;
    ctl->out_max = 0;
    const int cur = ctl->cur, nxt = cur ^ 1;
    const unsigned long long n_in = ctl->count[cur], n_out = ctl->count[nxt];
    if (abs_pattern(ctl->norm[nxt]) >= kInfBits) set_status(ctl, ST_STATE, 5);
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
            ctl->sel_cand_n = 0;
            ctl->sel_small = 0;
            ctl->sel_resolved = 0;
            for (int w = 0; w < 4; ++w) ctl->sel_tie_key[w] = 0;
            ctl->stat_cap += 1;
        }
    }
    ctl->sel_active = active;
    ctl->stat_out += kept;
    if (kept > ctl->stat_peak) ctl->stat_peak = kept;
    return active;
}

// ---------------------------------------------------------------------------
// Top-M select bodies (term bound with cap_policy 1): radix select of the
// cap_M-th largest |c| over its 63-bit pattern (monotone for non-negative
// doubles), 13 bits per pass from the top; when only some of the terms at
// that threshold fit, a second radix select over their keys (16 bits per
// pass, words x[0..W-1] then z[0..W-1]) finds the largest key to keep, so
// the kept set is "the cap_M largest |c|, ties by ascending key".
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double c) {
    return abs_pattern(c);
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

// Digit holding the k-th largest |c| (one block of 1024 threads).
// gather_max > 0: when the chosen digit of a pass before the last holds at
// most gather_max values, mark the select small (the values are gathered and
// the threshold resolved among them; see the batched select).
__device__ __forceinline__ void cap_pick_block(DevCtl* ctl, int shift, int last,
                                               unsigned long long* s_part,
                                               unsigned long long gather_max = 0) {
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
                } else if (gather_max && hv[j] <= gather_max) {
                    ctl->sel_small = 1;
                    ctl->sel_cand_n = 0;
                }
            }
            run += hv[j];
        }
    }
    __syncthreads();
    for (int b = t; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
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

__device__ __forceinline__ bool tie_select_needed(const DevCtl* ctl) {
    return ctl->sel_active && !ctl->status && ctl->sel_k != ctl->sel_ties;
}

// Histogram of 16-bit key digits over the tie list entries [lo, hi), stride.
template <int W>
__device__ __forceinline__ void tie_hist_range(DevCtl* ctl, const PKey<W>* tie_list, int p,
                                               unsigned long long lo, unsigned long long hi,
                                               unsigned long long stride) {
    uint64_t pre[2 * W];
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) pre[w] = ctl->sel_tie_key[w];
    const int wi = p / 4, shift = 48 - 16 * (p % 4);
    for (unsigned long long i = lo; i < hi; i += stride) {
        unsigned int digit = 0xffffffffu;
        const PKey<W> k = tie_list[i];
        if (tie_prefix_match<W>(k, pre, p))
            digit = (unsigned int)((key_word(k, wi) >> shift) & (kTieBins - 1));
        const unsigned int peers = __match_any_sync(__activemask(), digit);
        const int leader = __ffs(peers) - 1;
        if (digit != 0xffffffffu && (int)(threadIdx.x & 31) == leader)
            atomicAdd(&ctl->tie_hist[digit], (unsigned long long)__popc(peers));
    }
}

// Digit holding the k-th smallest key among the ties (one block of 1024).
template <int W>
__device__ __forceinline__ void tie_pick_block(DevCtl* ctl, int p, unsigned long long* s_part) {
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
__device__ __forceinline__ void tie_find_range(DevCtl* ctl, const PKey<W>* tie_list,
                                               unsigned long long lo, unsigned long long hi,
                                               unsigned long long stride) {
    uint64_t pre[2 * W];
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) pre[w] = ctl->sel_tie_key[w];
    const int p = ctl->sel_tie_pass;
    for (unsigned long long i = lo; i < hi; i += stride) {
        const PKey<W> k = tie_list[i];
        if (tie_prefix_match<W>(k, pre, p))
            for (int w = 0; w < 2 * W; ++w) ctl->sel_tie_key[w] = key_word(k, w);
    }
}

// Does a term survive the top-M select?
template <int W>
__device__ __forceinline__ bool cap_keep(const PKey<W>& K, double c, unsigned long long T,
                                         bool all_ties, const PKey<W>& tk) {
    const unsigned long long b = abs_bits(c);
    return (b > T) || (b == T && (all_ties || !key_less(tk, K)));
}

}  // namespace itpp
