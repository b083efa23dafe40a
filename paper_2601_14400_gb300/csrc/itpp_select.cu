// itpp_select.cu -- the top-M select of the partitioned merge (term bound,
// cap_policy 1; Sec. II.C "Practical considerations": keep the cap_M largest
// |c|, ties broken by ascending key).
//
// The values selected on are the 63-bit magnitude patterns b of the raw
// coefficients (monotone in |c|), offset by sel_lo: v = b - sel_lo.  Two ways
// to the threshold:
//   fast   the merge compared every kept child with a range [lo, hi] around
//          the previous gate's threshold, counted the children above hi and
//          listed those inside; when the cap_M-th largest lies inside
//          (above < cap_M <= above + listed), k_sel_begin compacts the
//          merge's per-CTA lists and the digits of v are resolved over that
//          list alone (sel_lo = lo);
//   full   otherwise (no range yet, the threshold moved outside it, a list
//          overflowed): k_sel_hist takes the first 13-bit digit over every
//          stored coefficient, with sel_lo = delta's pattern and the digit
//          scaled to the largest pattern the merge wrote (bits [sh, sh+13)
//          of v, sh = max(0, bitlen(hi - lo) - 13)), so the values spread over
//          thousands of bins; k_sel_gather lists the terms of the picked digit.
// Then, on the list: k_sel_vpass resolves the remaining digits of v;
// k_sel_tcollect / k_sel_tpass / k_sel_finish select among exact ties by key
// (a bitonic sort in shared memory, or 16-bit radix passes over a long tie
// list), and k_sel_finish records the kept set as the predicate (threshold,
// tie key) that the next gate's reads apply, and the next gate's range.  No
// CTA waits for another: each multi-block pass ends in its last CTA.
#include <cstring>

#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {

__device__ __forceinline__ int bit_length(unsigned long long v) {
    return v ? 64 - __clzll((long long)v) : 0;
}

// Shift of the full path's first digit: its top digit of v = b - lo, with
// the largest pattern the merge wrote as the top of the range.
__device__ __forceinline__ void sel_geometry(const DevCtl* ctl, unsigned long long lo,
                                             int* sh) {
    const unsigned long long hi = ctl->sel_hi;
    const int bits = bit_length(hi > lo ? hi - lo : 0ULL);
    *sh = bits > kSelBits ? bits - kSelBits : 0;
}

// Stored terms of the current buffer: chunk s is [off, off + cnt) when the
// buffer is segmented (a partitioned merge wrote it), else one run of n.
struct StateRuns {
    const ChunkDesc* din;
    bool seg;
    uint32_t P;
    uint64_t n;
};

__device__ __forceinline__ StateRuns state_runs(const DevCtl* ctl, const ChunkDesc* chunks0,
                                                const ChunkDesc* chunks1) {
    StateRuns r;
    const int cur = ctl->cur;
    r.din = cur ? chunks1 : chunks0;
    r.seg = ctl->seg != 0;
    r.P = ctl->nchunk[cur];
    r.n = live_count(ctl, cur);
    return r;
}

__device__ __forceinline__ unsigned long long sel_value(double c, unsigned long long lo) {
    const unsigned long long b = abs_bits(c);
    return b > lo ? b - lo : 0ULL;
}

// Inclusive scan of one value per thread over NT threads (s: NT slots).
template <int NT>
__device__ __forceinline__ unsigned long long scan_nt(unsigned long long v, unsigned long long* s) {
    const int t = threadIdx.x;
    s[t] = v;
    __syncthreads();
    for (int o = 1; o < NT; o <<= 1) {
        const unsigned long long a = t >= o ? s[t - o] : 0ULL;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    const unsigned long long r = s[t];
    __syncthreads();
    return r;
}

struct Pick {
    int digit;
    unsigned long long k_in;    // rank of the target inside the digit
    unsigned long long count;   // values in the digit
};

// The digit (in descending order) holding the k-th largest value, from a
// histogram of kSelBins counts (global 64-bit counts read through L2, or
// 32-bit shared ones); NT threads, result in *out (shared).
template <int NT, bool kGlobal>
__device__ __forceinline__ unsigned long long hist_at(const void* hist, int b) {
    return kGlobal ? __ldcg(static_cast<const unsigned long long*>(hist) + b)
                   : (unsigned long long)static_cast<const unsigned int*>(hist)[b];
}

template <int NT, bool kGlobal>
__device__ __forceinline__ void pick_digit(const void* hist, unsigned long long k,
                                           unsigned long long* s_part, Pick* out) {
    constexpr int PER = kSelBins / NT;
    const int t = threadIdx.x;
    if (t == 0) *out = Pick{0, 0, 0};
    // two passes over this thread's bins (sum, then find) instead of
    // holding PER counts in registers
    unsigned long long sum = 0;
    for (int j = 0; j < PER; ++j) sum += hist_at<NT, kGlobal>(hist, kSelBins - 1 - PER * t - j);
    const unsigned long long incl = scan_nt<NT>(sum, s_part);
    unsigned long long run = incl - sum;
    if (run < k && k <= incl) {
        for (int j = 0; j < PER; ++j) {
            const unsigned long long hv = hist_at<NT, kGlobal>(hist, kSelBins - 1 - PER * t - j);
            if (run < k && k <= run + hv) {
                out->digit = kSelBins - 1 - PER * t - j;
                out->k_in = k - run;
                out->count = hv;
            }
            run += hv;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// 0. Fast or full: when the cap_M-th largest value lies in the merge's
// candidate range, compact the merge's per-CTA lists into the candidate list
// (every CTA computes the region offsets and the decision from the same
// counts; block 0 alone writes the select state).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_sel_begin(DevCtl* ctl, CandRegions cr, unsigned long long* cand_v, uint32_t* cand_idx,
            uint64_t cand_cap, uint64_t cap_M, unsigned long long delta_bits) {
    __shared__ uint32_t s_scan[32];
    __shared__ uint32_t s_off[1024];
    if (!ctl->sel_active || ctl->status) return;
    const unsigned int nreg = ctl->cand_regions < 1024u ? ctl->cand_regions : 1024u;
    const uint32_t c = threadIdx.x < nreg ? cr.cnt[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t off = block_exclusive_scan<1024>(c, &tot, s_scan);
    s_off[threadIdx.x] = off;
    const unsigned long long above = ctl->sp_above;
    const int reason = ctl->sp_hi == 0ULL ? 1
                       : (ctl->sp_ovf || tot > cand_cap) ? 2
                       : above >= cap_M ? 3
                       : above + tot < cap_M ? 4 : 0;
    const bool fast = reason == 0;
    __syncthreads();
    if (fast) {
        for (unsigned int r = blockIdx.x; r < nreg; r += gridDim.x) {
            const uint32_t n = cr.cnt[r], o = s_off[r];
            const uint64_t rb = (uint64_t)r * cr.region;
            for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
                cand_v[o + j] = cr.v[rb + j];
                cand_idx[o + j] = cr.idx[rb + j];
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->sel_fast = fast ? 1 : 0;
        ctl->sp_reason = reason;
        ctl->sel_prefix = 0ULL;
        ctl->sel_mask = 0ULL;
        if (fast) {
            const int top = bit_length(ctl->sp_hi - ctl->sp_lo);
            ctl->sel_lo = ctl->sp_lo;
            ctl->sel_top = top;
            ctl->sel_k = cap_M - above;
            ctl->sel_cand_n = tot;
            if (top == 0) {          // a range of one value: every candidate ties
                ctl->sel_ties = tot;
                ctl->sel_tie_k = cap_M - above;
            }
        } else {
            ctl->sel_lo = delta_bits;
            ctl->sel_cand_n = 0ULL;
            ctl->stat_sel_full += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// 1. First digit (full path)
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256, 4)
k_sel_hist(Bufs<W> B, DevCtl* ctl, const ChunkDesc* desc0, const ChunkDesc* desc1) {
    __shared__ unsigned int h[kSelBins];
    __shared__ unsigned long long s_part[256];
    __shared__ int s_last;
    __shared__ Pick s_pick;
    if (!ctl->sel_active || ctl->status || ctl->sel_fast) return;
    const unsigned long long lo = ctl->sel_lo;
    int sh;
    sel_geometry(ctl, lo, &sh);
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const int cur = ctl->cur;
    const StateRuns rs = state_runs(ctl, desc0, desc1);
    // the coefficients' bit patterns, read as integers (no floating point)
    const unsigned long long* __restrict__ c =
        reinterpret_cast<const unsigned long long*>(B.coef(cur));
    auto count = [&](unsigned long long raw) {
        const unsigned long long b = raw & 0x7fffffffffffffffULL;   // |c| pattern
        unsigned long long d = (b > lo ? b - lo : 0ULL) >> sh;
        if (d > (unsigned long long)(kSelBins - 1)) d = kSelBins - 1;   // not reached: hi is the max
        atomicAdd(&h[d], 1u);
    };
    if (rs.seg) {
        for (uint32_t s = blockIdx.x; s < rs.P; s += gridDim.x) {
            const uint64_t off = rs.din[s].off;
            const uint32_t cnt = rs.din[s].cnt;
            for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) count(__ldcs(c + off + j));
        }
    } else {
        // eight independent loads in flight per thread, then their counts
        const uint64_t n = rs.n;
        constexpr int U = 8;
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
            unsigned long long v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = i0 + (uint64_t)u * stride;
                v[u] = i < n ? __ldcs(c + i) : 0ULL;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + (uint64_t)u * stride >= n) break;
                count(v[u]);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (h[b]) atomicAdd(&ctl->sel_hist[b], (unsigned long long)h[b]);
    // the last CTA to finish picks the digit (no CTA waits for another)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->sel_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    pick_digit<256, true>(ctl->sel_hist, ctl->sel_k, s_part, &s_pick);
    if (threadIdx.x == 0) {
        const Pick pk = s_pick;
        ctl->sel_prefix = (unsigned long long)pk.digit << sh;
        ctl->sel_mask = (unsigned long long)(kSelBins - 1) << sh;
        ctl->sel_k = pk.k_in;
        ctl->sel_top = sh;
        if (sh == 0) {          // every bit of v fixed: the digit's terms are exact ties
            ctl->sel_ties = pk.count;
            ctl->sel_tie_k = pk.k_in;
        }
        ctl->sel_done = 0u;
    }
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
}

// ---------------------------------------------------------------------------
// 2. Candidates (full path): the terms of the threshold's first digit.  A
// warp claims room for its hits in the CTA's shared stage (one shared atomic
// per warp and load round that has hits, no block barrier in the loop); once
// the stage is full, later hits go straight to the global list.  The
// successful claims form a prefix of the stage (after the first claim that
// does not fit, every later one starts past the end), which the CTA copies
// out at the end with one global claim.  The order of the candidates is
// immaterial: every later pass histograms them and the ties are sorted by key.
// ---------------------------------------------------------------------------
constexpr int kStage = 3072;      // staged candidates per CTA (36 KB)
constexpr int kVPasses = 5;       // 13-bit passes over v: 5 x 13 >= 63 bits
constexpr int kRangeShift0 = 45;  // the first candidate range: T +- about 1/128 of T

struct GatherStage {
    unsigned long long* st_v;
    uint32_t* st_i;
    unsigned int* s_claimed;
    unsigned int* s_staged;
};

// One round of up to 32 values per warp (every lane calls it).
__device__ __forceinline__ void gather_one(bool hit, unsigned long long x, uint64_t i,
                                           const GatherStage& gs, DevCtl* ctl,
                                           unsigned long long* cand_v, uint32_t* cand_idx,
                                           uint64_t cand_cap) {
    const unsigned int lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
    const unsigned int b = __ballot_sync(0xffffffffu, hit);
    if (!b) return;                                      // warp-uniform
    const int leader = __ffs(b) - 1;
    const unsigned int nb = __popc(b), r = __popc(b & lt);
    unsigned int q = 0u;
    if ((int)lane == leader) q = atomicAdd(gs.s_claimed, nb);
    q = __shfl_sync(0xffffffffu, q, leader);
    if (q + nb <= (unsigned int)kStage) {               // warp-uniform
        if (hit) {
            gs.st_v[q + r] = x;
            gs.st_i[q + r] = (uint32_t)i;
        }
        if ((int)lane == leader) atomicAdd(gs.s_staged, nb);
    } else {
        unsigned long long g = 0ULL;
        if ((int)lane == leader) g = atomicAdd(&ctl->sel_cand_n, (unsigned long long)nb);
        g = __shfl_sync(0xffffffffu, g, leader);
        if (hit) {
            if (g + r < cand_cap) {
                cand_v[g + r] = x;
                cand_idx[g + r] = (uint32_t)i;
            } else {
                set_status(ctl, ST_CAPACITY, 30);
            }
        }
    }
}

template <int W>
__global__ void __launch_bounds__(256)
k_sel_gather(Bufs<W> B, DevCtl* ctl, const ChunkDesc* desc0, const ChunkDesc* desc1,
             unsigned long long* cand_v, uint32_t* cand_idx, uint64_t cand_cap) {
    __shared__ unsigned long long st_v[kStage];
    __shared__ uint32_t st_i[kStage];
    __shared__ unsigned int s_claimed, s_staged;
    __shared__ unsigned long long s_base;
    if (!ctl->sel_active || ctl->status || ctl->sel_fast) return;
    const int cur = ctl->cur;
    const StateRuns rs = state_runs(ctl, desc0, desc1);
    const unsigned long long lo = ctl->sel_lo;
    const unsigned long long prefix = ctl->sel_prefix, mask = ctl->sel_mask;
    const double* __restrict__ c = B.coef(cur);
    const GatherStage gs{st_v, st_i, &s_claimed, &s_staged};
    if (threadIdx.x == 0) {
        s_claimed = 0u;
        s_staged = 0u;
    }
    __syncthreads();
    // whole warps iterate together (the claims are warp-wide)
    if (rs.seg) {
        for (uint32_t s = blockIdx.x; s < rs.P; s += gridDim.x) {
            const uint64_t off = rs.din[s].off;
            const uint32_t cnt = rs.din[s].cnt;
            for (uint32_t j0 = 0; j0 < cnt; j0 += blockDim.x) {
                const uint32_t j = j0 + threadIdx.x;
                const double v = j < cnt ? __ldcs(c + off + j) : 0.0;
                const unsigned long long x = sel_value(v, lo);
                gather_one(j < cnt && (x & mask) == prefix, x, off + j, gs, ctl, cand_v, cand_idx,
                           cand_cap);
            }
        }
    } else {
        const uint64_t n = rs.n;
        constexpr int U = 8;
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
             i0 - threadIdx.x < n; i0 += U * stride) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = i0 + (uint64_t)u * stride;
                v[u] = i < n ? __ldcs(c + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = i0 + (uint64_t)u * stride;
                const unsigned long long x = sel_value(v[u], lo);
                gather_one(i < n && (x & mask) == prefix, x, i, gs, ctl, cand_v, cand_idx,
                           cand_cap);
            }
        }
    }
    __syncthreads();
    const unsigned int m = s_staged;
    if (threadIdx.x == 0) s_base = m ? atomicAdd(&ctl->sel_cand_n, (unsigned long long)m) : 0ULL;
    __syncthreads();
    const unsigned long long base = s_base;
    for (unsigned int j = threadIdx.x; j < m; j += blockDim.x) {
        if (base + j < cand_cap) {
            cand_v[base + j] = st_v[j];
            cand_idx[base + j] = st_i[j];
        } else {
            set_status(ctl, ST_CAPACITY, 30);
        }
    }
}

// ---------------------------------------------------------------------------
// 3. The remaining digits of v over the candidates, one per launch; the
// last CTA picks.  Pass p covers bits [max(0, top - 13p), top - 13(p-1)),
// top = sel_top (the bits below the first digit on the full path, every bit
// of the range on the fast path).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_sel_vpass(DevCtl* ctl, const unsigned long long* cand_v, int p) {
    __shared__ unsigned int h[kSelBins];
    __shared__ unsigned long long s_part[1024];
    __shared__ int s_last;
    __shared__ Pick s_pick;
    if (!ctl->sel_active || ctl->status) return;
    const int sh = ctl->sel_top;
    if (sh - kSelBits * (p - 1) <= 0) return;          // every bit already fixed
    const int shift = sh - kSelBits * p > 0 ? sh - kSelBits * p : 0;
    const unsigned long long nc = ctl->sel_cand_n;
    const unsigned long long prefix = ctl->sel_prefix, mask = ctl->sel_mask;
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < nc;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long v = cand_v[j];
        if ((v & mask) == prefix) atomicAdd(&h[(v >> shift) & (kSelBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (h[b]) atomicAdd(&ctl->sel_hist[b], (unsigned long long)h[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->sel_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    pick_digit<1024, true>(ctl->sel_hist, ctl->sel_k, s_part, &s_pick);
    if (threadIdx.x == 0) {
        const Pick pk = s_pick;
        ctl->sel_prefix = prefix | ((unsigned long long)pk.digit << shift);
        ctl->sel_mask = mask | ((unsigned long long)(kSelBins - 1) << shift);
        ctl->sel_k = pk.k_in;
        if (shift == 0) {
            ctl->sel_ties = pk.count;
            ctl->sel_tie_k = pk.k_in;
        }
        ctl->sel_done = 0u;
    }
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
}

// ---------------------------------------------------------------------------
// 4. Ties: the keys of the candidates exactly at the threshold (only when
// some of them are dropped), staged per CTA like the candidates.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256)
k_sel_tcollect(Bufs<W> B, DevCtl* ctl, const unsigned long long* cand_v,
               const uint32_t* cand_idx, PKey<W>* tie_list, uint64_t tie_cap) {
    constexpr int kT = 1024;
    __shared__ PKey<W> st[kT];
    __shared__ unsigned int s_n;
    __shared__ unsigned long long s_base;
    if (!tie_select_needed(ctl)) return;
    const int cur = ctl->cur;
    const unsigned long long nc = ctl->sel_cand_n, T = ctl->sel_prefix;
    if (threadIdx.x == 0) s_n = 0u;
    __syncthreads();
    for (unsigned long long j0 = (unsigned long long)blockIdx.x * blockDim.x;
         j0 < nc; j0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long j = j0 + threadIdx.x;
        if (j < nc && cand_v[j] == T) {
            const unsigned int q = atomicAdd(&s_n, 1u);
            st[q] = load_key(B.key(cur) + cand_idx[j]);
        }
        __syncthreads();
        const unsigned int m = s_n;
        if (m > kT - 256) {
            if (threadIdx.x == 0) s_base = atomicAdd(&ctl->sel_tie_n, (unsigned long long)m);
            __syncthreads();
            for (unsigned int t = threadIdx.x; t < m; t += blockDim.x) {
                if (s_base + t < tie_cap) tie_list[s_base + t] = st[t];
                else set_status(ctl, ST_CAPACITY, 32);
            }
            __syncthreads();
            if (threadIdx.x == 0) s_n = 0u;
        }
        __syncthreads();
    }
    const unsigned int m = s_n;
    if (m) {
        if (threadIdx.x == 0) s_base = atomicAdd(&ctl->sel_tie_n, (unsigned long long)m);
        __syncthreads();
        for (unsigned int t = threadIdx.x; t < m; t += blockDim.x) {
            if (s_base + t < tie_cap) tie_list[s_base + t] = st[t];
            else set_status(ctl, ST_CAPACITY, 32);
        }
    }
}

// ---------------------------------------------------------------------------
// 5. Key passes over a long tie list (16-bit digits from word 0), one per
// launch, the last CTA picking; they stop once at most kSmallTies keys
// share the picked prefix (state 3), which the final block then sorts.
// ---------------------------------------------------------------------------
template <int W>
struct SmallTies {
    static constexpr int kMax = 2048 / W;    // 32 KB of keys
};

template <int W>
__global__ void __launch_bounds__(1024)
k_sel_tpass(DevCtl* ctl, const PKey<W>* tie_list, int p) {
    __shared__ unsigned long long s_part[1024];
    __shared__ int s_last;
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 0) return;
    if (p == 0 && ctl->sel_ties <= (unsigned long long)SmallTies<W>::kMax) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->sel_tie_state = 3;   // small already
        return;
    }
    tie_hist_range<W>(ctl, tie_list, p, (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x,
                      ctl->sel_tie_n, (unsigned long long)gridDim.x * blockDim.x);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->sel_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the digit (ascending) holding the sel_tie_k-th smallest key
    constexpr int PER = kTieBins / 1024;
    const int t = threadIdx.x;
    unsigned long long sum = 0;
    for (int j = 0; j < PER; ++j) sum += __ldcg(&ctl->tie_hist[PER * t + j]);
    const unsigned long long incl = scan_nt<1024>(sum, s_part);
    unsigned long long run = incl - sum;
    const unsigned long long k = ctl->sel_tie_k;
    const int wi = p / 4, shift = 48 - 16 * (p % 4);
    if (run < k && k <= incl) {
        for (int j = 0; j < PER; ++j) {
            const unsigned long long hv = __ldcg(&ctl->tie_hist[PER * t + j]);
            if (run < k && k <= run + hv) {
                ctl->sel_tie_k = k - run;
                ctl->sel_tie_key[wi] |= (unsigned long long)(PER * t + j) << shift;
                ctl->sel_tie_pass = p + 1;
                if (p == 8 * W - 1) ctl->sel_tie_state = 1;                 // every bit fixed
                else if (hv == 1) ctl->sel_tie_state = 2;                   // a unique key
                else if (hv <= (unsigned long long)SmallTies<W>::kMax) ctl->sel_tie_state = 3;
            }
            run += hv;
        }
    }
    __syncthreads();
    for (int b = t; b < kTieBins; b += blockDim.x) ctl->tie_hist[b] = 0ULL;
    if (t == 0) ctl->sel_done = 0u;
}

// ---------------------------------------------------------------------------
// 6. One block: the last key digits by a shared-memory sort, then the
// predicate.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ PKey<W> key_max() {
    PKey<W> k;
#pragma unroll
    for (int w = 0; w < W; ++w) { k.x[w] = ~0ULL; k.z[w] = ~0ULL; }
    return k;
}

// Ascending bitonic sort of n_pad (a power of two) keys in shared memory.
template <int W>
__device__ void bitonic_sort_keys(PKey<W>* a, int n_pad) {
    for (int k = 2; k <= n_pad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const PKey<W> x = a[i], y = a[l];
                    if (up ? key_less(y, x) : key_less(x, y)) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int W>
__global__ void __launch_bounds__(1024)
k_sel_finish(DevCtl* ctl, const PKey<W>* tie_list, uint64_t cap_M, uint64_t cand_hi,
             long long* drift, int n_drift, int gate) {
    __shared__ PKey<W> s_ties[SmallTies<W>::kMax];
    __shared__ unsigned int s_cnt;
    if (!ctl->sel_active) return;
    if (ctl->status) {
        __syncthreads();
        if (threadIdx.x == 0) ctl->sel_active = 0;
        return;
    }
    const bool all_ties = ctl->sel_k == ctl->sel_ties;
    if (!all_ties && ctl->sel_tie_state != 1) {
        // the keys sharing the picked prefix (state 3, or the unique key of
        // state 2), sorted; the tie_k-th smallest is the largest kept key
        const int p = ctl->sel_tie_pass;   // key digits fixed so far
        uint64_t pre[2 * W];
#pragma unroll
        for (int w = 0; w < 2 * W; ++w) pre[w] = ctl->sel_tie_key[w];
        if (threadIdx.x == 0) s_cnt = 0u;
        __syncthreads();
        const unsigned long long nt = ctl->sel_tie_n;
        for (unsigned long long j = threadIdx.x; j < nt; j += blockDim.x) {
            const PKey<W> k = tie_list[j];
            if (tie_prefix_match<W>(k, pre, p)) {
                const unsigned int q = atomicAdd(&s_cnt, 1u);
                if (q < (unsigned int)SmallTies<W>::kMax) s_ties[q] = k;
            }
        }
        __syncthreads();
        const unsigned int m = s_cnt;
        if (m > (unsigned int)SmallTies<W>::kMax || m == 0u) {
            if (threadIdx.x == 0) set_status(ctl, ST_STATE, 31);
        } else {
            int n_pad = 1;
            while (n_pad < (int)m) n_pad <<= 1;
            for (int i = (int)m + threadIdx.x; i < n_pad; i += blockDim.x) s_ties[i] = key_max<W>();
            __syncthreads();
            bitonic_sort_keys<W>(s_ties, n_pad);
            if (threadIdx.x == 0) {
                const unsigned long long r = ctl->sel_tie_state == 2 ? 1ULL : ctl->sel_tie_k;
                const PKey<W> tk = s_ties[r - 1];
                for (int w = 0; w < W; ++w) {
                    ctl->sel_tie_key[w] = tk.x[w];
                    ctl->sel_tie_key[W + w] = tk.z[w];
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int cur = ctl->cur;
        const unsigned long long lo = ctl->sel_lo;
        const unsigned long long T = ctl->sel_prefix + lo;   // the threshold's pattern
        // the kept set, applied where the next gate reads the state
        ctl->pend = 1;
        ctl->pend_n = ctl->count[cur];
        ctl->pend_T = T;
        ctl->pend_all_ties = all_ties;
        for (int w = 0; w < 4; ++w) ctl->pend_tie_key[w] = all_ties ? 0ULL : ctl->sel_tie_key[w];
        ctl->count[cur] = cap_M;   // the logical term count
        ctl->sel_active = 0;
        ctl->stat_cands += ctl->sel_cand_n;
        ctl->stat_range = ctl->sel_fast ? ctl->sp_hi - ctl->sp_lo
                                        : (ctl->sel_hi > lo ? ctl->sel_hi - lo : 0ULL);
        // the next gate's candidate range: C +- 2^s in pattern units (a
        // relative width of about 2^(s-52)), narrower when the list ran long
        // or overflowed, wider when the threshold fell outside.  Its centre C:
        // this threshold moved by what the next gate's threshold moved in the
        // last layer (the schedule repeats every layer), or, without that,
        // carried into the next gate's scale (the next gate reads the state
        // rescaled by 1/c_I, rnorm of the buffer this gate wrote).
        const unsigned long long Tp = ctl->sp_tprev;
        const int gi = n_drift > 0 ? gate % n_drift : 0;
        const int gn = n_drift > 0 ? (gate + 1) % n_drift : 0;
        if (n_drift > 0) drift[gi] = Tp ? (long long)(T - Tp) : 0LL;
        ctl->sp_tprev = T;
        int sft = ctl->sp_shift ? ctl->sp_shift : kRangeShift0;
        switch (ctl->sel_fast ? 0 : ctl->sp_reason) {
            case 0: if (ctl->sel_cand_n > cand_hi) sft -= 1; break;
            case 1: sft = kRangeShift0; break;
            case 2: sft -= 2; break;
            default: sft += 1; break;
        }
        sft = sft < 8 ? 8 : (sft > 60 ? 60 : sft);
        ctl->sp_shift = sft;
        const long long dn = n_drift > 0 ? drift[gn] : 0LL;
        unsigned long long C;
        if (dn != 0LL) {
            const long long c = (long long)T + dn;
            C = c > 0 ? (unsigned long long)c : 0ULL;
        } else {
            C = abs_pattern(__dmul_rn(__longlong_as_double((long long)T), ctl->rnorm[cur]));
        }
        const unsigned long long h = 1ULL << sft;
        ctl->sp_lo = C > h ? C - h : 0ULL;
        ctl->sp_hi = C + h;
    }
}

template <int W>
static Bufs<W> sel_bufs(const DeviceState& s) {
    Bufs<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    return b;
}

// The candidate list and the tie list in the merge table's memory (free on
// this path): v and idx of up to cand_cap candidates, then the tie keys.
template <int W>
struct SelScratch {
    unsigned long long* cand_v;
    uint32_t* cand_idx;
    uint64_t cand_cap;
    PKey<W>* ties;
    uint64_t tie_cap;
};

template <int W>
static SelScratch<W> sel_scratch(const DeviceState& s) {
    SelScratch<W> r;
    const uint64_t bytes = s.table_slots * sizeof(Slot<W>);
    char* base = static_cast<char*>(s.table);
    uint64_t cc = bytes / (12 + sizeof(PKey<W>));
    if (cc > s.buf_cap) cc = s.buf_cap;
    r.cand_cap = cc;
    r.cand_v = reinterpret_cast<unsigned long long*>(base);
    r.cand_idx = reinterpret_cast<uint32_t*>(base + cc * 8);
    const uint64_t toff = (cc * 12 + 255) / 256 * 256;
    r.ties = reinterpret_cast<PKey<W>*>(base + toff);
    r.tie_cap = (bytes - toff) / sizeof(PKey<W>);
    return r;
}

template <int W>
static cudaError_t select_w(const DeviceState& s, cudaStream_t st, int gate) {
    unsigned long long lo;
    std::memcpy(&lo, &s.delta, sizeof lo);   // delta >= +0: its pattern bounds every kept |c|
    const SelScratch<W> sc = sel_scratch<W>(s);
    const Bufs<W> B = sel_bufs<W>(s);
    k_sel_begin<<<s.num_sms, 1024, 0, st>>>(s.ctl, s.cand, sc.cand_v, sc.cand_idx, sc.cand_cap,
                                            s.cap_M, lo);
    k_sel_hist<W><<<s.num_sms * 4, 256, 0, st>>>(B, s.ctl, s.chunks[0], s.chunks[1]);
    k_sel_gather<W><<<s.num_sms * 4, 256, 0, st>>>(B, s.ctl, s.chunks[0], s.chunks[1],
                                                   sc.cand_v, sc.cand_idx, sc.cand_cap);
    for (int p = 1; p <= kVPasses; ++p)    // 13-bit digits cover any 63-bit range
        k_sel_vpass<<<s.num_sms, 1024, 0, st>>>(s.ctl, sc.cand_v, p);
    k_sel_tcollect<W><<<s.num_sms * 2, 256, 0, st>>>(B, s.ctl, sc.cand_v, sc.cand_idx, sc.ties,
                                                     sc.tie_cap);
    for (int p = 0; p < 8 * W; ++p)
        k_sel_tpass<W><<<s.num_sms, 1024, 0, st>>>(s.ctl, sc.ties, p);
    k_sel_finish<W><<<1, 1024, 0, st>>>(s.ctl, sc.ties, s.cap_M, s.cand_hi, s.sp_drift,
                                        s.sp_drift ? s.layer_gates : 0, gate);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_select_deferred(const DeviceState& s, cudaStream_t st, int gate) {
    return s.W == 1 ? select_w<1>(s, st, gate) : select_w<2>(s, st, gate);
}

int select_deferred_launches(int W) { return 4 + kVPasses + 8 * W + 1; }

}  // namespace itpp
