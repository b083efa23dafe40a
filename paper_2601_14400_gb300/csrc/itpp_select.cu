// itpp_select.cu -- the top-M select of the partitioned merge (term bound,
// cap_policy 1; Sec. II.C "Practical considerations": keep the cap_M largest
// |c|, ties broken by ascending key), in three launches per gate.
//
// The values selected on are the 63-bit magnitude patterns b of the raw
// coefficients (monotone in |c|).  Every kept output has b > delta's pattern
// (lo), and the merge records the largest pattern it wrote (hi), so the first
// radix digit is taken over v = b - lo scaled to 13 bits: bits [sh, sh+13)
// of v with sh = max(0, bitlen(hi - lo) - 13).  That spreads the values over
// thousands of bins (the raw pattern's top 13 bits would give four bins per
// binade), so the threshold's bin holds few terms:
//   k_sel_hist    histogram of the first digit; the last CTA to finish picks
//                 the digit holding the cap_M-th largest value;
//   k_sel_gather  the terms of that digit (v and index) into a candidate list;
//   k_sel_finish  one block: the remaining digits of v over the candidates,
//                 then the key select among exact ties (a bitonic sort in
//                 shared memory, or 16-bit radix passes over a long tie
//                 list), then the kept set is recorded as the predicate
//                 (threshold, tie key) that the next gate's reads apply.
#include <cstring>

#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {

// Offset and shift of the first digit.
__device__ __forceinline__ void sel_geometry(const DevCtl* ctl, unsigned long long lo,
                                             int* sh) {
    const unsigned long long hi = ctl->sel_hi;
    const unsigned long long range = hi > lo ? hi - lo : 0ULL;
    const int bits = range ? 64 - __clzll((long long)range) : 0;
    *sh = bits > kSelBits ? bits - kSelBits : 0;
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
// 1. First digit
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256, 4)
k_sel_hist(Bufs<W> B, DevCtl* ctl, unsigned long long lo) {
    __shared__ unsigned int h[kSelBins];
    __shared__ unsigned long long s_part[256];
    __shared__ int s_last;
    __shared__ Pick s_pick;
    if (!ctl->sel_active || ctl->status) return;
    int sh;
    sel_geometry(ctl, lo, &sh);
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    // the coefficients' bit patterns, read as integers (no floating point);
    // eight independent loads in flight per thread, then their counts
    const unsigned long long* __restrict__ c =
        reinterpret_cast<const unsigned long long*>(B.coef(cur));
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
            const unsigned long long b = v[u] & 0x7fffffffffffffffULL;   // |c| pattern
            unsigned long long d = (b > lo ? b - lo : 0ULL) >> sh;
            if (d > (unsigned long long)(kSelBins - 1)) d = kSelBins - 1;   // not reached: hi is the max
            atomicAdd(&h[d], 1u);
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
        if (sh == 0) {          // every bit of v fixed: the digit's terms are exact ties
            ctl->sel_ties = pk.count;
            ctl->sel_tie_k = pk.k_in;
        }
        ctl->sel_done = 0u;
    }
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
}

// ---------------------------------------------------------------------------
// 2. Candidates: the terms of the threshold's first digit.  A warp claims
// room for its hits in the CTA's shared stage (one shared atomic per warp and
// load round that has hits, no block barrier in the loop); once the stage is
// full, later hits go straight to the global list.  The successful claims
// form a prefix of the stage (after the first claim that does not fit, every
// later one starts past the end), which the CTA copies out at the end with
// one global claim.  The order of the candidates is immaterial: every later
// pass histograms them and the ties are sorted by key.
// ---------------------------------------------------------------------------
constexpr int kStage = 3072;      // staged candidates per CTA (36 KB)

template <int W>
__global__ void __launch_bounds__(256)
k_sel_gather(Bufs<W> B, DevCtl* ctl, unsigned long long lo, unsigned long long* cand_v,
             uint32_t* cand_idx, uint64_t cand_cap) {
    __shared__ unsigned long long st_v[kStage];
    __shared__ uint32_t st_i[kStage];
    __shared__ unsigned int s_claimed, s_staged;
    __shared__ unsigned long long s_base;
    if (!ctl->sel_active || ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const unsigned long long prefix = ctl->sel_prefix, mask = ctl->sel_mask;
    const double* __restrict__ c = B.coef(cur);
    constexpr int U = 8;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const unsigned int lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) {
        s_claimed = 0u;
        s_staged = 0u;
    }
    __syncthreads();
    // whole warps iterate together (the claims below are warp-wide)
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
            const bool hit = i < n && (x & mask) == prefix;
            const unsigned int b = __ballot_sync(0xffffffffu, hit);
            if (!b) continue;                                   // warp-uniform
            const int leader = __ffs(b) - 1;
            const unsigned int nb = __popc(b), r = __popc(b & lt);
            unsigned int q = 0u;
            if ((int)lane == leader) q = atomicAdd(&s_claimed, nb);
            q = __shfl_sync(0xffffffffu, q, leader);
            if (q + nb <= (unsigned int)kStage) {               // warp-uniform
                if (hit) {
                    st_v[q + r] = x;
                    st_i[q + r] = (uint32_t)i;
                }
                if ((int)lane == leader) atomicAdd(&s_staged, nb);
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
// last CTA picks.  Pass p covers bits [max(0, sh - 13p), sh - 13(p-1)).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_sel_vpass(DevCtl* ctl, unsigned long long lo, const unsigned long long* cand_v, int p) {
    __shared__ unsigned int h[kSelBins];
    __shared__ unsigned long long s_part[1024];
    __shared__ int s_last;
    __shared__ Pick s_pick;
    if (!ctl->sel_active || ctl->status) return;
    int sh;
    sel_geometry(ctl, lo, &sh);
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
               const uint32_t* cand_idx, PKey<W>* tie_list) {
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
            for (unsigned int t = threadIdx.x; t < m; t += blockDim.x) tie_list[s_base + t] = st[t];
            __syncthreads();
            if (threadIdx.x == 0) s_n = 0u;
        }
        __syncthreads();
    }
    const unsigned int m = s_n;
    if (m) {
        if (threadIdx.x == 0) s_base = atomicAdd(&ctl->sel_tie_n, (unsigned long long)m);
        __syncthreads();
        for (unsigned int t = threadIdx.x; t < m; t += blockDim.x) tie_list[s_base + t] = st[t];
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
k_sel_finish(DevCtl* ctl, unsigned long long lo, const PKey<W>* tie_list, uint64_t cap_M) {
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
        // the kept set, applied where the next gate reads the state
        ctl->pend = 1;
        ctl->pend_n = ctl->count[cur];
        ctl->pend_T = ctl->sel_prefix + lo;
        ctl->pend_all_ties = all_ties;
        for (int w = 0; w < 4; ++w) ctl->pend_tie_key[w] = all_ties ? 0ULL : ctl->sel_tie_key[w];
        ctl->count[cur] = cap_M;   // the logical term count
        ctl->sel_active = 0;
        ctl->stat_cands += ctl->sel_cand_n;
        ctl->stat_range = ctl->sel_hi > lo ? ctl->sel_hi - lo : 0ULL;
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

template <int W>
static cudaError_t select_w(const DeviceState& s, cudaStream_t st) {
    unsigned long long lo;
    std::memcpy(&lo, &s.delta, sizeof lo);   // delta >= +0: its pattern bounds every kept |c|
    // candidates and tie keys live in the merge table's memory (free after
    // the merge): 12 bytes per candidate plus the tie list
    char* scratch = static_cast<char*>(s.table);
    unsigned long long* cand_v = reinterpret_cast<unsigned long long*>(scratch);
    uint32_t* cand_idx = reinterpret_cast<uint32_t*>(cand_v + s.buf_cap);
    PKey<W>* ties = reinterpret_cast<PKey<W>*>(scratch + (s.buf_cap * 12 + 255) / 256 * 256);
    const Bufs<W> B = sel_bufs<W>(s);
    k_sel_hist<W><<<s.num_sms * 4, 256, 0, st>>>(B, s.ctl, lo);
    k_sel_gather<W><<<s.num_sms * 4, 256, 0, st>>>(B, s.ctl, lo, cand_v, cand_idx, s.buf_cap);
    for (int p = 1; p <= 4; ++p)    // 13-bit digits cover any 63-bit range
        k_sel_vpass<<<s.num_sms, 1024, 0, st>>>(s.ctl, lo, cand_v, p);
    k_sel_tcollect<W><<<s.num_sms * 2, 256, 0, st>>>(B, s.ctl, cand_v, cand_idx, ties);
    for (int p = 0; p < 8 * W; ++p)
        k_sel_tpass<W><<<s.num_sms, 1024, 0, st>>>(s.ctl, ties, p);
    k_sel_finish<W><<<1, 1024, 0, st>>>(s.ctl, lo, ties, s.cap_M);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_select_deferred(const DeviceState& s, cudaStream_t st) {
    return s.W == 1 ? select_w<1>(s, st) : select_w<2>(s, st);
}

}  // namespace itpp
