// itpp_sort.cu -- the sort-based merge (merge_path 1).
//
// The same gate as the hash paths (Sec. II.B, Algorithm 1 "Accumulate" then
// "Truncate"), with equal strings found by sorting instead of hashing:
//   1. expand: every stored term, normalised on load, is classified against
//      the gate string Q.  An anticommuting term has exactly one child, itself,
//      and no other child can share its string (the children of a string K
//      come from K and from QK, and QK commutes with Q iff K does), so it is
//      truncated and written out directly.  A commuting term emits the two
//      children (K, cosh(theta) c) and (QK, -sinh(theta) s c) into a child
//      buffer.
//   2. a least-significant-digit radix sort of the children on the whole key
//      (8-bit digits over x words then z words; digits above bit n are zero
//      for every key and are skipped), stable within and across tiles.
//   3. a segmented reduce over runs of equal keys: at most two addends per
//      run (the pair property above), one rounding, order-independent, then
//      the |c| > delta test, with the identity always kept (its merged value
//      is the new trace).
// Every result is bit-identical to the hash paths and to the oracle.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {

constexpr int kSB = 256;              // threads per CTA of the sort passes
constexpr int kSI = 16;               // items per thread per tile
constexpr int kSTile = kSB * kSI;     // items per tile
constexpr int kDig = 256;             // 8-bit digits
constexpr int kMaxPass = 32;          // 2W words x 8 digits, W <= 2

template <int W>
struct SortBufs {
    unsigned long long* n_child;      // [1] commuting children of this gate
    unsigned int* totals;             // [kMaxPass][256] digit totals per pass
    unsigned int* counts;             // [256][t_cap] per-tile digit counts -> offsets
    PKey<W>* k[2];                    // ping-pong child keys
    double* c[2];                     // ping-pong child coefficients
    uint64_t child_cap;
    uint64_t t_cap;
};

template <int W>
__host__ __device__ inline SortBufs<W> sort_layout(void* base, uint64_t buf_cap) {
    SortBufs<W> b;
    char* p = static_cast<char*>(base);
    b.child_cap = buf_cap;
    b.t_cap = (buf_cap + kSTile - 1) / kSTile;
    b.n_child = reinterpret_cast<unsigned long long*>(p);
    p += 256;
    b.totals = reinterpret_cast<unsigned int*>(p);
    p += (size_t)kMaxPass * kDig * 4;
    b.counts = reinterpret_cast<unsigned int*>(p);
    p += ((size_t)kDig * b.t_cap * 4 + 255) / 256 * 256;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(p);
        p += ((size_t)buf_cap * sizeof(PKey<W>) + 255) / 256 * 256;
        b.c[i] = reinterpret_cast<double*>(p);
        p += ((size_t)buf_cap * 8 + 255) / 256 * 256;
    }
    return b;
}

template <int W>
uint64_t sort_bytes_w(uint64_t buf_cap) {
    const uint64_t t_cap = (buf_cap + kSTile - 1) / kSTile;
    uint64_t b = 256 + (uint64_t)kMaxPass * kDig * 4;
    b += ((uint64_t)kDig * t_cap * 4 + 255) / 256 * 256;
    b += 2 * (((uint64_t)buf_cap * sizeof(PKey<W>) + 255) / 256 * 256);
    b += 2 * (((uint64_t)buf_cap * 8 + 255) / 256 * 256);
    return b;
}

struct PassArg {
    int word;    // 0..W-1: x[word]; W..2W-1: z[word-W]
    int shift;   // bit offset of the digit in the word
};

template <int W>
__device__ __forceinline__ uint32_t digit_of(const PKey<W>& k, PassArg a) {
    const uint64_t v = a.word < W ? k.x[a.word] : k.z[a.word - W];
    return (uint32_t)(v >> a.shift) & 0xffu;
}

// Reset the per-gate counters.
__global__ void k_sort_begin(DevCtl* ctl, unsigned long long* n_child, unsigned int* totals,
                             int npass) {
    if (ctl->status) return;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctl->count[ctl->cur ^ 1] = 0ULL;
        *n_child = 0ULL;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npass * kDig; i += gridDim.x * blockDim.x)
        totals[i] = 0u;
}

// 1. Expand: pass-through of anticommuting terms, children of commuting ones.
template <int W>
__global__ void __launch_bounds__(kSB)
k_sort_expand(Bufs<W> B, DevCtl* ctl, GateArg<W> g, SortBufs<W> sb, double delta,
              uint64_t cap_out) {
    __shared__ uint32_t s_scan[kSB / 32];
    __shared__ unsigned long long s_base[2];
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rnorm = ctl->rnorm[cur];
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    const uint64_t tiles = (n + kSB - 1) / kSB;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t i = t * kSB + threadIdx.x;
        PKey<W> K;
#pragma unroll
        for (int w = 0; w < W; ++w) { K.x[w] = 0; K.z[w] = 0; }
        double raw = 0.0;
        bool live = i < n, comm = false, neg = false;
        if (live) {
            K = load_key_stream(B.key(cur) + i);
            raw = __ldcs(B.coef(cur) + i);
            comm = commutes(K, g);
            neg = comm && product_negative(K, g);
        }
        const double c = key_is_zero(K) ? 1.0 : __dmul_rn(raw, rnorm);
        const double m = __longlong_as_double(
            __double_as_longlong(g.msh) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
        const double a1 = __dmul_rn(c, g.ch);     // cosh(theta) K
        const double b1 = __dmul_rn(c, m);        // -sinh(theta) s QK
        // the identity commutes with every gate, so a pass-through is never it
        const bool pass = live && !comm && above(c, dbits) && light(K, g.maxw);
        const bool kids = live && comm;
        uint32_t tot_p, tot_k;
        const uint32_t off_p = block_exclusive_scan<kSB>(pass ? 1u : 0u, &tot_p, s_scan);
        const uint32_t off_k = block_exclusive_scan<kSB>(kids ? 2u : 0u, &tot_k, s_scan);
        if (threadIdx.x == 0) {
            s_base[0] = tot_p ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot_p) : 0ULL;
            s_base[1] = tot_k ? atomicAdd(sb.n_child, (unsigned long long)tot_k) : 0ULL;
        }
        __syncthreads();
        const unsigned long long bp = s_base[0], bk = s_base[1];
        __syncthreads();
        if (bp + tot_p > cap_out || bk + tot_k > sb.child_cap) {
            if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 50);
            return;
        }
        if (pass) {
            store_key_stream(B.key(cur ^ 1) + bp + off_p, K);
            __stcs(B.coef(cur ^ 1) + bp + off_p, c);
        }
        if (kids) {
            const uint64_t q = bk + off_k;
            store_key_stream(sb.k[0] + q, K);
            sb.c[0][q] = a1;
            store_key_stream(sb.k[0] + q + 1, key_xor(K, g));
            sb.c[0][q + 1] = b1;
        }
    }
}

// 2a. Per-tile digit counts (row-major [digit][tile]) and per-pass totals.
template <int W>
__global__ void __launch_bounds__(kSB)
k_rs_count(DevCtl* ctl, SortBufs<W> sb, int src, PassArg pa, int pass) {
    __shared__ unsigned int h[kDig];
    if (ctl->status) return;
    const uint64_t n = *sb.n_child;
    const uint64_t tiles = (n + kSTile - 1) / kSTile;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        h[threadIdx.x] = 0u;
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < kSI; ++j) {
            const uint64_t i = t * kSTile + (uint64_t)j * kSB + threadIdx.x;
            if (i < n) atomicAdd(&h[digit_of(sb.k[src][i], pa)], 1u);
        }
        __syncthreads();
        const unsigned int v = h[threadIdx.x];
        sb.counts[(uint64_t)threadIdx.x * sb.t_cap + t] = v;
        if (v) atomicAdd(&sb.totals[pass * kDig + threadIdx.x], v);
        __syncthreads();
    }
}

// 2b. Offsets: row d of the count matrix becomes the exclusive prefix over
// tiles plus the number of items with a smaller digit.
__global__ void __launch_bounds__(1024)
k_rs_rowscan(DevCtl* ctl, unsigned long long* n_child, unsigned int* counts,
             const unsigned int* totals, uint64_t t_cap, int pass) {
    __shared__ unsigned int s_w[32];
    __shared__ unsigned int s_carry;
    if (ctl->status) return;
    const uint64_t n = *n_child;
    const uint64_t tiles = (n + kSTile - 1) / kSTile;
    const int d = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        unsigned int base = 0;
        for (int e = 0; e < d; ++e) base += totals[pass * kDig + e];
        s_carry = base;
    }
    __syncthreads();
    unsigned int* row = counts + (uint64_t)d * t_cap;
    for (uint64_t c0 = 0; c0 < tiles; c0 += 1024) {
        const uint64_t i = c0 + threadIdx.x;
        const unsigned int v = i < tiles ? row[i] : 0u;
        unsigned int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned int w = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const unsigned int before = (warp ? s_w[warp - 1] : 0u) + x - v;
        if (i < tiles) row[i] = s_carry + before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_w[31];
        __syncthreads();
    }
}

// 2c. Stable scatter: items of a tile in index order (j, then thread), each
// to its digit's offset plus its rank among the tile's earlier items with
// the same digit.
template <int W>
__global__ void __launch_bounds__(kSB)
k_rs_scatter(DevCtl* ctl, SortBufs<W> sb, int src, PassArg pa) {
    constexpr int kWarps = kSB / 32;
    __shared__ unsigned int s_off[kDig];
    __shared__ unsigned int s_wc[kWarps][kDig];
    if (ctl->status) return;
    const uint64_t n = *sb.n_child;
    const uint64_t tiles = (n + kSTile - 1) / kSTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int lt = (1u << lane) - 1u;
    const int dst = src ^ 1;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        s_off[threadIdx.x] = sb.counts[(uint64_t)threadIdx.x * sb.t_cap + t];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s_wc[w][threadIdx.x] = 0u;
        __syncthreads();
        for (int j = 0; j < kSI; ++j) {
            const uint64_t i = t * kSTile + (uint64_t)j * kSB + threadIdx.x;
            const bool live = i < n;
            PKey<W> K;
            double c = 0.0;
            uint32_t d = kDig;            // a key no live item has
            if (live) {
                K = sb.k[src][i];
                c = sb.c[src][i];
                d = digit_of(K, pa);
            }
            const unsigned int peers = __match_any_sync(0xffffffffu, d);
            const unsigned int rank = __popc(peers & lt);
            if (live && rank == 0) s_wc[warp][d] = __popc(peers);
            __syncthreads();
            if (live) {
                unsigned int before = 0;
                for (int w = 0; w < warp; ++w) before += s_wc[w][d];
                const uint64_t q = (uint64_t)s_off[d] + before + rank;
                sb.k[dst][q] = K;
                sb.c[dst][q] = c;
            }
            __syncthreads();
            unsigned int sum = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) { sum += s_wc[w][threadIdx.x]; s_wc[w][threadIdx.x] = 0u; }
            s_off[threadIdx.x] += sum;
            __syncthreads();
        }
    }
}

// 3. Segmented reduce of the sorted children, truncation, output.
template <int W>
__global__ void __launch_bounds__(kSB)
k_sort_reduce(Bufs<W> B, DevCtl* ctl, SortBufs<W> sb, int src, GateArg<W> g, double delta,
              uint64_t cap_out) {
    __shared__ uint32_t s_scan[kSB / 32];
    __shared__ unsigned long long s_base;
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = *sb.n_child;
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    const PKey<W>* __restrict__ k = sb.k[src];
    const double* __restrict__ c = sb.c[src];
    const uint64_t tiles = (n + kSB - 1) / kSB;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t i = t * kSB + threadIdx.x;
        PKey<W> K;
        double v = 0.0;
        bool keep = false;
        if (i < n) {
            K = k[i];
            const bool start = i == 0 || !key_eq(k[i - 1], K);
            if (start) {
                v = c[i];
                if (i + 1 < n && key_eq(k[i + 1], K)) {
                    v = __dadd_rn(v, c[i + 1]);        // the two addends of K
                    if (i + 2 < n && key_eq(k[i + 2], K)) set_status(ctl, ST_STATE, 51);
                }
                keep = above(v, dbits) && light(K, g.maxw);
                if (key_is_zero(K)) {
                    ctl->norm[cur ^ 1] = v;            // the merged identity: new trace
                    if (!keep) set_status(ctl, ST_TRACE_ZERO, 52);
                    keep = true;
                }
            }
        }
        uint32_t tot;
        const uint32_t off = block_exclusive_scan<kSB>(keep ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
        __syncthreads();
        const unsigned long long base = s_base;
        __syncthreads();
        if (base + tot > cap_out) {
            if (threadIdx.x == 0) set_status(ctl, ST_CAPACITY, 53);
            return;
        }
        if (keep) {
            store_key_stream(B.key(cur ^ 1) + base + off, K);
            __stcs(B.coef(cur ^ 1) + base + off, v);
        }
    }
}

template <int W>
static Bufs<W> sbufs_of(const DeviceState& s) {
    Bufs<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    return b;
}

// The digit passes that can see a nonzero digit: bits >= n are zero in
// every key.
template <int W>
static int plan_passes(int n, PassArg* out) {
    int np = 0;
    for (int plane = 0; plane < 2; ++plane)
        for (int w = 0; w < W; ++w) {
            const int bits = n - 64 * w < 64 ? n - 64 * w : 64;
            for (int sh = 0; sh < bits; sh += 8) out[np++] = PassArg{plane * W + w, sh};
        }
    return np;
}

template <int W>
static cudaError_t sorted_w(const DeviceState& s, const HostGate& h, void* scratch,
                            cudaStream_t st) {
    GateArg<W> g;
    for (int w = 0; w < W; ++w) { g.qx[w] = h.qx[w]; g.qz[w] = h.qz[w]; }
    g.ch = h.ch;
    g.msh = h.msh;
    g.qyy = h.qyy;
    g.maxw = h.maxw;
    const SortBufs<W> sb = sort_layout<W>(scratch, s.buf_cap);
    PassArg pa[kMaxPass];
    const int npass = plan_passes<W>(s.n, pa);
    const Bufs<W> B = sbufs_of<W>(s);
    k_sort_begin<<<8, 1024, 0, st>>>(s.ctl, sb.n_child, sb.totals, npass);
    uint64_t ge = (s.buf_cap + kSB - 1) / kSB;
    const uint64_t lim = (uint64_t)s.num_sms * 8;
    if (ge > lim) ge = lim;
    if (ge < 1) ge = 1;
    k_sort_expand<W><<<(int)ge, kSB, 0, st>>>(B, s.ctl, g, sb, s.delta, s.buf_cap);
    uint64_t gt = sb.t_cap;
    const uint64_t lim_t = (uint64_t)s.num_sms * 4;
    if (gt > lim_t) gt = lim_t;
    if (gt < 1) gt = 1;
    int src = 0;
    for (int q = 0; q < npass; ++q) {
        k_rs_count<W><<<(int)gt, kSB, 0, st>>>(s.ctl, sb, src, pa[q], q);
        k_rs_rowscan<<<kDig, 1024, 0, st>>>(s.ctl, sb.n_child, sb.counts, sb.totals, sb.t_cap, q);
        k_rs_scatter<W><<<(int)gt, kSB, 0, st>>>(s.ctl, sb, src, pa[q]);
        src ^= 1;
    }
    k_sort_reduce<W><<<(int)ge, kSB, 0, st>>>(B, s.ctl, sb, src, g, s.delta, s.buf_cap);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gate_sorted(const DeviceState& s, const HostGate& g, void* scratch,
                               uint64_t scratch_bytes, cudaStream_t st) {
    if (scratch_bytes < sorted_scratch_bytes(s.W, s.buf_cap)) return cudaErrorInvalidValue;
    return s.W == 1 ? sorted_w<1>(s, g, scratch, st) : sorted_w<2>(s, g, scratch, st);
}

uint64_t sorted_scratch_bytes(int W, uint64_t buf_cap) {
    return W == 1 ? sort_bytes_w<1>(buf_cap) : sort_bytes_w<2>(buf_cap);
}

int sorted_launches(int n, int W) {
    PassArg pa[kMaxPass];
    const int np = W == 1 ? plan_passes<1>(n, pa) : plan_passes<2>(n, pa);
    return 3 + 3 * np;
}

}  // namespace itpp
