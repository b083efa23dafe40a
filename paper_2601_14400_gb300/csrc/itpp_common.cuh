// itpp_common.cuh -- device data layout and Pauli bit algebra shared by the
// sm_103a kernels of the imaginary-time Pauli propagation library.
//
// Layout in HBM (one propagation):
//   state buffers 0 and 1, each 2*cap_M terms:
//     keys  PKey<W>[2*cap_M]  AoS, 16*W bytes per term: x[0..W-1], z[0..W-1]
//     coef  double[2*cap_M]   raw (un-normalised) coefficients
//   merge table  Slot<W>[2^t]  open addressing, 32 B (W=1) / 64 B (W=2) slots
//   DevCtl       counters, the current-buffer index, normalisers, status
// The stored coefficient of term i is raw[i]; its value is raw[i] * rnorm[cur]
// with rnorm = 1 / (raw identity coefficient), and exactly 1 for the identity
// (the trace normalisation of Sec. II.C -- identify the identity coefficient
// and rescale every coefficient -- applied when the term is next read).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace itpp {

// Device status codes (same numbering as itpp_status in include/itpp.h).
enum : int {
    ST_OK = 0, ST_ARG = 1, ST_ALLOC = 2, ST_CAPACITY = 3, ST_HASH_PROBE = 4,
    ST_TIMEOUT = 5, ST_TRACE_ZERO = 6, ST_CUDA = 7, ST_STATE = 8
};

template <int W>
struct alignas(16) PKey {
    uint64_t x[W];
    uint64_t z[W];
};

// Merge-table slot: the key, its raw coefficient, the generation tag that
// marks the slot as occupied in the current gate, and the source index.
template <int W>
struct alignas(W == 1 ? 32 : 64) Slot {
    uint64_t x[W];
    uint64_t z[W];
    double c;
    uint32_t tag;
    uint32_t idx;
};
static_assert(sizeof(Slot<1>) == 32, "slot size");
static_assert(sizeof(Slot<2>) == 64, "slot size");

// Per-gate constants, passed by value.
template <int W>
struct GateArg {
    uint64_t qx[W];
    uint64_t qz[W];
    double ch;    // cosh(theta), theta = alpha * dtau
    double msh;   // -sinh(theta)
    int qyy;      // popcount(qx & qz) mod 4 (number of Y letters in Q)
    int maxw = 1 << 30;   // Pauli weight cutoff (Sec. II.B): keep weight <= maxw
};

constexpr int kSelBits = 13;                 // radix digit of the top-M select
constexpr int kSelBins = 1 << kSelBits;
constexpr int kTieBits = 16;                 // radix digit of the tie (key) select
constexpr int kTieBins = 1 << kTieBits;

// Device-resident control block: everything that changes from gate to gate
// lives here, so a sequence of gates can be launched (or captured) without
// the host knowing any count.
struct DevCtl {
    unsigned long long count[2];   // term count of state buffer 0 / 1
    unsigned long long buf_cap;    // capacity of each state buffer (terms)
    double norm[2];                // normaliser of buffer 0 / 1 (raw identity coefficient)
    double rnorm[2];               // its reciprocal, 1.0 / norm (one division per gate)
    int cur;                       // buffer holding the state
    int status;                    // first device error (ST_*), sticky
    unsigned int gen;              // merge-table generation of the current gate
    unsigned int err_info;
    // statistics
    unsigned long long stat_gates, stat_in, stat_out, stat_peak, stat_cap;
    unsigned long long stat_probes;
    unsigned long long stat_scatters;
    unsigned long long stat_cands, stat_range;
    // top-M select state
    int sel_active;
    int sel_pass;
    unsigned long long sel_k;        // rank still to place among the prefix matches
    unsigned long long sel_prefix;   // |c| bit pattern fixed so far
    unsigned long long sel_mask;
    unsigned long long sel_ties;     // number of terms with |c| == threshold
    unsigned long long sel_tie_keep; // how many of them to keep
    unsigned long long sel_tie_n;    // tie list length (compacted)
    unsigned long long sel_tie_k;    // rank still to place in the tie select
    int sel_tie_state;               // 0 running, 1 key known, 2 unique prefix found
    int sel_small, sel_resolved;     // batched select: few values share the prefix
                                     // (gathered and resolved at once), resolved
    int sel_tie_pass;
    unsigned long long sel_cand_n;   // candidates gathered after the first digit
    // deferred top-M compaction: the state buffer holds pend_n terms of which
    // the select's kept set (sel_prefix / tie key) is the state; the next
    // gate's scatter or an explicit materialisation applies it
    int pend;
    int pend_all_ties;
    unsigned long long pend_n;
    unsigned long long pend_T;
    uint64_t pend_tie_key[4];
    uint64_t sel_tie_key[4];         // largest kept tie key (x..., z...)
    // partitioned merge: where the next merge finds its partitions
    unsigned int part_P;             // partitions of the current state
    int part_from_scatter;           // 1: in the scatter buffer; 0: segments of the state
    int part_over;                   // this gate's partitions hold for this gate only
    int need_scatter;                // ... so the next gate re-partitions
    // segmented state: the merge writes every partition's children as one
    // segment of a chunk its CTA claimed (alloc[] is the chunk allocator of
    // each buffer); the buffer then holds seg_P segments, described by the
    // partition descriptors, with unused room between them
    int seg;                         // 1: the current buffer is segmented
    unsigned int seg_P;
    unsigned long long alloc[2];
    unsigned int nchunk[2];          // output chunks in use per buffer (contiguous runs)
    // top-M select folded into the merge: the merge counts its kept
    // children above sp_hi and lists those in [sp_lo, sp_hi] (a range around
    // the previous gate's threshold); the select then reads only that list
    unsigned long long sp_lo, sp_hi; // candidate range (sp_hi == 0: none)
    unsigned long long sp_above;     // kept children with pattern > sp_hi
    unsigned long long sp_tprev;     // the last select's threshold pattern (0: none)
    int sp_ovf;                      // a CTA's candidate region overflowed
    int sp_shift;                    // log2 of the range's half-width (0: unset)
    unsigned int cand_regions;       // regions of the candidate list in use
    int sel_fast;                    // this select reads the merge's candidates
    int sp_reason;                   // why not: 1 no range, 2 list too long, 3 threshold
                                     // above the range, 4 below it
    int sel_top;                     // bits of v = pattern - sel_lo still to resolve
    unsigned long long sel_lo;       // offset of the select's values
    unsigned long long stat_sel_full, stat_long;
    // children below the candidate range left unwritten by this gate's merge
    // (drop_on); the merge is run again in full when fewer than cap_M were
    // kept (retry), counted in stat_retry
    int drop_on, retry;
    unsigned long long stat_retry;
    int scatter_over;                // a window's partition stride overflowed: the
                                     // gate scatters again by its pair key
    // top-M select geometry: largest |c| pattern the gate wrote (partitioned
    // merge), the value the select uses, and the last-CTA counter
    unsigned long long out_max;
    unsigned long long sel_hi;
    unsigned int sel_done;
    unsigned long long sel_hist[kSelBins];
    unsigned long long tie_hist[kTieBins];
};

// Terms held by buffer b, clamped to the buffer (after a device error the
// counters may run past it; every kernel also returns early on an error).
__device__ __forceinline__ uint64_t live_count(const DevCtl* ctl, int b) {
    const unsigned long long n = ctl->count[b];
    return n < ctl->buf_cap ? n : ctl->buf_cap;
}

// The 63-bit magnitude pattern of a double.  The mask is applied in inline
// PTX so that the compiler does not turn it into a floating-point |x|, which
// would run on the (slow, shared) double-precision pipe.
__device__ __forceinline__ unsigned long long abs_pattern(double c) {
    unsigned long long r;
    asm("and.b64 %0, %1, 0x7fffffffffffffff;" : "=l"(r) : "l"(__double_as_longlong(c)));
    return r;
}

// |c| > delta for delta >= 0, decided on the bit patterns: for non-negative
// doubles the unsigned order of the patterns is the numeric order, so this is
// exact (NaN patterns exceed +inf and count as kept, where fabs(c) > delta
// would drop them; the propagation produces no NaN from finite inputs).
__device__ __forceinline__ bool above(double c, unsigned long long delta_bits) {
    return abs_pattern(c) > delta_bits;
}

// Normalised value of a stored coefficient.
__device__ __forceinline__ double normalised(double raw, double rnorm, bool identity) {
    return identity ? 1.0 : __dmul_rn(raw, rnorm);
}

__device__ __forceinline__ void set_status(DevCtl* ctl, int code, unsigned int info = 0) {
    if (atomicCAS(&ctl->status, 0, code) == 0) ctl->err_info = info;
}

// ---------------------------------------------------------------------------
// Pauli bit algebra (Sec. II.C and App. A)
// ---------------------------------------------------------------------------

// [P, Q] = 0 iff the symplectic product sum_i (xP_i zQ_i + zP_i xQ_i) is even.
template <int W>
__device__ __forceinline__ bool commutes(const PKey<W>& k, const GateArg<W>& g) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += __popcll((k.x[w] & g.qz[w]) ^ (k.z[w] & g.qx[w]));
    return (s & 1) == 0;
}

// For a commuting pair, Q P = s R with R = (xQ^xP, zQ^zP) and s = +-1.
// With sigma(a,b) = i^{ab} X^a Z^b per site the phase exponent is
// e = #Y(Q) + #Y(P) - #Y(R) + 2 popc(zQ & xP) (mod 4), and e is 0 or 2
// when P and Q commute.  Returns true when s = -1.
template <int W>
__device__ __forceinline__ bool product_negative(const PKey<W>& k, const GateArg<W>& g) {
    int e = g.qyy;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t x3 = k.x[w] ^ g.qx[w], z3 = k.z[w] ^ g.qz[w];
        e += __popcll(k.x[w] & k.z[w]) - __popcll(x3 & z3) + 2 * __popcll(g.qz[w] & k.x[w]);
    }
    return (e & 3) == 2;
}

template <int W>
__device__ __forceinline__ PKey<W> key_xor(const PKey<W>& k, const GateArg<W>& g) {
    PKey<W> r;
#pragma unroll
    for (int w = 0; w < W; ++w) { r.x[w] = k.x[w] ^ g.qx[w]; r.z[w] = k.z[w] ^ g.qz[w]; }
    return r;
}

template <int W>
__device__ __forceinline__ bool key_is_zero(const PKey<W>& k) {
    uint64_t a = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) a |= k.x[w] | k.z[w];
    return a == 0;
}

// Within the Pauli weight cutoff: at most maxw non-identity letters,
// popc(x | z) <= maxw (a bound of 64W or more never drops a string).
template <int W>
__device__ __forceinline__ bool light(const PKey<W>& k, int maxw) {
    if (maxw >= 64 * W) return true;
    int w = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) w += __popcll(k.x[i] | k.z[i]);
    return w <= maxw;
}

// Whether k * Q (Q the gate's string) is the identity, i.e. k == Q.
template <int W>
__device__ __forceinline__ bool key_is_zero_xor(const PKey<W>& k, const GateArg<W>& g) {
    uint64_t a = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) a |= (k.x[w] ^ g.qx[w]) | (k.z[w] ^ g.qz[w]);
    return a == 0;
}

template <int W>
__device__ __forceinline__ bool key_eq(const PKey<W>& a, const PKey<W>& b) {
    uint64_t d = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) d |= (a.x[w] ^ b.x[w]) | (a.z[w] ^ b.z[w]);
    return d == 0;
}

// a < b in the export order: x[0..W-1] then z[0..W-1], unsigned.
template <int W>
__device__ __forceinline__ bool key_less(const PKey<W>& a, const PKey<W>& b) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (a.x[w] != b.x[w]) return a.x[w] < b.x[w];
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (a.z[w] != b.z[w]) return a.z[w] < b.z[w];
    return false;
}

// ---------------------------------------------------------------------------
// Hashing of keys: MurmurHash3 (x86, 32-bit) over the 4W 32-bit halves of
// the key.  Only 32-bit multiplies: on GB300 the 64-bit integer multiply of
// a 64-bit mixer competes with the FP64 arithmetic for the same slow pipe.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

__device__ __forceinline__ uint32_t murmur_mix(uint32_t h, uint32_t k) {
    k *= 0xcc9e2d51u;
    k = rotl32(k, 15);
    k *= 0x1b873593u;
    h ^= k;
    h = rotl32(h, 13);
    return h * 5u + 0xe6546b64u;
}

template <int W>
__device__ __forceinline__ uint64_t key_hash(const PKey<W>& k) {
    uint32_t h = 0x9747b28cu;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h = murmur_mix(h, (uint32_t)k.x[w]);
        h = murmur_mix(h, (uint32_t)(k.x[w] >> 32));
        h = murmur_mix(h, (uint32_t)k.z[w]);
        h = murmur_mix(h, (uint32_t)(k.z[w] >> 32));
    }
    h ^= 16u * W;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return (uint64_t)h;
}

// Slots of the table used when the input holds n terms (load <= load_pct%).
__device__ __forceinline__ uint64_t table_mask(uint64_t n, uint64_t alloc_slots, int load_pct) {
    uint64_t need = (n * 100ULL + (uint64_t)load_pct - 1) / (uint64_t)load_pct;
    if (need < 256) need = 256;
    uint64_t s = 1;
    while (s < need) s <<= 1;
    if (s > alloc_slots) s = alloc_slots;
    return s - 1;
}

// ---------------------------------------------------------------------------
// Global memory access helpers
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ PKey<W> load_key_stream(const PKey<W>* p) {
    PKey<W> k;
    const ulonglong2* v = reinterpret_cast<const ulonglong2*>(p);
    if constexpr (W == 1) {
        ulonglong2 a = __ldcs(v);
        k.x[0] = a.x;
        k.z[0] = a.y;
    } else {
        ulonglong2 a = __ldcs(v), b = __ldcs(v + 1);
        k.x[0] = a.x; k.x[1] = a.y;
        k.z[0] = b.x; k.z[1] = b.y;
    }
    return k;
}

template <int W>
__device__ __forceinline__ PKey<W> load_key(const PKey<W>* p) {
    PKey<W> k;
    const ulonglong2* v = reinterpret_cast<const ulonglong2*>(p);
    if constexpr (W == 1) {
        ulonglong2 a = __ldg(v);
        k.x[0] = a.x;
        k.z[0] = a.y;
    } else {
        ulonglong2 a = __ldg(v), b = __ldg(v + 1);
        k.x[0] = a.x; k.x[1] = a.y;
        k.z[0] = b.x; k.z[1] = b.y;
    }
    return k;
}

template <int W>
__device__ __forceinline__ void store_key(PKey<W>* p, const PKey<W>& k) {
    ulonglong2* v = reinterpret_cast<ulonglong2*>(p);
    if constexpr (W == 1) {
        *v = make_ulonglong2(k.x[0], k.z[0]);
    } else {
        v[0] = make_ulonglong2(k.x[0], k.x[1]);
        v[1] = make_ulonglong2(k.z[0], k.z[1]);
    }
}

template <int W>
__device__ __forceinline__ void store_key_stream(PKey<W>* p, const PKey<W>& k) {
    ulonglong2* v = reinterpret_cast<ulonglong2*>(p);
    if constexpr (W == 1) {
        __stcs(v, make_ulonglong2(k.x[0], k.z[0]));
    } else {
        __stcs(v, make_ulonglong2(k.x[0], k.x[1]));
        __stcs(v + 1, make_ulonglong2(k.z[0], k.z[1]));
    }
}

// Exclusive block scan of one 32-bit value per thread; *total gets the sum.
// smem needs BLOCK/32 entries.  Ends with a barrier.
template <int BLOCK>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total,
                                                         uint32_t* smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < BLOCK / 32) ? smem[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < BLOCK / 32) smem[lane] = w;
    }
    __syncthreads();
    const uint32_t before = (warp == 0) ? 0u : smem[warp - 1];
    *total = smem[BLOCK / 32 - 1];
    __syncthreads();
    return before + x - v;
}

}  // namespace itpp
