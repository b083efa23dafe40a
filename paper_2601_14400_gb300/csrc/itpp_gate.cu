// itpp_gate.cu -- the per-gate kernels of one propagation on sm_103a: one
// elementary step of Algorithm 1 (propagate every term with
// Eq. (ITPP_PropRules), accumulate equal strings, truncate, normalise), and
// the top-M select of the term bound.  The bodies live in itpp_gate_body.cuh.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

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
    g.maxw = h.maxw;
    return g;
}

__device__ __forceinline__ void flush_probes(DevCtl* ctl, int probes) {
    for (int o = 16; o > 0; o >>= 1) probes += __shfl_down_sync(0xffffffffu, probes, o);
    if ((threadIdx.x & 31) == 0 && probes) atomicAdd(&ctl->stat_probes, (unsigned long long)probes);
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
    int probes = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        insert_one(B.key(cur), B.coef(cur), i, ctl, table, mask, gen, g, probe_limit, &probes);
    flush_probes(ctl, probes);
}

// ---------------------------------------------------------------------------
// k_gate_main: branch, emit, merge (partner lookup), truncate, compact.
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
    constexpr uint64_t TILE = (uint64_t)BLOCK * IPT;
    const uint64_t tiles = (n + TILE - 1) / TILE;
    int probes = 0;
    const GlobalLookup<W> lk{table, mask, gen, probe_limit, ctl, &probes};
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x)
        gate_tile<W, BLOCK, IPT>(t, n, B.key(cur), B.coef(cur), B.key(cur ^ 1), B.coef(cur ^ 1), ctl, cur,
                                 lk, g, rnorm, dbits, cap_out, s_scan, &s_base);
    flush_probes(ctl, probes);
}

// ---------------------------------------------------------------------------
// k_gate_post: buffer switch, normaliser, generation, statistics, bound.
// ---------------------------------------------------------------------------
__global__ void k_gate_post(DevCtl* ctl, uint64_t cap_M, int cap_policy) {
    __shared__ int s_active;
    if (ctl->status) return;
    if (threadIdx.x == 0) s_active = post_one(ctl, cap_M, cap_policy);
    __syncthreads();
    if (s_active)
        for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) ctl->sel_hist[b] = 0ULL;
}

// ---------------------------------------------------------------------------
// Top-M select chain (every kernel returns at once when the bound holds).
// ---------------------------------------------------------------------------
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
    const double* __restrict__ c = B.coef(cur);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = abs_bits(__ldg(c + i));
        if ((b & mask) == prefix) atomicAdd(&h[(b >> shift) & (kSelBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (h[b]) atomicAdd(&ctl->sel_hist[b], (unsigned long long)h[b]);
}

__global__ void __launch_bounds__(1024) k_cap_pick(DevCtl* ctl, int shift, int last) {
    if (!ctl->sel_active || ctl->status) return;
    __shared__ unsigned long long s_part[1024];
    cap_pick_block(ctl, shift, last, s_part);
}

// Compact the keys of the terms at the threshold into the tie list (only
// when some of them are dropped); prepare the output buffer.
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
        const bool tie = i < n && abs_bits(__ldg(B.coef(cur) + i)) == T;
        uint32_t tot;
        const uint32_t off = block_exclusive_scan<BLOCK>(tie ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->sel_tie_n, (unsigned long long)tot) : 0ULL;
        __syncthreads();
        if (tie) tie_list[s_base + off] = load_key(B.key(cur) + i);
    }
}

template <int W>
__global__ void __launch_bounds__(256)
k_tie_hist(DevCtl* ctl, const PKey<W>* tie_list, int p) {
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 0) return;
    tie_hist_range<W>(ctl, tie_list, p, (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x,
                      ctl->sel_tie_n, (unsigned long long)gridDim.x * blockDim.x);
}

template <int W>
__global__ void __launch_bounds__(1024) k_tie_pick(DevCtl* ctl, int p) {
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 0) return;
    __shared__ unsigned long long s_part[1024];
    tie_pick_block<W>(ctl, p, s_part);
}

template <int W>
__global__ void __launch_bounds__(256) k_tie_find(DevCtl* ctl, const PKey<W>* tie_list) {
    if (!tie_select_needed(ctl) || ctl->sel_tie_state != 2) return;
    tie_find_range<W>(ctl, tie_list, (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x,
                      ctl->sel_tie_n, (unsigned long long)gridDim.x * blockDim.x);
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
            K = load_key_stream(B.key(cur) + i);
            c = __ldcs(B.coef(cur) + i);
            keep = cap_keep(K, c, T, all_ties, tk);
            if (key_is_zero(K) && !keep) set_status(ctl, ST_TRACE_ZERO, 2);
        }
        uint32_t tot;
        const uint32_t off = block_exclusive_scan<BLOCK>(keep ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
        __syncthreads();
        if (keep) {
            store_key_stream(B.key(cur ^ 1) + s_base + off, K);
            __stcs(B.coef(cur ^ 1) + s_base + off, c);
        }
    }
}

__global__ void k_cap_end(DevCtl* ctl) {
    if (threadIdx.x == 0 && ctl->sel_active) {
        if (!ctl->status) ctl->cur ^= 1;
        ctl->sel_active = 0;
    }
}

template <int W>
__device__ __forceinline__ PKey<W> pend_tie_key(const DevCtl* ctl) {
    PKey<W> tk;
#pragma unroll
    for (int w = 0; w < W; ++w) { tk.x[w] = ctl->pend_tie_key[w]; tk.z[w] = ctl->pend_tie_key[W + w]; }
    return tk;
}

// Materialise the state of the partitioned merge for a reader that wants a
// contiguous run: apply a deferred select (its kept set), and gather the
// segments of a segmented buffer, into the other buffer (normaliser
// unchanged), then switch to it.
__device__ __forceinline__ bool mat_needed(const DevCtl* ctl) { return ctl->pend || ctl->seg; }

__global__ void k_mat_begin(DevCtl* ctl) {
    if (threadIdx.x != 0 || !mat_needed(ctl) || ctl->status) return;
    const int cur = ctl->cur;
    ctl->count[cur ^ 1] = 0ULL;
    ctl->norm[cur ^ 1] = ctl->norm[cur];
    ctl->rnorm[cur ^ 1] = ctl->rnorm[cur];
}

// One round of up to BLOCK terms [i0, i0 + BLOCK) of a run of n (every
// thread calls it).
template <int W, int BLOCK>
__device__ __forceinline__ void mat_round(const Bufs<W>& B, DevCtl* ctl, int cur, uint64_t off,
                                          uint64_t n, uint64_t i0, bool pend, unsigned long long T,
                                          bool all_ties, const PKey<W>& tk, uint32_t* s_scan,
                                          unsigned long long* s_base) {
    const uint64_t i = i0 + threadIdx.x;
    PKey<W> K;
    double c = 0;
    bool keep = false;
    if (i < n) {
        K = load_key_stream(B.key(cur) + off + i);
        c = __ldcs(B.coef(cur) + off + i);
        keep = !pend || cap_keep(K, c, T, all_ties, tk);
        if (key_is_zero(K) && !keep) set_status(ctl, ST_TRACE_ZERO, 3);
    }
    uint32_t tot;
    const uint32_t o = block_exclusive_scan<BLOCK>(keep ? 1u : 0u, &tot, s_scan);
    if (threadIdx.x == 0)
        *s_base = tot ? atomicAdd(&ctl->count[cur ^ 1], (unsigned long long)tot) : 0ULL;
    __syncthreads();
    if (keep) {
        store_key_stream(B.key(cur ^ 1) + *s_base + o, K);
        __stcs(B.coef(cur ^ 1) + *s_base + o, c);
    }
}

template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_materialize(Bufs<W> B, DevCtl* ctl, const ChunkDesc* chunks0, const ChunkDesc* chunks1) {
    if (!mat_needed(ctl) || ctl->status) return;
    __shared__ uint32_t s_scan[BLOCK / 32];
    __shared__ unsigned long long s_base;
    const int cur = ctl->cur;
    const bool pend = ctl->pend != 0;
    const unsigned long long T = ctl->pend_T;
    const bool all_ties = ctl->pend_all_ties;
    const PKey<W> tk = pend_tie_key<W>(ctl);
    if (ctl->seg) {
        const ChunkDesc* din = cur ? chunks1 : chunks0;
        const uint32_t P = ctl->nchunk[cur];
        for (uint32_t p = blockIdx.x; p < P; p += gridDim.x) {
            const uint64_t off = din[p].off, n = din[p].cnt;
            for (uint64_t i0 = 0; i0 < n; i0 += BLOCK)
                mat_round<W, BLOCK>(B, ctl, cur, off, n, i0, pend, T, all_ties, tk, s_scan, &s_base);
        }
    } else {
        uint64_t n = pend ? ctl->pend_n : ctl->count[cur];
        if (n > ctl->buf_cap) n = ctl->buf_cap;
        const uint64_t tiles = (n + BLOCK - 1) / BLOCK;
        for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x)
            mat_round<W, BLOCK>(B, ctl, cur, 0, n, t * BLOCK, pend, T, all_ties, tk, s_scan, &s_base);
    }
}

__global__ void k_mat_end(DevCtl* ctl) {
    if (threadIdx.x != 0 || !mat_needed(ctl)) return;
    if (!ctl->status) ctl->cur ^= 1;
    ctl->pend = 0;
    ctl->seg = 0;
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
static cudaError_t cap_select_w(const DeviceState& s, cudaStream_t st) {
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
    return cudaGetLastError();
}

template <int W>
static cudaError_t cap_w(const DeviceState& s, cudaStream_t st) {
    cudaError_t e = cap_select_w<W>(s, st);
    if (e != cudaSuccess) return e;
    const int g = stream_grid(s, 256, 8);
    k_cap_compact<W, 256><<<g, 256, 0, st>>>(bufs_of<W>(s), s.ctl);
    k_cap_end<<<1, 32, 0, st>>>(s.ctl);
    return cudaGetLastError();
}

cudaError_t launch_cap_select(const DeviceState& s, cudaStream_t st) {
    return s.W == 1 ? cap_select_w<1>(s, st) : cap_select_w<2>(s, st);
}

int cap_launches(const DeviceState& s) {
    return s.merge_deferred ? select_deferred_launches(s.W) : 5 * 2 + 1 + 8 * s.W * 2 + 3;
}

template <int W>
static cudaError_t materialize_w(const DeviceState& s, cudaStream_t st) {
    k_mat_begin<<<1, 32, 0, st>>>(s.ctl);
    k_materialize<W, 256><<<stream_grid(s, 256, 8), 256, 0, st>>>(bufs_of<W>(s), s.ctl,
                                                                  s.chunks[0], s.chunks[1]);
    k_mat_end<<<1, 32, 0, st>>>(s.ctl);
    return cudaGetLastError();
}

cudaError_t launch_materialize(const DeviceState& s, cudaStream_t st) {
    if (!s.merge_deferred) return cudaSuccess;
    return s.W == 1 ? materialize_w<1>(s, st) : materialize_w<2>(s, st);
}

cudaError_t launch_cap(const DeviceState& s, cudaStream_t st, int gate) {
    if (s.merge_deferred) return launch_select_deferred(s, st, gate);
    return s.W == 1 ? cap_w<1>(s, st) : cap_w<2>(s, st);
}

}  // namespace itpp
