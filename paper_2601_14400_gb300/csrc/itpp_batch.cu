// itpp_batch.cu -- many independent propagations advanced together.
//
// B instances (each its own Hamiltonian, gate count, state, merge table and
// control block) take their gate g of the current Trotter layer in the same
// launches: a plan kernel lays the active instances' terms and tiles out in
// one index space (exclusive prefix over instances), and the table-build,
// branch-emit and top-M kernels map each item or tile back to its instance.
// Every instance runs the device bodies of the single propagation
// (itpp_gate_body.cuh), so its state is bit-identical to a plain run.
// Instances with fewer gates per layer sit out the later steps.  A whole
// layer (all steps) is captured once into a CUDA graph by the C ABI and
// replayed, since every quantity that changes between layers lives on the
// device.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {

constexpr int kIpt = 2;                               // branch-emit items per thread
constexpr uint64_t kTileH = 4096;                     // histogram tile
constexpr uint64_t kTileC = 256;                      // compaction tile

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
    return b;
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
        const unsigned long long tiles = (items + kTile - 1) / kTile;
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
    if (!ctl->sel_active || ctl->status) return;
    __shared__ unsigned long long s_part[1024];
    cap_pick_block(ctl, shift, last, s_part);
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
template <int W>
static cudaError_t batch_step_w(const BatchState& s, int step, cudaStream_t st) {
    const BatchBufs<W> S = batch_bufs<W>(s);
    const int grid = s.num_sms * 8;
    k_b_plan<W><<<1, 1024, 0, st>>>(S, step, (uint64_t)s.main_block * kIpt);
    k_b_insert<W><<<s.num_sms * s.insert_grid, 256, 0, st>>>(S, step, s.load_pct, s.probe_limit);
    const int gm = s.num_sms * s.main_grid;
    switch (s.main_block) {
        case 128: k_b_main<W, 128><<<gm, 128, 0, st>>>(S, step, s.delta, s.load_pct, s.probe_limit); break;
        case 512: k_b_main<W, 512><<<gm, 512, 0, st>>>(S, step, s.delta, s.load_pct, s.probe_limit); break;
        default:  k_b_main<W, 256><<<gm, 256, 0, st>>>(S, step, s.delta, s.load_pct, s.probe_limit); break;
    }
    k_b_post<W><<<1, 1024, 0, st>>>(S, s.cap_M, s.cap_policy);
    if (s.cap_policy == 1) {
        const int shifts[5] = {50, 37, 24, 11, 0};
        for (int p = 0; p < 5; ++p) {
            k_b_cap_hist<W><<<grid, 256, 0, st>>>(S, shifts[p]);
            k_b_cap_pick<W><<<s.B, 1024, 0, st>>>(S, shifts[p], p == 4 ? 1 : 0);
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
    return 4 + (s.cap_policy == 1 ? 5 * 2 + 1 + 8 * s.W * 2 + 3 : 0);
}

}  // namespace itpp
