// itpp_aux.cu -- sm_103a kernels around the gate: expectation values read
// from the propagated operator (Sec. II.C), explicit threshold truncation,
// normalised export, import with validation, and the identity initial state
// (Algorithm 1, "Initialize rho = I").
#include "itpp_common.cuh"
#include "itpp_launch.h"

namespace itpp {

template <int W>
struct BufsA {
    PKey<W>* k[2];
    double* c[2];
    // by compare-select (a dynamic index copies the array to local memory)
    __device__ __forceinline__ PKey<W>* key(int i) const { return i ? k[1] : k[0]; }
    __device__ __forceinline__ double* coef(int i) const { return i ? c[1] : c[0]; }
};

template <int W>
static BufsA<W> bufsa_of(const DeviceState& s) {
    BufsA<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    return b;
}

static int grid_for(const DeviceState& s, uint64_t n, int block, int per_sm) {
    uint64_t g = (n + block - 1) / block;
    uint64_t lim = (uint64_t)s.num_sms * per_sm;
    if (g > lim) g = lim;
    if (g < 1) g = 1;
    return (int)g;
}

template <int W>
__device__ __forceinline__ PKey<W> key_from_planes(const uint64_t* x, const uint64_t* z,
                                                   uint64_t j) {
    PKey<W> k;
#pragma unroll
    for (int w = 0; w < W; ++w) { k.x[w] = x[j * W + w]; k.z[w] = z[j * W + w]; }
    return k;
}

// ---------------------------------------------------------------------------
// Expectation values: <O> = sum_j w_j c_{P_j} (identity coefficient one).
// ---------------------------------------------------------------------------

// One CTA: deterministic open-addressing table of the observable strings
// (first occurrence of each distinct string), zeroed value slots.
template <int W>
__global__ void k_obs_prep(const uint64_t* ox, const uint64_t* oz, int m, int tsize, int* tab,
                           int* first, double* vals, DevCtl* ctl) {
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) tab[t] = -1;
    for (int j = threadIdx.x; j < m; j += blockDim.x) vals[j] = 0.0;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const uint64_t mask = (uint64_t)tsize - 1;
    for (int j = 0; j < m; ++j) {
        const PKey<W> K = key_from_planes<W>(ox, oz, (uint64_t)j);
        uint64_t h = key_hash(K) & mask;
        int p = 0;
        for (; p < tsize; ++p) {
            const int e = tab[h];
            if (e < 0) { tab[h] = j; first[j] = j; break; }
            if (key_eq(key_from_planes<W>(ox, oz, (uint64_t)e), K)) { first[j] = e; break; }
            h = (h + 1) & mask;
        }
        if (p == tsize) set_status(ctl, ST_HASH_PROBE, 3);
    }
}

// Stream the state once; each term looks its key up in the observable
// table and, on a hit, writes its normalised coefficient to the slot of the
// first occurrence (a key occurs at most once in the state).
template <int W>
__global__ void __launch_bounds__(256)
k_obs_scan(BufsA<W> B, DevCtl* ctl, const uint64_t* __restrict__ ox,
           const uint64_t* __restrict__ oz, int tsize, const int* __restrict__ tab,
           double* vals) {
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rnorm = ctl->rnorm[cur];
    const uint64_t mask = (uint64_t)tsize - 1;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = load_key(B.key(cur) + i);
        uint64_t h = key_hash(K) & mask;
        for (int p = 0; p < tsize; ++p) {
            const int e = __ldg(tab + h);
            if (e < 0) break;
            if (key_eq(key_from_planes<W>(ox, oz, (uint64_t)e), K)) {
                vals[e] = normalised(__ldg(B.coef(cur) + i), rnorm, key_is_zero(K));
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

// One CTA of 256 threads: out[j] = c_{P_j}; out[m] = sum_j w_j c_{P_j},
// Kahan-compensated per thread over a fixed stride, then combined in a fixed
// tree order (deterministic).
__global__ void __launch_bounds__(256)
k_obs_reduce(int m, const int* __restrict__ first, const double* __restrict__ vals,
             const double* __restrict__ w, double* out) {
    __shared__ double s_sum[256], s_cmp[256];
    double sum = 0.0, cmp = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double c = vals[first[j]];
        out[j] = c;
        if (w) {
            const double y = __dsub_rn(__dmul_rn(w[j], c), cmp);
            const double t = __dadd_rn(sum, y);
            cmp = __dsub_rn(__dsub_rn(t, sum), y);
            sum = t;
        }
    }
    s_sum[threadIdx.x] = sum;
    s_cmp[threadIdx.x] = cmp;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            // add (sum_b - cmp_b) into (sum_a, cmp_a) with one compensated step
            const double a = s_sum[threadIdx.x], ca = s_cmp[threadIdx.x];
            const double b = s_sum[threadIdx.x + o], cb = s_cmp[threadIdx.x + o];
            const double y = __dsub_rn(b, __dadd_rn(ca, cb));
            const double t = __dadd_rn(a, y);
            s_cmp[threadIdx.x] = __dsub_rn(__dsub_rn(t, a), y);
            s_sum[threadIdx.x] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[m] = s_sum[0];
}

template <int W>
static cudaError_t expect_w(const DeviceState& s, const uint64_t* ox, const uint64_t* oz,
                            const double* ow, int m, int tsize, int* tab, int* first,
                            double* vals, double* out, cudaStream_t st) {
    k_obs_prep<W><<<1, 256, 0, st>>>(ox, oz, m, tsize, tab, first, vals, s.ctl);
    k_obs_scan<W><<<grid_for(s, s.buf_cap, 256, 8), 256, 0, st>>>(
        bufsa_of<W>(s), s.ctl, ox, oz, tsize, tab, vals);
    k_obs_reduce<<<1, 256, 0, st>>>(m, first, vals, ow, out);
    return cudaGetLastError();
}

cudaError_t launch_expect(const DeviceState& s, const uint64_t* ox, const uint64_t* oz,
                          const double* ow, int m, int tsize, int* tab, int* first,
                          double* vals, double* out, cudaStream_t st) {
    return s.W == 1 ? expect_w<1>(s, ox, oz, ow, m, tsize, tab, first, vals, out, st)
                    : expect_w<2>(s, ox, oz, ow, m, tsize, tab, first, vals, out, st);
}

// ---------------------------------------------------------------------------
// Export: x plane, z plane and normalised coefficients of the current state.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256)
k_export(BufsA<W> B, const DevCtl* ctl, uint64_t* xo, uint64_t* zo, double* co) {
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rnorm = ctl->rnorm[cur];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = load_key(B.key(cur) + i);
#pragma unroll
        for (int w = 0; w < W; ++w) { xo[i * W + w] = K.x[w]; zo[i * W + w] = K.z[w]; }
        co[i] = normalised(B.coef(cur)[i], rnorm, key_is_zero(K));
    }
}

cudaError_t launch_export(const DeviceState& s, uint64_t* x, uint64_t* z, double* c,
                          cudaStream_t st) {
    const int g = grid_for(s, s.buf_cap, 256, 8);
    if (s.W == 1) k_export<1><<<g, 256, 0, st>>>(bufsa_of<1>(s), s.ctl, x, z, c);
    else k_export<2><<<g, 256, 0, st>>>(bufsa_of<2>(s), s.ctl, x, z, c);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Import: planes -> buffer 0, with checks (bits >= n clear, the identity
// present with c != 0, keys distinct via the merge table).
// ---------------------------------------------------------------------------
__global__ void k_import_begin(DevCtl* ctl, uint64_t count) {
    if (threadIdx.x == 0) {
        ctl->cur = 0;
        ctl->count[0] = count;
        ctl->count[1] = 0;
        ctl->norm[0] = 1.0;
        ctl->norm[1] = 1.0;
        ctl->rnorm[0] = 1.0;
        ctl->rnorm[1] = 1.0;
        ctl->status = 0;
        ctl->err_info = 0;
        ctl->gen = ctl->gen + 1u;
        ctl->sel_active = 0;
        ctl->sel_tie_n = 0;
        ctl->stat_gates = ctl->stat_in = ctl->stat_out = ctl->stat_cap = ctl->stat_probes = 0;
        ctl->stat_scatters = 0;
        ctl->stat_cands = 0;
        ctl->stat_range = 0;
        ctl->stat_peak = count;
        ctl->stat_sel_full = ctl->stat_long = ctl->stat_retry = 0;
        ctl->drop_on = ctl->retry = ctl->scatter_over = 0;
        ctl->sel_k = 0;   // reused below as "identity seen" flag
        ctl->pend = 0;
        ctl->seg = 0;
        ctl->sp_lo = ctl->sp_hi = 0;
        ctl->sp_shift = 0;
        ctl->sp_tprev = 0;
    }
}

template <int W>
__global__ void __launch_bounds__(256)
k_import(BufsA<W> B, DevCtl* ctl, const uint64_t* x, const uint64_t* z, const double* c,
         uint64_t count, int n_sites, Slot<W>* table, uint64_t alloc_slots, int probe_limit) {
    const unsigned gen = ctl->gen;
    const uint64_t mask = table_mask(count, alloc_slots, 50);
    uint64_t top[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int lo = 64 * w;
        top[w] = (n_sites >= lo + 64) ? 0ULL
                 : (n_sites <= lo ? ~0ULL : (~0ULL << (n_sites - lo)));
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = key_from_planes<W>(x, z, i);
        const double ci = c[i];
        bool bad = false;
#pragma unroll
        for (int w = 0; w < W; ++w) bad |= ((K.x[w] | K.z[w]) & top[w]) != 0;
        if (bad) set_status(ctl, ST_ARG, 10);
        if (key_is_zero(K)) {
            if (ci == 0.0) set_status(ctl, ST_TRACE_ZERO, 10);
            atomicAdd(&ctl->sel_k, 1ULL);
        }
        B.key(0)[i] = K;
        B.coef(0)[i] = ci;
        // table insert for the duplicate check (key -> index)
        uint64_t h = key_hash(K) & mask;
        int p = 0;
        for (; p < probe_limit; ++p) {
            Slot<W>* s = table + h;
            unsigned t = __ldcg(&s->tag);
            bool done = false;
            while (t != gen) {
                const unsigned old = atomicCAS(&s->tag, t, gen);
                if (old == t) {
                    for (int w = 0; w < W; ++w) { s->x[w] = K.x[w]; s->z[w] = K.z[w]; }
                    s->idx = (uint32_t)i;
                    done = true;
                    break;
                }
                t = old;
            }
            if (done) break;
            h = (h + 1) & mask;
        }
        if (p == probe_limit) set_status(ctl, ST_HASH_PROBE, 10);
    }
}

template <int W>
__global__ void __launch_bounds__(256)
k_import_check(const BufsA<W> B, DevCtl* ctl, uint64_t count, const Slot<W>* table,
               uint64_t alloc_slots, int probe_limit) {
    const unsigned gen = ctl->gen;
    const uint64_t mask = table_mask(count, alloc_slots, 50);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = B.key(0)[i];
        uint64_t h = key_hash(K) & mask;
        for (int p = 0; p < probe_limit; ++p) {
            const Slot<W>* s = table + h;
            if (s->tag != gen) break;
            PKey<W> k2;
            for (int w = 0; w < W; ++w) { k2.x[w] = s->x[w]; k2.z[w] = s->z[w]; }
            if (key_eq(k2, K)) {
                if (s->idx != (uint32_t)i) set_status(ctl, ST_ARG, 11);   // duplicate key
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__global__ void k_import_end(DevCtl* ctl) {
    if (threadIdx.x == 0) {
        if (ctl->sel_k != 1ULL) set_status(ctl, ST_TRACE_ZERO, 12);   // identity missing
        ctl->sel_k = 0;
        ctl->gen = ctl->gen + 1u;
    }
}

template <int W>
static cudaError_t import_w(const DeviceState& s, const uint64_t* x, const uint64_t* z,
                            const double* c, uint64_t count, cudaStream_t st) {
    const int g = grid_for(s, count, 256, 8);
    k_import_begin<<<1, 32, 0, st>>>(s.ctl, count);
    k_import<W><<<g, 256, 0, st>>>(bufsa_of<W>(s), s.ctl, x, z, c, count, s.n,
                                   reinterpret_cast<Slot<W>*>(s.table), s.table_slots,
                                   s.probe_limit);
    k_import_check<W><<<g, 256, 0, st>>>(bufsa_of<W>(s), s.ctl, count,
                                         reinterpret_cast<const Slot<W>*>(s.table),
                                         s.table_slots, s.probe_limit);
    k_import_end<<<1, 32, 0, st>>>(s.ctl);
    return cudaGetLastError();
}

cudaError_t launch_import(const DeviceState& s, const uint64_t* x, const uint64_t* z,
                          const double* c, uint64_t count, cudaStream_t st) {
    return s.W == 1 ? import_w<1>(s, x, z, c, count, st) : import_w<2>(s, x, z, c, count, st);
}

// ---------------------------------------------------------------------------
// Identity state (Algorithm 1 initialisation).
// ---------------------------------------------------------------------------
template <int W>
__global__ void k_reset_identity(BufsA<W> B, DevCtl* ctl) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        PKey<W> I;
        for (int w = 0; w < W; ++w) { I.x[w] = 0; I.z[w] = 0; }
        B.key(0)[0] = I;
        B.coef(0)[0] = 1.0;
        ctl->cur = 0;
        ctl->count[0] = 1;
        ctl->count[1] = 0;
        ctl->norm[0] = 1.0;
        ctl->norm[1] = 1.0;
        ctl->rnorm[0] = 1.0;
        ctl->rnorm[1] = 1.0;
        ctl->status = 0;
        ctl->err_info = 0;
        ctl->gen = ctl->gen + 1u;
        ctl->sel_active = 0;
        ctl->sel_tie_n = 0;
        ctl->sel_k = 0;
        ctl->pend = 0;
        ctl->seg = 0;
        ctl->sp_lo = ctl->sp_hi = 0;
        ctl->sp_shift = 0;
        ctl->sp_tprev = 0;
        ctl->stat_gates = ctl->stat_in = ctl->stat_out = ctl->stat_cap = ctl->stat_probes = 0;
        ctl->stat_scatters = 0;
        ctl->stat_cands = 0;
        ctl->stat_range = 0;
        ctl->stat_sel_full = ctl->stat_long = ctl->stat_retry = 0;
        ctl->drop_on = ctl->retry = ctl->scatter_over = 0;
        ctl->stat_peak = 1;
    }
}

cudaError_t launch_reset_identity(const DeviceState& s, cudaStream_t st) {
    if (s.W == 1) k_reset_identity<1><<<1, 32, 0, st>>>(bufsa_of<1>(s), s.ctl);
    else k_reset_identity<2><<<1, 32, 0, st>>>(bufsa_of<2>(s), s.ctl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Explicit truncation: keep |c| > delta of the normalised state, write the
// normalised values into the other buffer (normaliser one).
// ---------------------------------------------------------------------------
__global__ void k_trunc_begin(DevCtl* ctl) {
    if (ctl->status) return;
    if (threadIdx.x == 0) {
        const int cur = ctl->cur;
        ctl->count[cur ^ 1] = 0;
        ctl->norm[cur ^ 1] = 1.0;
        ctl->rnorm[cur ^ 1] = 1.0;
    }
}

template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_trunc(BufsA<W> B, DevCtl* ctl, double delta) {
    __shared__ uint32_t s_scan[BLOCK / 32];
    __shared__ unsigned long long s_base;
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rnorm = ctl->rnorm[cur];
    const uint64_t tiles = (n + BLOCK - 1) / BLOCK;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t i = t * BLOCK + threadIdx.x;
        PKey<W> K;
        double c = 0;
        bool keep = false;
        if (i < n) {
            K = load_key_stream(B.key(cur) + i);
            c = normalised(__ldcs(B.coef(cur) + i), rnorm, key_is_zero(K));
            keep = above(c, (unsigned long long)__double_as_longlong(delta));
            if (key_is_zero(K) && !keep) {
                set_status(ctl, ST_TRACE_ZERO, 20);
                keep = true;
            }
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

__global__ void k_flip(DevCtl* ctl) {
    if (threadIdx.x == 0 && !ctl->status) ctl->cur ^= 1;
}

cudaError_t launch_truncate(const DeviceState& s, double delta, cudaStream_t st) {
    const int g = grid_for(s, s.buf_cap, 256, 8);
    k_trunc_begin<<<1, 32, 0, st>>>(s.ctl);
    if (s.W == 1) k_trunc<1, 256><<<g, 256, 0, st>>>(bufsa_of<1>(s), s.ctl, delta);
    else k_trunc<2, 256><<<g, 256, 0, st>>>(bufsa_of<2>(s), s.ctl, delta);
    k_flip<<<1, 32, 0, st>>>(s.ctl);
    return cudaGetLastError();
}

}  // namespace itpp
