// itpp_adjoint.cu -- gradients of a propagated expectation value with respect
// to every gate coefficient alpha_k, by a reverse sweep over the steps with
// the kept support of every step frozen (the paper has no such step; this is
// the linear algebra of Eq. (ITPP_PropRules) and the per-step normalisation).
//
// With u_s the normalised state after step s (support S_s), D_s its identity
// coefficient before normalisation and f = sum_j w_j u_L[P_j]:
//   nu_s[K] = mu_s[K] / D_s (K != I),  nu_s[I] = -sum_{K != I} mu_s[K] u_s[K] / D_s
//   mu_{s-1}[P] = nu_s[P]                                ({P,Q} = 0)
//               = cosh nu_s[P] + s (-sinh) nu_s[Q P]    ([P,Q] = 0)
//   df/dtheta_s = sum_{[P,Q]=0} u_{s-1}[P] (sinh nu_s[P] - s cosh nu_s[Q P])
// where mu_s = df/du_s, nu_s = 0 outside S_s and theta_s = alpha_k dtau.
// S_s is the kept set of step s: after the threshold and, with the top-M
// bound, after the select.
//
// Memory: the forward saves a snapshot every ckpt_every layers; each segment
// is recomputed from its snapshot into an arena that keeps every step's state
// and, per input term, the output positions of its children (itself, a new
// partner string, or the partner that was present).  The reverse sweep then
// gathers through those positions -- no atomics, fixed-order reductions.
// Output order inside a recomputed segment need not match the first forward,
// so the adjoint vector is carried across a segment boundary by key (a
// table lookup into the snapshot's keys).
#include <cmath>
#include <cstring>
#include <vector>

#include "itpp.h"
#include "itpp_common.cuh"
#include "itpp_ctx.h"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

using namespace itpp;

namespace {

constexpr int kRB = 256;      // reduction block
constexpr int kRGrid = 512;   // fixed reduction grid: deterministic partial order

template <int W>
GateArg<W> gate_arg_of(const HostGate& h) {
    GateArg<W> g;
    for (int w = 0; w < W; ++w) { g.qx[w] = h.qx[w]; g.qz[w] = h.qz[w]; }
    g.ch = h.ch;
    g.msh = h.msh;
    g.qyy = h.qyy;
    g.maxw = h.maxw;
    return g;
}

__device__ __forceinline__ double block_sum(double v, double* s) {
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] = __dadd_rn(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

__global__ void k_adj_log(const DevCtl* ctl, unsigned long long* log, int s) {
    if (threadIdx.x == 0) log[s] = ctl->status ? ~0ULL : ctl->count[ctl->cur];
}

// Snapshot of the current state: AoS keys and normalised coefficients.
template <int W>
__global__ void __launch_bounds__(256)
k_adj_snapshot(const PKey<W>* k0, const double* c0, const PKey<W>* k1, const double* c1,
               const DevCtl* ctl, PKey<W>* keys, double* coef) {
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rn = ctl->rnorm[cur];
    const PKey<W>* ks = cur ? k1 : k0;
    const double* cs = cur ? c1 : c0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = ks[i];
        keys[i] = K;
        coef[i] = normalised(cs[i], rn, key_is_zero(K));
    }
}

// Before recomputing step r: input region r-1 holds cnt[r-1] terms scaled by
// rn[r-1]; outputs go to region r.
__global__ void k_adj_prep(DevCtl* ctl, const unsigned long long* cnt, const double* rn, int r,
                           unsigned long long cap) {
    if (threadIdx.x != 0) return;
    ctl->cur = 0;
    ctl->count[0] = cnt[r - 1];
    ctl->count[1] = 0;
    ctl->rnorm[0] = rn[r - 1];
    ctl->norm[0] = 1.0;
    ctl->buf_cap = cap;
    ctl->sel_active = 0;
}

template <int W>
__global__ void __launch_bounds__(256)
k_adj_insert(const PKey<W>* kin, const double* cin, DevCtl* ctl, Slot<W>* table,
             uint64_t alloc_slots, GateArg<W> g, int probe_limit) {
    if (ctl->status) return;
    const uint64_t n = live_count(ctl, 0);
    const uint64_t mask = table_mask(n, alloc_slots, 50);
    const unsigned gen = ctl->gen;
    int probes = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        insert_one(kin, cin, i, ctl, table, mask, gen, g, probe_limit, &probes);
}

template <int W>
__global__ void __launch_bounds__(256)
k_adj_main(const PKey<W>* kin, const double* cin, PKey<W>* kout, double* cout, DevCtl* ctl,
           const Slot<W>* table, uint64_t alloc_slots, GateArg<W> g, double delta,
           uint64_t cap_out, int probe_limit, StepMaps maps) {
    __shared__ uint32_t s_scan[256 / 32];
    __shared__ unsigned long long s_base;
    if (ctl->status) return;
    const uint64_t n = live_count(ctl, 0);
    const double rnorm = ctl->rnorm[0];
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    const unsigned gen = ctl->gen;
    const uint64_t mask = table_mask(n, alloc_slots, 50);
    const uint64_t tiles = (n + 511) / 512;
    int probes = 0;
    const GlobalLookup<W> lk{table, mask, gen, probe_limit, ctl, &probes};
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x)
        gate_tile<W, 256, 2, true>(t, n, kin, cin, kout, cout, ctl, 0, lk, g, rnorm, dbits,
                                   cap_out, s_scan, &s_base, maps);
}

__global__ void k_adj_post(DevCtl* ctl, uint64_t cap_M, int cap_policy) {
    if (threadIdx.x != 0 || ctl->status) return;
    post_one(ctl, cap_M, cap_policy);   // output (buffer 1) above the bound -> select
    ctl->count[0] = 0;                  // the compacted copy is counted here
    ctl->norm[0] = ctl->norm[1];
    ctl->rnorm[0] = ctl->rnorm[1];
}

// Kept terms of step r (all of them, or the top-M select's when it fired)
// copied from the step's output into its compact region, recording the
// compaction map and the identity's position.
template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_adj_compact(const PKey<W>* kpre, const double* cpre, PKey<W>* kout, double* cout,
              DevCtl* ctl, int* cmap, unsigned long long* id_pos) {
    __shared__ uint32_t s_scan[BLOCK / 32];
    __shared__ unsigned long long s_base;
    if (ctl->status) return;
    const uint64_t n = live_count(ctl, 1);
    const bool active = ctl->sel_active;
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
            K = kpre[i];
            c = cpre[i];
            keep = !active || cap_keep(K, c, T, all_ties, tk);
            if (key_is_zero(K) && !keep) set_status(ctl, ST_TRACE_ZERO, 32);
        }
        uint32_t tot;
        const uint32_t off = block_exclusive_scan<BLOCK>(keep ? 1u : 0u, &tot, s_scan);
        if (threadIdx.x == 0)
            s_base = tot ? atomicAdd(&ctl->count[0], (unsigned long long)tot) : 0ULL;
        __syncthreads();
        if (i < n) {
            const uint64_t pos = s_base + off;
            cmap[i] = keep ? (int)pos : -1;
            if (keep) {
                kout[pos] = K;
                cout[pos] = c;
                if (key_is_zero(K)) *id_pos = pos;
            }
        }
    }
}

__global__ void k_adj_after(DevCtl* ctl, unsigned long long* cnt, double* rn, int r) {
    if (threadIdx.x != 0) return;
    cnt[r] = ctl->count[0];
    rn[r] = ctl->rnorm[1];
    ctl->sel_active = 0;
}

// Seed: mu[i] = sum of the weights of the observable strings equal to key i.
template <int W>
__global__ void __launch_bounds__(256)
k_adj_seed(const PKey<W>* keys, uint64_t n, const uint64_t* ox, const uint64_t* oz,
           const double* wsum, const int* tab, int tsize, double* mu) {
    const uint64_t mask = (uint64_t)tsize - 1;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = keys[i];
        double v = 0.0;
        uint64_t h = key_hash(K) & mask;
        for (int p = 0; p < tsize; ++p) {
            const int e = tab[h];
            if (e < 0) break;
            PKey<W> o;
            for (int w = 0; w < W; ++w) { o.x[w] = ox[(size_t)e * W + w]; o.z[w] = oz[(size_t)e * W + w]; }
            if (key_eq(o, K)) { v = wsum[e]; break; }
            h = (h + 1) & mask;
        }
        mu[i] = v;
    }
}

// Per distinct observable string (first occurrence), the sum of its weights.
__global__ void k_adj_wsum(const int* first, const double* w, int m, double* wsum) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int j = 0; j < m; ++j) wsum[j] = 0.0;
    for (int j = 0; j < m; ++j) wsum[first[j]] = __dadd_rn(wsum[first[j]], w[j]);
}

// dot = sum_{j != idpos} mu[j] u[j], u = raw * rn; block partials.
__global__ void __launch_bounds__(kRB)
k_adj_dot(const double* raw, const double* mu, uint64_t n, const unsigned long long* idpos,
          const double* rn, double* partials) {
    __shared__ double s[kRB];
    const unsigned long long id = *idpos;
    const double r = *rn;
    double acc = 0.0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x)
        if (j != id) acc = __dadd_rn(acc, __dmul_rn(mu[j], __dmul_rn(raw[j], r)));
    const double b = block_sum(acc, s);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// nu_I = -dot / D = -dot * rn (one block).
__global__ void __launch_bounds__(kRB)
k_adj_dot_final(const double* partials, int np, const double* rn, double* nu_i) {
    __shared__ double s[kRB];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc = __dadd_rn(acc, partials[i]);
    const double b = block_sum(acc, s);
    if (threadIdx.x == 0) *nu_i = -__dmul_rn(b, *rn);
}

// mu_{s-1} from nu_s through the recorded output positions; partial sums of
// df/dtheta_s.
template <int W>
__global__ void __launch_bounds__(kRB)
k_adj_back(const PKey<W>* kin, const double* cin, uint64_t n_in, const double* rn_in,
           const int* self_out, const int* emit_out, const int* part_src, const int* cmap,
           const double* mu_out, const unsigned long long* idpos_out, const double* rn_out,
           const double* nu_i, GateArg<W> g, double sh, double chd, double* mu_in,
           double* partials) {
    __shared__ double s[kRB];
    const double ri = *rn_in, ro = *rn_out, nI = *nu_i;
    const long long id = (long long)*idpos_out;
    // nu at an output position of the step (before the term bound)
    auto nu = [&](int pre) -> double {
        if (pre < 0) return 0.0;
        const int c = cmap[pre];
        return c < 0 ? 0.0 : (c == id ? nI : __dmul_rn(mu_out[c], ro));
    };
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_in;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = kin[i];
        const double vs = nu(self_out[i]);
        if (!commutes(K, g)) {
            mu_in[i] = vs;
        } else {
            const double sg = product_negative(K, g) ? -1.0 : 1.0;
            int po = emit_out[i];
            if (po < 0 && part_src[i] >= 0) po = self_out[part_src[i]];
            const double vp = nu(po);
            mu_in[i] = __dadd_rn(__dmul_rn(g.ch, vs), __dmul_rn(sg * g.msh, vp));
            const double u = normalised(cin[i], ri, key_is_zero(K));
            acc = __dadd_rn(acc, __dmul_rn(u, __dsub_rn(__dmul_rn(sh, vs),
                                                        __dmul_rn(sg * chd, vp))));
        }
    }
    const double b = block_sum(acc, s);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void __launch_bounds__(kRB)
k_adj_gsum(const double* partials, int np, double* gstep, long long s) {
    __shared__ double sh[kRB];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc = __dadd_rn(acc, partials[i]);
    const double b = block_sum(acc, sh);
    if (threadIdx.x == 0) gstep[s] = b;
}

template <int W>
__global__ void __launch_bounds__(256)
k_adj_remap_insert(const PKey<W>* keys, const double* mu, uint64_t n, Slot<W>* table,
                   uint64_t alloc_slots, DevCtl* ctl, int probe_limit) {
    const uint64_t mask = table_mask(n, alloc_slots, 50);
    const unsigned gen = ctl->gen;
    int probes = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (!table_insert(table, mask, gen, keys[i], mu[i], (uint32_t)i, probe_limit, &probes))
            set_status(ctl, ST_HASH_PROBE, 30);
}

template <int W>
__global__ void __launch_bounds__(256)
k_adj_remap_lookup(const PKey<W>* keys, uint64_t n, uint64_t n_table, double* mu,
                   const Slot<W>* table, uint64_t alloc_slots, DevCtl* ctl, int probe_limit) {
    const uint64_t mask = table_mask(n_table, alloc_slots, 50);
    const unsigned gen = ctl->gen;
    int probes = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (!table_find(table, mask, gen, keys[i], &v, probe_limit, ctl, &probes))
            set_status(ctl, ST_STATE, 31);   // the sets at a boundary must agree
        mu[i] = v;
    }
}

__global__ void k_adj_bump_gen(DevCtl* ctl) {
    if (threadIdx.x == 0) ctl->gen = ctl->gen + 1u;
}

// The adjoint shares the handle's merge table: its generations continue the
// handle's, and the handle continues after the adjoint's, so no stale slot
// ever reads as occupied.
__global__ void k_adj_gen_copy(DevCtl* dst, const DevCtl* src) {
    if (threadIdx.x == 0) dst->gen = src->gen + 1u;
}

// Frozen forward with other gate weights: one step of the linear map of
// Eq. (ITPP_PropRules) on the kept support recorded by the recompute (the
// output positions of every input's children, and which were kept), before
// the step's normalisation.  Every kept position receives exactly one write.
template <int W>
__global__ void __launch_bounds__(256)
k_frz_step(const PKey<W>* kin, const double* u_in, uint64_t n_in, const int* self_out,
           const int* emit_out, const int* part_src, const int* cmap, GateArg<W> g,
           double* u_out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_in;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = kin[i];
        const double u = u_in[i];
        const int so = self_out[i];
        const int ks = so >= 0 ? cmap[so] : -1;
        if (!commutes(K, g)) {
            if (ks >= 0) u_out[ks] = u;
            continue;
        }
        const double m = product_negative(K, g) ? -g.msh : g.msh;   // s (-sinh)
        const int ps = part_src[i];
        const double a = __dmul_rn(g.ch, u);
        if (ks >= 0) u_out[ks] = ps >= 0 ? __dadd_rn(a, __dmul_rn(m, u_in[ps])) : a;
        const int eo = emit_out[i];
        const int ke = eo >= 0 ? cmap[eo] : -1;
        if (ke >= 0) u_out[ke] = __dmul_rn(m, u);
    }
}

// The step's normalisation: every kept value divided by the identity's (the
// identity then exactly one).  d receives the identity's value first.
__global__ void k_frz_trace(const double* u, const unsigned long long* id_pos, double* d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d = u[*id_pos];
}

__global__ void __launch_bounds__(256)
k_frz_scale(double* u, uint64_t n, const unsigned long long* id_pos, const double* d) {
    const unsigned long long id = *id_pos;
    const double r = __ddiv_rn(1.0, *d);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        u[i] = i == id ? 1.0 : __dmul_rn(u[i], r);
}

// sum_i mu[i] u[i] (block partials; fixed grid, fixed order).
__global__ void __launch_bounds__(kRB)
k_frz_dot(const double* mu, const double* u, uint64_t n, double* partials) {
    __shared__ double s[kRB];
    double acc = 0.0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x)
        acc = __dadd_rn(acc, __dmul_rn(mu[j], u[j]));
    const double b = block_sum(acc, s);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// grad_alpha[k] = dtau * sum over layers of df/dtheta at gate k.
__global__ void k_adj_params(const double* gstep, int n_layers, int n_gates, double dtau,
                             double* grad) {
    for (int k = threadIdx.x; k < n_gates; k += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < n_layers; ++l)
            acc = __dadd_rn(acc, gstep[(size_t)l * n_gates + k]);
        grad[k] = __dmul_rn(acc, dtau);
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    bool alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16) == cudaSuccess; }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Weights of a frozen evaluation: per elementary gate of the schedule.
struct FrozenEval {
    std::vector<double> ch, msh;
};

// The adjoint sweep (ev == nullptr), or the frozen forward evaluated with the
// weights of ev on the support the handle's own coefficients produce (ev:
// value receives f, grad_alpha is not written).
template <int W>
itpp_status adjoint_w(itpp_ctx* h, int L, int K, const uint64_t* obs_x, const uint64_t* obs_z,
                      const double* seed, int m, double* grad_alpha, double* value,
                      const FrozenEval* ev = nullptr) {
    DeviceState& s = h->s;
    cudaStream_t st = h->stream;
    const int G = (int)h->gates.size();
    const long long S = (long long)L * G;
    const int n_seg = (L + K - 1) / K;
    const size_t kb = sizeof(PKey<W>);
    const int grid = s.num_sms * 8;
    auto chk = [&](cudaError_t e) { return e == cudaSuccess; };

    // ---- forward from the identity, logging counts, snapshot per segment
    DevBuf log;
    if (!log.alloc((size_t)(S + 1) * 8)) return ITPP_ERR_ALLOC;
    itpp_detail_touch(h);
    if (!chk(launch_reset_identity(s, st))) return ITPP_ERR_CUDA;
    std::vector<DevBuf> snap((size_t)n_seg);
    std::vector<uint64_t> snap_n((size_t)n_seg);
    for (int j = 0; j < n_seg; ++j) {
        itpp_status stt = itpp_detail_sync_ctl(h);
        if (stt) return stt;
        const uint64_t c = h->h_ctl->count[h->h_ctl->cur];
        snap_n[(size_t)j] = c;
        if (!snap[(size_t)j].alloc((size_t)c * (kb + 8))) return ITPP_ERR_ALLOC;
        PKey<W>* sk = snap[(size_t)j].as<PKey<W>>();
        double* sc = reinterpret_cast<double*>(sk + c);
        if (!chk((itpp_detail_touch(h), launch_materialize(s, st)))) return ITPP_ERR_CUDA;
        k_adj_snapshot<W><<<grid, 256, 0, st>>>(
            static_cast<const PKey<W>*>(s.keys[0]), s.coef[0],
            static_cast<const PKey<W>*>(s.keys[1]), s.coef[1], s.ctl, sk, sc);
        if (j == 0) k_adj_log<<<1, 32, 0, st>>>(s.ctl, log.as<unsigned long long>(), 0);
        const int l_end = (j + 1) * K < L ? (j + 1) * K : L;
        for (int l = j * K; l < l_end; ++l)
            for (int k = 0; k < G; ++k) {
                itpp_status e = itpp_detail_launch_gate(h, k);
                if (e) return e;
                k_adj_log<<<1, 32, 0, st>>>(s.ctl, log.as<unsigned long long>(),
                                            (int)((long long)l * G + k + 1));
            }
    }
    itpp_status stt = itpp_detail_sync_ctl(h);
    if (stt) return stt;
    std::vector<unsigned long long> cnt_log((size_t)S + 1);
    if (!chk(cudaMemcpy(cnt_log.data(), log.p, (size_t)(S + 1) * 8, cudaMemcpyDeviceToHost)))
        return ITPP_ERR_CUDA;

    // ---- value f and the observable table for the seed
    const size_t tsize = [&] { size_t t = 1; while (t < (size_t)2 * m) t <<= 1; return t; }();
    DevBuf obs;
    if (!obs.alloc((size_t)m * W * 16 + (size_t)m * 8 * 4 + tsize * 4 + (size_t)m * 4 + 64))
        return ITPP_ERR_ALLOC;
    char* op = obs.as<char>();
    uint64_t* d_ox = reinterpret_cast<uint64_t*>(op); op += (size_t)m * W * 8;
    uint64_t* d_oz = reinterpret_cast<uint64_t*>(op); op += (size_t)m * W * 8;
    double* d_w = reinterpret_cast<double*>(op); op += (size_t)m * 8;
    double* d_vals = reinterpret_cast<double*>(op); op += (size_t)m * 8;
    double* d_out = reinterpret_cast<double*>(op); op += (size_t)(m + 1) * 8;
    double* d_wsum = reinterpret_cast<double*>(op); op += (size_t)m * 8;
    int* d_tab = reinterpret_cast<int*>(op); op += tsize * 4;
    int* d_first = reinterpret_cast<int*>(op);
    if (!chk(cudaMemcpyAsync(d_ox, obs_x, (size_t)m * W * 8, cudaMemcpyHostToDevice, st)) ||
        !chk(cudaMemcpyAsync(d_oz, obs_z, (size_t)m * W * 8, cudaMemcpyHostToDevice, st)) ||
        !chk(cudaMemcpyAsync(d_w, seed, (size_t)m * 8, cudaMemcpyHostToDevice, st)))
        return ITPP_ERR_CUDA;
    if (!chk((itpp_detail_touch(h), launch_materialize(s, st))) ||
        !chk(launch_expect(s, d_ox, d_oz, d_w, m, (int)tsize, d_tab, d_first, d_vals, d_out, st)))
        return ITPP_ERR_CUDA;
    k_adj_wsum<<<1, 32, 0, st>>>(d_first, d_w, m, d_wsum);
    double fval = 0;
    if (!chk(cudaMemcpyAsync(&fval, d_out + m, 8, cudaMemcpyDeviceToHost, st)) ||
        !chk(cudaStreamSynchronize(st)))
        return ITPP_ERR_CUDA;

    // ---- arena for the largest segment.  Per step r >= 1: the step's output
    // before the term bound ("pre", at most 2 * inputs), its kept terms
    // ("comp", the next step's input), the three output-position maps of the
    // inputs and the compaction map of the pre terms; region 0 holds the
    // snapshot.
    auto round256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t arena_max = 0, reg_max = 1;
    for (int j = 0; j < n_seg; ++j) {
        const long long s0 = (long long)j * K * G;
        const long long s1 = ((long long)(j + 1) * K < L ? (long long)(j + 1) * K : L) * G;
        size_t bytes = 0;
        for (long long q = s0; q <= s1; ++q) {
            const size_t c = cnt_log[(size_t)q];
            bytes += round256(c * kb) + round256(c * 8);
            if (q > s0) {
                const size_t ci = cnt_log[(size_t)(q - 1)];
                bytes += round256(2 * ci * kb) + round256(2 * ci * 8) + round256(ci * 12) +
                         round256(2 * ci * 4);
                reg_max = 2 * ci > reg_max ? 2 * ci : reg_max;
            }
            reg_max = c > reg_max ? c : reg_max;
        }
        arena_max = bytes > arena_max ? bytes : arena_max;
    }
    const int steps_max = K * G;
    DevBuf arena, mu0, mu1, musave, ctl2, arrs, part, gst, grad;
    if (!arena.alloc(arena_max) || !mu0.alloc(reg_max * 8) || !mu1.alloc(reg_max * 8) ||
        !musave.alloc(reg_max * 8) || !ctl2.alloc(sizeof(DevCtl)) ||
        !arrs.alloc((size_t)(steps_max + 1) * 8 * 4) || !part.alloc((size_t)kRGrid * 8 + 64) ||
        !gst.alloc((size_t)S * 8) || !grad.alloc((size_t)G * 8))
        return ITPP_ERR_ALLOC;
    unsigned long long* a_cnt = arrs.as<unsigned long long>();
    double* a_rn = reinterpret_cast<double*>(a_cnt + steps_max + 1);
    unsigned long long* a_id = reinterpret_cast<unsigned long long*>(a_rn + steps_max + 1);
    unsigned long long* a_idpre = a_id + steps_max + 1;   // identity position before the bound
    double* nu_i = part.as<double>() + kRGrid;
    DevCtl* c2 = ctl2.as<DevCtl>();
    if (!chk(cudaMemsetAsync(c2, 0, sizeof(DevCtl), st))) return ITPP_ERR_CUDA;
    k_adj_gen_copy<<<1, 32, 0, st>>>(c2, s.ctl);
    double* mu_cur = mu0.as<double>();
    double* mu_prev = mu1.as<double>();

    // frozen evaluation: the state carried across segment boundaries (on
    // the next snapshot's order) and the identity's value of a step
    DevBuf u_snap, d_tr;
    if (ev && (!u_snap.alloc(reg_max * 8) || !d_tr.alloc(64))) return ITPP_ERR_ALLOC;
    if (ev) {
        const double one = 1.0;   // segment 0 starts from the identity alone
        if (!chk(cudaMemcpyAsync(u_snap.p, &one, 8, cudaMemcpyHostToDevice, st)))
            return ITPP_ERR_CUDA;
    }
    for (int jj = 0; jj < n_seg; ++jj) {
        const int j = ev ? jj : n_seg - 1 - jj;
        const long long s0 = (long long)j * K * G;
        const long long s1 = ((long long)(j + 1) * K < L ? (long long)(j + 1) * K : L) * G;
        const int R = (int)(s1 - s0);
        // region layout
        std::vector<PKey<W>*> rk((size_t)R + 1), pk((size_t)R + 1, nullptr);
        std::vector<double*> rc((size_t)R + 1), pc((size_t)R + 1, nullptr);
        std::vector<int*> rmap((size_t)R + 1, nullptr), cmap((size_t)R + 1, nullptr);
        char* ap = arena.as<char>();
        for (int r = 0; r <= R; ++r) {
            const size_t c = cnt_log[(size_t)(s0 + r)];
            rk[(size_t)r] = reinterpret_cast<PKey<W>*>(ap);
            ap += round256(c * kb);
            rc[(size_t)r] = reinterpret_cast<double*>(ap);
            ap += round256(c * 8);
            if (r > 0) {
                const size_t ci = cnt_log[(size_t)(s0 + r - 1)];
                pk[(size_t)r] = reinterpret_cast<PKey<W>*>(ap);
                ap += round256(2 * ci * kb);
                pc[(size_t)r] = reinterpret_cast<double*>(ap);
                ap += round256(2 * ci * 8);
                rmap[(size_t)r] = reinterpret_cast<int*>(ap);
                ap += round256(ci * 12);
                cmap[(size_t)r] = reinterpret_cast<int*>(ap);
                ap += round256(2 * ci * 4);
            }
        }
        // restore the snapshot into region 0 (normalised values, rn = 1)
        const uint64_t c0 = snap_n[(size_t)j];
        const PKey<W>* sk = snap[(size_t)j].as<PKey<W>>();
        const double* sc = reinterpret_cast<const double*>(sk + c0);
        const unsigned long long c0u = c0;
        const double one = 1.0;
        if (!chk(cudaMemcpyAsync(rk[0], sk, c0 * kb, cudaMemcpyDeviceToDevice, st)) ||
            !chk(cudaMemcpyAsync(rc[0], sc, c0 * 8, cudaMemcpyDeviceToDevice, st)) ||
            !chk(cudaMemcpyAsync(a_cnt, &c0u, 8, cudaMemcpyHostToDevice, st)) ||
            !chk(cudaMemcpyAsync(a_rn, &one, 8, cudaMemcpyHostToDevice, st)))
            return ITPP_ERR_CUDA;
        // recompute the segment, recording output positions
        for (int r = 1; r <= R; ++r) {
            const HostGate& hg = h->gates[(size_t)((s0 + r - 1) % G)];
            const GateArg<W> g = gate_arg_of<W>(hg);
            const size_t ci = cnt_log[(size_t)(s0 + r - 1)];
            StepMaps maps{rmap[(size_t)r], rmap[(size_t)r] + ci, rmap[(size_t)r] + 2 * ci,
                          a_idpre + r};
            k_adj_prep<<<1, 32, 0, st>>>(c2, a_cnt, a_rn, r, reg_max);
            k_adj_insert<W><<<grid, 256, 0, st>>>(rk[(size_t)r - 1], rc[(size_t)r - 1], c2,
                                                  static_cast<Slot<W>*>(s.table), s.table_slots,
                                                  g, s.probe_limit);
            k_adj_main<W><<<s.num_sms * 4, 256, 0, st>>>(
                rk[(size_t)r - 1], rc[(size_t)r - 1], pk[(size_t)r], pc[(size_t)r], c2,
                static_cast<const Slot<W>*>(s.table), s.table_slots, g, s.delta, 2 * ci,
                s.probe_limit, maps);
            k_adj_post<<<1, 32, 0, st>>>(c2, s.cap_M, s.cap_policy);
            if (s.cap_policy == 1) {
                DeviceState v = s;
                v.keys[0] = rk[(size_t)r];
                v.coef[0] = rc[(size_t)r];
                v.keys[1] = pk[(size_t)r];
                v.coef[1] = pc[(size_t)r];
                v.ctl = c2;
                v.buf_cap = reg_max;
                if (!chk(launch_cap_select(v, st))) return ITPP_ERR_CUDA;
            }
            k_adj_compact<W, 256><<<grid, 256, 0, st>>>(pk[(size_t)r], pc[(size_t)r],
                                                        rk[(size_t)r], rc[(size_t)r], c2,
                                                        cmap[(size_t)r], a_id + r);
            k_adj_after<<<1, 32, 0, st>>>(c2, a_cnt, a_rn, r);
        }
        const size_t cR = cnt_log[(size_t)s1];
        if (ev) {
            // the recorded maps with the evaluation's weights, from the state
            // carried into this segment (on the snapshot's order)
            if (!chk(cudaMemcpyAsync(mu_prev, u_snap.p, c0 * 8, cudaMemcpyDeviceToDevice, st)))
                return ITPP_ERR_CUDA;
            for (int r = 1; r <= R; ++r) {
                const size_t gi = (size_t)((s0 + r - 1) % G);
                GateArg<W> g = gate_arg_of<W>(h->gates[gi]);
                g.ch = ev->ch[gi];
                g.msh = ev->msh[gi];
                const size_t ci = cnt_log[(size_t)(s0 + r - 1)];
                const size_t co = cnt_log[(size_t)(s0 + r)];
                k_frz_step<W><<<grid, 256, 0, st>>>(rk[(size_t)r - 1], mu_prev, ci,
                                                    rmap[(size_t)r], rmap[(size_t)r] + ci,
                                                    rmap[(size_t)r] + 2 * ci, cmap[(size_t)r], g,
                                                    mu_cur);
                k_frz_trace<<<1, 32, 0, st>>>(mu_cur, a_id + r, d_tr.as<double>());
                k_frz_scale<<<grid, 256, 0, st>>>(mu_cur, co, a_id + r, d_tr.as<double>());
                double* t = mu_cur; mu_cur = mu_prev; mu_prev = t;
            }
            // mu_prev: the evaluated state on this segment's last order
            if (j < n_seg - 1) {
                const uint64_t cn = snap_n[(size_t)j + 1];
                const PKey<W>* nk = snap[(size_t)j + 1].as<PKey<W>>();
                k_adj_remap_insert<W><<<grid, 256, 0, st>>>(rk[(size_t)R], mu_prev, cR,
                                                            static_cast<Slot<W>*>(s.table),
                                                            s.table_slots, c2, s.probe_limit);
                k_adj_remap_lookup<W><<<grid, 256, 0, st>>>(nk, cn, cR, u_snap.as<double>(),
                                                            static_cast<const Slot<W>*>(s.table),
                                                            s.table_slots, c2, s.probe_limit);
                k_adj_bump_gen<<<1, 32, 0, st>>>(c2);
            } else {
                k_adj_seed<W><<<grid, 256, 0, st>>>(rk[(size_t)R], cR, d_ox, d_oz, d_wsum, d_tab,
                                                    (int)tsize, mu_cur);
                k_frz_dot<<<kRGrid, kRB, 0, st>>>(mu_cur, mu_prev, cR, part.as<double>());
                k_adj_gsum<<<1, kRB, 0, st>>>(part.as<double>(), kRGrid, d_tr.as<double>(), 1);
            }
            if (!chk(cudaGetLastError())) return ITPP_ERR_CUDA;
            continue;
        }
        // seed of this segment's last state
        if (j == n_seg - 1) {
            k_adj_seed<W><<<grid, 256, 0, st>>>(rk[(size_t)R], cR, d_ox, d_oz, d_wsum, d_tab,
                                                (int)tsize, mu_cur);
        } else {
            // carry mu across the boundary by key: the next segment's snapshot
            const uint64_t cn = snap_n[(size_t)j + 1];
            const PKey<W>* nk = snap[(size_t)j + 1].as<PKey<W>>();
            k_adj_remap_insert<W><<<grid, 256, 0, st>>>(nk, musave.as<double>(), cn,
                                                        static_cast<Slot<W>*>(s.table),
                                                        s.table_slots, c2, s.probe_limit);
            k_adj_remap_lookup<W><<<grid, 256, 0, st>>>(rk[(size_t)R], cR, cn, mu_cur,
                                                        static_cast<const Slot<W>*>(s.table),
                                                        s.table_slots, c2, s.probe_limit);
            k_adj_bump_gen<<<1, 32, 0, st>>>(c2);
        }
        // reverse sweep over the segment
        for (int r = R; r >= 1; --r) {
            const HostGate& hg = h->gates[(size_t)((s0 + r - 1) % G)];
            const size_t ci = cnt_log[(size_t)(s0 + r - 1)];
            const size_t co = cnt_log[(size_t)(s0 + r)];
            k_adj_dot<<<kRGrid, kRB, 0, st>>>(rc[(size_t)r], mu_cur, co, a_id + r, a_rn + r,
                                              part.as<double>());
            k_adj_dot_final<<<1, kRB, 0, st>>>(part.as<double>(), kRGrid, a_rn + r, nu_i);
            k_adj_back<W><<<kRGrid, kRB, 0, st>>>(
                rk[(size_t)r - 1], rc[(size_t)r - 1], ci, a_rn + r - 1, rmap[(size_t)r],
                rmap[(size_t)r] + ci, rmap[(size_t)r] + 2 * ci, cmap[(size_t)r], mu_cur,
                a_id + r, a_rn + r, nu_i, gate_arg_of<W>(hg), hg.sh, hg.chd, mu_prev,
                part.as<double>());
            k_adj_gsum<<<1, kRB, 0, st>>>(part.as<double>(), kRGrid, gst.as<double>(),
                                          s0 + r - 1);
            double* t = mu_cur; mu_cur = mu_prev; mu_prev = t;
        }
        // mu on the snapshot order, for the previous segment
        if (!chk(cudaMemcpyAsync(musave.p, mu_cur, c0 * 8, cudaMemcpyDeviceToDevice, st)))
            return ITPP_ERR_CUDA;
        if (!chk(cudaGetLastError())) return ITPP_ERR_CUDA;
    }
    if (ev) {
        k_adj_gen_copy<<<1, 32, 0, st>>>(s.ctl, c2);
        double fe = 0.0;
        int c2_status = 0;
        if (!chk(cudaMemcpyAsync(&fe, d_tr.as<double>() + 1, 8, cudaMemcpyDeviceToHost, st)) ||
            !chk(cudaMemcpyAsync(&c2_status, &c2->status, sizeof(int), cudaMemcpyDeviceToHost,
                                 st)) ||
            !chk(cudaStreamSynchronize(st)))
            return ITPP_ERR_CUDA;
        if (c2_status) return (itpp_status)c2_status;
        *value = fe;
        return ITPP_OK;
    }
    k_adj_params<<<1, 256, 0, st>>>(gst.as<double>(), L, G, h->dtau, grad.as<double>());
    k_adj_gen_copy<<<1, 32, 0, st>>>(s.ctl, c2);
    int c2_status = 0;
    if (!chk(cudaMemcpyAsync(grad_alpha, grad.p, (size_t)G * 8, cudaMemcpyDeviceToHost, st)) ||
        !chk(cudaMemcpyAsync(&c2_status, &c2->status, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        !chk(cudaStreamSynchronize(st)))
        return ITPP_ERR_CUDA;
    if (c2_status) return (itpp_status)c2_status;
    if (value) *value = fval;
    return ITPP_OK;
}

}  // namespace

extern "C" itpp_status itpp_adjoint(itpp_handle h, int n_layers, int ckpt_every,
                                    const uint64_t* obs_x, const uint64_t* obs_z,
                                    const double* seed, int m, double* grad_alpha,
                                    double* value) {
    if (!h || n_layers < 1 || ckpt_every < 1 || !obs_x || !obs_z || !seed || !grad_alpha ||
        m < 1 || m > 65536)
        return ITPP_ERR_ARG;
    if (h->gates.empty()) return ITPP_ERR_ARG;
    if (h->sticky) return h->sticky;
    // gradients per elementary gate of the schedule, then folded onto the
    // Hamiltonian's coefficients (d alpha_gate / d alpha = src_scale)
    std::vector<double> g_sched(h->gates.size(), 0.0);
    itpp_status st = h->s.W == 1
        ? adjoint_w<1>(h, n_layers, ckpt_every, obs_x, obs_z, seed, m, g_sched.data(), value)
        : adjoint_w<2>(h, n_layers, ckpt_every, obs_x, obs_z, seed, m, g_sched.data(), value);
    if (st == ITPP_ERR_CUDA) h->sticky = st;
    if (st == ITPP_OK) {
        for (int k = 0; k < h->user_gates; ++k) grad_alpha[k] = 0.0;
        for (size_t j = 0; j < g_sched.size(); ++j)
            grad_alpha[h->src_gate[j]] += g_sched[j] * h->src_scale[j];
    }
    return st;
}

extern "C" itpp_status itpp_frozen_value(itpp_handle h, int n_layers, int ckpt_every,
                                         const double* alpha_eval, const uint64_t* obs_x,
                                         const uint64_t* obs_z, const double* w, int m,
                                         double* value) {
    if (!h || n_layers < 1 || ckpt_every < 1 || !alpha_eval || !obs_x || !obs_z || !w ||
        !value || m < 1 || m > 65536)
        return ITPP_ERR_ARG;
    if (h->gates.empty()) return ITPP_ERR_ARG;
    if (h->sticky) return h->sticky;
    FrozenEval ev;
    ev.ch.resize(h->gates.size());
    ev.msh.resize(h->gates.size());
    for (size_t j = 0; j < h->gates.size(); ++j) {
        const double a = alpha_eval[h->src_gate[j]];
        if (!std::isfinite(a)) return ITPP_ERR_ARG;
        const double theta = (a * h->src_scale[j]) * h->dtau;
        ev.ch[j] = std::cosh(theta);
        ev.msh[j] = -std::sinh(theta);
        if (!std::isfinite(ev.ch[j]) || !std::isfinite(ev.msh[j])) return ITPP_ERR_ARG;
    }
    itpp_status st = h->s.W == 1
        ? adjoint_w<1>(h, n_layers, ckpt_every, obs_x, obs_z, w, m, nullptr, value, &ev)
        : adjoint_w<2>(h, n_layers, ckpt_every, obs_x, obs_z, w, m, nullptr, value, &ev);
    if (st == ITPP_ERR_CUDA) h->sticky = st;
    return st;
}

extern "C" itpp_status itpp_set_alpha(itpp_handle h, const double* alpha) {
    if (!h || !alpha) return ITPP_ERR_ARG;
    for (int k = 0; k < h->user_gates; ++k)
        if (!std::isfinite(alpha[k])) return ITPP_ERR_ARG;
    for (size_t k = 0; k < h->gates.size(); ++k) {   // cosh / sinh overflow
        const double theta = (alpha[h->src_gate[k]] * h->src_scale[k]) * h->dtau;
        if (!std::isfinite(std::cosh(theta)) || !std::isfinite(std::sinh(theta))) return ITPP_ERR_ARG;
    }
    cudaStreamSynchronize(h->stream);
    for (size_t k = 0; k < h->gates.size(); ++k) {
        HostGate& g = h->gates[k];
        const double theta = (alpha[h->src_gate[k]] * h->src_scale[k]) * h->dtau;
        g.ch = std::cosh(theta);
        g.msh = -std::sinh(theta);
        g.sh = std::sinh(theta);
        g.chd = std::cosh(theta);
    }
    return ITPP_OK;
}
