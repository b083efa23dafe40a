// itpp_psd.cu -- the positive-semidefinite-restored observable (Sec. II.C):
//
//   <O>_{2 tau} ~= Tr[(O rho) rho] / Tr[rho^2],   rho = sum_P c_P P, c_I = 1,
//
// for O = sum_j w_j O_j.  With Tr(P_a P_b) = 2^n delta_ab the purity is
// Tr[rho^2] / 2^n = sum_P c_P^2 (the squared l2 norm of the coefficients),
// and Tr[(O_j P) R] is nonzero only for R = O_j.P.  When O_j and P
// anticommute the product carries a factor +-i and the pair (P, O_j.P) is
// met again as (O_j.P, P) with the opposite factor, so those terms cancel;
// when they commute O_j P = s O_j.P with s = +-1 (the sign of the
// propagation rule), so
//
//   Tr[(O rho) rho] / 2^n = sum_j w_j sum_{P : [P, O_j] = 0} s(O_j, P) c_P c_{O_j.P}.
//
// That is a partner lookup: every term of the state goes into the merge
// table (under a generation of its own), then one pass over the state
// looks up O_j.P for every commuting observable string.  Sums are
// compensated per thread, then reduced in a fixed order, so the result does
// not depend on scheduling.
#include "itpp_common.cuh"
#include "itpp_gate_body.cuh"
#include "itpp_launch.h"

namespace itpp {

namespace {

constexpr int kPB = 256;

template <int W>
static Bufs<W> psd_bufs(const DeviceState& s) {
    Bufs<W> b;
    for (int i = 0; i < 2; ++i) {
        b.k[i] = reinterpret_cast<PKey<W>*>(s.keys[i]);
        b.c[i] = s.coef[i];
    }
    return b;
}

// A fresh table generation for the state's terms (never equal to a gate's).
__global__ void k_psd_begin(DevCtl* ctl) {
    if (threadIdx.x != 0 || ctl->status) return;
    ctl->gen = ctl->gen + 1u;
    if (ctl->gen == 0u) set_status(ctl, ST_STATE, 60);
}

// Every term of the state, normalised, into the table.
template <int W>
__global__ void __launch_bounds__(kPB)
k_psd_build(Bufs<W> B, DevCtl* ctl, Slot<W>* table, uint64_t slots, int load_pct,
            int probe_limit) {
    if (ctl->status) return;
    const int cur = ctl->cur;
    const uint64_t n = live_count(ctl, cur);
    const double rnorm = ctl->rnorm[cur];
    const unsigned gen = ctl->gen;
    const uint64_t mask = table_mask(n, slots, load_pct);
    int probes = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const PKey<W> K = load_key(B.key(cur) + i);
        const double c = normalised(B.coef(cur)[i], rnorm, key_is_zero(K));
        if (!table_insert(table, mask, gen, K, c, (uint32_t)i, probe_limit, &probes))
            set_status(ctl, ST_HASH_PROBE, 61);
    }
}

__device__ __forceinline__ void kahan_add(double& s, double& comp, double v) {
    const double y = __dsub_rn(v, comp);
    const double t = __dadd_rn(s, y);
    comp = __dsub_rn(__dsub_rn(t, s), y);
    s = t;
}

// One pass over the state: purity and the commuting-pair overlap; per-block
// partials (numerator, purity) in a fixed-order tree.
template <int W>
__global__ void __launch_bounds__(kPB)
k_psd_pairs(Bufs<W> B, DevCtl* ctl, const Slot<W>* table, uint64_t slots, int load_pct,
            int probe_limit, const uint64_t* __restrict__ ox, const uint64_t* __restrict__ oz,
            const double* __restrict__ ow, int m, double* partials) {
    __shared__ double s_num[kPB], s_den[kPB];
    double num = 0.0, cn = 0.0, den = 0.0, cd = 0.0;
    if (!ctl->status) {
        const int cur = ctl->cur;
        const uint64_t n = live_count(ctl, cur);
        const double rnorm = ctl->rnorm[cur];
        const unsigned gen = ctl->gen;
        const uint64_t mask = table_mask(n, slots, load_pct);
        int probes = 0;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (uint64_t)gridDim.x * blockDim.x) {
            const PKey<W> P = load_key(B.key(cur) + i);
            const double cp = normalised(B.coef(cur)[i], rnorm, key_is_zero(P));
            kahan_add(den, cd, __dmul_rn(cp, cp));
            for (int j = 0; j < m; ++j) {
                GateArg<W> o;
                int yy = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    o.qx[w] = __ldg(ox + (size_t)j * W + w);
                    o.qz[w] = __ldg(oz + (size_t)j * W + w);
                    yy += __popcll(o.qx[w] & o.qz[w]);
                }
                o.qyy = yy & 3;
                if (!commutes(P, o)) continue;
                double cr;
                if (!table_find(table, mask, gen, key_xor(P, o), &cr, probe_limit, ctl, &probes))
                    continue;
                const double pair = __dmul_rn(cp, cr);
                const double v = __dmul_rn(__ldg(ow + j), pair);
                kahan_add(num, cn, product_negative(P, o) ? -v : v);
            }
        }
    }
    s_num[threadIdx.x] = num;
    s_den[threadIdx.x] = den;
    __syncthreads();
    for (int o = kPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_num[threadIdx.x] = __dadd_rn(s_num[threadIdx.x], s_num[threadIdx.x + o]);
            s_den[threadIdx.x] = __dadd_rn(s_den[threadIdx.x], s_den[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s_num[0];
        partials[2 * blockIdx.x + 1] = s_den[0];
    }
}

// The blocks' partials in block order (compensated); the ratio; the next
// gate gets a fresh table generation.
__global__ void k_psd_final(DevCtl* ctl, const double* partials, int n_part, double* out) {
    if (threadIdx.x != 0) return;
    double num = 0.0, cn = 0.0, den = 0.0, cd = 0.0;
    for (int b = 0; b < n_part; ++b) {
        kahan_add(num, cn, partials[2 * b]);
        kahan_add(den, cd, partials[2 * b + 1]);
    }
    out[0] = __ddiv_rn(num, den);
    out[1] = num;
    out[2] = den;
    if (!ctl->status) {
        ctl->gen = ctl->gen + 1u;
        if (ctl->gen == 0u) set_status(ctl, ST_STATE, 62);
    }
}

template <int W>
static cudaError_t psd_w(const DeviceState& s, const uint64_t* d_ox, const uint64_t* d_oz,
                         const double* d_ow, int m, double* d_partials, int n_part,
                         double* d_out, cudaStream_t st) {
    // stale contents (the top-M select borrows this memory) must not read as
    // tags: clear the table first
    const size_t slot = W == 1 ? 32 : 64;
    cudaError_t e = cudaMemsetAsync(s.table, 0, (size_t)s.table_slots * slot, st);
    if (e != cudaSuccess) return e;
    k_psd_begin<<<1, 32, 0, st>>>(s.ctl);
    Slot<W>* table = static_cast<Slot<W>*>(s.table);
    k_psd_build<W><<<s.num_sms * 8, kPB, 0, st>>>(psd_bufs<W>(s), s.ctl, table, s.table_slots,
                                                 s.load_pct, s.probe_limit);
    k_psd_pairs<W><<<n_part, kPB, 0, st>>>(psd_bufs<W>(s), s.ctl, table, s.table_slots,
                                          s.load_pct, s.probe_limit, d_ox, d_oz, d_ow, m,
                                          d_partials);
    k_psd_final<<<1, 32, 0, st>>>(s.ctl, d_partials, n_part, d_out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_expect_psd(const DeviceState& s, const uint64_t* d_ox, const uint64_t* d_oz,
                              const double* d_ow, int m, double* d_partials, int n_part,
                              double* d_out, cudaStream_t st) {
    return s.W == 1 ? psd_w<1>(s, d_ox, d_oz, d_ow, m, d_partials, n_part, d_out, st)
                    : psd_w<2>(s, d_ox, d_oz, d_ow, m, d_partials, n_part, d_out, st);
}

}  // namespace itpp
