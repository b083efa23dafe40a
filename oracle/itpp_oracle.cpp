// ITPP oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously correct CPU restatement of imaginary-time Pauli
// propagation (Algorithm 1 of "Pauli Propagation for Imaginary-Time
// Evolution").  Only the tests, the smoke check and the bench's CPU-baseline
// leg may load this file's library; the product (the CUDA library) never
// does, and this file shares no code with it.
//
// Build: g++ -O2 -ffp-contract=off -shared -fPIC (no FMA contraction, so every
// product and sum below is rounded once, in the order written).
//
// Representation (Eq. (Observable_Pauli)): a Pauli string is a pair of bit
// masks x, z of W words (site i = bit i%64 of word i/64); (x_i, z_i) = (0,0)
// I, (1,0) X, (0,1) Z, (1,1) Y.  An operator is a std::map from string to
// real coefficient; the identity is the all-zero string.
//
// Functions and the passages they follow:
//   commutes / pauli_product ... Sec. II.C (commute vs anticommute cases) and
//                                App. A (Eq. (ITE_Pauli_rules)); phase from
//                                sigma(x,z) = i^{x z} X^x Z^z.
//   apply_gate .................. Algorithm 1 inner loop: propagate every term
//                                with Eq. (ITPP_PropRules), accumulate,
//                                truncate |c| > delta and, when set, the
//                                Pauli weight cutoff (Sec. II.B), cap (the
//                                term bound of the "Practical considerations"
//                                paragraph, Sec. II.C), normalise by the
//                                identity coefficient: identify it and
//                                rescale every coefficient by its reciprocal
//                                (Sec. II.C).
//   expect ...................... <O> = Tr[O rho] with the identity
//                                coefficient equal to one (Sec. II.C, the
//                                expectation from the propagated operator).
//   expect_psd .................. <O>_{2 tau} of the squared (positive
//                                semidefinite) state, Sec. II.C: the Pauli
//                                expansion of O rho first, then its overlap
//                                with rho, over the purity (l2 norm).
//   frozen forward / adjoint .... gradients of the propagated expectation with
//                                the support of every gate held fixed; the
//                                paper has no such step, it is the linear
//                                algebra of Eq. (ITPP_PropRules) and the
//                                per-gate normalisation.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <complex>
#include <map>
#include <vector>

namespace {

constexpr int MAXW = 4;  // up to 256 sites

struct Key {
    // words 0..W-1 hold x, words MAXW..MAXW+W-1 hold z; unused words are 0.
    std::array<uint64_t, 2 * MAXW> w{};
    bool operator<(const Key& o) const { return w < o.w; }
    bool operator==(const Key& o) const { return w == o.w; }
    bool is_identity() const {
        for (uint64_t v : w) if (v) return false;
        return true;
    }
};

int popcount64(uint64_t v) {
    int c = 0;
    while (v) { v &= v - 1; ++c; }
    return c;
}

// Pauli weight: the number of non-identity letters, popc(x | z).
int weight(int W, const Key& k) {
    int w = 0;
    for (int i = 0; i < W; ++i) w += popcount64(k.w[i] | k.w[MAXW + i]);
    return w;
}

Key make_key(int W, const uint64_t* x, const uint64_t* z) {
    Key k;
    for (int i = 0; i < W; ++i) { k.w[i] = x[i]; k.w[MAXW + i] = z[i]; }
    return k;
}

// P and Q anticommute iff the symplectic form sum_i (xP_i zQ_i + zP_i xQ_i)
// is odd (each site where the letters differ and neither is I contributes one
// sign flip).
bool commutes(int W, const Key& P, const Key& Q) {
    int s = 0;
    for (int i = 0; i < W; ++i)
        s += popcount64(P.w[i] & Q.w[MAXW + i]) + popcount64(P.w[MAXW + i] & Q.w[i]);
    return (s & 1) == 0;
}

// Q*P = i^e R with R = (xQ^xP, zQ^zP).  Site by site,
// sigma(a,b) = i^{ab} X^a Z^b and Z^b X^c = (-1)^{bc} X^c Z^b give
// e = ab(Q) + ab(P) - ab(R) + 2 b(Q) c(P)  (mod 4).
int pauli_product(int W, const Key& Q, const Key& P, Key* R) {
    int e = 0;
    for (int i = 0; i < W; ++i) {
        uint64_t xq = Q.w[i], zq = Q.w[MAXW + i], xp = P.w[i], zp = P.w[MAXW + i];
        uint64_t xr = xq ^ xp, zr = zq ^ zp;
        R->w[i] = xr;
        R->w[MAXW + i] = zr;
        e += popcount64(xq & zq) + popcount64(xp & zp) - popcount64(xr & zr)
             + 2 * popcount64(zq & xp);
    }
    return ((e % 4) + 4) % 4;
}

enum Status { OK = 0, ERR_ARG = 1, ERR_CAPACITY = 3, ERR_TRACE_ZERO = 6, ERR_STATE = 8 };

struct Frozen;

struct Oracle {
    int n = 0, W = 0;
    std::vector<Key> Q;        // gates in Trotter order
    std::vector<double> alpha; // their coefficients
    double dtau = 0, delta = 0;
    uint64_t cap_M = 0;
    int cap_policy = 0;
    int max_weight = 0;        // Pauli weight cutoff (Sec. II.B); 0: none
    std::map<Key, double> rho;
    // per applied gate: the support kept and the normaliser (for the frozen
    // forward used by the adjoint check)
    bool record = false;
    std::vector<std::vector<Key>> support;
    std::vector<int> gate_of_step;
};

// One elementary step of Algorithm 1 (the body of the loop over Hamiltonian
// terms): rho' <- sum over terms of V^dagger P V, then rho <- T(rho')/Tr T(rho').
int apply_gate(Oracle& o, int k) {
    const Key& Q = o.Q[k];
    const double theta = o.alpha[k] * o.dtau;       // V = exp(-(theta/2) Q)
    const double ch = std::cosh(theta);
    const double msh = -std::sinh(theta);
    std::map<Key, double> next;                      // rho' <- 0
    for (const auto& [P, c] : o.rho) {
        if (!commutes(o.W, P, Q)) {
            next[P] += c;                            // {P,Q} = 0: P unchanged
        } else {                                     // [P,Q] = 0
            next[P] += c * ch;                       //   cosh(theta) P
            Key R;
            int e = pauli_product(o.W, Q, P, &R);    //   Q P = i^e R, e in {0,2}
            double s = (e == 0) ? 1.0 : -1.0;
            next[R] += (c * msh) * s;                //   - sinh(theta) Q P
        }
    }
    // threshold truncation: keep |c| > delta, on the accumulated coefficients;
    // with a weight cutoff k, also drop strings with more than k non-identity
    // letters (Sec. II.B "Pauli weight cutoff"; the identity has weight 0)
    for (auto it = next.begin(); it != next.end();) {
        const bool heavy = o.max_weight > 0 && weight(o.W, it->first) > o.max_weight;
        if (std::fabs(it->second) > o.delta && !heavy) ++it;
        else {
            if (it->first.is_identity()) return ERR_TRACE_ZERO;
            it = next.erase(it);
        }
    }
    Key I;
    if (next.find(I) == next.end()) return ERR_TRACE_ZERO;
    // term bound: keep the cap_M largest |c| (ties: smaller key first)
    if (o.cap_M && next.size() > o.cap_M) {
        if (o.cap_policy == 0) return ERR_CAPACITY;
        std::vector<std::pair<Key, double>> v(next.begin(), next.end());
        std::sort(v.begin(), v.end(), [](const auto& a, const auto& b) {
            double fa = std::fabs(a.second), fb = std::fabs(b.second);
            if (fa != fb) return fa > fb;
            return a.first < b.first;
        });
        v.resize(o.cap_M);
        next.clear();
        for (auto& kv : v) next.insert(kv);
        if (next.find(I) == next.end()) return ERR_TRACE_ZERO;
    }
    // normalise by the trace: rescale every coefficient by the reciprocal of
    // the identity coefficient (one division per step), the identity itself
    // becoming exactly one
    const double cI = next[I];
    const double inv = 1.0 / cI;
    for (auto& kv : next) kv.second = kv.first.is_identity() ? 1.0 : kv.second * inv;
    o.rho.swap(next);
    if (o.record) {
        std::vector<Key> s;
        s.reserve(o.rho.size());
        for (auto& kv : o.rho) s.push_back(kv.first);
        o.support.push_back(std::move(s));
        o.gate_of_step.push_back(k);
    }
    return OK;
}


// ---------------------------------------------------------------------------
// Frozen-support forward and its adjoint (gradients with respect to the gate
// coefficients).  The paper has no such step; this is the linear algebra of
// Eq. (ITPP_PropRules) and the per-step normalisation with the kept support
// of every step held fixed:
//   raw_s[K] = a_K u_{s-1}[K] + [K commutes] s(Q,K) (-sinh) u_{s-1}[Q K],
//              a_K = cosh(theta) if [K,Q] = 0 else 1, for K in S_s,
//   u_s = raw_s / raw_s[I],   f = sum_j w_j u_L[P_j].
// ---------------------------------------------------------------------------
struct Frozen {
    std::vector<int> gate;                          // gate index of step s (1-based steps)
    std::vector<std::vector<Key>> support;          // S_s, s = 1..L
};

// One frozen step: u_prev on S_{s-1} -> raw on S_s.
std::map<Key, double> frozen_step(int W, const std::map<Key, double>& u_prev, const Key& Q,
                                  double ch, double msh, const std::vector<Key>& S) {
    std::map<Key, double> raw;
    for (const Key& K : S) raw[K] = 0.0;
    for (const auto& [P, c] : u_prev) {
        if (!commutes(W, P, Q)) {
            auto it = raw.find(P);
            if (it != raw.end()) it->second += c;
        } else {
            auto it = raw.find(P);
            if (it != raw.end()) it->second += c * ch;
            Key R;
            int e = pauli_product(W, Q, P, &R);
            auto jt = raw.find(R);
            if (jt != raw.end()) jt->second += (c * msh) * (e == 0 ? 1.0 : -1.0);
        }
    }
    return raw;
}

std::map<Key, double> normalise(const std::map<Key, double>& raw, double* D) {
    Key I;
    *D = raw.at(I);
    const double inv = 1.0 / *D;
    std::map<Key, double> u;
    for (const auto& [K, v] : raw) u[K] = K.is_identity() ? 1.0 : v * inv;
    return u;
}

double observe(const Oracle& o, const std::map<Key, double>& u, const uint64_t* ox,
               const uint64_t* oz, const double* w, int m) {
    double f = 0.0;
    for (int j = 0; j < m; ++j) {
        auto it = u.find(make_key(o.W, ox + (size_t)j * o.W, oz + (size_t)j * o.W));
        if (it != u.end()) f += w[j] * it->second;
    }
    return f;
}

// Frozen forward over the recorded supports; keeps every state when asked.
int frozen_forward(const Oracle& o, const double* alpha, std::vector<std::map<Key, double>>* states,
                   std::vector<double>* Ds, std::map<Key, double>* last) {
    std::map<Key, double> u;
    u[Key{}] = 1.0;
    if (states) states->push_back(u);
    for (size_t s = 0; s < o.support.size(); ++s) {
        const int k = o.gate_of_step[s];
        const double theta = alpha[k] * o.dtau;
        std::map<Key, double> raw = frozen_step(o.W, u, o.Q[k], std::cosh(theta),
                                                -std::sinh(theta), o.support[s]);
        double D = 0;
        if (raw.find(Key{}) == raw.end()) return ERR_TRACE_ZERO;
        u = normalise(raw, &D);
        if (Ds) Ds->push_back(D);
        if (states) states->push_back(u);
    }
    if (last) *last = u;
    return OK;
}

}  // namespace

extern "C" {

void* oracle_create(int n, int n_gates, const uint64_t* gx, const uint64_t* gz,
                    const double* alpha, double dtau, double delta,
                    uint64_t cap_M, int cap_policy) {
    if (n < 1 || n > 64 * MAXW || n_gates < 0 || !(delta >= 0)) return nullptr;
    Oracle* o = new Oracle;
    o->n = n;
    o->W = (n + 63) / 64;
    o->dtau = dtau;
    o->delta = delta;
    o->cap_M = cap_M;
    o->cap_policy = cap_policy;
    for (int k = 0; k < n_gates; ++k) {
        o->Q.push_back(make_key(o->W, gx + (size_t)k * o->W, gz + (size_t)k * o->W));
        o->alpha.push_back(alpha[k]);
    }
    o->rho[Key{}] = 1.0;  // initialise rho = I (the 1/2^n cancels, Sec. II.C)
    return o;
}

void oracle_destroy(void* h) { delete static_cast<Oracle*>(h); }

int oracle_apply_gate(void* h, int k) {
    Oracle& o = *static_cast<Oracle*>(h);
    if (k < 0 || k >= (int)o.Q.size()) return ERR_ARG;
    return apply_gate(o, k);
}

// n_layers Trotter steps, each the gates in their stored order.
int oracle_apply_layers(void* h, int n_layers) {
    Oracle& o = *static_cast<Oracle*>(h);
    for (int l = 0; l < n_layers; ++l)
        for (int k = 0; k < (int)o.Q.size(); ++k) {
            int st = apply_gate(o, k);
            if (st) return st;
        }
    return OK;
}

uint64_t oracle_count(void* h) { return static_cast<Oracle*>(h)->rho.size(); }

// Terms in ascending key order (x words, then z words), normalised.
void oracle_get_terms(void* h, uint64_t* x, uint64_t* z, double* c) {
    Oracle& o = *static_cast<Oracle*>(h);
    size_t i = 0;
    for (const auto& [P, v] : o.rho) {
        for (int w = 0; w < o.W; ++w) {
            x[i * o.W + w] = P.w[w];
            z[i * o.W + w] = P.w[MAXW + w];
        }
        c[i] = v;
        ++i;
    }
}

// Replace the state (used for one-gate checks on synthetic states).
// Pauli weight cutoff k for every later gate (0: none).
int oracle_set_max_weight(void* h, int k) {
    if (k < 0) return ERR_ARG;
    static_cast<Oracle*>(h)->max_weight = k;
    return OK;
}

int oracle_set_terms(void* h, uint64_t count, const uint64_t* x, const uint64_t* z,
                     const double* c) {
    Oracle& o = *static_cast<Oracle*>(h);
    o.rho.clear();
    for (uint64_t i = 0; i < count; ++i) {
        Key k = make_key(o.W, x + i * o.W, z + i * o.W);
        if (o.rho.count(k)) return ERR_ARG;
        o.rho[k] = c[i];
    }
    return OK;
}

// Coefficient of each requested string (0 when absent).
void oracle_coeffs(void* h, const uint64_t* ox, const uint64_t* oz, int m, double* out) {
    Oracle& o = *static_cast<Oracle*>(h);
    for (int j = 0; j < m; ++j) {
        auto it = o.rho.find(make_key(o.W, ox + (size_t)j * o.W, oz + (size_t)j * o.W));
        out[j] = (it == o.rho.end()) ? 0.0 : it->second;
    }
}

// <O> = sum_j w_j c_{P_j}: Tr(P_a P_b) = 2^n delta_ab and the identity
// coefficient is one, so Tr[O rho]/Tr[rho] is this plain sum.
double oracle_expect(void* h, const uint64_t* ox, const uint64_t* oz, const double* ow,
                     int m) {
    Oracle& o = *static_cast<Oracle*>(h);
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
        auto it = o.rho.find(make_key(o.W, ox + (size_t)j * o.W, oz + (size_t)j * o.W));
        if (it != o.rho.end()) s += ow[j] * it->second;
    }
    return s;
}

// <O>_{2 tau} ~= Tr[(O rho) rho] / Tr[rho^2] (Sec. II.C, restoring positive
// semidefiniteness by squaring the state).  The product O rho is expanded in
// the Pauli basis (O_j P = i^e S, complex coefficients summed per string),
// then overlapped with rho: Tr[S R] = 2^n delta_SR, so Tr[(O rho) rho] / 2^n
// = sum_S [O rho]_S c_S.  The purity Tr[rho^2] / 2^n is the squared l2 norm
// of the coefficients.  out: [0] the ratio, [1] the numerator / 2^n, [2] the
// purity / 2^n, [3] the imaginary part of the numerator (zero up to
// rounding for Hermitian O and rho).
int oracle_expect_psd(void* h, const uint64_t* ox, const uint64_t* oz, const double* ow, int m,
                      double* out) {
    Oracle& o = *static_cast<Oracle*>(h);
    std::map<Key, std::complex<double>> prod;                 // O rho
    const std::complex<double> ipow[4] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    for (int j = 0; j < m; ++j) {
        const Key Oj = make_key(o.W, ox + (size_t)j * o.W, oz + (size_t)j * o.W);
        for (const auto& [P, c] : o.rho) {
            Key S;
            const int e = pauli_product(o.W, Oj, P, &S);      // O_j P = i^e S
            prod[S] += ow[j] * c * ipow[e & 3];
        }
    }
    std::complex<double> num = 0.0;
    for (const auto& [S, v] : prod) {
        auto it = o.rho.find(S);
        if (it != o.rho.end()) num += v * it->second;
    }
    double purity = 0.0;
    for (const auto& kv : o.rho) purity += kv.second * kv.second;
    out[0] = num.real() / purity;
    out[1] = num.real();
    out[2] = purity;
    out[3] = num.imag();
    return OK;
}

// Run n_layers Trotter layers from the identity, recording the kept support
// of every step (for the frozen-support forward and its adjoint).
int oracle_record(void* h, int n_layers) {
    Oracle& o = *static_cast<Oracle*>(h);
    o.rho.clear();
    o.rho[Key{}] = 1.0;
    o.record = true;
    o.support.clear();
    o.gate_of_step.clear();
    int st = oracle_apply_layers(h, n_layers);
    o.record = false;
    return st;
}

// f = sum_j w_j u_L[P_j] of the frozen forward with gate coefficients alpha
// (n_gates values; the Hamiltonian's own when alpha is NULL).
int oracle_frozen_value(void* h, const double* alpha, const uint64_t* ox, const uint64_t* oz,
                        const double* w, int m, double* f) {
    Oracle& o = *static_cast<Oracle*>(h);
    std::map<Key, double> u;
    int st = frozen_forward(o, alpha ? alpha : o.alpha.data(), nullptr, nullptr, &u);
    if (st) return st;
    *f = observe(o, u, ox, oz, w, m);
    return OK;
}

// Gradient of the frozen f with respect to every gate coefficient alpha_k
// (summed over the layers).  Reverse sweep: mu_s = df/du_s, then
//   nu_s[K] = mu_s[K] / D_s (K != I),  nu_s[I] = -sum_{K != I} mu_s[K] u_s[K] / D_s,
//   mu_{s-1}[P] = nu_s[P]                                  ({P,Q} = 0),
//               = cosh nu_s[P] + s (-sinh) nu_s[Q P]      ([P,Q] = 0),
//   df/dtheta_s = sum_{[P,Q]=0} u_{s-1}[P] (sinh nu_s[P] - s cosh nu_s[Q P]),
// with nu_s = 0 outside S_s and theta_s = alpha_k dtau.
int oracle_adjoint(void* h, const uint64_t* ox, const uint64_t* oz, const double* w, int m,
                   double* grad_alpha, double* f) {
    Oracle& o = *static_cast<Oracle*>(h);
    std::vector<std::map<Key, double>> U;
    std::vector<double> D;
    int st = frozen_forward(o, o.alpha.data(), &U, &D, nullptr);
    if (st) return st;
    const size_t L = o.support.size();
    *f = observe(o, U[L], ox, oz, w, m);
    for (size_t k = 0; k < o.Q.size(); ++k) grad_alpha[k] = 0.0;
    std::map<Key, double> mu;
    for (const auto& kv : U[L]) mu[kv.first] = 0.0;
    for (int j = 0; j < m; ++j) {
        auto it = mu.find(make_key(o.W, ox + (size_t)j * o.W, oz + (size_t)j * o.W));
        if (it != mu.end()) it->second += w[j];
    }
    for (size_t s = L; s >= 1; --s) {
        const int k = o.gate_of_step[s - 1];
        const Key& Q = o.Q[k];
        const double theta = o.alpha[k] * o.dtau;
        const double ch = std::cosh(theta), sh = std::sinh(theta), msh = -sh;
        double dot = 0.0;
        for (const auto& [K, v] : U[s])
            if (!K.is_identity()) dot += mu[K] * v;
        std::map<Key, double> nu;
        for (const auto& [K, v] : mu) nu[K] = K.is_identity() ? -dot / D[s - 1] : v / D[s - 1];
        auto nu_of = [&](const Key& K) {
            auto it = nu.find(K);
            return it == nu.end() ? 0.0 : it->second;
        };
        std::map<Key, double> mu_prev;
        double g = 0.0;
        for (const auto& [P, up] : U[s - 1]) {
            if (!commutes(o.W, P, Q)) {
                mu_prev[P] = nu_of(P);
            } else {
                Key R;
                const double sg = pauli_product(o.W, Q, P, &R) == 0 ? 1.0 : -1.0;
                mu_prev[P] = ch * nu_of(P) + sg * msh * nu_of(R);
                g += up * (sh * nu_of(P) - sg * ch * nu_of(R));
            }
        }
        grad_alpha[k] += g * o.dtau;
        mu.swap(mu_prev);
    }
    return OK;
}

// Bit algebra exposed for the pin tests.
int oracle_commutes(int W, const uint64_t* px, const uint64_t* pz, const uint64_t* qx,
                    const uint64_t* qz) {
    return commutes(W, make_key(W, px, pz), make_key(W, qx, qz)) ? 1 : 0;
}

int oracle_pauli_product(int W, const uint64_t* qx, const uint64_t* qz, const uint64_t* px,
                         const uint64_t* pz, uint64_t* rx, uint64_t* rz) {
    Key R;
    int e = pauli_product(W, make_key(W, qx, qz), make_key(W, px, pz), &R);
    for (int i = 0; i < W; ++i) { rx[i] = R.w[i]; rz[i] = R.w[MAXW + i]; }
    return e;
}

}  // extern "C"
