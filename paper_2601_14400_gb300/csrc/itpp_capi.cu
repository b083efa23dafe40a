// itpp_capi.cu -- the C ABI (include/itpp.h): argument checks, allocation,
// per-gate weights, launch ordering, synchronising reads.  No step of the
// propagation itself runs here; every one is a kernel in itpp_gate.cu /
// itpp_aux.cu.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "itpp.h"
#include "itpp_common.cuh"
#include "itpp_ctx.h"
#include "itpp_launch.h"

using namespace itpp;

namespace {

itpp_status cuda_fail(itpp_ctx* h) {
    if (h && h->sticky == ITPP_OK) h->sticky = ITPP_ERR_CUDA;
    return ITPP_ERR_CUDA;
}

bool bits_ok(int n, int W, const uint64_t* x) {
    for (int w = 0; w < W; ++w) {
        const int lo = 64 * w;
        if (n >= lo + 64) continue;
        const uint64_t top = (n <= lo) ? ~0ULL : (~0ULL << (n - lo));
        if (x[w] & top) return false;
    }
    return true;
}

int popc64(uint64_t v) {
    int c = 0;
    while (v) { v &= v - 1; ++c; }
    return c;
}

uint64_t next_pow2(uint64_t v) {
    uint64_t s = 1;
    while (s < v) s <<= 1;
    return s;
}

size_t slot_bytes(int W) { return W == 1 ? 32 : 64; }

void free_all(itpp_ctx* h) {
    for (int i = 0; i < 2; ++i) {
        if (h->s.keys[i]) cudaFree(h->s.keys[i]);
        if (h->s.coef[i]) cudaFree(h->s.coef[i]);
    }
    if (h->s.table) cudaFree(h->s.table);
    if (h->s.part_keys) cudaFree(h->s.part_keys);
    if (h->s.part_coef) cudaFree(h->s.part_coef);
    if (h->s.part_cursor) cudaFree(h->s.part_cursor);
    for (int i = 0; i < 2; ++i) {
        if (h->s.part_desc[i]) cudaFree(h->s.part_desc[i]);
        if (h->s.chunks[i]) cudaFree(h->s.chunks[i]);
    }
    if (h->s.ctl) cudaFree(h->s.ctl);
    if (h->obs_mem) cudaFree(h->obs_mem);
    if (h->sort_mem) cudaFree(h->sort_mem);
    if (h->psd_mem) cudaFree(h->psd_mem);
    if (h->s.cand.cnt) cudaFree(h->s.cand.cnt);
    if (h->s.sp_drift) cudaFree(h->s.sp_drift);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    for (int k = 0; k < kKinds; ++k)
        for (auto& e : h->ev[k]) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
}

// Fold finished event pairs into the totals (synchronises the stream).
void prof_fold(itpp_ctx* h) {
    cudaStreamSynchronize(h->stream);
    for (int k = 0; k < kKinds; ++k) {
        for (size_t i = 0; i < h->ev_used[k]; ++i) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, h->ev[k][i].a, h->ev[k][i].b) == cudaSuccess) {
                h->prof_ms[k] += ms;
                h->prof_n[k] += 1;
            }
        }
        h->ev_used[k] = 0;
    }
}

EventPair* prof_begin(itpp_ctx* h, int kind) {
    if (!h->prof) return nullptr;
    if (h->ev_used[kind] >= 8192) prof_fold(h);
    if (h->ev_used[kind] == h->ev[kind].size()) {
        EventPair e;
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
        h->ev[kind].push_back(e);
    }
    EventPair* e = &h->ev[kind][h->ev_used[kind]++];
    cudaEventRecord(e->a, h->stream);
    return e;
}

void prof_end(itpp_ctx* h, EventPair* e) {
    if (e) cudaEventRecord(e->b, h->stream);
}

// Read the head of the control block and fold the device status into the
// handle's sticky status.
itpp_status sync_ctl(itpp_ctx* h) {
    if (cudaMemcpyAsync(h->h_ctl, h->s.ctl, kCtlHead, cudaMemcpyDeviceToHost, h->stream) !=
        cudaSuccess)
        return cuda_fail(h);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h);
    if (h->sticky == ITPP_OK && h->h_ctl->status != 0) h->sticky = (itpp_status)h->h_ctl->status;
    return h->sticky;
}

itpp_status launch_one_gate(itpp_ctx* h, int k) {
    const HostGate& g = h->gates[(size_t)k];
    cudaError_t e = cudaSuccess;
    if (h->p.merge_path == 0) {
        // a window's first gate (or any gate after the state changed
        // elsewhere) re-partitions; later gates of the window read the
        // previous gate's segments unless a partition outgrew the limit
        const int force = g.win_start || h->part_epoch != h->state_epoch ||
                          h->part_last != k - 1;
        EventPair* ev0 = prof_begin(h, 0);
        e = launch_part_scatter(h->s, g, force, h->stream);
        prof_end(h, ev0);
        h->part_epoch = h->state_epoch;
        h->part_last = k;
        if (e == cudaSuccess) {
            EventPair* ev1 = prof_begin(h, 1);
            e = launch_part_merge(h->s, g, h->stream);
            prof_end(h, ev1);
        }
    } else if (h->p.merge_path == 1) {
        EventPair* ev1 = prof_begin(h, 1);
        e = launch_gate_sorted(h->s, g, h->sort_mem, h->sort_bytes, h->stream);
        prof_end(h, ev1);
        h->launches += sorted_launches(h->s.n, h->s.W) - 2;
    } else {
        EventPair* ev0 = prof_begin(h, 0);
        e = launch_gate_insert(h->s, g, h->stream);
        prof_end(h, ev0);
        if (e == cudaSuccess) {
            EventPair* ev1 = prof_begin(h, 1);
            e = launch_gate_main(h->s, g, h->stream);
            prof_end(h, ev1);
        }
    }
    if (e == cudaSuccess) e = launch_gate_post(h->s, h->stream);
    // scatter, merge, post (partitioned: also the scatter's clear and second
    // launch, the merge's check and second launch, which return at once
    // unless the scatter or the merge must be redone)
    h->launches += h->p.merge_path == 0 ? 7 : 3;
    if (e == cudaSuccess && h->s.cap_policy == 1) {
        EventPair* ev2 = prof_begin(h, 2);
        e = launch_cap(h->s, h->stream, k);
        prof_end(h, ev2);
        h->launches += cap_launches(h->s);
    }
    return e == cudaSuccess ? ITPP_OK : cuda_fail(h);
}

itpp_status ensure_obs(itpp_ctx* h, int m, int W) {
    const size_t tsize = next_pow2((uint64_t)2 * m);
    const size_t need = (size_t)m * W * 16 + (size_t)m * 8 + tsize * 4 + (size_t)m * 4 +
                        (size_t)m * 8 + (size_t)(m + 1) * 8 + 256;
    if (need <= h->obs_bytes) return ITPP_OK;
    if (h->obs_mem) cudaFree(h->obs_mem);
    h->obs_mem = nullptr;
    h->obs_bytes = 0;
    if (cudaMalloc(&h->obs_mem, need) != cudaSuccess) return ITPP_ERR_ALLOC;
    h->obs_bytes = need;
    return ITPP_OK;
}

struct ObsPtrs {
    uint64_t *ox, *oz;
    double *ow, *vals, *out;
    int *tab, *first;
    int tsize;
};

ObsPtrs obs_layout(itpp_ctx* h, int m, int W) {
    ObsPtrs o;
    char* b = static_cast<char*>(h->obs_mem);
    o.tsize = (int)next_pow2((uint64_t)2 * m);
    o.ox = reinterpret_cast<uint64_t*>(b);
    b += (size_t)m * W * 8;
    o.oz = reinterpret_cast<uint64_t*>(b);
    b += (size_t)m * W * 8;
    o.ow = reinterpret_cast<double*>(b);
    b += (size_t)m * 8;
    o.vals = reinterpret_cast<double*>(b);
    b += (size_t)m * 8;
    o.out = reinterpret_cast<double*>(b);
    b += (size_t)(m + 1) * 8;
    o.tab = reinterpret_cast<int*>(b);
    b += (size_t)o.tsize * 4;
    o.first = reinterpret_cast<int*>(b);
    return o;
}

itpp_status check_obs_args(itpp_ctx* h, const uint64_t* ox, const uint64_t* oz, int m) {
    if (!h || !ox || !oz || m < 1 || m > 65536) return ITPP_ERR_ARG;
    for (int j = 0; j < m; ++j)
        if (!bits_ok(h->s.n, h->s.W, ox + (size_t)j * h->s.W) ||
            !bits_ok(h->s.n, h->s.W, oz + (size_t)j * h->s.W))
            return ITPP_ERR_ARG;
    return ITPP_OK;
}

}  // namespace

itpp_status itpp_detail_sync_ctl(itpp_ctx* h) { return sync_ctl(h); }
itpp_status itpp_detail_launch_gate(itpp_ctx* h, int k) { return launch_one_gate(h, k); }

// ---------------------------------------------------------------------------
// Canonical order and checkpoints (host side)
// ---------------------------------------------------------------------------
namespace {

template <int W>
struct HostTerm {
    uint64_t k[2 * W];   // x words, then z words: the comparison order
    double c;
};

template <int W>
itpp_status sort_terms_w(uint64_t* x, uint64_t* z, double* c, uint64_t count) {
    std::vector<HostTerm<W>> t;
    try {
        t.resize(count);
    } catch (...) {
        return ITPP_ERR_ALLOC;
    }
    for (uint64_t i = 0; i < count; ++i) {
        for (int w = 0; w < W; ++w) {
            t[i].k[w] = x[i * W + w];
            t[i].k[W + w] = z[i * W + w];
        }
        t[i].c = c[i];
    }
    std::sort(t.begin(), t.end(), [](const HostTerm<W>& a, const HostTerm<W>& b) {
        for (int w = 0; w < 2 * W; ++w)
            if (a.k[w] != b.k[w]) return a.k[w] < b.k[w];
        return false;
    });
    for (uint64_t i = 0; i < count; ++i) {
        for (int w = 0; w < W; ++w) {
            x[i * W + w] = t[i].k[w];
            z[i * W + w] = t[i].k[W + w];
        }
        c[i] = t[i].c;
    }
    return ITPP_OK;
}

constexpr char kStateMagic[8] = {'I', 'T', 'P', 'P', 'S', 'T', '0', '1'};

struct FileCloser {
    FILE* f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};

}  // namespace

extern "C" {

const char* itpp_status_string(itpp_status s) {
    switch (s) {
        case ITPP_OK: return "ok";
        case ITPP_ERR_ARG: return "invalid argument";
        case ITPP_ERR_ALLOC: return "allocation failed";
        case ITPP_ERR_CAPACITY: return "term bound or buffer capacity exceeded";
        case ITPP_ERR_HASH_PROBE: return "merge table probe limit reached";
        case ITPP_ERR_TIMEOUT: return "device wait timed out";
        case ITPP_ERR_TRACE_ZERO: return "identity coefficient truncated or missing";
        case ITPP_ERR_CUDA: return "CUDA runtime error";
        case ITPP_ERR_STATE: return "invalid state";
        case ITPP_ERR_IO: return "state file unreadable, unwritable or of another size";
    }
    return "unknown status";
}

const char* itpp_version(void) { return "itpp-gb300 0.1"; }

itpp_status itpp_create(int n, const uint64_t* gate_x, const uint64_t* gate_z,
                        const double* alpha, int n_gates, double dtau, const itpp_params* p,
                        void* cuda_stream, itpp_handle* out) {
    if (!out || !p || n < 1 || n > 128 || n_gates < 0) return ITPP_ERR_ARG;
    if (n_gates > 0 && (!gate_x || !gate_z || !alpha)) return ITPP_ERR_ARG;
    if (!std::isfinite(dtau) || !(p->delta >= 0.0) || !std::isfinite(p->delta)) return ITPP_ERR_ARG;
    if (p->cap_M < 1 || p->cap_M > (1ULL << 31)) return ITPP_ERR_ARG;
    if (p->cap_policy != 0 && p->cap_policy != 1) return ITPP_ERR_ARG;
    if (p->merge_path < 0 || p->merge_path > 2) return ITPP_ERR_ARG;
    if (p->max_weight < 0 || p->max_weight > 128) return ITPP_ERR_ARG;
    if (p->trotter_order < 0 || p->trotter_order > 2) return ITPP_ERR_ARG;
    if (p->partition_target != 0 && (p->partition_target < 64 || p->partition_target > 2048))
        return ITPP_ERR_ARG;
    if (p->table_load_pct != 0 && (p->table_load_pct < 10 || p->table_load_pct > 75))
        return ITPP_ERR_ARG;
    if (p->block_threads != 0 && p->block_threads != 128 && p->block_threads != 256 &&
        p->block_threads != 512)
        return ITPP_ERR_ARG;
    if (p->items_per_thread != 0 && p->items_per_thread != 1 && p->items_per_thread != 2 &&
        p->items_per_thread != 4)
        return ITPP_ERR_ARG;
    const int W = (n + 63) / 64;
    for (int k = 0; k < n_gates; ++k) {
        if (!std::isfinite(alpha[k])) return ITPP_ERR_ARG;
        if (!bits_ok(n, W, gate_x + (size_t)k * W) || !bits_ok(n, W, gate_z + (size_t)k * W))
            return ITPP_ERR_ARG;
    }

    itpp_ctx* h = new (std::nothrow) itpp_ctx;
    if (!h) return ITPP_ERR_ALLOC;
    h->p = *p;
    h->dtau = dtau;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&h->device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return ITPP_ERR_CUDA;
    }
    DeviceState& s = h->s;
    s.n = n;
    s.W = W;
    s.num_sms = sms;
    s.cap_M = p->cap_M;
    s.buf_cap = 2 * p->cap_M;
    s.max_ctas = std::min(8 * sms, 1024);   // the select reads at most 1024 candidate regions
    if (p->merge_path == 0) {
        // merge CTAs claim output chunks: room for what the chunks leave
        // unused, and an even count (the L2 bulk prefetch rounds byte ranges
        // to 16 bytes); candidate positions are 32-bit
        s.chunk = merge_chunk(p->cap_M, s.max_ctas, W);
        s.buf_cap += merge_slack(p->cap_M, s.max_ctas, W);
        s.buf_cap += s.buf_cap & 1ULL;
        if (s.buf_cap >= (1ULL << 32)) {
            delete h;
            return ITPP_ERR_ARG;
        }
    }
    s.cap_policy = p->cap_policy;
    s.delta = p->delta + 0.0;   // -0 becomes +0 (the threshold compares bit patterns)
    s.load_pct = p->table_load_pct ? p->table_load_pct : 50;
    // defaults: 512 x 2 for the partitioned merge (a whole partition in
    // registers), 256 x 2 for the global-table merge
    s.block = p->block_threads ? p->block_threads : 256;
    s.ipt = p->items_per_thread ? p->items_per_thread : 2;
    s.merge_deferred = p->merge_path == 0;
    s.probe_limit = 4096;
    const int load_for_size = s.load_pct < 50 ? s.load_pct : 50;
    uint64_t need = (p->cap_M * 100 + load_for_size - 1) / load_for_size;
    s.table_slots = next_pow2(need < 256 ? 256 : need);

    // the layer's schedule: the first-order product, or the symmetric
    // (Strang) product with half angles around the last term
    h->user_gates = n_gates;
    if (p->trotter_order == 2 && n_gates > 1) {
        for (int k = 0; k < n_gates - 1; ++k) { h->src_gate.push_back(k); h->src_scale.push_back(0.5); }
        h->src_gate.push_back(n_gates - 1);
        h->src_scale.push_back(1.0);
        for (int k = n_gates - 2; k >= 0; --k) { h->src_gate.push_back(k); h->src_scale.push_back(0.5); }
    } else {
        for (int k = 0; k < n_gates; ++k) { h->src_gate.push_back(k); h->src_scale.push_back(1.0); }
    }
    // per-gate weights: theta = alpha * dtau, the angle of Eq. (ITPP_PropRules)
    h->gates.resize(h->src_gate.size());
    for (size_t j = 0; j < h->gates.size(); ++j) {
        const int k = h->src_gate[j];
        HostGate& g = h->gates[j];
        int yy = 0;
        for (int w = 0; w < W; ++w) {
            g.qx[w] = gate_x[(size_t)k * W + w];
            g.qz[w] = gate_z[(size_t)k * W + w];
            yy += popc64(g.qx[w] & g.qz[w]);
        }
        const double theta = (alpha[k] * h->src_scale[j]) * dtau;
        g.ch = std::cosh(theta);
        g.msh = -std::sinh(theta);
        g.sh = std::sinh(theta);
        g.chd = std::cosh(theta);
        g.qyy = yy & 3;
        g.maxw = p->max_weight ? p->max_weight : (1 << 30);
        if (!std::isfinite(g.ch) || !std::isfinite(g.msh)) {   // |alpha dtau| beyond ~710
            delete h;
            return ITPP_ERR_ARG;
        }
    }

    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) {
        ok &= cudaMalloc(&s.keys[i], s.buf_cap * 16 * W) == cudaSuccess;
        ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.coef[i]), s.buf_cap * 8) == cudaSuccess;
    }
    ok &= ok && cudaMalloc(&s.table, s.table_slots * slot_bytes(W)) == cudaSuccess;
    ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.ctl), sizeof(DevCtl)) == cudaSuccess;
    ok &= ok && cudaMallocHost(reinterpret_cast<void**>(&h->h_ctl), sizeof(DevCtl)) == cudaSuccess;
    if (ok && p->merge_path == 0) {
        // the scatter buffer: partitions of a fixed stride, 2.5x the mean
        // partition at the bound (a window group adds up to 4^sites terms)
        s.part_cap = 2 * p->cap_M + p->cap_M / 2 + (1ULL << 18);   // even
        s.part_target = p->partition_target ? p->partition_target : partition_target_default(W);
        // the scatter aims at half the target at most (after gates whose
        // stored children outnumber the kept ones)
        s.part_max = partition_max(p->cap_M, (s.part_target + 1) / 2);
        ok &= cudaMalloc(&s.part_keys, s.part_cap * 16 * W) == cudaSuccess;
        ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.part_coef), s.part_cap * 8) == cudaSuccess;
        ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.part_cursor),
                               (size_t)s.part_max * sizeof(unsigned int)) == cudaSuccess;
        for (int i = 0; i < 2; ++i)
            ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.part_desc[i]),
                                   (size_t)s.part_max * sizeof(PartDesc)) == cudaSuccess;
        // output chunks: every claim takes at least one chunk of the buffer
        // or (exact claims) one partition's children, and each CTA leaves
        // one partly used
        s.max_chunks = (uint32_t)((s.chunk ? s.buf_cap / s.chunk : 0ULL) + s.part_max +
                                  2ULL * (uint64_t)s.max_ctas + 64);
        for (int i = 0; i < 2; ++i)
            ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.chunks[i]),
                                   (size_t)s.max_chunks * sizeof(ChunkDesc)) == cudaSuccess;
        // the merge's candidate regions for the top-M select: about half the
        // bound's worth of entries over the merge's CTAs
        uint64_t region = p->cap_M / (2ULL * (uint64_t)s.max_ctas);
        if (region < 64) region = 64;
        const uint64_t ent = region * (uint64_t)s.max_ctas;
        const size_t cnt_bytes = ((size_t)s.max_ctas * 4 + 255) / 256 * 256;
        void* cm = nullptr;
        ok &= ok && cudaMalloc(&cm, cnt_bytes + (size_t)ent * 12) == cudaSuccess;
        if (cm) {
            s.cand.cnt = static_cast<uint32_t*>(cm);
            s.cand.v = reinterpret_cast<unsigned long long*>(static_cast<char*>(cm) + cnt_bytes);
            s.cand.idx = reinterpret_cast<uint32_t*>(s.cand.v + ent);
            s.cand.region = region;
        }
        // the candidate range narrows while the merge lists more than this
        s.cand_hi = std::max<uint64_t>(16384, std::min<uint64_t>(p->cap_M / 16, ent / 8));
        s.layer_gates = (int)h->gates.size();
        ok &= ok && cudaMalloc(reinterpret_cast<void**>(&s.sp_drift),
                               (size_t)(s.layer_gates + 1) * sizeof(long long)) == cudaSuccess;
        ok &= ok && cudaMemsetAsync(s.sp_drift, 0, (size_t)(s.layer_gates + 1) * sizeof(long long),
                                    h->stream) == cudaSuccess;
        plan_windows(W, h->gates);
    }
    if (ok && p->merge_path == 1) {
        h->sort_bytes = sorted_scratch_bytes(W, s.buf_cap);
        ok &= cudaMalloc(&h->sort_mem, h->sort_bytes) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return ITPP_ERR_ALLOC;
    }
    ok &= cudaMemsetAsync(s.table, 0, s.table_slots * slot_bytes(W), h->stream) == cudaSuccess;
    ok &= cudaMemsetAsync(s.ctl, 0, sizeof(DevCtl), h->stream) == cudaSuccess;
    ok &= cudaMemcpyAsync(&s.ctl->buf_cap, &s.buf_cap, sizeof(s.buf_cap),
                          cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
    ok &= launch_reset_identity(s, h->stream) == cudaSuccess;
    ok &= cudaStreamSynchronize(h->stream) == cudaSuccess;
    if (!ok) {
        free_all(h);
        delete h;
        return ITPP_ERR_CUDA;
    }
    *out = h;
    return ITPP_OK;
}

itpp_status itpp_destroy(itpp_handle h) {
    if (!h) return ITPP_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return ITPP_OK;
}

itpp_status itpp_apply_gate(itpp_handle h, int k) {
    if (!h) return ITPP_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (k < 0 || k >= (int)h->gates.size()) return ITPP_ERR_ARG;
    return launch_one_gate(h, k);
}

itpp_status itpp_apply_trotter_layer(itpp_handle h, int n_layers) {
    if (!h || n_layers < 0) return ITPP_ERR_ARG;
    if (h->sticky) return h->sticky;
    for (int l = 0; l < n_layers; ++l)
        for (int k = 0; k < (int)h->gates.size(); ++k) {
            itpp_status st = launch_one_gate(h, k);
            if (st) return st;
        }
    return ITPP_OK;
}

itpp_status itpp_reset(itpp_handle h) {
    if (!h) return ITPP_ERR_ARG;
    if (h->sticky == ITPP_ERR_CUDA) return h->sticky;
    h->sticky = ITPP_OK;
    itpp_detail_touch(h);
    return launch_reset_identity(h->s, h->stream) == cudaSuccess ? ITPP_OK : cuda_fail(h);
}

itpp_status itpp_truncate(itpp_handle h, double delta) {
    if (!h || !(delta >= 0.0) || !std::isfinite(delta)) return ITPP_ERR_ARG;
    if (h->sticky) return h->sticky;
    if ((itpp_detail_touch(h), launch_materialize(h->s, h->stream)) != cudaSuccess) return cuda_fail(h);
    return launch_truncate(h->s, delta + 0.0, h->stream) == cudaSuccess ? ITPP_OK : cuda_fail(h);
}

itpp_status itpp_synchronize(itpp_handle h) {
    if (!h) return ITPP_ERR_ARG;
    return sync_ctl(h);
}

itpp_status itpp_get_count(itpp_handle h, uint64_t* count) {
    if (!h || !count) return ITPP_ERR_ARG;
    itpp_status st = sync_ctl(h);
    *count = h->h_ctl->count[h->h_ctl->cur];
    return st;
}

itpp_status itpp_get_stats(itpp_handle h, itpp_stats* o) {
    if (!h || !o) return ITPP_ERR_ARG;
    itpp_status st = sync_ctl(h);
    const DevCtl& c = *h->h_ctl;
    o->gates_applied = c.stat_gates;
    o->terms_in = c.stat_in;
    o->terms_out = c.stat_out;
    o->peak_terms = c.stat_peak;
    o->cap_events = c.stat_cap;
    o->count = c.count[c.cur];
    o->table_probes = c.stat_probes;
    o->repartitions = c.stat_scatters;
    o->select_candidates = c.stat_cands;
    o->select_range = c.stat_range;
    o->select_full = c.stat_sel_full;
    o->long_partitions = c.stat_long;
    o->merge_retries = c.stat_retry;
    o->error_site = c.status ? c.err_info : 0;
    o->kernel_launches = h->launches;
    return st;
}

itpp_status itpp_get_terms(itpp_handle h, uint64_t* x, uint64_t* z, double* c,
                           uint64_t capacity, uint64_t* count) {
    if (!h || !count) return ITPP_ERR_ARG;
    if (!h->sticky && (itpp_detail_touch(h), launch_materialize(h->s, h->stream)) != cudaSuccess) return cuda_fail(h);
    itpp_status st = sync_ctl(h);
    if (st) return st;
    const uint64_t n = h->h_ctl->count[h->h_ctl->cur];
    *count = n;
    if (capacity < n) return ITPP_ERR_CAPACITY;
    if (n == 0) return ITPP_OK;
    if (!x || !z || !c) return ITPP_ERR_ARG;
    const int o = h->h_ctl->cur ^ 1;   // the other buffer is free between gates
    uint64_t* dx = static_cast<uint64_t*>(h->s.keys[o]);
    uint64_t* dz = dx + n * h->s.W;
    double* dc = h->s.coef[o];
    if (launch_export(h->s, dx, dz, dc, h->stream) != cudaSuccess) return cuda_fail(h);
    const size_t kb = (size_t)n * h->s.W * 8;
    if (cudaMemcpyAsync(x, dx, kb, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(z, dz, kb, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(c, dc, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return cuda_fail(h);
    return sync_ctl(h);
}

itpp_status itpp_sort_terms(int W, uint64_t* x, uint64_t* z, double* c, uint64_t count) {
    if (W != 1 && W != 2) return ITPP_ERR_ARG;
    if (count == 0) return ITPP_OK;
    if (!x || !z || !c) return ITPP_ERR_ARG;
    return W == 1 ? sort_terms_w<1>(x, z, c, count) : sort_terms_w<2>(x, z, c, count);
}

itpp_status itpp_get_terms_sorted(itpp_handle h, uint64_t* x, uint64_t* z, double* c,
                                  uint64_t capacity, uint64_t* count) {
    itpp_status st = itpp_get_terms(h, x, z, c, capacity, count);
    if (st) return st;
    return itpp_sort_terms(h->s.W, x, z, c, *count);
}

itpp_status itpp_save(itpp_handle h, const char* path) {
    if (!h || !path) return ITPP_ERR_ARG;
    uint64_t n = 0;
    itpp_status st = itpp_get_count(h, &n);
    if (st) return st;
    const int W = h->s.W;
    std::vector<uint64_t> x, z;
    std::vector<double> c;
    try {
        x.resize(n * W);
        z.resize(n * W);
        c.resize(n);
    } catch (...) {
        return ITPP_ERR_ALLOC;
    }
    uint64_t got = 0;
    st = itpp_get_terms_sorted(h, x.data(), z.data(), c.data(), n, &got);
    if (st) return st;
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) return ITPP_ERR_IO;
    const int32_t hdr[2] = {h->s.n, W};
    bool ok = fwrite(kStateMagic, 1, 8, fc.f) == 8 && fwrite(hdr, 4, 2, fc.f) == 2 &&
              fwrite(&got, 8, 1, fc.f) == 1 &&
              fwrite(x.data(), 8, got * W, fc.f) == got * W &&
              fwrite(z.data(), 8, got * W, fc.f) == got * W &&
              fwrite(c.data(), 8, got, fc.f) == got;
    ok = fclose(fc.f) == 0 && ok;
    fc.f = nullptr;
    return ok ? ITPP_OK : ITPP_ERR_IO;
}

itpp_status itpp_load(itpp_handle h, const char* path) {
    if (!h || !path) return ITPP_ERR_ARG;
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) return ITPP_ERR_IO;
    char magic[8];
    int32_t hdr[2];
    uint64_t count = 0;
    if (fread(magic, 1, 8, fc.f) != 8 || memcmp(magic, kStateMagic, 8) != 0 ||
        fread(hdr, 4, 2, fc.f) != 2 || fread(&count, 8, 1, fc.f) != 1)
        return ITPP_ERR_IO;
    const int W = h->s.W;
    if (hdr[0] != h->s.n || hdr[1] != W || count < 1 || count > h->s.cap_M) return ITPP_ERR_IO;
    std::vector<uint64_t> x, z;
    std::vector<double> c;
    try {
        x.resize(count * W);
        z.resize(count * W);
        c.resize(count);
    } catch (...) {
        return ITPP_ERR_ALLOC;
    }
    if (fread(x.data(), 8, count * W, fc.f) != count * W ||
        fread(z.data(), 8, count * W, fc.f) != count * W ||
        fread(c.data(), 8, count, fc.f) != count)
        return ITPP_ERR_IO;
    return itpp_set_terms(h, x.data(), z.data(), c.data(), count);
}

itpp_status itpp_set_terms(itpp_handle h, const uint64_t* x, const uint64_t* z, const double* c,
                           uint64_t count) {
    if (!h || !x || !z || !c || count < 1 || count > h->s.cap_M) return ITPP_ERR_ARG;
    for (uint64_t i = 0; i < count; ++i)
        if (!std::isfinite(c[i])) return ITPP_ERR_ARG;   // a NaN or inf coefficient
    if (h->sticky == ITPP_ERR_CUDA) return h->sticky;
    cudaStreamSynchronize(h->stream);
    // stage the planes in buffer 1, import into buffer 0
    uint64_t* dx = static_cast<uint64_t*>(h->s.keys[1]);
    uint64_t* dz = dx + count * h->s.W;
    double* dc = h->s.coef[1];
    const size_t kb = (size_t)count * h->s.W * 8;
    if (cudaMemcpyAsync(dx, x, kb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(dz, z, kb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(dc, c, (size_t)count * 8, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return cuda_fail(h);
    itpp_detail_touch(h);
    if (launch_import(h->s, dx, dz, dc, count, h->stream) != cudaSuccess) return cuda_fail(h);
    h->sticky = ITPP_OK;
    itpp_status st = sync_ctl(h);
    if (st != ITPP_OK && st != ITPP_ERR_CUDA) {
        // invalid input: restore a valid (identity) state and report
        h->sticky = ITPP_OK;
        launch_reset_identity(h->s, h->stream);
        sync_ctl(h);
        return st;
    }
    return st;
}

itpp_status itpp_expect_device(itpp_handle h, const uint64_t* d_ox, const uint64_t* d_oz,
                               const double* d_ow, int m, double* d_out) {
    if (!h || !d_ox || !d_oz || !d_out || m < 1 || m > 65536) return ITPP_ERR_ARG;
    if (h->sticky) return h->sticky;
    itpp_status st = ensure_obs(h, m, h->s.W);
    if (st) return st;
    ObsPtrs o = obs_layout(h, m, h->s.W);
    if ((itpp_detail_touch(h), launch_materialize(h->s, h->stream)) != cudaSuccess) return cuda_fail(h);
    EventPair* ev = prof_begin(h, 3);
    cudaError_t e = launch_expect(h->s, d_ox, d_oz, d_ow, m, o.tsize, o.tab, o.first, o.vals,
                                  d_out, h->stream);
    prof_end(h, ev);
    return e == cudaSuccess ? ITPP_OK : cuda_fail(h);
}

static itpp_status expect_host(itpp_handle h, const uint64_t* ox, const uint64_t* oz,
                               const double* ow, int m, double* coeffs, double* total) {
    itpp_status st = check_obs_args(h, ox, oz, m);
    if (st) return st;
    if (h->sticky) return h->sticky;
    st = ensure_obs(h, m, h->s.W);
    if (st) return st;
    ObsPtrs o = obs_layout(h, m, h->s.W);
    const size_t kb = (size_t)m * h->s.W * 8;
    if (cudaMemcpyAsync(o.ox, ox, kb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(o.oz, oz, kb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return cuda_fail(h);
    if (ow && cudaMemcpyAsync(o.ow, ow, (size_t)m * 8, cudaMemcpyHostToDevice, h->stream) !=
                  cudaSuccess)
        return cuda_fail(h);
    if ((itpp_detail_touch(h), launch_materialize(h->s, h->stream)) != cudaSuccess) return cuda_fail(h);
    EventPair* ev = prof_begin(h, 3);
    cudaError_t e = launch_expect(h->s, o.ox, o.oz, ow ? o.ow : nullptr, m, o.tsize, o.tab,
                                  o.first, o.vals, o.out, h->stream);
    prof_end(h, ev);
    if (e != cudaSuccess) return cuda_fail(h);
    std::vector<double> buf((size_t)m + 1);
    if (cudaMemcpyAsync(buf.data(), o.out, ((size_t)m + 1) * 8, cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
        return cuda_fail(h);
    st = sync_ctl(h);
    if (st) return st;
    if (coeffs) std::memcpy(coeffs, buf.data(), (size_t)m * 8);
    if (total) *total = buf[(size_t)m];
    return ITPP_OK;
}

itpp_status itpp_expect(itpp_handle h, const uint64_t* obs_x, const uint64_t* obs_z,
                        const double* obs_w, int m, double* out) {
    if (!h || !obs_w || !out) return ITPP_ERR_ARG;
    return expect_host(h, obs_x, obs_z, obs_w, m, nullptr, out);
}

itpp_status itpp_expect_psd(itpp_handle h, const uint64_t* obs_x, const uint64_t* obs_z,
                            const double* obs_w, int m, double* out) {
    if (!h || !obs_w || !out) return ITPP_ERR_ARG;
    itpp_status st = check_obs_args(h, obs_x, obs_z, m);
    if (st) return st;
    if (h->sticky) return h->sticky;
    st = ensure_obs(h, m, h->s.W);
    if (st) return st;
    const int n_part = h->s.num_sms * 8;
    if (!h->psd_mem && cudaMalloc(reinterpret_cast<void**>(&h->psd_mem),
                                  ((size_t)2 * n_part + 4) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return ITPP_ERR_ALLOC;
    }
    ObsPtrs o = obs_layout(h, m, h->s.W);
    const size_t kb = (size_t)m * h->s.W * 8;
    if (cudaMemcpyAsync(o.ox, obs_x, kb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(o.oz, obs_z, kb, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(o.ow, obs_w, (size_t)m * 8, cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess)
        return cuda_fail(h);
    if ((itpp_detail_touch(h), launch_materialize(h->s, h->stream)) != cudaSuccess) return cuda_fail(h);
    double* d_out = h->psd_mem + 2 * (size_t)n_part;
    EventPair* ev = prof_begin(h, 3);
    cudaError_t e = launch_expect_psd(h->s, o.ox, o.oz, o.ow, m, h->psd_mem, n_part, d_out,
                                      h->stream);
    prof_end(h, ev);
    if (e != cudaSuccess) return cuda_fail(h);
    if (cudaMemcpyAsync(out, d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream) !=
        cudaSuccess)
        return cuda_fail(h);
    return sync_ctl(h);
}

itpp_status itpp_coeffs(itpp_handle h, const uint64_t* obs_x, const uint64_t* obs_z, int m,
                        double* out) {
    if (!h || !out) return ITPP_ERR_ARG;
    return expect_host(h, obs_x, obs_z, nullptr, m, out, nullptr);
}

itpp_status itpp_profile_enable(itpp_handle h, int enable) {
    if (!h) return ITPP_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    for (int k = 0; k < kKinds; ++k) {
        h->ev_used[k] = 0;
        h->prof_ms[k] = 0;
        h->prof_n[k] = 0;
    }
    h->prof = enable != 0;
    return ITPP_OK;
}

itpp_status itpp_profile_read(itpp_handle h, int kid, uint64_t* launches, double* total_ms) {
    if (!h || kid < 0 || kid >= kKinds || !launches || !total_ms) return ITPP_ERR_ARG;
    prof_fold(h);
    *launches = h->prof_n[kid];
    *total_ms = h->prof_ms[kid];
    return ITPP_OK;
}

}  // extern "C"
