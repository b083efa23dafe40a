// itpp_noalloc.cu -- one elementary gate without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a gate:
// code running under a memory pool or arena that owns every byte of the
// device, code inside a framework's allocator-free region, or a host that
// must not trigger an implicit synchronisation by calling cudaMalloc or
// cudaFree.  itpp_gate_apply_noalloc serves them: the caller passes its own
// input and output buffers, and the scratch the gate needs (the merge table
// and the control block) lives in the file-scope array below, which every
// GPU that loads this library holds until the process exits.
//
// The scratch is shared by every call on a device and keeps the last call's
// contents.  The merge table needs no clearing between calls: each call takes
// a new generation number and slots tagged with an older one count as free
// (the array starts zeroed and generations start at one); when the 32-bit
// generation wraps, the call's first kernel zeroes the whole table once.  The
// counters that must start at zero are reset by that kernel too.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on this scratch and corrupt each other's results; serialise
// them.  With CUDA's lazy module loading, the first call on a device may be
// the one that loads this library's module and sets the array aside (which
// allocates and can synchronise): callers that must not allocate make one
// call, or create any handle of this library, on that device beforehand.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "itpp.h"
#include "itpp_common.cuh"
#include "itpp_launch.h"

namespace {

using itpp::DevCtl;

constexpr size_t kCtlBytes = (sizeof(DevCtl) + 255) / 256 * 256;
constexpr size_t kTableBytes = size_t(16) << 20;           // 16 MiB merge table
constexpr size_t kScratchBytes = kCtlBytes + kTableBytes;  // about 17 MiB in all

// The scratch: control block first, merge table after it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device; looked up once per
// device (host code cannot use the array's name as a device address).
itpp_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return ITPP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ITPP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ITPP_OK;
}

// The normaliser's value before the gate's merge writes it: a NaN pattern
// that no merge produces, so a call whose input lacks the identity (and
// which therefore never writes it) is told apart.
constexpr unsigned long long kNoIdentity = 0x7ff80000deadbeefULL;

// Reset the control block for a call: input in buffer 0 with n_in terms,
// output in buffer 1, a fresh table generation.  When the generation counter
// wraps, every slot is cleared (tag 0 = free) before generation 1 is used,
// so a slot last written about 2^32 calls earlier cannot pass for a live one.
__global__ void __launch_bounds__(256) k_noalloc_begin(uint64_t n_in, uint64_t buf_cap) {
    __shared__ int s_wrap;
    DevCtl* ctl = reinterpret_cast<DevCtl*>(g_noalloc_scratch);
    if (threadIdx.x == 0) {
        ctl->status = 0;
        ctl->err_info = 0;
        ctl->cur = 0;
        ctl->count[0] = n_in;
        ctl->count[1] = 0;
        ctl->buf_cap = buf_cap;
        ctl->norm[0] = 1.0;
        ctl->rnorm[0] = 1.0;
        ctl->norm[1] = __longlong_as_double((long long)kNoIdentity);
        ctl->rnorm[1] = 1.0;
        const unsigned int g = ctl->gen + 1u;
        s_wrap = g == 0u;
        ctl->gen = g ? g : 1u;
    }
    __syncthreads();
    if (s_wrap) {
        uint4* t = reinterpret_cast<uint4*>(g_noalloc_scratch + kCtlBytes);
        for (size_t i = threadIdx.x; i < kTableBytes / sizeof(uint4); i += blockDim.x)
            t[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Count and trace of the output; an error (or an input without the
// identity) leaves count = UINT64_MAX and trace = NaN.
__global__ void k_noalloc_end(uint64_t* d_n_out, double* d_trace_out) {
    if (threadIdx.x != 0) return;
    DevCtl* ctl = reinterpret_cast<DevCtl*>(g_noalloc_scratch);
    if (!ctl->status &&
        (unsigned long long)__double_as_longlong(ctl->norm[1]) == kNoIdentity)
        itpp::set_status(ctl, itpp::ST_TRACE_ZERO, 50);
    if (ctl->status) {
        *d_n_out = ~0ULL;
        if (d_trace_out) *d_trace_out = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    ctl->rnorm[1] = __ddiv_rn(1.0, ctl->norm[1]);
    *d_n_out = ctl->count[1];
    if (d_trace_out) *d_trace_out = ctl->norm[1];
}

// Rescale the output by the reciprocal of its identity coefficient (the
// trace normalisation), the identity becoming exactly one.
template <int W>
__global__ void __launch_bounds__(256)
k_noalloc_normalise(itpp::PKey<W>* keys, double* coef) {
    const DevCtl* ctl = reinterpret_cast<const DevCtl*>(g_noalloc_scratch);
    if (ctl->status) return;
    const uint64_t n = ctl->count[1];
    const double r = ctl->rnorm[1];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        coef[i] = itpp::normalised(coef[i], r, itpp::key_is_zero(keys[i]));
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

}  // namespace

extern "C" itpp_status itpp_gate_apply_noalloc(
    int n, const uint64_t* gate_x, const uint64_t* gate_z, double alpha, double dtau,
    double delta, const uint64_t* d_keys_in, const double* d_coef_in, uint64_t n_in,
    uint64_t* d_keys_out, double* d_coef_out, uint64_t out_capacity, uint64_t* d_n_out,
    double* d_trace_out, void* cuda_stream) {
    if (n < 1 || n > 128 || !gate_x || !gate_z || !d_keys_in || !d_coef_in || !d_keys_out ||
        !d_coef_out || !d_n_out || n_in < 1)
        return ITPP_ERR_ARG;
    if (!std::isfinite(alpha) || !std::isfinite(dtau) || !(delta >= 0.0) || !std::isfinite(delta))
        return ITPP_ERR_ARG;
    const int W = (n + 63) / 64;
    if (!bits_ok(n, W, gate_x) || !bits_ok(n, W, gate_z)) return ITPP_ERR_ARG;
    const uint64_t slot_bytes = W == 1 ? 32 : 64;
    const uint64_t slots = kTableBytes / slot_bytes;
    if (n_in > ITPP_NOALLOC_MAX_TERMS(W)) return ITPP_ERR_CAPACITY;
    if (out_capacity < 2 * n_in) return ITPP_ERR_CAPACITY;

    void* scratch = nullptr;
    itpp_status st = scratch_address(&scratch);
    if (st) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    itpp::DeviceState s;
    s.n = n;
    s.W = W;
    s.keys[0] = const_cast<uint64_t*>(d_keys_in);
    s.coef[0] = const_cast<double*>(d_coef_in);
    s.keys[1] = d_keys_out;
    s.coef[1] = d_coef_out;
    s.ctl = reinterpret_cast<DevCtl*>(scratch);
    s.table = static_cast<unsigned char*>(scratch) + kCtlBytes;
    s.table_slots = slots;
    s.cap_M = 0;
    s.buf_cap = out_capacity > n_in ? out_capacity : n_in;
    s.cap_policy = 0;
    s.delta = delta + 0.0;   // -0 becomes +0 (the threshold compares bit patterns)
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s.num_sms = sms;

    itpp::HostGate g;
    int yy = 0;
    for (int w = 0; w < W; ++w) {
        g.qx[w] = gate_x[w];
        g.qz[w] = gate_z[w];
        uint64_t v = gate_x[w] & gate_z[w];
        while (v) { v &= v - 1; ++yy; }
    }
    const double theta = alpha * dtau;
    g.ch = std::cosh(theta);
    g.msh = -std::sinh(theta);
    g.qyy = yy & 3;

    k_noalloc_begin<<<1, 256, 0, stream>>>(n_in, s.buf_cap);
    if (itpp::launch_gate_insert(s, g, stream) != cudaSuccess) return ITPP_ERR_CUDA;
    if (itpp::launch_gate_main(s, g, stream) != cudaSuccess) return ITPP_ERR_CUDA;
    k_noalloc_end<<<1, 32, 0, stream>>>(d_n_out, d_trace_out);
    const int grid = sms * 8;
    if (W == 1)
        k_noalloc_normalise<1><<<grid, 256, 0, stream>>>(
            reinterpret_cast<itpp::PKey<1>*>(d_keys_out), d_coef_out);
    else
        k_noalloc_normalise<2><<<grid, 256, 0, stream>>>(
            reinterpret_cast<itpp::PKey<2>*>(d_keys_out), d_coef_out);
    return cudaGetLastError() == cudaSuccess ? ITPP_OK : ITPP_ERR_CUDA;
}
