// itpp_ctx.h -- the handle behind itpp_handle (internal; shared by the C ABI
// translation units).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "itpp.h"
#include "itpp_common.cuh"
#include "itpp_launch.h"

namespace itpp_detail {

constexpr int kKinds = 4;
constexpr size_t kCtlHead = offsetof(itpp::DevCtl, sel_hist);

struct EventPair {
    cudaEvent_t a, b;
};

}  // namespace itpp_detail

using itpp_detail::EventPair;
using itpp_detail::kKinds;
using itpp_detail::kCtlHead;

struct itpp_ctx {
    itpp::DeviceState s;
    std::vector<itpp::HostGate> gates;   // the elementary gates of one layer
    // gate j of the layer is Hamiltonian term src_gate[j] with coefficient
    // alpha * src_scale[j] (the first-order product: j, 1; Strang: halves)
    std::vector<int> src_gate;
    std::vector<double> src_scale;
    int user_gates = 0;
    double dtau = 0;
    itpp_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    itpp_status sticky = ITPP_OK;
    itpp::DevCtl* h_ctl = nullptr;   // pinned mirror of the control block head
    // expectation scratch
    void* obs_mem = nullptr;
    size_t obs_bytes = 0;
    // PSD-restored observable: block partials and the result
    double* psd_mem = nullptr;
    // sorted merge scratch
    void* sort_mem = nullptr;
    uint64_t sort_bytes = 0;
    uint64_t launches = 0;   // kernels launched by this handle
    // partitioned merge: the state's partitions are valid for the window of
    // gate part_last while part_epoch == state_epoch; anything else that
    // changes the state bumps state_epoch
    uint64_t state_epoch = 1, part_epoch = 0;
    int part_last = -1;
    // profiling
    bool prof = false;
    std::vector<EventPair> ev[kKinds];
    size_t ev_used[kKinds] = {0, 0, 0, 0};
    double prof_ms[kKinds] = {0, 0, 0, 0};
    uint64_t prof_n[kKinds] = {0, 0, 0, 0};
};


// Helpers of the C ABI used by more than one translation unit.
itpp_status itpp_detail_sync_ctl(itpp_ctx* h);
itpp_status itpp_detail_launch_gate(itpp_ctx* h, int k);
// The state changed outside a window's merges (partitions must be rebuilt).
inline void itpp_detail_touch(itpp_ctx* h) { ++h->state_epoch; }
