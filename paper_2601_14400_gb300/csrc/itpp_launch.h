// itpp_launch.h -- host-side launchers of the sm_103a kernels (internal).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace itpp {

struct DevCtl;

// One partition of the state as a gate of a window wrote it (a contiguous
// segment of the state buffer).
struct PartDesc {
    unsigned long long off;   // first term in the state buffer
    unsigned int cnt;         // terms stored
    unsigned int pad;
};

// One output chunk of a partitioned merge: a contiguous run of stored terms
// (the partitions' segments the CTA packed into it), for readers that walk
// the whole state rather than its partitions.
struct ChunkDesc {
    unsigned long long off;   // first term in the state buffer
    unsigned int cnt;         // terms stored
    unsigned int pad;
};

// The candidate list the partitioned merge fills for the top-M select: CTA r
// of the merge owns entries [r * region, (r + 1) * region) of v (the
// candidate's |c| pattern minus the range's low end) and idx (its position
// in the output buffer), and writes how many it used to cnt[r].
struct CandRegions {
    unsigned long long* v = nullptr;
    uint32_t* idx = nullptr;
    uint32_t* cnt = nullptr;
    uint64_t region = 0;
};

// Device resources of one propagation (or of one batch instance table).
struct DeviceState {
    int n = 0, W = 1;
    void* keys[2] = {nullptr, nullptr};   // PKey<W>[buf_cap]
    double* coef[2] = {nullptr, nullptr}; // double[buf_cap]
    void* table = nullptr;                // Slot<W>[table_slots]
    uint64_t table_slots = 0;
    DevCtl* ctl = nullptr;
    uint64_t cap_M = 0, buf_cap = 0;
    int cap_policy = 0;
    double delta = 0;
    // launch shape
    int num_sms = 1;
    int block = 256, ipt = 2, load_pct = 50, probe_limit = 4096;
    // partitioned merge (itpp_part.cu): scatter buffer and cursors
    void* part_keys = nullptr;        // PKey<W>[part_cap]
    double* part_coef = nullptr;      // double[part_cap]
    unsigned int* part_cursor = nullptr;   // [part_max]
    PartDesc* part_desc[2] = {nullptr, nullptr};   // [part_max] per state buffer
    uint64_t part_cap = 0;
    uint32_t part_max = 0;
    int part_target = 0;              // mean partition size of the scatter
    uint64_t chunk = 0;               // output chunk a merge CTA claims at a time (terms)
    ChunkDesc* chunks[2] = {nullptr, nullptr};   // [max_chunks] per state buffer
    uint32_t max_chunks = 0;
    int max_ctas = 0;                 // CTAs of the merge and select grids at most
    CandRegions cand;                 // one allocation: cnt[max_ctas], then v, then idx
    uint64_t cand_hi = 0;             // candidate count above which the range narrows
    // per gate of a layer: how the select's threshold pattern moved at that
    // gate (the prediction of the next layer's), and the number of gates
    long long* sp_drift = nullptr;
    int layer_gates = 0;
    // top-M select leaves its kept set as a predicate for the next scatter
    bool merge_deferred = false;
};

// Per-gate host constants (computed once in itpp_create).
struct HostGate {
    uint64_t qx[2] = {0, 0}, qz[2] = {0, 0};
    double ch = 1, msh = 0;  // cosh(theta), -sinh(theta)
    double sh = 0, chd = 1;  // d ch / d theta = sinh(theta), -d msh / d theta = cosh(theta)
    int qyy = 0;
    int maxw = 1 << 30;      // Pauli weight cutoff (off by default)
    // the window of consecutive gates this gate belongs to (partitioned merge)
    uint64_t keep_x[2] = {~0ULL, ~0ULL}, keep_z[2] = {~0ULL, ~0ULL};   // key bits hashed
    int pair_mode = 1;       // 1: the gate alone, partitioned by its pair key
    int win_sites = 0;       // sites of the window (mask mode)
    int win_start = 1;       // first gate of its window
};

// One elementary gate: merge-table build, branch-emit-merge-truncate, post.
cudaError_t launch_gate_insert(const DeviceState& s, const HostGate& g, cudaStream_t st);
cudaError_t launch_gate_main(const DeviceState& s, const HostGate& g, cudaStream_t st);
cudaError_t launch_gate_post(const DeviceState& s, cudaStream_t st);
// Partitioned merge: scatter by the window's masked key (or the pair key),
// then one shared-memory table per partition (the default merge of a single
// propagation).  force = 1 re-partitions unconditionally (first gate of a
// window, or the state changed outside the window); force = 0 only when the
// previous gate's partitions held for that gate alone (pair-key mode).
cudaError_t launch_part_scatter(const DeviceState& s, const HostGate& g, int force,
                                cudaStream_t st);
cudaError_t launch_part_merge(const DeviceState& s, const HostGate& g, cudaStream_t st);
uint32_t partition_max(uint64_t cap_M, int target);
int partition_target_default(int W);
// Output chunk of the partitioned merge for a term bound, and the room the
// chunks may leave unused in a state buffer (added to its capacity).
uint64_t merge_chunk(uint64_t cap_M, int max_ctas, int W);
uint64_t merge_slack(uint64_t cap_M, int max_ctas, int W);
// Group consecutive gates into windows of at most a few sites (sets the
// window fields of every gate).
void plan_windows(int W, std::vector<HostGate>& gates);
// Top-M select and compaction (no-ops on the device when the bound holds).
// gate: the gate's index in the layer's schedule (the partitioned merge's
// select predicts the next threshold from the same gate of the last layer).
cudaError_t launch_cap(const DeviceState& s, cudaStream_t st, int gate = 0);
int cap_launches(const DeviceState& s);
// The select part only (threshold and tie key in the control block, no
// compaction): used where the kept set is compacted elsewhere.
cudaError_t launch_cap_select(const DeviceState& s, cudaStream_t st);
// The top-M select of the partitioned merge (itpp_select.cu): leaves the
// kept set as a predicate for the next gate's reads.
cudaError_t launch_select_deferred(const DeviceState& s, cudaStream_t st, int gate);
int select_deferred_launches(int W);
// Apply a deferred top-M select and gather a segmented state into one
// contiguous run (compaction); a no-op when neither is there.
cudaError_t launch_materialize(const DeviceState& s, cudaStream_t st);
// Sort-based merge path (children buffer, radix sort, segmented reduce).
cudaError_t launch_gate_sorted(const DeviceState& s, const HostGate& g, void* scratch,
                               uint64_t scratch_bytes, cudaStream_t st);
uint64_t sorted_scratch_bytes(int W, uint64_t buf_cap);
int sorted_launches(int n, int W);

// Expectation: obs table build, state scan, reduction.  d_tab holds
// tsize ints, d_first m ints, d_vals m doubles.
cudaError_t launch_expect(const DeviceState& s, const uint64_t* d_ox, const uint64_t* d_oz,
                          const double* d_ow, int m, int tsize, int* d_tab, int* d_first,
                          double* d_vals, double* d_out, cudaStream_t st);
// <O>_{2 tau} of the squared state (itpp_psd.cu): d_partials holds
// 2 * n_part doubles, d_out three (ratio, numerator / 2^n, purity / 2^n).
cudaError_t launch_expect_psd(const DeviceState& s, const uint64_t* d_ox, const uint64_t* d_oz,
                              const double* d_ow, int m, double* d_partials, int n_part,
                              double* d_out, cudaStream_t st);
// Normalised export into the other buffer's memory: x plane, z plane, c.
cudaError_t launch_export(const DeviceState& s, uint64_t* d_x, uint64_t* d_z, double* d_c,
                          cudaStream_t st);
// Import from x/z planes and c into buffer 0, with bit and duplicate checks.
cudaError_t launch_import(const DeviceState& s, const uint64_t* d_x, const uint64_t* d_z,
                          const double* d_c, uint64_t count, cudaStream_t st);
// Explicit threshold truncation + normalisation of the current state.
cudaError_t launch_truncate(const DeviceState& s, double delta, cudaStream_t st);
// Reset the control block (state = identity in buffer 0).
cudaError_t launch_reset_identity(const DeviceState& s, cudaStream_t st);

// Many independent propagations sharing launches (itpp_batch.cu).  Instance
// b owns the slices [b*buf_cap, (b+1)*buf_cap) of both state buffers,
// [b*table_slots, ...) of the table and control block ctls[b].
struct BatchState {
    int B = 0, W = 1, max_gates = 0;
    void* keys[2] = {nullptr, nullptr};
    double* coef[2] = {nullptr, nullptr};
    void* table = nullptr;
    DevCtl* ctls = nullptr;
    void* gates = nullptr;               // GateArg<W>[B * max_gates]
    int* n_gates = nullptr;              // [B]
    unsigned long long* item_prefix = nullptr;   // [B + 1] each
    unsigned long long* tile_prefix = nullptr;
    unsigned long long* cap_prefix = nullptr;
    unsigned long long* ccap_prefix = nullptr;
    uint64_t cap_M = 0, buf_cap = 0, table_slots = 0;
    int cap_policy = 0;
    double delta = 0;
    int num_sms = 1, load_pct = 50, probe_limit = 4096;
    // launch shape (autotuned): branch-emit block (x2 items per thread), grid
    // multipliers (CTAs per SM) of the branch-emit and table-build kernels
    int main_block = 256, main_grid = 4, insert_grid = 8;
    // merge_path 0 (partitioned merge): per instance a scatter buffer of
    // part_cap terms in at most part_max pair-key partitions; the merge's
    // CTAs per SM (0: as many as fit) and the scatter's, and the mean
    // partition size (autotuned); merge_path 2: the global table above
    int merge_path = 0;
    void* part_keys = nullptr;                    // [B * part_cap] keys
    double* part_coef = nullptr;                  // [B * part_cap + 2]
    unsigned int* part_cursor = nullptr;          // [B * part_max]
    uint64_t part_cap = 0;
    uint32_t part_max = 0;
    int part_target = 0, merge_ctas = 0, scatter_grid = 8;
};

// Gate `step` of the layer for every instance that has one.
cudaError_t launch_batch_step(const BatchState& s, int step, cudaStream_t st);
// CTAs per SM of the batch's partition merge that fit, for W mask words and
// `block` threads per CTA (sets the kernel's shared-memory attributes: call
// it before capturing a layer).
int batch_merge_fit(int W, int block);
int batch_step_launches(const BatchState& s);

}  // namespace itpp
