/*
 * itpp.h -- C ABI of the GB300 imaginary-time Pauli propagation library.
 *
 * The library propagates the identity operator through a first-order Trotter
 * product of imaginary-time Pauli gates (Algorithm 1 of "Pauli Propagation
 * for Imaginary-Time Evolution", arXiv 2601.14400) and reads thermal
 * expectation values from the propagated operator.  Every step of the
 * method runs in hand-written sm_103a CUDA kernels; the host side only
 * validates arguments, computes the per-gate weights once and orders the
 * launches.
 *
 * Representation (Eq. (Observable_Pauli), Sec. II.B):
 *   A Pauli string on n sites is a pair of masks (x, z) of W = ceil(n/64)
 *   uint64 words; site i is bit i%64 of word i/64.  (x_i, z_i) = (0,0) I,
 *   (1,0) X, (0,1) Z, (1,1) Y (the Hermitian Y, not XZ).  Bits >= n must be
 *   zero.  Host arrays of strings are row-major: string j occupies words
 *   [j*W, (j+1)*W) of the x array and of the z array.  1 <= n <= 128.
 *
 * Conventions shared by every call:
 *   - Every call returns itpp_status.  Calls that launch work are
 *     asynchronous on the handle's CUDA stream; an error detected on the
 *     device (capacity, hash probe limit, trace collapse) is stored in the
 *     handle and returned by the next synchronising call (itpp_synchronize,
 *     itpp_get_count, itpp_get_terms, itpp_expect, itpp_coeffs).  Once a
 *     handle holds an error every later call returns it; destroy still works.
 *   - The library owns all device memory it allocates for a handle and frees
 *     it in itpp_destroy.  Caller pointers are only read or written during
 *     the call (host arrays) or until the stream reaches the work (device
 *     arrays of the *_device calls).
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef ITPP_H
#define ITPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct itpp_ctx* itpp_handle;
typedef struct itpp_batch_ctx* itpp_batch_handle;

typedef enum {
    ITPP_OK = 0,
    ITPP_ERR_ARG = 1,         /* invalid argument (checked on the host)            */
    ITPP_ERR_ALLOC = 2,       /* a device or host allocation failed                */
    ITPP_ERR_CAPACITY = 3,    /* more terms than cap_M with cap_policy 0, or a
                                 buffer would overflow                              */
    ITPP_ERR_HASH_PROBE = 4,  /* the merge table's probe limit was reached          */
    ITPP_ERR_TIMEOUT = 5,     /* a device-side wait gave up (bounded spin)          */
    ITPP_ERR_TRACE_ZERO = 6,  /* the identity coefficient was truncated or is
                                 missing, so the trace cannot be normalised         */
    ITPP_ERR_CUDA = 7,        /* a CUDA runtime call failed                         */
    ITPP_ERR_STATE = 8,       /* call not valid in the handle's current state       */
    ITPP_ERR_IO = 9           /* a state file could not be opened, read or written,
                                 or is not a state of this handle's n             */
} itpp_status;

/* Propagation parameters.  Zero-initialise and set what you need. */
typedef struct {
    /* Coefficient threshold: after each gate keep a term iff |c| > delta
     * (Sec. II.B "Coefficient threshold"; Algorithm 1, "Truncate").  The test
     * is applied to the merged coefficients before the trace normalisation.
     * Must be >= 0; 0 keeps every nonzero coefficient. */
    double delta;
    /* Term bound (Sec. II.C, "Practical considerations"): the most terms the
     * state may hold after a gate.  Sizes the device buffers
     * (2 * cap_M terms each, two of them) and the merge table. >= 1. */
    uint64_t cap_M;
    /* 0: a gate that leaves more than cap_M terms is an ITPP_ERR_CAPACITY
     *    error ("terminating").
     * 1: keep the cap_M largest |c| (ties: ascending key, words x[0..W-1]
     *    then z[0..W-1] compared as unsigned), the K-truncation of Sec. II.C
     *    applied only when the bound is exceeded ("adapting").  With
     *    delta = 0 this is the paper's K-truncation proper (K = cap_M, the K
     *    largest coefficients after every step); each step that dropped
     *    terms counts in itpp_stats.cap_events. */
    int cap_policy;
    /* How the children of equal strings are found and summed; every path
     * gives bit-identical states.
     * 0: partitioned merge (default): the state is scattered into hash
     *    partitions of the key with a window's sites cleared (consecutive
     *    gates acting on a few sites share one scatter) or of the pair key
     *    {K, Q.K}, and each partition is merged through an open-addressing
     *    table in shared memory.
     * 1: sort fallback: the commuting terms' children are radix-sorted on
     *    the whole key (8-bit digits, digits above bit n skipped) and runs of
     *    equal keys are summed by a segmented reduce; anticommuting terms,
     *    which never share a string with another child, bypass the sort.
     *    Needs a scratch of about 2 * (2 cap_M) children.
     * 2: one open-addressing table in global memory for the whole state. */
    int merge_path;
    /* Tuning (0 = library default or the autotuned value):
     * table_load_pct: highest load of the merge table, in percent (10..75).
     * block_threads: threads per CTA of the gate kernels (128, 256, 512).
     * items_per_thread: terms per thread per tile (1, 2, 4; the partitioned
     * merge holds at most two). */
    int table_load_pct;
    int block_threads;
    int items_per_thread;
    /* Pauli weight cutoff (Sec. II.B, "Pauli weight cutoff"): after every
     * gate, also drop the strings with more than max_weight non-identity
     * letters (popc(x | z) > max_weight), together with the |c| > delta
     * test; the identity (weight 0) always stays.  0: no cutoff; 0..128. */
    int max_weight;
    /* Product formula of a Trotter layer (Sec. II.C): 1 (default, or 0) the
     * first-order product of the gates in order; 2 the symmetric second-order
     * (Strang) product, gates 1..G-1 with half angles, gate G with the full
     * angle, then gates G-1..1 with half angles (2G-1 elementary gates per
     * layer; itpp_apply_gate indexes that schedule, while itpp_set_alpha and
     * itpp_adjoint keep taking and returning the G coefficients). */
    int trotter_order;
    /* Partitioned merge (merge_path 0): the mean partition size the scatter
     * aims for, 64..2048 terms (0: the library default).  Larger partitions
     * amortise the per-partition work; a partition above one CTA's staging
     * capacity (1,024 terms at W = 1, 512 at W = 2) is merged in slower
     * sub-passes. */
    int partition_target;
    int reserved[2];
} itpp_params;

/* Counters kept on the device and read by itpp_get_stats (synchronising). */
typedef struct {
    uint64_t gates_applied;   /* elementary gates since create / last load      */
    uint64_t terms_in;        /* sum over gates of the input term count N_in    */
    uint64_t terms_out;       /* sum over gates of the kept term count          */
    uint64_t peak_terms;      /* largest kept term count after any gate         */
    uint64_t cap_events;      /* gates where the cap_M bound fired              */
    uint64_t count;           /* current term count                             */
    uint64_t table_probes;    /* merge-table slots visited (build + lookups)    */
    uint64_t kernel_launches; /* kernels this handle has launched (host count)  */
    uint64_t repartitions;    /* partitioned merge: scatters run (window starts,
                               * state changes, gates partitioned by pair key)   */
    uint64_t select_candidates; /* top-M selects: terms listed around the
                                 * threshold, summed over gates                  */
    uint64_t select_range;    /* last top-M select: width of the |c| pattern range
                               * its candidates were listed from                 */
    uint64_t select_full;     /* top-M selects that passed over every stored
                               * coefficient (the threshold lay outside the range
                               * the merge listed, or no range was known yet)    */
    uint64_t long_partitions; /* partitioned merge: partitions above one CTA's
                               * staging capacity, merged in sub-passes          */
    uint64_t error_site;      /* where the first device error was raised (a code
                               * of the library's kernels; 0 while status is ok),
                               * reported together with the status by
                               * itpp_get_stats even when the status is an error */
    uint64_t merge_retries;   /* partitioned merge with top-M: gates whose merge
                               * ran twice (it leaves children below the select's
                               * predicted range unwritten, and runs again in full
                               * when fewer than cap_M children were kept)        */
} itpp_stats;

/* ---------------------------------------------------------------------------
 * Lifetime
 * ------------------------------------------------------------------------- */

/* Create a propagation of the Hamiltonian H = sum_k alpha_k Q_k
 * (Algorithm 1, "Input"), with gates applied in the given order inside every
 * Trotter layer.  The gate of term k is V_k = exp(-(dtau/2) alpha_k Q_k)
 * (Sec. II.C, first-order Trotter product), whose propagation rule
 * (Eq. (ITPP_PropRules)) uses the angle theta_k = alpha_k * dtau; the host
 * computes cosh(theta_k) and sinh(theta_k) once here.  The state starts as
 * the identity operator (Algorithm 1, "Initialize rho = I"; Sec. II.C: the
 * 1/2^n of the maximally mixed state cancels).
 *   n           number of sites, 1..128.
 *   gate_x/z    host, n_gates * W words each, row-major; bits >= n zero.
 *   alpha       host, n_gates real coefficients.
 *   dtau        Trotter step, finite.
 *   p           host; copied.  NULL is ITPP_ERR_ARG.
 *   cuda_stream cudaStream_t to run on (NULL = the legacy default stream).
 *   out         receives the handle; untouched on error.
 * Errors: ITPP_ERR_ARG (bad sizes, bits >= n, delta < 0, cap_M == 0,
 * non-finite alpha or dtau), ITPP_ERR_ALLOC, ITPP_ERR_CUDA. */
itpp_status itpp_create(int n, const uint64_t* gate_x, const uint64_t* gate_z,
                        const double* alpha, int n_gates, double dtau,
                        const itpp_params* p, void* cuda_stream, itpp_handle* out);

/* Free every device and host resource of the handle (synchronises its
 * stream first).  NULL is accepted. */
itpp_status itpp_destroy(itpp_handle h);

/* ---------------------------------------------------------------------------
 * The hot path
 * ------------------------------------------------------------------------- */

/* Apply n_layers Trotter layers (Algorithm 1, loop over Trotter steps): for
 * every gate in order, each term P with coefficient c becomes
 *   P (coefficient c)                              if {P, Q} = 0,
 *   cosh(theta) c P  and  -sinh(theta) c (Q P)     if [P, Q] = 0
 * (Eq. (ITPP_PropRules), derived in App. A), where Q P = s R with s = +-1 and
 * R the string (xQ^xP, zQ^zP); children with the same string are summed
 * (Algorithm 1, "Accumulate"), terms with |c| <= delta are dropped, the cap
 * policy is applied, and every coefficient is divided by the identity's
 * ("Truncate and normalize", Sec. II.C per-step trace normalisation).
 * Asynchronous.  n_layers >= 0. */
itpp_status itpp_apply_trotter_layer(itpp_handle h, int n_layers);

/* Apply the single gate k (0 <= k < n_gates) of the Trotter order; the same
 * elementary step as inside itpp_apply_trotter_layer.  Asynchronous. */
itpp_status itpp_apply_gate(itpp_handle h, int k);

/* Reset the state to the identity operator (Algorithm 1, "Initialize
 * rho = I") and clear the statistics and a stored device error.
 * Asynchronous. */
itpp_status itpp_reset(itpp_handle h);

/* Threshold truncation of the current (normalised) state: keep |c| > delta,
 * then renormalise (Sec. II.B "Coefficient threshold"; Algorithm 1
 * "Truncate and normalize").  delta >= 0; a delta >= 1 would drop the
 * identity and is ITPP_ERR_TRACE_ZERO.  Asynchronous. */
itpp_status itpp_truncate(itpp_handle h, double delta);

/* Expectation value <O> = Tr[O rho] / Tr[rho] = sum_j w_j c_{P_j} of
 * O = sum_j w_j P_j (Sec. II.C, expectation from the propagated operator;
 * Tr(P_a P_b) = 2^n delta_ab and the identity coefficient is one).
 *   obs_x/z  host, m * W words; obs_w host, m weights; 1 <= m <= 65536.
 *   out      host; receives <O>.
 * Synchronising.  The sum over j is compensated (Kahan). */
itpp_status itpp_expect(itpp_handle h, const uint64_t* obs_x, const uint64_t* obs_z,
                        const double* obs_w, int m, double* out);

/* Expectation value of the positive-semidefinite restored state (Sec. II.C,
 * squaring the approximate operator): <O>_{2 tau} ~= Tr[(O rho) rho] /
 * Tr[rho^2], the estimate at imaginary time 2 tau from the state at tau.
 * The product O rho is never expanded: only commuting pairs contribute,
 * Tr[(O rho) rho] / 2^n = sum_j w_j sum_{[P,O_j]=0} s(O_j,P) c_P c_{O_j P},
 * found by a lookup of O_j.P in a hash table of the state; the purity
 * Tr[rho^2] / 2^n is the squared l2 norm of the coefficients.
 *   obs_x/z, obs_w  host, as itpp_expect; 1 <= m <= 65536.
 *   out             host, three doubles: <O>_{2 tau}, Tr[(O rho) rho] / 2^n,
 *                   Tr[rho^2] / 2^n.
 * Cost: one table build plus m commutation tests per term.  Uses the merge
 * table's memory (cleared first); the state is unchanged.  Synchronising;
 * sums are compensated (Kahan) and reduced in a fixed order. */
itpp_status itpp_expect_psd(itpp_handle h, const uint64_t* obs_x, const uint64_t* obs_z,
                            const double* obs_w, int m, double* out);

/* The coefficient c_{P_j} of each string (0 where the string is absent).
 * Host arrays; out has m entries.  Synchronising. */
itpp_status itpp_coeffs(itpp_handle h, const uint64_t* obs_x, const uint64_t* obs_z,
                        int m, double* out);

/* Device-pointer form of itpp_coeffs + itpp_expect, fully asynchronous:
 * d_obs_x/z (m*W words), d_obs_w (m) and d_out (m+1 doubles: the m
 * coefficients, then the weighted sum) are device memory that must stay valid
 * until the stream reaches the work. */
itpp_status itpp_expect_device(itpp_handle h, const uint64_t* d_obs_x, const uint64_t* d_obs_z,
                               const double* d_obs_w, int m, double* d_out);

/* ---------------------------------------------------------------------------
 * State access
 * ------------------------------------------------------------------------- */

/* Wait for the stream and return the handle's status. */
itpp_status itpp_synchronize(itpp_handle h);

/* Current number of terms.  Synchronising. */
itpp_status itpp_get_count(itpp_handle h, uint64_t* count);

/* Copy the current normalised state to host buffers x, z (capacity * W words
 * each) and c (capacity doubles).  The order of the terms is unspecified.
 * *count receives the term count; ITPP_ERR_CAPACITY if capacity < count
 * (nothing copied).  Synchronising. */
itpp_status itpp_get_terms(itpp_handle h, uint64_t* x, uint64_t* z, double* c,
                           uint64_t capacity, uint64_t* count);

/* Replace the state by count terms from host buffers (checkpoint resume,
 * synthetic states).  Keys must be distinct, bits >= n zero, and the
 * identity must be present with a nonzero coefficient; count <= cap_M.
 * Clears the stored device status.  Synchronising. */
itpp_status itpp_set_terms(itpp_handle h, const uint64_t* x, const uint64_t* z,
                           const double* c, uint64_t count);

/* Sort count terms held in host arrays into the canonical order: ascending
 * by x word 0, x word 1, ..., then z word 0, z word 1, ... (unsigned 64-bit
 * comparisons), the (x, z, c) triple of a term moving together.  This is the
 * order in which exported states are compared term by term.  Equal keys keep
 * an unspecified relative order (a state has none).  Runs on the host only:
 * no handle, no device.  x, z: count * W words each, c: count doubles, all
 * in place.  Errors: ITPP_ERR_ARG (W not 1 or 2; a NULL array with
 * count > 0), ITPP_ERR_ALLOC (the host scratch, 8 + 16W bytes a term). */
itpp_status itpp_sort_terms(int W, uint64_t* x, uint64_t* z, double* c, uint64_t count);

/* itpp_get_terms, then itpp_sort_terms on the copied terms: the normalised
 * state in the canonical order.  Arguments and errors as itpp_get_terms
 * (plus ITPP_ERR_ALLOC).  Synchronising. */
itpp_status itpp_get_terms_sorted(itpp_handle h, uint64_t* x, uint64_t* z, double* c,
                                  uint64_t capacity, uint64_t* count);

/* Checkpoint the normalised state to a file (resume with itpp_load).  The
 * file holds, little-endian: the 8 bytes "ITPPST01", int32 n, int32 W,
 * uint64 count, then the x words (count * W uint64), the z words (same)
 * and the coefficients (count doubles), terms in the canonical order of
 * itpp_sort_terms, so equal states give equal files.  path: host string.
 * Errors: ITPP_ERR_ARG (NULL handle or path), ITPP_ERR_IO, ITPP_ERR_ALLOC,
 * the handle's stored error.  Synchronising. */
itpp_status itpp_save(itpp_handle h, const char* path);

/* Replace the state by the one a file written by itpp_save holds (the same
 * n is required; the gates, dtau and parameters stay those of h), as
 * itpp_set_terms does; continuing from a loaded state gives the same terms
 * and coefficients, bit for bit, as continuing the saved handle.  Errors:
 * ITPP_ERR_ARG (NULL arguments), ITPP_ERR_IO (unreadable, truncated, wrong
 * magic, another n or W, more than cap_M terms), the errors of
 * itpp_set_terms.  Synchronising. */
itpp_status itpp_load(itpp_handle h, const char* path);

/* Device counters (see itpp_stats).  Synchronising. */
itpp_status itpp_get_stats(itpp_handle h, itpp_stats* out);

/* Kernel timing with CUDA events recorded on the handle's stream around the
 * launches of the gate kernels.  itpp_profile_enable(h, 1) starts (and
 * clears) the accumulation; itpp_profile_read synchronises and returns, for
 * kernel class kid, the number of launches and their total device time in
 * milliseconds.  kid 0: the state scatter (merge_path 0) or the global
 * merge-table build (merge_path 2); 1: branch-emit-merge-truncate (the whole
 * sorted merge for merge_path 1); 2: the top-M select; 3: expectation. */
itpp_status itpp_profile_enable(itpp_handle h, int enable);
itpp_status itpp_profile_read(itpp_handle h, int kid, uint64_t* launches, double* total_ms);

/* ---------------------------------------------------------------------------
 * Gradients (adjoint of the frozen-support propagation)
 * ------------------------------------------------------------------------- */

/* Replace the gate coefficients alpha_k (n_gates values, host) of a handle;
 * the host recomputes the per-gate weights.  The state is unchanged. */
itpp_status itpp_set_alpha(itpp_handle h, const double* alpha);

/* Gradient of f = sum_j w_j c_{P_j}(beta) with respect to every gate
 * coefficient alpha_k, where c is the normalised state after n_layers Trotter
 * layers from the identity and the kept support of every elementary step is
 * held at what the forward produced ("frozen support").  The paper has no
 * such step; it is the linear algebra of Eq. (ITPP_PropRules) and the
 * per-step trace normalisation (Sec. II.C), evaluated by a reverse sweep.
 * The call resets the handle to the identity, runs the forward (saving a
 * snapshot every ckpt_every layers), then for each segment from the last
 * recomputes its steps from the snapshot and sweeps them backwards.
 *   obs_x/z, w   host, m observable strings and weights (w_j = df/dc_{P_j}).
 *   grad_alpha   host, n_gates: df/dalpha_k summed over the layers.
 *   value        host or NULL: f.
 * The kept support includes the term bound: with cap_policy 1 the frozen
 * support of a step is its top-M set.  Device memory: one snapshot per
 * segment plus, for every step of the largest segment, its output before and
 * after the bound and four int32 maps, allocated for the call.  After the call the handle
 * holds the forward's final state.  Synchronising. */
itpp_status itpp_adjoint(itpp_handle h, int n_layers, int ckpt_every, const uint64_t* obs_x,
                         const uint64_t* obs_z, const double* w, int m, double* grad_alpha,
                         double* value);

/* The frozen-support forward that itpp_adjoint differentiates, evaluated at
 * other coefficients: the kept support of every step is the one the handle's
 * own coefficients produce (as in itpp_adjoint), and the linear maps of the
 * propagation rule (Eq. (ITPP_PropRules)) and the per-step trace
 * normalisation (Sec. II.C) on it are applied with
 * theta = alpha_eval[k] * dtau.  value receives f = sum_j w_j c_{P_j} after
 * n_layers layers from the identity.  The paper has no counterpart: this is
 * the function whose derivative at alpha_eval = alpha the adjoint returns,
 * so that a central difference of it checks the gradient at any size.
 * alpha_eval: host, one finite value per Hamiltonian term.  Other arguments,
 * memory, state and synchronisation as itpp_adjoint. */
itpp_status itpp_frozen_value(itpp_handle h, int n_layers, int ckpt_every,
                              const double* alpha_eval, const uint64_t* obs_x,
                              const uint64_t* obs_z, const double* w, int m, double* value);

/* ---------------------------------------------------------------------------
 * Batched propagation: many independent instances in shared launches
 * ------------------------------------------------------------------------- */

/* Create B independent propagations (Algorithm 1 for each), advanced
 * together: in every Trotter layer, gate g of every instance that has one
 * runs in the same kernel launches, and the whole layer is one CUDA graph
 * launch.  Each instance's state is bit-identical to a plain run of the same
 * Hamiltonian with the same parameters.  p->merge_path 0 (default): every
 * gate scatters each instance's terms into hash partitions of its pair key
 * and merges the partitions of all instances in one launch of the
 * shared-memory merge (p->partition_target as in itpp_create); 2: one global
 * merge table per instance; 1 is not offered for batches (ITPP_ERR_ARG).
 *   B            1..65535 instances.
 *   n[B]         sites per instance (1..128); all instances use
 *                W = ceil(max n / 64) mask words.
 *   n_gates[B]   gates per layer per instance (instances with fewer gates sit
 *                out the later steps of a layer).
 *   gate_x/z     host, concatenated over instances in order (instance b's
 *                gates follow instance b-1's), W words per gate.
 *   alpha        host, concatenated likewise.
 *   dtau, p      as in itpp_create; cap_M bounds every instance separately.
 *   cuda_stream  stream to run on; NULL makes the library create its own
 *                (graph capture needs a non-legacy stream).
 * Memory: per instance two buffers of 2*cap_M terms, a table and a control
 * block (about 0.6 MB), and for merge_path 0 a scatter buffer of about
 * 2.5*cap_M terms.  Errors: as itpp_create. */
itpp_status itpp_batch_create(int B, const int* n, const int* n_gates, const uint64_t* gate_x,
                              const uint64_t* gate_z, const double* alpha, double dtau,
                              const itpp_params* p, void* cuda_stream, itpp_batch_handle* out);
itpp_status itpp_batch_destroy(itpp_batch_handle h);

/* n_layers Trotter layers for every instance.  Asynchronous.  An instance
 * that meets a device error (bound, probe limit) stops; the others go on. */
itpp_status itpp_batch_apply_trotter_layer(itpp_batch_handle h, int n_layers);

/* Wait; ITPP_OK if every instance is healthy, else the first error. */
itpp_status itpp_batch_synchronize(itpp_batch_handle h);

/* The launch shape of a batch, chosen by timing (the autotuner of the
 * batched path).  Partitioned merge (merge_path 0): threads per CTA of the
 * partition merge (128, 256, 512), its CTAs per SM (2, 4, or as many as fit),
 * the scatter's CTAs per SM (4, 8, 16) and the mean partition size (350,
 * 500, 700, 1000 terms at W = 1; 150, 300, 450 at W = 2; not tried when
 * itpp_batch_create was given a partition_target).  Global table
 * (merge_path 2): threads per CTA of the branch-emit kernel (128, 256, 512;
 * two terms per thread), its CTAs per SM (2, 4, 8), the table build's CTAs
 * per SM (4, 8, 16) and the merge table's highest load (25..65 %;
 * itpp_batch_create with table_load_pct 0 sizes the tables for 25 %,
 * otherwise loads below the requested one are not tried).
 * Each candidate is timed with CUDA events over probe_layers Trotter layers
 * from the identity, replayed as the layer graph; coordinate descent from
 * the default shape, one parameter at a time.  The fastest shape stays
 * installed.  Every instance is reset to the identity before each timing
 * and after the search (statistics cleared), so results never depend on the
 * tuning: every shape gives bit-identical states.  Synchronising.
 *   probe_layers  >= 1.
 *   out           host, may be NULL. */
typedef struct {
    int main_block;              /* threads per CTA of the merge kernel          */
    int main_grid;               /* its CTAs per SM                              */
    int insert_grid;             /* CTAs per SM of the scatter / table build     */
    int table_load_pct;          /* global table: highest load (%); else 0       */
    double ms_per_probe;         /* the chosen shape: probe_layers layers (ms)   */
    double ms_per_probe_default; /* the default shape (partitioned: 256 threads,
                                  * as many CTAs as fit, 8, the default size;
                                  * global table: 256, 4, 8, 50 %)              */
    int candidates;              /* shapes timed                                 */
    int partition_target;        /* partitioned: mean partition size; else 0     */
    int reserved[2];
} itpp_tune_result;
itpp_status itpp_batch_autotune(itpp_batch_handle h, int probe_layers, itpp_tune_result* out);

/* Term count (and, when statuses != NULL, the status) of every instance;
 * host arrays of B entries.  Synchronising. */
itpp_status itpp_batch_get_counts(itpp_batch_handle h, uint64_t* counts, int* statuses);

/* Instance b: statistics, normalised terms (as itpp_get_terms) and an
 * expectation value (as itpp_expect).  Synchronising. */
itpp_status itpp_batch_get_stats(itpp_batch_handle h, int b, itpp_stats* out);
itpp_status itpp_batch_get_terms(itpp_batch_handle h, int b, uint64_t* x, uint64_t* z,
                                 double* c, uint64_t capacity, uint64_t* count);
itpp_status itpp_batch_expect(itpp_batch_handle h, int b, const uint64_t* obs_x,
                              const uint64_t* obs_z, const double* obs_w, int m, double* out);

/* ---------------------------------------------------------------------------
 * One gate without device allocation
 * ------------------------------------------------------------------------- */

/* Largest input term count of itpp_gate_apply_noalloc for W = ceil(n/64)
 * mask words: its merge table is a fixed 16 MiB, filled at most half. */
#define ITPP_NOALLOC_MAX_TERMS(W) ((W) == 1 ? 262144ULL : 131072ULL)

/* One elementary gate (the same step as itpp_apply_gate: propagate, merge,
 * truncate |c| > delta, rescale by the identity coefficient) on buffers the
 * caller owns, allocating nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc at that point -- code
 * running inside a memory pool or arena that owns all device memory, or a
 * host path that must not pay the implicit synchronisation of cudaMalloc /
 * cudaFree.  Its scratch (merge table and control block, about 17 MiB) is a
 * file-scope device array that every GPU loading the library holds until the
 * process exits; no cudaMalloc, cudaFree or allocating library routine is
 * called.
 *   n, gate_x, gate_z  sites and the gate string Q (host, W words each).
 *   alpha, dtau        Q's coefficient and the step: theta = alpha * dtau.
 *   delta              threshold (>= 0).
 *   d_keys_in          device, n_in terms, each 2W words: x[0..W-1] then
 *                      z[0..W-1]; distinct strings, the identity present
 *                      (an input without it is reported through d_n_out).
 *   d_coef_in          device, n_in finite normalised coefficients (the
 *                      identity's is taken as exactly one).
 *   n_in               1 .. ITPP_NOALLOC_MAX_TERMS(W); larger is
 *                      ITPP_ERR_CAPACITY.
 *   d_keys_out/_coef_out  device, room for out_capacity >= 2 * n_in terms
 *                      (smaller is ITPP_ERR_CAPACITY); receive the kept terms
 *                      in an unspecified order, normalised.
 *   d_n_out            device, receives the kept count, or UINT64_MAX when a
 *                      device-side error (merge-table probe limit, identity
 *                      truncated or absent from the input) occurred.
 *   d_trace_out        device or NULL: the identity coefficient before the
 *                      rescaling.
 *   cuda_stream        stream to run on.
 * Asynchronous.  The first call on a device looks up the scratch's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Under CUDA's lazy module loading (the
 * default), that first call may also be what loads this library's module on
 * the device and sets the scratch aside, which allocates device memory and
 * can synchronise: a caller that must not allocate makes one warm-up call
 * (or creates any handle of this library) on each device before entering its
 * allocation-free region.  All calls share the scratch and it keeps the last
 * call's contents (each call takes a fresh generation of the merge table, and
 * the table is cleared once when the 32-bit generation wraps): calls whose
 * work overlaps on the GPU race and corrupt each other; serialise them. */
itpp_status itpp_gate_apply_noalloc(int n, const uint64_t* gate_x, const uint64_t* gate_z,
                                    double alpha, double dtau, double delta,
                                    const uint64_t* d_keys_in, const double* d_coef_in,
                                    uint64_t n_in, uint64_t* d_keys_out, double* d_coef_out,
                                    uint64_t out_capacity, uint64_t* d_n_out,
                                    double* d_trace_out, void* cuda_stream);

/* Human-readable name of a status code (static storage). */
const char* itpp_status_string(itpp_status s);

/* Library version, e.g. "itpp-gb300 0.1". */
const char* itpp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ITPP_H */
