/*
 * bf.h -- C ABI of libbf: exhaustive low-spectrum search for Ising spin
 * glasses on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Jalowiecki, Rams, Gardas, "Brute-forcing spin-glass problems with
 * CUDA", Sec. 2, Eq. (1), and Algorithm 1 of Sec. 3): for an Ising instance on
 * n spins s_i in {-1, +1}, evaluate
 *
 *     E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i
 *
 * for all 2^n configurations and return the S lowest (energy, configuration)
 * pairs.  The paper's H of Eq. (1) carries an overall minus sign; negate J and
 * h to obtain it.
 *
 * Conventions (fixed by this library where the paper is silent):
 *   - Configuration integer (Sec. 3, Eqs. (4)-(5)): c = sum_i q_i 2^i with
 *     q_i = (s_i + 1) / 2, i.e. bit i of c (least significant bit = spin 0)
 *     is 1 iff s_i = +1.  n <= 64.
 *   - J is a dense row-major n x n matrix; only its strict upper triangle
 *     (i < j) is read.  The diagonal and lower triangle are ignored.
 *   - Output order: ascending energy, ties broken by ascending c.  The result
 *     is therefore unique.
 *   - Integer instances (BF_I32) are exact.  Float instances (BF_F32, BF_F64)
 *     are screened in exact fixed point with a rigorous quantisation bound and
 *     every surviving candidate is re-evaluated from the input values: an FP64
 *     sum of Eq. (1), or (spaces of at most 2^20 configurations, the batched
 *     search) the quantised energy plus the rounding residuals summed exactly in
 *     64-bit fixed point and rounded once to FP64.  Returned energies are FP64
 *     values of Eq. (1) and the final order is taken on them.
 *
 * Memory and streams: every pointer argument named "device" is device memory
 * owned by the caller and must stay valid until the work queued on `stream`
 * has completed.  The library never allocates device memory: the caller
 * provides a workspace of at least bf_*_workspace_size() bytes, aligned to
 * 256 bytes.  Calls on one workspace must not overlap in time.  The library
 * keeps per-device state for the life of the process (kernel attributes,
 * events that order its constant tables between streams): after a
 * cudaDeviceReset() of a device it must not be used on that device again.
 *
 * Errors: argument errors are detected on the host before anything is
 * launched and reported by the return value.  Conditions found on the device
 * (candidate storage exhausted) are recorded in the workspace and returned by
 * bf_workspace_status(), which synchronises the stream.  On any error the
 * outputs are undefined.  bf_last_error_detail() gives a per-thread message.
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BF_OK = 0,
    BF_EINVAL = 1,        /* invalid argument (detected on the host) */
    BF_ECUDA = 2,         /* a CUDA runtime call failed */
    BF_EOVERFLOW = 3,     /* candidate storage in the workspace exhausted */
    BF_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    BF_EUNSUPPORTED = 5,  /* valid but outside what this build supports */
    BF_EWORKSPACE = 6     /* workspace too small or misaligned */
} bf_status;

typedef enum {
    BF_I32 = 0,  /* int32 couplings and fields; energies returned as int64 */
    BF_F32 = 1,  /* float couplings and fields; energies returned as double */
    BF_F64 = 2   /* double couplings and fields; energies returned as double */
} bf_dtype;

/* Screening kernel choice for bf_low_spectrum. */
typedef enum {
    BF_VARIANT_AUTO = 0,   /* library default (Gray-code walk) */
    BF_VARIANT_GRAY = 1,   /* Gray-code walk: exact int32 fixed point with a
                              two-lane 16-bit pre-filter, one flip per step */
    BF_VARIANT_TC = 2      /* tensor-core screening: 128 x 256 energies per
                              tcgen05 MMA (BF16 hi+lo splits, FP32 accumulation),
                              exact int32 rescans; needs n - fixed_bits >= 15 */
} bf_variant;

/*
 * Options; a NULL pointer or zero fields select the defaults.
 *   variant      one of bf_variant
 *   fixed_bits   number of most significant configuration bits held fixed
 *                (0 = enumerate all 2^n); the enumerated subspace is
 *                c = (fixed_value << (n - fixed_bits)) + x, x in [0, 2^(n-fixed_bits)),
 *                the paper's chunk offset of Sec. 3, Eq. (6)
 *   fixed_value  value of those bits, < 2^fixed_bits
 *   task_log2    log2 of the number of configurations one thread walks
 *                per task (0 = automatic)
 *   grid_blocks  persistent grid size of the enumeration kernel (0 = automatic)
 *   spill_log2   log2 of the number of spill records in the workspace
 *                (0 = default 21); a smaller area makes BF_EOVERFLOW reachable
 *                in tests
 *   profile      nonzero: record CUDA events around the enumeration kernel on
 *                the call's stream (read back with bf_last_profile)
 *   stall_test   testing only: nonzero makes the tensor-core kernel's MMA warps
 *                issue nothing, so the epilogue's bounded waits (0.2 s) run out;
 *                the kernel then stops, frees its tensor memory and the call's
 *                workspace status is BF_ETIMEOUT.  The CUDA context stays
 *                usable.  Ignored by the other kernels.
 *   inner_bits   spins walked by the fully unrolled block of the Gray-code walk:
 *                0 = automatic (10 for searches of at least 2^42 configurations
 *                and 9 below; spaces of at most 2^20 configurations are then
 *                enumerated exactly by the small-space kernels, without a walk), or 9 or
 *                10 (10 needs n >= 14), which always walks.  Results do not
 *                depend on it.  Ignored by the tensor-core variant.
 * When variant, inner_bits, task_log2 and grid_blocks are all 0 and bf_autotune
 * has run for this device and (n, n - fixed_bits, S, dtype), its choice is used.
 */
typedef struct {
    int32_t variant;
    int32_t fixed_bits;
    uint64_t fixed_value;
    int32_t task_log2;
    int32_t grid_blocks;
    int32_t spill_log2;
    int32_t profile;
    int32_t stall_test;
    int32_t inner_bits;
    int32_t reserved[4];
} bf_options;

/* Largest S accepted by bf_low_spectrum. */
#define BF_MAX_S 2048

/*
 * Workspace bytes needed by bf_low_spectrum for (n, S, dtype, options).
 * Returns 0 for arguments bf_low_spectrum would reject.
 */
size_t bf_workspace_size(int n, int S, bf_dtype dtype, const bf_options* opt);

/*
 * bf_low_spectrum -- the S lowest (energy, configuration) pairs of one
 * instance (Algorithm 1, Sec. 3; energy of Eq. (1), Sec. 2).
 *   J          device, n*n values of `dtype`, row-major; strict upper triangle read
 *   h          device, n values of `dtype`
 *   n          number of spins, 1 <= n <= 64; n - fixed_bits <= 62
 *   S          number of states returned, 1 <= S <= min(BF_MAX_S, 2^(n-fixed_bits))
 *   energies   device out, S values: int64 for BF_I32, double otherwise
 *   states     device out, S configuration integers
 *   workspace  device, >= bf_workspace_size(...) bytes, 256-byte aligned
 *   stream     cudaStream_t (NULL = legacy default stream)
 * Queues the whole search on `stream` and returns without synchronising
 * (BF_OK when the work was queued); the call can be captured in a CUDA graph
 * and replayed with new values in J and h (same n, S, dtype and options).
 * Instances outside the int32 fixed-point range are reported by
 * bf_workspace_status (BF_EUNSUPPORTED).
 * Zero fields: when every h_i is 0, E(c) = E(~c); a search over the whole
 * space (fixed_bits = 0) of more than 2^20 configurations with the Gray walk
 * and S <= 1 + n + n(n-1)/2 then enumerates only the configurations with spin
 * n-1 at -1 and adds the mirrors c ^ (2^n - 1) to the result.  The output is
 * the same as that of the full enumeration.
 * Streams: the enumeration kernel reads its per-instance step increments from
 * one table per device, which the call fills from the workspace just before
 * the kernel.  Searches queued on different streams are ordered around that
 * table by the library (the next fill waits for the previous enumeration
 * kernel on the device).  Work queued while a stream is being captured is not
 * ordered that way: a graph holding this call must not run at the same time
 * as another search on the same device.
 */
bf_status bf_low_spectrum(const void* J, const void* h, int n, int S, bf_dtype dtype,
                          void* energies, uint64_t* states,
                          void* workspace, size_t workspace_bytes,
                          const bf_options* opt, void* stream);

/*
 * bf_autotune -- choose the screening kernel and launch shape of bf_low_spectrum
 * for one search size by timing candidates on this GPU (CUDA events on
 * `stream`), as the paper chooses its launch configuration by measurement
 * (Sec. 4.2).  Candidates: for spaces of at most 2^20 configurations the
 * exact small-space enumeration without a walk (the default there); the
 * Gray-code walk with 9 and 10 inner spins, the default task length
 * (task_log2) and lengths 2^2 and 2^4 shorter and 2^2 longer (at most 2^14
 * blocks per task), 1 or 2 blocks per SM; the tensor-core variant with three
 * task lengths where n - fixed_bits >= 15.  Each candidate runs
 * bf_low_spectrum's plan on J, h (arguments as for bf_low_spectrum; `base` supplies fixed_bits,
 * fixed_value and spill_log2, may be NULL).  Searches of more than 2^39
 * configurations time only the end of the task queue: at least 2^39
 * configurations and two batches of tasks per block (same task shape as the
 * full search), starting from the threshold an untimed run of the same part
 * reached, as most of a full search runs near its final threshold; a full
 * n = 48 tuning takes a few seconds.  Smaller searches run whole.  Candidates whose workspace exceeds
 * workspace_bytes are skipped (bf_workspace_size with default options fits
 * them all).  Writes the fastest options to *best (fixed_bits / fixed_value
 * as given) and, if best_rate is not NULL, its configurations per second, and
 * caches the choice for this device and (n, n - fixed_bits, S, dtype): later
 * bf_low_spectrum / bf_workspace_size calls that leave variant, inner_bits,
 * task_log2 and grid_blocks at 0 use it.  Results never depend on the choice.
 * If records is not NULL, up to records_cap candidates and their rates are
 * written there and *records_count (may be NULL) receives their number.
 * Synchronises the stream; energies / states / workspace hold no result
 * afterwards.
 */
typedef struct {
    bf_options opt;           /* a candidate */
    double configs_per_s;     /* its measured rate (0 if it did not run: workspace, overflow) */
} bf_tune_record;

bf_status bf_autotune(const void* J, const void* h, int n, int S, bf_dtype dtype, void* energies, uint64_t* states,
                      void* workspace, size_t workspace_bytes, const bf_options* base, void* stream,
                      bf_options* best, double* best_rate, bf_tune_record* records, int records_cap,
                      int* records_count);

/*
 * bf_low_spectrum_noalloc -- bf_low_spectrum for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is an
 * interface convenience.
 * Some callers must not allocate when they search: code running under a
 * framework whose caching allocator owns the free device memory, callbacks
 * and real-time loops where an allocation's implicit device synchronisation
 * is not acceptable, or hosts whose memory budget is fixed at start-up.  This
 * entry point takes inputs and outputs only (same meaning, layout and
 * ownership as bf_low_spectrum) and uses a workspace held in a 4 MiB device
 * array of the library, which every GPU that loads the library keeps until
 * the process exits.  It calls no cudaMalloc / cudaFree.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address once; make that first call before any stream
 *     capture.  The address is kept for the life of the process: after a
 *     cudaDeviceReset() of that device, which destroys the array with the
 *     context, this entry point must not be called again in the process.
 *   - Searches needing more than 4 MiB (at the default grid roughly S > 256,
 *     or a spill area larger than opt->spill_log2, default 16 here) return
 *     BF_EUNSUPPORTED without launching anything.
 *   - Every call shares the array: calls whose work overlaps on the GPU race
 *     and give undefined results.  Each call clears what it needs.
 *   - Unlike bf_low_spectrum, every call synchronises `stream`: it waits
 *     for its work to finish and returns the device-side status
 *     (BF_EOVERFLOW etc.) directly.
 */
bf_status bf_low_spectrum_noalloc(const void* J, const void* h, int n, int S, bf_dtype dtype,
                                  void* energies, uint64_t* states,
                                  const bf_options* opt, void* stream);

/* Limits of the batched search. */
#define BF_BATCHED_MIN_N 10
#define BF_BATCHED_MAX_N 32
#define BF_BATCHED_MAX_S 64

/*
 * Workspace bytes needed by bf_low_spectrum_batched for B instances of at most
 * n_max spins; 0 for arguments it would reject.
 */
size_t bf_batched_workspace_size(int B, int n_max, int S, bf_dtype dtype, const bf_options* opt);

/*
 * bf_low_spectrum_batched -- the S lowest (energy, configuration) pairs of
 * each of B independent instances (Algorithm 1, Sec. 3, applied per
 * instance; energy of Eq. (1), Sec. 2), in one persistent launch over an
 * (instance, chunk) work queue.
 *   J_packed   device, instance b's n[b] x n[b] row-major couplings start at
 *              element J_offsets[b] (strict upper triangle read)
 *   J_offsets  device, B element offsets (int64)
 *   h_packed   device, instance b's fields start at element h_offsets[b]
 *   h_offsets  device, B element offsets (int64)
 *   n          device, B spin counts, each in [BF_BATCHED_MIN_N, n_max]
 *   n_max      host, upper bound of n[] (<= BF_BATCHED_MAX_N); sizes the workspace
 *   S          1 <= S <= BF_BATCHED_MAX_S (and <= 2^n[b])
 *   energies   device out, B x S row-major: int64 for BF_I32, double otherwise
 *   states     device out, B x S configuration integers
 *   workspace  device, >= bf_batched_workspace_size(...) bytes, 256-byte aligned
 * opt->task_log2 sets log2 of the configurations per work unit (default 25),
 * opt->grid_blocks the persistent grid.  No host synchronisation and no
 * allocation: the call is capturable in a CUDA graph.  Instances with n out
 * of range are reported by bf_workspace_status as BF_EINVAL (their output
 * rows are left unwritten).  Instances with all h_i = 0 and n >= 11 enumerate
 * only the configurations with spin n-1 at -1 (E(c) = E(~c)); their rows
 * include the mirrors c ^ (2^n - 1) and equal those of the full enumeration.
 */
bf_status bf_low_spectrum_batched(int B, const void* J_packed, const int64_t* J_offsets,
                                  const void* h_packed, const int64_t* h_offsets, const int32_t* n,
                                  int n_max, int S, bf_dtype dtype, void* energies, uint64_t* states,
                                  void* workspace, size_t workspace_bytes, const bf_options* opt,
                                  void* stream);

/*
 * bf_autotune_batched -- pick the work-unit size (opt->task_log2) and the
 * persistent grid (opt->grid_blocks) of bf_low_spectrum_batched for this
 * batch by timing candidate launches (CUDA events on `stream`), as the
 * paper tunes its launch configuration by measurement (Sec. 4.2).  Arguments
 * as for bf_low_spectrum_batched; candidates whose workspace exceeds
 * workspace_bytes are skipped (size the workspace with task_log2 = 21 to
 * allow them all).  Writes the fastest options to *best and its time in ms to
 * *best_ms (may be NULL) and caches them for this device and (B, n_max, S,
 * dtype): later bf_low_spectrum_batched / bf_batched_workspace_size calls
 * that leave task_log2 and grid_blocks at 0 use the cached choice.  Runs the
 * batched search several times and synchronises the stream.
 */
bf_status bf_autotune_batched(int B, const void* J_packed, const int64_t* J_offsets, const void* h_packed,
                              const int64_t* h_offsets, const int32_t* n, int n_max, int S, bf_dtype dtype,
                              void* energies, uint64_t* states, void* workspace, size_t workspace_bytes,
                              void* stream, bf_options* best, float* best_ms);

/*
 * bf_low_spectrum_backward -- gradient of L = sum_b sum_k g[b,k] E_b(s^(b,k))
 * with respect to each instance's couplings and fields.  Eq. (1) (Sec. 2) is
 * linear in J and h, so dL/dJ_ij = sum_k g_k s_i s_j (i < j) and
 * dL/dh_i = sum_k g_k s_i over the given states (FP64 accumulation, k in
 * ascending order).
 *   states     device, B x S configuration integers (e.g. a forward's output)
 *   grad_E     device, B x S doubles (dL/dE of each returned energy)
 *   n          device, B spin counts (1..64)
 *   J_offsets  device, B int64 element offsets of each instance's n x n block in dJ
 *   h_offsets  device, B int64 element offsets of each instance's n fields in dh
 *   dJ, dh     device out, float or double per out_dtype (BF_F32 / BF_F64);
 *              entries on and below the diagonal of each dJ block are set to 0
 *   S          1 <= S <= 4096
 * No host synchronisation, no allocation; capturable.
 */
bf_status bf_low_spectrum_backward(const uint64_t* states, const double* grad_E, const int32_t* n, int B, int S,
                                   const int64_t* J_offsets, const int64_t* h_offsets, void* dJ, void* dh,
                                   bf_dtype out_dtype, void* stream);

/*
 * Workspace bytes needed by bf_low_spectrum_qubo; 0 for arguments it would
 * reject.
 */
size_t bf_qubo_workspace_size(int n, int S, bf_dtype dtype, const bf_options* opt);

/*
 * bf_low_spectrum_qubo -- the S lowest (value, configuration) pairs of the
 * QUBO form of the problem (Sec. 2, Eqs. (2)-(3)) over binary q in {0,1}^n:
 *
 *     F(q) = sum_{i<j} a_ij q_i q_j + sum_i b_i q_i
 *
 * (the paper's Eq. (2) with the overall sign flipped, as for Eq. (1)).  The
 * configuration integer is c = sum_i q_i 2^i, the paper's coding of Eq. (4);
 * ties are broken by ascending c.  The library maps the problem exactly onto
 * its Ising search: J'_ij = a_ij, h'_i = 2 b_i + sum_{j != i} a_ij (Eq. (3)
 * scaled by 4) and F = (E' + sum_{i<j} a_ij + 2 sum_i b_i) / 4.
 *   a          device, n*n values of `dtype`, row-major; strict upper triangle read
 *   b          device, n values of `dtype`
 *   F          device out, S values: int64 for BF_I32 (exact), double otherwise
 *   states     device out, S configuration integers (bit i = q_i)
 *   workspace  device, >= bf_qubo_workspace_size(...) bytes, 256-byte aligned
 * Other arguments and options as for bf_low_spectrum (float inputs are
 * converted to a double Ising instance first).  BF_I32 inputs whose
 * 2 b_i + sum_j a_ij leaves int32 are reported by bf_workspace_status
 * (BF_EUNSUPPORTED).  Like bf_low_spectrum the call does not synchronise.
 */
bf_status bf_low_spectrum_qubo(const void* a, const void* b, int n, int S, bf_dtype dtype, void* F, uint64_t* states,
                               void* workspace, size_t workspace_bytes, const bf_options* opt, void* stream);

/*
 * q-state Potts model -- one of the other classical spin-glass models to
 * which Sec. 2 says the method extends (its Ref. Wu82).  Energy, with the
 * same sign convention as Eq. (1) here:
 *
 *     E(sigma) = sum_{i<j} J_ij [sigma_i == sigma_j] + sum_i h_i(sigma_i),
 *
 * sigma_i in {0, ..., q-1}, 2 <= q <= 8, configuration integer
 * c = sum_i sigma_i q^i (base-q digits; the binary coding of Sec. 3, Eq. (4)
 * for q = 2).  q^n <= 2^62.  Ties are broken by ascending c.  For q = 2 the
 * model is an Ising instance: with J' = J, h'_i = h_i(1) - h_i(0) and
 * C = sum_{i<j} J_ij + sum_i (h_i(0) + h_i(1)), 2 E(sigma) = E'(s) + C, and
 * q = 2 searches above 4096 configurations run as that Ising search (integer
 * h_i(1) - h_i(0) outside int32: BF_EUNSUPPORTED from bf_workspace_status).
 *   J          device, n*n values of `dtype`, row-major; strict upper triangle read
 *   h          device, n*q values of `dtype`, row-major: h[i*q + v] = h_i(v)
 *   energies   device out, S values: int64 for BF_I32 (exact), double otherwise
 *              (every candidate re-evaluated in FP64, as for bf_low_spectrum)
 *   states     device out, S configuration integers
 *   workspace  device, >= bf_potts_workspace_size(...) bytes, 256-byte aligned
 * Options: task/grid/spill/profile fields as for bf_low_spectrum; fixed_bits
 * and the tensor-core variant are not supported (BF_EINVAL).  The call does
 * not synchronise (graph-capturable, with the same stream rule as
 * bf_low_spectrum for its per-device tables); instances outside the int32
 * fixed-point range are reported by bf_workspace_status (BF_EUNSUPPORTED).
 */
size_t bf_potts_workspace_size(int n, int q, int S, bf_dtype dtype, const bf_options* opt);

bf_status bf_low_spectrum_potts(const void* J, const void* h, int n, int q, int S, bf_dtype dtype, void* energies,
                                uint64_t* states, void* workspace, size_t workspace_bytes, const bf_options* opt,
                                void* stream);

/*
 * Resumable search (checkpoint / restart).  Algorithm 1 (Sec. 3) processes the
 * configuration space in chunks, c = offset + index (Eq. (6)), keeping the S
 * lowest records seen so far.  A cursor holds that state between chunks: the
 * 2^chunk_bits chunks are the subspaces whose top chunk_bits configuration
 * bits equal the chunk number, and the cursor records the next chunk and the
 * running list.  It is a caller-owned host buffer of bf_cursor_bytes(S)
 * bytes, self-describing and position independent (128-byte header with a
 * checksum, then S energies and S states), so it can be written to a file
 * and passed back after a restart.  The final list equals bf_low_spectrum's
 * result for the whole space (every candidate's energy is evaluated per
 * configuration, so chunking changes nothing).
 */

/* FNV-1a 64 digest of an instance (n, dtype, strict upper triangle of J, h); host memory. */
uint64_t bf_instance_digest(const void* J_host, const void* h_host, int n, bf_dtype dtype);

/* Bytes of a cursor for S states (0 if S is outside [1, BF_MAX_S]). */
size_t bf_cursor_bytes(int S);

/*
 * Initialises a cursor for an n-spin instance of `dtype` whose digest is
 * `digest` (bf_instance_digest), split into 2^chunk_bits chunks
 * (0 <= chunk_bits <= min(n, 40), S <= 2^(n - chunk_bits)).  Host only.
 */
bf_status bf_cursor_init(void* cursor, size_t cursor_bytes, int n, int S, bf_dtype dtype, int chunk_bits,
                         uint64_t digest);

/* Workspace bytes bf_cursor_step needs with these options (0 if rejected; fixed_bits must be 0). */
size_t bf_cursor_workspace_size(const void* cursor, size_t cursor_bytes, const bf_options* opt);

/*
 * Searches up to max_chunks further chunks on the GPU and merges each chunk's S
 * records into the cursor (host), which is consistent (checksum resealed)
 * after every chunk.  J, h: device, the instance the cursor was made for (its
 * digest is checked, after a device-to-host copy).  Synchronises the stream
 * after every chunk.  Device-side conditions are returned directly.
 */
bf_status bf_cursor_step(void* cursor, size_t cursor_bytes, const void* J, const void* h, int max_chunks,
                         void* workspace, size_t workspace_bytes, const bf_options* opt, void* stream);

/*
 * Reads a cursor (host): next chunk, number of chunks, and the current list
 * (count records, ascending by (E, c); int64 energies for BF_I32, double
 * otherwise).  Any output pointer may be NULL.
 */
bf_status bf_cursor_state(const void* cursor, size_t cursor_bytes, uint64_t* next_chunk, uint64_t* total_chunks,
                          void* energies_host, uint64_t* states_host, int* count);

/*
 * Synchronises `stream` and returns the status recorded on the device by the
 * last call that used `workspace` (BF_OK, BF_EOVERFLOW or BF_ETIMEOUT).
 */
bf_status bf_workspace_status(const void* workspace, void* stream);

/*
 * Duration in milliseconds of the enumeration kernel of the last call made on
 * this host thread with opt->profile != 0 (CUDA events recorded on that
 * call's stream immediately around the kernel).  Waits for the end event.
 * Returns BF_EINVAL if no profiled call was made.
 */
bf_status bf_last_profile(float* enumeration_ms);

/* Number of kernels this library has launched in the process so far. */
int64_t bf_launch_count(void);

/*
 * Measured issue rates of this GPU (measurement hook, no counterpart in the
 * paper): the denominators of the enumeration kernels' roofline, whose work
 * is counted in integer-ALU lane-instructions per configuration.  Each rate is
 * lane-instructions per clock per SM of one instruction class, from one
 * 1024-thread block per SM running 8 independent dependency chains per
 * thread (x_t = op(x_{t-1}, x_{t-2}, x_{t-4})), cycles read on the SM.
 */
typedef struct {
    int32_t sms;                  /* multiprocessors (device query) */
    double sm_clock_mhz;          /* SM cycles / CUDA-event time of the probe launches */
    double iadd3_lanes_per_clk;   /* 3-input 32-bit integer add */
    double lop3_lanes_per_clk;    /* 3-input logic operation (integer ALU only) */
    double vmnmx_lanes_per_clk;   /* 16x2 minimum / maximum */
    double ffma_lanes_per_clk;    /* FP32 fused multiply-add (for comparison) */
} bf_issue_rates;

/* Device workspace bytes bf_measure_issue_rates needs. */
size_t bf_issue_rates_workspace_size(void);

/*
 * Runs the probe kernels on `stream` (two launches per class, about 10 ms in
 * all) and fills *out.  workspace: device, >= bf_issue_rates_workspace_size()
 * bytes.  Synchronises the stream.
 */
bf_status bf_measure_issue_rates(void* workspace, size_t workspace_bytes, bf_issue_rates* out, void* stream);

/*
 * bf_merge_lists -- the S lowest records of k result lists (host memory).
 * A search split across processes or GPUs by fixed_bits / fixed_value
 * (disjoint subspaces, the chunk offset of Sec. 3, Eq. (6)) gives one sorted
 * list per shard; the S lowest records overall are the first S of their union
 * under the order (E, c) of Algorithm 1 (Sec. 3).
 *   energies   host, k pointers to S_each values (int64 for BF_I32, double otherwise)
 *   states     host, k pointers to S_each configuration integers
 *   out_*      host, S values each
 * A configuration listed more than once is kept once.  Pure host code.
 */
bf_status bf_merge_lists(int k, const void* const* energies, const uint64_t* const* states, int S_each,
                         bf_dtype dtype, int S, void* out_energies, uint64_t* out_states);

/* Human-readable name of a status code. */
const char* bf_status_string(bf_status s);

/* Detail of the last error raised on the calling host thread ("" if none). */
const char* bf_last_error_detail(void);

/* Library version string. */
const char* bf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BF_H */
