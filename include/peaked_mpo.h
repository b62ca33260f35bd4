/*
 * peaked_mpo.h -- C ABI of the GB300 middle-out MPO contraction library.
 *
 * The library computes, on one GPU, the iterative cancellation of a mirrored circuit
 * C = C_L . C_R into a Matrix Product Operator M (Kremer & Dupuis, "Efficient Classical
 * Simulation of Heuristic Peaked Quantum Circuits", Algorithm 1):
 *   - transpile to a line and split at the midpoint (Sec. II.A),
 *   - absorb the innermost layers of C_L (from the left) and C_R (from the right) into M,
 *     each gate followed by an SVD with relative cutoff eps (Sec. II.B.1),
 *   - when size(M) >= tau, unswap: try SWAPs on bonds from the left, right or both sides
 *     and keep those that lower the bond dimension (Sec. II.B.2; parallel variant App. A.1;
 *     non-strict acceptance App. A.2), recording M = P_L M~ P_R (Eq. 1),
 *   - rewire: route the remaining gates with the updated qubit layouts (Sec. II.B.3),
 *   - apply M to |0...0> and extract the peak / sample / evaluate amplitudes (Sec. II.C).
 *
 * Conventions shared by every call:
 *   - All pointers in signatures are HOST pointers unless a name ends in _dev.  Inputs are
 *     copied; the caller keeps ownership of every buffer it passes.  Output buffers are
 *     caller-allocated host memory of the stated size.
 *   - Complex numbers are stored as interleaved (re, im) float64 pairs.
 *   - A two-qubit gate on the logical pair (a, b) is a 4x4 row-major matrix in the basis
 *     index 2*x_a + x_b.  A bitstring is uint8[n] indexed by logical qubit; its integer
 *     value is sum_q x_q 2^q.
 *   - Every call returns a pc_status.  0 is success, negative values are errors, positive
 *     values are warnings.  No C++ exception crosses this boundary.  After an error,
 *     pc_last_error() on the owning context describes it.
 *   - Calls on one circuit handle are not thread-safe; distinct handles may be used from
 *     distinct host threads.  Each circuit owns one CUDA stream.
 */
#ifndef PEAKED_MPO_H
#define PEAKED_MPO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pc_status;

#define PC_OK               0
#define PC_ERR_INVALID_ARG (-1)   /* bad pointer, size, qubit index or config value      */
#define PC_ERR_NONUNITARY  (-2)   /* a gate with max|G^dagger G - I| > 1e-6              */
#define PC_ERR_OOM         (-3)   /* device allocation failed                            */
#define PC_ERR_NOCONVERGE  (-4)   /* a Jacobi factorisation hit its sweep cap            */
#define PC_ERR_TIMEOUT     (-5)   /* a bounded device wait gave up                       */
#define PC_ERR_NOT_PEAKED  (-6)   /* the exact peak search hit its expansion cap         */
#define PC_ERR_CUDA        (-7)   /* a CUDA runtime call failed                          */
#define PC_ERR_STATE       (-8)   /* call out of order (e.g. peak before contract)       */
#define PC_WARN_STALLED     1     /* size(M) stayed >= tau after unswapping (Sec. III.A) */

#define PC_UNSWAP_PARALLEL   0    /* App. A.1: six (side, parity) batches per cycle      */
#define PC_UNSWAP_SEQUENTIAL 1    /* Algorithm 1: largest available bond, one at a time  */
#define PC_UNSWAP_OFF        2    /* no unswapping (the plain Middle-MPO attack, Sec. I) */

#define PC_PRECISION_FP64    0    /* every step in FP64                                   */
#define PC_PRECISION_TF32X3  1    /* merges as complex 3xTF32 on tcgen05 tensor cores with */
                                  /* FP32 accumulation; factorisation and truncation FP64  */

#define PC_SIDE_ALTERNATE    0    /* Algorithm 1: each step absorbs a layer of C_L, then of C_R */
#define PC_SIDE_ADAPTIVE     1    /* App. A.3: each step tentatively absorbs the next layer of  */
                                  /* either side and keeps the smaller size(M) (ties: left)    */

#define PC_SIDE_LEFT  0           /* out-legs: M <- g M   */
#define PC_SIDE_RIGHT 1           /* in-legs:  M <- M h   */
#define PC_SIDE_BOTH  2

typedef struct pc_ctx pc_ctx;
typedef struct pc_circuit pc_circuit;

/* Hyperparameters of App. A.4 plus the library's own settings. */
typedef struct pc_config {
  double eps;                /* SVD cutoff: keep s_k > eps * s_0 (relative, strict)       */
  int32_t chi_max;           /* hard cap on every bond dimension, 1..1024                 */
  double tau;                /* size(M) threshold (total tensor elements) for unswapping  */
  int32_t max_unswap_iter;   /* cap on unswap cycles per stage (paper: 20)                */
  int32_t accept_equal;      /* 0 strict (paper default), 1 also accept equal dimension   */
  int32_t unswap_mode;       /* PC_UNSWAP_*                                               */
  int32_t jacobi_max_sweeps; /* cap on one-sided Jacobi sweeps per factorisation (>= 1)   */
  int32_t device;            /* CUDA device ordinal                                       */
  int32_t fp32_precondition; /* 1: bond matrices with >= 64 vectors first run FP32 Jacobi  */
                             /* sweeps; the accumulated rotation is made unitary in FP64   */
                             /* (two Newton-Schulz steps) and applied, then FP64 sweeps    */
                             /* finish.  The result keeps FP64 accuracy.  0: FP64 only.     */
  int32_t precision;         /* PC_PRECISION_*: arithmetic of the two-site merge          */
  int32_t precondition_sweeps; /* cap on FP32 preconditioning sweeps (>= 1); the FP64 sweeps */
                             /* that follow run to convergence whatever this cap           */
  int32_t side_mode;         /* PC_SIDE_ALTERNATE or PC_SIDE_ADAPTIVE                      */
  int32_t certify_trials;    /* 1: an unswap trial is first decided without its full      */
                             /* factorisation when a rigorous lower bound shows that its   */
                             /* count reaches the rejection threshold (the k-th singular   */
                             /* value of a randomised FP64 projection, Sec. II.B.2 needs   */
                             /* only the count), the projection's Jacobi run in FP32 and,  */
                             /* for trials that bound leaves open, in FP64; decisions are  */
                             /* those of full factorisations; 0: every trial is factorised */
  int32_t deflate;           /* 1: when the chi_max cap decides the count, the FP64 sweeps */
                             /* orthogonalise only what the kept vectors need (a floor set */
                             /* from the FP32 sweeps, verified afterwards); 0: off         */
  double fp32_dead_rel;      /* FP32 sweep floor (rows below sqrt(fp32_dead_rel) |X|_F are */
                             /* left to the FP64 sweeps); 0: 1e-12 / rows                  */
  int32_t recanonicalise;    /* 1 (default): after each absorption step, compress M to     */
                             /* canonical form (Algorithm 1): a left-to-right QR sweep and */
                             /* a right-to-left SVD sweep with the cutoff, restoring the   */
                             /* Vidal/Hastings form that truncating updates drift from     */
  int32_t pad_;
} pc_config;

/* Counters filled by pc_contract. */
typedef struct pc_stats {
  int64_t n_updates;         /* two-site updates from absorption (gates + routing SWAPs)  */
  int64_t n_trials;          /* unswap trials evaluated                                   */
  int64_t n_accepted;        /* unswap trials accepted                                    */
  int64_t n_stages;          /* outer iterations of Algorithm 1                           */
  int64_t n_waves;           /* batched launches of independent updates                   */
  int64_t final_size;        /* size(M) at the end                                        */
  int32_t max_chi;           /* largest bond dimension seen                               */
  int32_t stalled;           /* 1 if PC_WARN_STALLED was raised                           */
  int32_t max_sweeps;        /* largest Jacobi sweep count used by one factorisation      */
  int32_t fallbacks;         /* waves redone in FP64 only after a failed norm check of   */
                             /* the FP32 preconditioning                                  */
  double seconds;            /* host wall time of the call                                */
  int32_t max_sweeps_fp32;   /* largest FP32 preconditioning sweep count of one update     */
  int32_t pad_;
  int64_t n_trials_certified; /* unswap trials rejected by the lower-bound certificate     */
  int64_t n_deflated;        /* factorisations finished with the deflation floor          */
  int64_t n_full;            /* full factorisations (absorption updates and trials that   */
                             /* ran the whole SVD)                                        */
  int64_t n_recanon;         /* recanonicalisation sweeps (Algorithm 1 compression)        */
  double alg_flops;          /* algorithmic work of the call's two-site updates: per       */
                             /* absorption update 4(4 L^2 v + 22 v^3) (thin SVD with both  */
                             /* vector sets, complex, L >= v the bond matrix sides), per   */
                             /* unswap trial the values-only 4(4 L v^2 - 4 v^3 / 3), plus   */
                             /* 8 m chi_m n + 2048 chi_l chi_r for every merge and gate     */
} pc_stats;

/* Fills cfg with the paper's defaults except eps/chi_max (1e-10 / 256) and tau (1e6). */
void pc_default_config(pc_config* cfg);

/* Creates a context on cfg->device.  *out receives the handle; pc_destroy frees it.
 * Errors: PC_ERR_INVALID_ARG for out-of-range settings, PC_ERR_CUDA. */
pc_status pc_create(const pc_config* cfg, pc_ctx** out);
pc_status pc_destroy(pc_ctx* ctx);
const char* pc_last_error(pc_ctx* ctx);

/* Loads a circuit (Algorithm 1 Require: circuit C on N qubits) and allocates its device MPO
 * store, initialised to the identity with bond dimension 1 (Algorithm 1, M <- I).
 *   pairs       int32[n_gates][2]      logical qubits (a, b), a != b, 0 <= a,b < n_qubits
 *   mats        float64[n_gates][4][4][2]  gate matrices, time order
 *   split_index gates [0, split) form the earlier half C_R, the rest C_L (Sec. II.A);
 *               -1 selects n_gates / 2
 *   oneq_*      n_oneq one-qubit gates applied after every two-qubit gate (e.g. X^s):
 *               oneq_qubits int32[n_oneq], oneq_mats float64[n_oneq][2][2][2]
 * Gates are checked for unitarity (PC_ERR_NONUNITARY).  2 <= n_qubits <= 4096. */
pc_status pc_load_gates(pc_ctx* ctx, int32_t n_qubits, int64_t n_gates, const int32_t* pairs,
                        const double* mats, int64_t split_index, int64_t n_oneq,
                        const int32_t* oneq_qubits, const double* oneq_mats, pc_circuit** out);
pc_status pc_destroy_circuit(pc_circuit* c);

/* Runs Algorithm 1 to the end: every layer absorbed, unswap stages when size(M) >= tau.
 * Returns PC_WARN_STALLED (> 0) when the progress rule had to force absorption.
 * stats may be NULL. */
pc_status pc_contract(pc_circuit* c, pc_stats* stats);

/* At most max_iterations outer iterations of Algorithm 1 (each: absorb layer pairs while
 * size(M) < tau, at least one pair; then one unswap stage).  Returns PC_OK while layers
 * remain as well as when done; *done (may be NULL) is set to 1 once every layer is absorbed.
 * stats (may be NULL) receives the counters of this call only. */
pc_status pc_contract_iterations(pc_circuit* c, int32_t max_iterations, pc_stats* stats, int32_t* done);

/* Telemetry of the contraction (the quantities of the paper's Fig. 3: MPO size against the
 * unitaries absorbed and against time, by phase): one record after each absorption phase and
 * one after each unswap stage, since the circuit was loaded. */
typedef struct pc_trace_record {
  int32_t stage;             /* outer iteration of Algorithm 1                              */
  int32_t phase;             /* 0 after absorption, 1 after unswapping                      */
  int64_t gates;             /* two-qubit gates of C absorbed so far (both sides)           */
  int64_t size;              /* size(M), total tensor elements                             */
  int32_t max_chi;
  int32_t accepted;          /* swaps accepted in this stage (0 after absorption)          */
  double seconds;            /* host wall time since pc_load_gates                         */
} pc_trace_record;
/* rec[cap] receives up to cap records; *n_rec the full count. */
pc_status pc_get_trace(pc_circuit* c, int64_t cap, pc_trace_record* rec, int64_t* n_rec);

/* The counters of the circuit's work since its last pc_contract / pc_contract_iterations
 * call began (updates run through pc_apply_updates included). */
pc_status pc_get_stats(pc_circuit* c, pc_stats* stats);

/* Layer cursors of the two fronts (number of layers of C_L / C_R already absorbed). */
pc_status pc_get_cursors(pc_circuit* c, int64_t* left, int64_t* right);
pc_status pc_set_cursors(pc_circuit* c, int64_t left, int64_t right);

/* Device-side checkpoint of the contraction state: the MPO (sites, spectra, bond
 * dimensions), both layouts and both cursors.  pc_snapshot copies the state into a buffer
 * owned by the circuit (allocated on first use); pc_restore copies it back.  Both are
 * device-to-device copies on the circuit's stream. */
pc_status pc_snapshot(pc_circuit* c);
pc_status pc_restore(pc_circuit* c);

/* Host-file checkpoint of the contraction state: bond dimensions, site tensors, spectra,
 * both layouts, both cursors, the one-qubit-layer flag and the stage counter (the MPO and
 * the permutations P_L, P_R of Eq. 1 plus where the two fronts stand).  The gate list is not
 * stored: pc_checkpoint_read restores into a circuit loaded with the same gates (same n and
 * layer counts, checked) and chi_max at least the stored bond dimensions.  Binary format,
 * little-endian, versioned; PC_ERR_INVALID_ARG for a file that does not match,
 * PC_ERR_STATE for an unreadable / unwritable path. */
pc_status pc_checkpoint_write(pc_circuit* c, const char* path);
pc_status pc_checkpoint_read(pc_circuit* c, const char* path);

/* One unswap stage (Sec. II.B.2) on the current MPO, in the configured mode.
 * *n_accepted (may be NULL) receives the number of accepted swaps. */
pc_status pc_unswap(pc_circuit* c, int32_t* n_accepted);

/* Algorithm 1 Ensure + Sec. II.C: exact argmax_x |<x|C|0>|^2 by best-first search over
 * prefix marginals.  bits uint8[n]; *p_peak the probability normalised by ||M|0>||^2;
 * *norm2 (may be NULL) = ||M|0>||^2 (1 for a unitary circuit without truncation).
 * PC_ERR_NOT_PEAKED if more than max_expansions prefixes had to be expanded. */
pc_status pc_extract_peak(pc_circuit* c, int64_t max_expansions, uint8_t* bits, double* p_peak,
                          double* norm2);

/* Sec. II.C: n_samples bitstrings drawn site by site from the conditionals of M|0>.
 * The uniforms are u[s][j] = (splitmix64(seed, s*n + j) >> 11) * 2^-53 (site j), and a
 * site's bit is 1 iff u >= P(0 | prefix).  bits uint8[n_samples][n] (logical order). */
pc_status pc_sample(pc_circuit* c, int64_t n_samples, uint64_t seed, uint8_t* bits);

/* <x|C|0> for k bitstrings (uint8[k][n] logical order) into amp float64[k][2]. */
pc_status pc_amplitudes(pc_circuit* c, int64_t k, const uint8_t* bits, double* amp);

/* Inspection.  chi int32[n-1]; layout_l / layout_r int32[n] (logical qubit -> site, the
 * permutations P_L / P_R of Eq. 1); s float64[cap] the normalised spectrum of one bond. */
pc_status pc_get_bond_dims(pc_circuit* c, int32_t* chi);
pc_status pc_get_layouts(pc_circuit* c, int32_t* layout_l, int32_t* layout_r);
pc_status pc_get_spectrum(pc_circuit* c, int32_t bond, int32_t cap, double* s, int32_t* len);

/* Site tensor B_j as float64[chi_{j-1}][4][chi_j][2] (p = 2*out + in), Hastings/Vidal form:
 * |M>> = B_0 B_1 ... B_{n-1}, Frobenius norm 1.  dims int32[2] receives (chi_{j-1}, chi_j);
 * cap is the capacity of out in complex elements. */
pc_status pc_get_site(pc_circuit* c, int32_t j, int64_t cap, double* out, int32_t* dims);

/* Replaces the MPO with caller-given tensors (for per-kernel tests and microbenchmarks).
 * chi int32[n+1] with chi[0] = chi[n] = 1 and 1 <= chi[b] <= chi_max otherwise;
 * sites: the n tensors B_j[chi[j]][4][chi[j+1]] concatenated (complex, interleaved);
 * lam: the n-1 bond spectra lam_b[chi[b+1]] concatenated.  Layouts reset to identity. */
pc_status pc_set_state(pc_circuit* c, const int32_t* chi, const double* sites, const double* lam);

/* Applies two-site updates (merge, 16x16 operator, factorise, truncate, split; Sec. II.B.1)
 * to n_ops bonds that must be pairwise non-adjacent (|b_i - b_k| >= 2), as one batch.
 *   bonds int32[n_ops], ops float64[n_ops][16][16][2] acting on (p_j, p_{j+1}) with
 *   p = 2*out + in, row index 4*p_j' + p_{j+1}'.  chi_out int32[n_ops] (may be NULL). */
pc_status pc_apply_updates(pc_circuit* c, int32_t n_ops, const int32_t* bonds, const double* ops,
                           int32_t* chi_out);

/* The absorption plan with unswapping off: the sequence of updates the router emits
 * (Sec. II.A transpilation interleaved with absorption; Algorithm 1 order).  Host-only,
 * needs no GPU.  rec int32[cap][4] = (side, bond, kind 0 swap / 1 gate, gate index or -1);
 * *n_rec receives the full count (may exceed cap; then only cap records are written). */
pc_status pc_plan_routing(int32_t n_qubits, int64_t n_gates, const int32_t* pairs,
                          int64_t split_index, int64_t cap, int32_t* rec, int64_t* n_rec);

/* The log of pc_contract: plan records int32[cap][5] = (side, bond, kind 0 swap / 1 gate /
 * 2 accepted unswap, gate or -1, chi after) and unswap records int32[cap][4] = (stage,
 * iteration, side, bond). */
pc_status pc_get_plan(pc_circuit* c, int64_t cap, int32_t* rec, int64_t* n_rec);
pc_status pc_get_unswap_log(pc_circuit* c, int64_t cap, int32_t* rec, int64_t* n_rec);

/* Kernel accounting since the last pc_reset_kernel_timers.  Per kernel class (0 merge and
 * gate, 1 Jacobi factorisation, 2 truncation, 3 split, 4 everything else: environments,
 * peak search, sampling, one-qubit gates, accumulator set-up, 5 unswap-trial certificates:
 * projection, FP32 and FP64 sweeps and norms) the number of kernel launches and, when timing is
 * enabled, the total milliseconds measured with CUDA events on the circuit's stream (class 4
 * is counted, not timed) and the floating-point work:
 * class 0: 8 * 4chi_l * chi_m * 4chi_r + 8 * 256 * chi_l * chi_r (complex merge + gate);
 * class 1: 4 * (4 M^2 N + 22 N^3) with M >= N the bond matrix sides (textbook thin SVD
 * with both singular-vector sets, complex, per full factorisation); class 3: 8 * m * n * k
 * (B_j = T0 V); class 5: the projection (8 r v L) and the rotations performed.
 * launches, ms, flops: arrays of length 6 (any may be NULL). */
pc_status pc_kernel_timers(pc_circuit* c, int64_t* launches, double* ms, double* flops);

/* Measured arithmetic peaks of the device (the denominators of the library's FP64 and FP32
 * rooflines): an FMA-chain kernel over every SM (8 blocks of 256 threads per SM, 8
 * independent chains per thread), best of three timed launches after a warm-up, CUDA
 * events.  Writes TFLOP/s (2 flops per FMA) to the two host doubles.  Not in the paper. */
pc_status pc_measure_alu_peaks(int32_t device, double* fp64_tflops, double* fp32_tflops);

/* Autotuner of the FP64 one-sided Jacobi launch (the library's choice, not the paper's): for
 * each shape i (lens[i] x lens[i] complex bond matrices, batches[i] of them in one launch;
 * 4 <= lens <= 4096, 1 <= batches <= 64) it times two sweeps of seeded random matrices with 1,
 * 2 and 4 warps per row pair (CUDA events, best of two after a warm-up), installs the fastest
 * width in the process-wide table the launches consult (keyed by ceil(log2 row length) and
 * floor(log2 row pairs per round)), and appends the table entries to the text file `path`
 * (NULL: no file).  ms_out (may be NULL): double[n_shapes][3], milliseconds per width.  The
 * width changes the speed only: the sweeps sum every inner product in one fixed order that
 * depends on the row length alone, so a factorisation is bit-identical at every width (and in
 * every launch it shares with other factorisations). */
pc_status pc_autotune(int32_t device, int32_t n_shapes, const int32_t* lens, const int32_t* batches,
                      const char* path, double* ms_out);
/* Installs a table written by pc_autotune (lines "len_bucket pairs_bucket width ...", '#'
 * lines are comments); a width of 0 restores the built-in choice for that entry.  Returns
 * PC_ERR_INVALID_ARG if the file cannot be read or holds no valid line. */
pc_status pc_load_tuning(const char* path);
pc_status pc_reset_kernel_timers(pc_circuit* c, int32_t enable);

/* One bond factorisation that allocates no device memory.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc (a program that fixes its device
 * footprint at start-up, a plugin inside a framework that owns all device allocations,
 * code running where allocation is not allowed).  It runs the library's one-sided Jacobi,
 * truncation (keep s_k > eps * s_0, at most chi_max, renormalised) and V^dagger extraction
 * on the caller's buffers, with all scratch in one fixed device array (about 2.1 MB, held
 * by every GPU that loads the library until exit).
 *   x_dev   DEVICE float64[m][n][2], the bond matrix, row-major; 1 <= m, n <= 256
 *   s_dev   DEVICE float64[min(m, n, chi_max)]: kept singular values, normalised to unit 2-norm
 *   vh_dev  DEVICE float64[min(m, n, chi_max)][n][2]: kept right singular vectors as rows
 *   count   HOST: number of values kept
 *   stream  a cudaStream_t, or NULL for the default stream; the call is synchronous: it
 *           copies the count back and returns after it has synchronised that stream.
 * Sizes beyond 256 return PC_ERR_INVALID_ARG.  Every call shares the one array and leaves
 * its contents there; calls that overlap on the GPU (concurrent streams, threads) race.
 * The first call on a device looks up the array's address with that device current:
 * make it before any stream capture.  The address is cached per device for the life of
 * the process and is stale after a cudaDeviceReset of that device. */
pc_status pc_factorise_noalloc(const double* x_dev, int32_t m, int32_t n, double eps, int32_t chi_max,
                               double* s_dev, double* vh_dev, int32_t* count, void* stream);

/* ---- Batching: the waves of several circuits in one set of launches -------------------
 * A batch owns a launcher thread and one factorisation workspace.  A circuit attached to a
 * batch posts each of its waves (absorption updates, unswap trials) to the launcher instead
 * of launching them itself; the launcher combines the waves posted by every attached
 * circuit that is contracting into launches of at most max_tasks factorisations of any mix
 * of bond dimensions, precisions and configurations (one persistent Jacobi launch for all),
 * waiting at most about 2 ms for a circuit that has not posted yet.  Results per circuit
 * are the ones it gets alone, up to the rounding order of the shared launch (the Jacobi
 * group width depends on the launch's total work).  The paper runs one circuit at a time
 * (Sec. III); this is the library's own scheduling. */
typedef struct pc_batch pc_batch;

/* A batch on ctx's device: max_tasks factorisations per launch (1..256), scratch arena of at
 * most arena_bytes (0: 8 GiB), allocated as needed.  Destroy it only after every circuit
 * has been detached. */
pc_status pc_batch_create(pc_ctx* ctx, int32_t max_tasks, int64_t arena_bytes, pc_batch** out);
pc_status pc_batch_destroy(pc_batch* b);
/* Routes c's waves through the batch (attach) or back to the circuit's own workspace. */
pc_status pc_batch_attach(pc_batch* b, pc_circuit* c);
pc_status pc_batch_detach(pc_batch* b, pc_circuit* c);
/* pc_contract on n distinct circuits at once, one host thread each, their waves combined.
 * statuses[k] receives circuit k's status, stats[k] (stats may be NULL) its counters.
 * Returns the most recent error status among them, else PC_OK. */
pc_status pc_batch_contract(pc_batch* b, int32_t n, pc_circuit* const* circuits, pc_status* statuses,
                            pc_stats* stats);
/* Combined launches so far, factorisations they ran, the largest launch, and per kernel
 * class (as pc_kernel_timers) the milliseconds (when timing is on) and algorithmic flops. */
pc_status pc_batch_counters(pc_batch* b, int64_t* launches, int64_t* tasks, int32_t* max_tasks, double* ms,
                            double* flops);
pc_status pc_batch_set_timing(pc_batch* b, int32_t enable);

/* Device bytes a circuit of n_qubits at chi_max keeps resident while served: site store,
 * spectra, right environments, peak-search pool and the buffers of n_samples samples.
 * Host-only.  -1 for invalid sizes. */
int64_t pc_projected_bytes(int32_t n_qubits, int32_t chi_max, int64_t n_samples);

/* ---- Serving: a request loop with continuous batching ----------------------------------
 * Requests (a circuit and its configuration) may be submitted at any time.  The server
 * admits them in arrival order as soon as a slot is free and the circuit's projected bytes
 * (pc_projected_bytes at its chi_max) fit in memory_budget next to the resident ones; each
 * admitted circuit stays resident until its peak (and samples) are ready, and the
 * factorisations of all contracting circuits run in shared launches of one batch.
 * Time-to-peak of a request = completion - submission on the server clock. */
typedef struct pc_server pc_server;

typedef struct pc_server_config {
  int32_t device;
  int32_t max_resident;      /* circuits admitted at once (slots), >= 1                     */
  int64_t memory_budget;     /* bytes for the resident circuits' stores, > 0                */
  int32_t max_tasks;         /* factorisations per combined launch, 1..256                  */
  int64_t arena_bytes;       /* shared factorisation scratch (0: 8 GiB), besides the budget */
} pc_server_config;

typedef struct pc_request {
  pc_config cfg;             /* eps, chi_max, tau, precision, ...; cfg.device is ignored     */
  int32_t n_qubits;
  int64_t n_gates;
  const int32_t* pairs;      /* as pc_load_gates; copied by pc_server_submit                */
  const double* mats;
  int64_t split_index;
  int64_t n_oneq;
  const int32_t* oneq_qubits;
  const double* oneq_mats;
  int64_t n_samples;         /* samples to draw from the result (0: none), as pc_sample     */
  uint64_t seed;
} pc_request;

typedef struct pc_result {
  pc_status status;          /* of the request's contraction, peak and sampling            */
  int32_t n_qubits;
  double p_peak;             /* as pc_extract_peak                                          */
  double norm2;
  double t_submit, t_admit, t_done;   /* seconds on the server clock                       */
  int64_t n_updates, n_trials, n_accepted;
  int32_t max_chi;
  int64_t store_bytes;       /* projected bytes it held while resident                      */
} pc_result;

typedef struct pc_server_stats {
  int64_t submitted, admitted, completed, failed;
  int32_t resident, max_resident_seen;
  int64_t bytes_resident, max_bytes_seen;
  double p50_s, p99_s, mean_s;   /* time-to-peak of the completed requests (nearest rank)   */
  double circuits_per_hour;      /* completed / (last completion - first submission)        */
  int64_t launches, tasks;       /* combined factorisation launches and their tasks         */
  int32_t max_tasks_per_launch;
} pc_server_stats;

pc_status pc_server_create(const pc_server_config* cfg, pc_server** out);
/* Copies the request; *ticket identifies it.  A request whose projected bytes exceed
 * memory_budget completes with PC_ERR_OOM without being admitted. */
pc_status pc_server_submit(pc_server* s, const pc_request* req, int64_t* ticket);
/* Waits for a request (timeout_s < 0: without limit; PC_ERR_TIMEOUT when it is not done in
 * time) and copies its result: bits uint8[n] (the peak, may be NULL), samples
 * uint8[n_samples][n] (may be NULL). */
pc_status pc_server_wait(pc_server* s, int64_t ticket, double timeout_s, pc_result* res, uint8_t* bits,
                         uint8_t* samples);
pc_status pc_server_get_stats(pc_server* s, pc_server_stats* out);
/* Seconds since pc_server_create. */
double pc_server_clock(pc_server* s);
/* Finishes every submitted request, then frees the server. */
pc_status pc_server_destroy(pc_server* s);

/* The CUDA stream (a cudaStream_t) every kernel of this circuit runs on, for callers that
 * time or order their own work against it.  The circuit keeps ownership. */
pc_status pc_get_stream(pc_circuit* c, void** stream);

/* Library version string. */
const char* pc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PEAKED_MPO_H */
