/*
 * qsim_gb300.h — C ABI of the GB300 (sm_103a) dense state-vector simulator.
 *
 * The library applies a gate sequence to a dense 2^n complex state vector
 * held in GPU memory (Section 2.1, Eq. 1), either one gate at a time
 * (Algorithms 1-4, Eq. 3-4) or after dependency-aware gate contraction into
 * dense k-qubit blocks (Section 3.4, Eq. 6-7) grouped into shared-memory tile
 * passes. It also evaluates Pauli-sum expectation values and their adjoint
 * gradients, which the paper does not cover (textbook definitions, stated at
 * each entry point).
 *
 * Conventions used by every entry point:
 *   - Qubit q is bit q of the amplitude index (Eq. 2: U on qubit k is
 *     I^{(x) n-k-1} (x) U (x) I^{(x) k}); qubit 0 is the least significant bit.
 *   - Amplitudes are interleaved complex numbers: QS_C64 = (float re, float im)
 *     = 8 bytes, QS_C128 = (double re, double im) = 16 bytes, index-major.
 *   - All arrays passed in (gates, parameters, Pauli terms, host buffers) are
 *     owned by the caller and only read during the call; nothing keeps a
 *     pointer to them after return.
 *   - Outputs are written only when the call returns QS_OK.
 *   - Device work is ordered on the state's stream. Calls that return host
 *     values (norm, expectation, gradient, copies to host) synchronise that
 *     stream before returning. A call on two states whose streams differ
 *     orders them with events: its work waits for what was queued on both,
 *     and a state written by the call is ready on its own stream afterwards.
 *   - A plan holds device tables (gate matrices, parameter rows, a CUDA graph)
 *     that each execution rewrites: one thread at a time may use a plan.
 *     Executions of one plan on states with different streams are ordered by
 *     the plan itself (each waits for the previous one's device work).
 *   - Errors: a negative qs_status; qs_last_error() returns a message for the
 *     calling thread. Invalid arguments (qubit >= n, repeated qubit in a gate,
 *     unknown kind, size mismatch) give QS_ERR_ARG before any device work.
 *   - The library fails (QS_ERR_CUDA) when no CUDA device is present: there is
 *     no CPU fallback.
 */
#ifndef QSIM_GB300_H
#define QSIM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qs_status;
#define QS_OK 0
#define QS_ERR_ARG (-1)
#define QS_ERR_OOM (-2)
#define QS_ERR_CUDA (-3)
#define QS_ERR_TIMEOUT (-4)
#define QS_ERR_UNSUPPORTED (-5)

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Gate kinds. Single-target: H, X, Y, Z, S, SDG, T, TDG, RX, RY, RZ, P, U1.
 * Two-target: SWAP, U2. Any kind may carry up to two controls (the gate acts
 * on the subspace where every control bit is 1, Section 2.1's CU form). */
typedef enum {
  QS_GATE_H = 1, QS_GATE_X, QS_GATE_Y, QS_GATE_Z, QS_GATE_S, QS_GATE_SDG,
  QS_GATE_T, QS_GATE_TDG, QS_GATE_RX, QS_GATE_RY, QS_GATE_RZ, QS_GATE_P,
  QS_GATE_U1, QS_GATE_SWAP, QS_GATE_U2
} qs_gate_kind;

/* One gate. Rotations are R_P(a) = exp(-i a P / 2); P(a) = diag(1, e^{ia}).
 * angle = param + scale * theta[param_index] when param_index >= 0, else param.
 * mat: U1 = 2x2, U2 = 4x4 complex row-major (re, im); for U2 local index bit 0
 * belongs to q[0] and bit 1 to q[1] (the ordering of Eq. 6). */
typedef struct {
  int32_t kind;
  int32_t nq;            /* number of targets: 1 or 2 */
  int32_t q[2];          /* target qubits */
  int32_t nctrl;         /* 0..2 */
  int32_t ctrl[2];       /* control qubits */
  int32_t param_index;   /* -1 = fixed angle */
  double param;
  double scale;
  double mat[32];
} qs_gate;

/* Pauli string with coefficient: X on bits of xmask only, Z on zmask only,
 * Y where both are set; qubits >= n must be clear. */
typedef struct {
  double coeff;
  uint64_t xmask;
  uint64_t zmask;
} qs_pauli_term;

/* Execution modes for plans. */
typedef enum {
  QS_MODE_PER_GATE = 0,  /* one kernel launch per gate (Algorithms 1-4) */
  QS_MODE_FUSED = 1,     /* DAG contraction into k-qubit blocks + tile passes */
  QS_MODE_TENSOR = 2,    /* as FUSED, with blocks applied as dense complex GEMMs on tensor cores
                            (tcgen05), each its own pass over the state.
                            QS_C64: 6-qubit contraction (fuse_k = 4 or 5: that width, the blocks
                            padded to 6 qubits), blocks of >= reserved[0] gates (default 10) as
                            64x64 complex blocks with FP32 accumulation (tc_precision), n >= 13
                            (smaller states plan as FUSED).
                            QS_C128: 5-qubit contraction (fuse_k = 4: that width, padded to 5),
                            blocks of >= reserved[0] gates (default 1: every block) as 32x32
                            complex blocks computed exactly: each row of 64 reals shares a
                            power-of-two scale, amplitudes are cut into six 9-bit integer
                            digits and W into six (fp16), the 21 digit products of levels 0-5
                            accumulate in FP32, one accumulator per level (levels 0-2 exactly)
                            and are combined in FP32 pairs without FP64 instructions; per pass
                            and output the error is at most 2^-46 times the 2-norm of the
                            32-amplitude row plus 2^-49 of its scale (2^-48 of the norm between
                            passes, which hand the state over as FP32 pairs). n >= 12 (smaller
                            states plan as FUSED); tc_precision must be 0. */
  QS_MODE_SMGP = 3       /* staggered multi-gate parallelism (Section 3.3, Tab. 3): runs of 2, 4 or 8
                            consecutive uncontrolled one-target gates on distinct qubits become a
                            group; the state is cut into S segments by qubits no member targets,
                            and S launches of a two-dimensional block (x = amplitude pairs, y =
                            member) let member j update segment (T + j) mod S at step T; other
                            gates run one launch each as in QS_MODE_PER_GATE. Introspection and
                            batched execution treat the plan as a per-gate plan. */
} qs_mode;

/* Planner and kernel options. Zero-initialised fields take the defaults. */
typedef struct {
  int32_t mode;          /* qs_mode */
  int32_t fuse_k;        /* max qubits per fused block (1..5 on CUDA cores; tensor mode: 6 for
                            QS_C64, or 5 when fuse_k = 5; always 5 for QS_C128); 0 = auto */
  int32_t tile_qubits;   /* m: qubits staged per shared-memory tile (6..14); 0 = auto */
  int32_t low_qubits;    /* L: qubits 0..L-1 always in the tile (coalescing); 0 = auto */
  int32_t paper_mode;    /* 1 = contract only the merges of Section 3.4 (1q(x)1q, same-qubit, same-(c,t) CU) */
  int32_t tc_precision;  /* tensor mode, QS_C64: 4 = fp16 hi/lo split with three products and a power-of-two
                            pre-scale of the amplitudes (default; about 2^-22 relative per pass),
                            3 = bf16 hi/lo split, three products (about 2^-16), 1 = bf16, one product */
  int32_t threads;       /* CUDA threads per tile CTA; 0 = auto */
  int32_t fuse_parametric; /* 1 = parametric gates may join dense blocks, whose matrices are then
                              rebuilt from theta on the device at every execution (per batch row).
                              0 = they stay separate ops resolved from theta on the device. */
  int32_t reserved[8];   /* reserved[0]: tensor mode, least gates per tensor-core block (0 = 10).
                            reserved[1]: tensor mode, tensor-core pass pipeline (single and batched
                            executions): 0 = tiles staged in shared memory by bulk asynchronous
                            copies (default), 1 = tiles staged in registers by the computing
                            threads.
                            reserved[2]: fused and tensor modes, n >= 12: least gates in a
                            diagonal phase run (0 = max(16, 2n), < 0 = no phase runs). A phase
                            run is a contiguous stretch of CNOTs, SWAPs and diagonal gates
                            (Z, S, T, RZ, P and their one-control forms) whose permutation of
                            the basis composes to the identity, such as a QAOA cost layer; it
                            runs as one sweep multiplying amplitude x by
                            prod_j exp(i alpha_j (-1)^popcount(mask_j & x)) (qs_plan_phase_terms).
                            reserved[3]: QS_C128 fused and tensor-core plans, arithmetic of the
                            CUDA-core passes (tile, phase and adjoint reverse-sweep passes):
                            0 (default) or 1 = FP32 pairs ("double-float": each real held as
                            h + l with two floats, error-free sum and product transformations,
                            about 46 significant bits, relative error near 2^-46 per
                            operation); 2 = FP64. The state stays complex128 in memory, split
                            into pairs when a tile is loaded and joined when it is stored.
                            GB300's FP32 rate is about 64x its FP64 rate.
                            reserved[4]: qs_plan_execute_batched schedule: 0 = every pass covers
                            the whole batch (default), 1 = when at least two states fit in 64 MiB
                            (about half the L2), every pass runs on one wave of such states
                            before the next wave (passes then read L2, not HBM; more launches).
                            reserved[5]: tile passes' staging: 0 (default) or 1 = every thread
                            loads and stores 16-byte vectors; 2 = the bulk-copy (TMA) engine
                            moves each run of 2^low_qubits amplitudes into one of two
                            shared-memory tile buffers (the next tile loads while the ops run
                            on this one) and back, where the runs are at least 16 bytes and two
                            tiles fit (complex64 and FP64 tiles; FP32-pair tiles keep the
                            vector path). Its waits are bounded like the tensor-core passes'. */
} qs_plan_opts;

/* Statistics of a plan (Fig. 16's compression ratio uses gates/blocks). */
typedef struct {
  int64_t gates;         /* gates in the input circuit */
  int64_t blocks;        /* fused blocks (or gates, per-gate mode) */
  int64_t passes;        /* HBM sweeps-worth of kernel launches per execution */
  int64_t launches;      /* kernel launches per execution */
  double sweeps;         /* algorithmic state sweeps (read + write of 2^n amplitudes) */
  double per_gate_sweeps;/* sweeps the same circuit costs one gate at a time */
  double flops_per_amp;  /* real floating-point operations per amplitude per execution */
  int32_t max_block_qubits;
  int32_t tile_qubits;
  int32_t low_qubits;
  int32_t reserved[5];   /* reserved[0]: tile passes staged by bulk copies (qs_plan_opts reserved[5]) */
} qs_plan_info;

typedef struct qs_state_s* qs_state_t;
typedef struct qs_plan_s* qs_plan_t;

/* ---------------- state ---------------- */

/* Allocates an n-qubit state (1 <= n <= 40) on the current CUDA device and
 * sets it to |0...0> (Section 3.1: the simulator builds the initial state).
 * stream: a cudaStream_t (NULL = the legacy default stream) on which all work
 * on this state is ordered. QS_ERR_OOM when the device cannot hold 2^n amps. */
qs_status qs_state_alloc(int n, qs_dtype dtype, void* stream, qs_state_t* out);

/* Wraps caller-owned device memory of 2^n amplitudes (not initialised, not
 * freed by qs_state_free). dev_ptr must be 16-byte aligned. (The state
 * vector of Eq. 1.) */
qs_status qs_state_wrap(void* dev_ptr, int n, qs_dtype dtype, void* stream, qs_state_t* out);

qs_status qs_state_free(qs_state_t s);
qs_status qs_state_info(qs_state_t s, int* n, qs_dtype* dtype, void** dev_ptr);
qs_status qs_state_set_stream(qs_state_t s, void* stream);

/* Sets the computational basis state |x> (x < 2^n). (|x> of Eq. 1: qubit q is bit q of x.) */
qs_status qs_state_set_basis(qs_state_t s, uint64_t x);

/* Copies 2^n amplitudes (bytes = 2^n * amp size) between host and device;
 * host memory may be pageable or pinned. (Data movement: no counterpart in
 * the paper.) */
qs_status qs_state_copy_from_host(qs_state_t s, const void* host, size_t bytes);
qs_status qs_state_copy_to_host(qs_state_t s, void* host, size_t bytes);
/* dst <- src (same n and dtype), device to device. (No counterpart in the paper.) */
qs_status qs_state_copy(qs_state_t dst, qs_state_t src);

/* Reads `count` amplitudes psi[idx[k]] (idx host array, each < 2^n) into
 * host memory `out` (count complex values of the state's dtype, interleaved
 * re/im), gathered on the device: sampling a state without copying all 2^n
 * amplitudes (Eq. 1 indexing: qubit q is bit q of the index). An index >= 2^n
 * gives QS_ERR_ARG before any device work. Synchronises the state's stream.
 * (An access helper with no counterpart in the paper.) */
qs_status qs_state_get_amplitudes(qs_state_t s, const uint64_t* idx, size_t count, void* out);

/* ---------------- circuits ---------------- */

/* Plans a circuit for n qubits: resolves gate matrices (FP64), builds the gate
 * DAG (Section 3.4: an edge from each earlier gate sharing a qubit, controls
 * included), contracts it greedily into blocks of <= fuse_k qubits whose
 * unitary is the ordered product (Eq. 7 for distinct qubits, M2 M1 for the
 * same qubit), and groups blocks into tile passes. opts NULL = per-gate mode.
 * Parametric gates are resolved at execution time from theta. More than 2^30
 * gates give QS_ERR_ARG. */
qs_status qs_plan_create(int n, qs_dtype dtype, const qs_gate* gates, size_t ngates,
                         const qs_plan_opts* opts, qs_plan_t* out);
qs_status qs_plan_info_get(qs_plan_t p, qs_plan_info* info);
qs_status qs_plan_free(qs_plan_t p);

/* Applies a plan to a state in place: psi <- G_N ... G_1 psi. theta holds
 * ntheta parameters (may be NULL when the circuit has none). Per gate the
 * update of Eq. 3-4 (Algorithms 1-4); fused blocks apply their product
 * matrix (Eq. 6-7, Section 3.4). */
qs_status qs_plan_execute(qs_plan_t p, qs_state_t s, const double* theta, size_t ntheta);

/* Runs the plan on `count` independent states held in host memory (page-locked
 * for overlap): host_in[i] (2^n amplitudes, read) -> host_out[i] (written; the
 * pointer arrays may repeat a buffer, and host_out may be NULL to keep only
 * the norms), norms[i] = ||psi_i||^2 after the circuit (may be NULL). The
 * states pass through the nwork >= 1 device states in `work` (same n and
 * dtype as the plan) round robin: the copy of input i+1 into one work state
 * and the copy of result i-1 out of another run on their own streams while
 * input i is computed, so with nwork >= 2 the host link hides behind the
 * circuit (norms are gathered on the device and read once at the end).
 * theta as for qs_plan_execute, shared by all inputs. Blocks until every
 * result is in host memory. QS_ERR_ARG for a NULL input, work states of
 * another n or dtype, or a work state listed twice. The overlap of copies
 * with compute follows Section 3.2's multi-buffering (Tab. 2). */
qs_status qs_plan_execute_host(qs_plan_t p, qs_state_t* work, int nwork, const void* const* host_in,
                               void* const* host_out, int count, const double* theta, size_t ntheta,
                               double* norms);

/* Autotuner (no counterpart in the paper): plans the circuit under a built-in
 * grid of options (per-gate; CUDA-core contraction width 1..4 with two tile
 * shapes; for complex64 with n >= 13, tensor-core plans with three block
 * thresholds), runs each once to warm up and once timed with CUDA events on
 * the state's stream (the state's contents are overwritten), and writes the
 * fastest options to *best and its time to *best_ms (may be NULL). Results
 * are cached per (n, dtype, gate list): a cached circuit is not timed again,
 * and the cache can be saved to and loaded from a file (below). Synchronises. */
qs_status qs_plan_autotune(qs_state_t scratch, const qs_gate* gates, size_t ngates, const double* theta,
                           size_t ntheta, qs_plan_opts* best, double* best_ms);

/* The autotuner's cache, kept across processes (no counterpart in the paper).
 * Entries are keyed by (n, dtype, gate count, a hash of the fields each gate
 * uses: targets up to nq, controls up to nctrl, the angle and parameter
 * binding of rotations, the matrix of U1/U2), so unused fields do not matter.
 *   qs_tune_cache_lookup: host only; *found = 1 and *best / *best_ms (each may
 *     be NULL) when the circuit has an entry, else *found = 0.
 *   qs_tune_cache_put: records options for a circuit (a deployment's known
 *     choice); they must plan it (else the qs_plan_create error); ms >= 0.
 *   qs_tune_cache_save: writes every entry as text (path: a file name;
 *     *entries may be NULL); QS_ERR_ARG when the file cannot be written.
 *   qs_tune_cache_load: merges a saved file into the cache (its entries
 *     replace equal keys); a malformed file or out-of-range value gives
 *     QS_ERR_ARG and leaves the cache unchanged.
 *   qs_tune_cache_clear: empties the cache.
 * All are thread-safe. */
qs_status qs_tune_cache_lookup(int n, qs_dtype dtype, const qs_gate* gates, size_t ngates, qs_plan_opts* best,
                               double* best_ms, int* found);
qs_status qs_tune_cache_put(int n, qs_dtype dtype, const qs_gate* gates, size_t ngates,
                            const qs_plan_opts* opts, double ms);
qs_status qs_tune_cache_save(const char* path, int64_t* entries);
qs_status qs_tune_cache_load(const char* path, int64_t* entries);
qs_status qs_tune_cache_clear(void);

/* One-shot: plan, execute, free. (Eq. 3-4 per gate, as qs_plan_execute.) */
qs_status qs_apply_circuit(qs_state_t s, const qs_gate* gates, size_t ngates,
                           const double* theta, size_t ntheta, const qs_plan_opts* opts);

/* ---------------- observables ---------------- */

/* *out = sum_i |psi_i|^2, accumulated in FP64. (No counterpart in the paper.) */
qs_status qs_norm(qs_state_t s, double* out);

/* *out = sum_j c_j <psi|P_j|psi> with P|i> = i^{#Y} (-1)^{popcount(i & z)} |i xor x>,
 * accumulated in FP64 (terms with equal xmask share one sweep). (No
 * counterpart in the paper: the textbook expectation value of a Pauli sum.) */
qs_status qs_expval_pauli_sum(qs_state_t s, const qs_pauli_term* terms, size_t nterms, double* out);

/* out <- sum_j c_j P_j psi (out must not alias s). (No counterpart in the paper.) */
qs_status qs_apply_pauli_sum(qs_state_t s, const qs_pauli_term* terms, size_t nterms, qs_state_t out);

/* max_i |a_i - b_i| and ||a - b||_2 in FP64 for two states of equal n (dtypes
 * may differ: the error of a complex64 result against a complex128 run).
 * (No counterpart in the paper.) */
qs_status qs_state_diff(qs_state_t a, qs_state_t b, double* max_abs, double* l2);

/* <a|b> in FP64: (*re, *im). (No counterpart in the paper.) */
qs_status qs_inner(qs_state_t a, qs_state_t b, double* re, double* im);

/* Adjoint-method gradient (Jones and Gacon, arXiv:2009.02823) of
 * E(theta) = <psi|H|psi>, psi = C(theta) psi0, psi0 = the state s (left
 * unchanged). grad has ntheta entries. Allocates two scratch states. */
qs_status qs_adjoint_grad(qs_state_t s, const qs_gate* gates, size_t ngates,
                          const double* theta, size_t ntheta,
                          const qs_pauli_term* terms, size_t nterms,
                          double* expval_out, double* grad_out);
/* Same, with plan options (may be NULL = the defaults above): they plan the
 * forward execution (any fused or tensor mode); their complex128 arithmetic
 * (reserved[3], FP32 pairs) applies to the reverse sweep as well.
 * (Jones and Gacon, as qs_adjoint_grad.) */
qs_status qs_adjoint_grad_opts(qs_state_t s, const qs_gate* gates, size_t ngates, const double* theta,
                               size_t ntheta, const qs_pauli_term* terms, size_t nterms,
                               const qs_plan_opts* opts, double* expval_out, double* grad_out);

/* ---------------- batched execution ---------------- */

/* Applies one planned circuit to B states with B parameter vectors (row b of
 * theta, B x ntheta row-major, drives state b) and, when terms != NULL,
 * writes <H> of each final state to expvals[b]. All states must share n,
 * dtype and stream. The launch sequence is captured once into a CUDA graph
 * and replayed.
 * (No counterpart in the paper: the many parameter vectors of one circuit
 * that a variational loop evaluates.) */
qs_status qs_plan_execute_batched(qs_plan_t p, qs_state_t* states, int B,
                                  const double* theta, size_t ntheta,
                                  const qs_pauli_term* terms, size_t nterms, double* expvals);

/* One-shot batched apply: plans the circuit for the states' n and dtype with
 * opts (NULL = per-gate mode, as for qs_plan_create), applies it to the B
 * states with row b of theta (B x ntheta, row-major; NULL when the circuit
 * has no parameters) driving state b, synchronises the states' stream and
 * frees the plan. The states must share n, dtype and stream (QS_ERR_ARG
 * otherwise). For repeated batches keep a plan and call
 * qs_plan_execute_batched, which replays its captured graph. (No counterpart in the paper.) */
qs_status qs_apply_circuit_batched(qs_state_t* states, int B, const qs_gate* gates, size_t ngates,
                                   const double* theta, size_t ntheta, const qs_plan_opts* opts);

/* ---------------- allocation-free expectation value ----------------
 * The paper has no counterpart: this is a deployment variant of
 * qs_expval_pauli_sum for callers that cannot allocate device memory while
 * they evaluate an observable (a host program that owns all device memory
 * and gives this library a fixed region, an inference or control loop with a
 * pre-reserved memory budget, code running under another framework's
 * allocator). It computes the same value with the same kernels, but keeps all
 * temporaries in one array compiled into the library (80 KiB of device memory
 * on every GPU that loads it, held until the process exits) and never calls
 * cudaMalloc or cudaFree.
 *   dev_state: the caller's 2^n amplitudes in device memory (16-byte aligned),
 *              read only; stream: cudaStream_t the work is ordered on (NULL =
 *              legacy default stream); terms: host array of nterms <= 1024
 *              Pauli strings (more gives QS_ERR_ARG before any device work);
 *   *out: the FP64 expectation value; the call synchronises `stream`.
 * Every call looks up the array's device address in the current CUDA context
 * (make the state's device current), so the address stays right after a
 * device reset or a switch of context; the first call on a device loads the
 * library's device code there, so make it before any stream capture. All
 * calls share the one array: calls whose device work overlaps
 * (other threads, other streams) race on it and must be serialised by the
 * caller. Every slot a call reads is written earlier in the same call, so no
 * clearing is needed between calls. */
qs_status qs_expval_pauli_sum_noalloc(const void* dev_state, int n, qs_dtype dtype, void* stream,
                                      const qs_pauli_term* terms, size_t nterms, double* out);

/* ---------------- plan introspection (host only, no device work) ----------------
 * A plan executes ops in order: gate ops (one input gate, applied by itself)
 * and block ops (a contracted block: a dense 2^nq x 2^nq matrix, or 2^nq
 * diagonal entries, over `qubits` in ascending order, local bit j = qubits[j],
 * the Eq. 7 ordering). In per-gate mode every op is a gate op and every pass
 * one op. */
qs_status qs_plan_op_count(qs_plan_t p, int64_t* nops, int64_t* npasses);
/* type: 0 = gate op, 1 = dense block, 2 = diagonal block, 3 = dense block applied on tensor
 * cores (its own pass: 6 qubits over 13-qubit tiles for QS_C64, 5 qubits over 12-qubit tiles
 * for QS_C128), 4 = diagonal phase run (its own pass; its
 * terms via qs_plan_phase_terms). qubits: capacity 6, or n for a phase run.
 * gate_index: the input gate of a gate op (-1 for blocks). mat (optional,
 * capacity 2 * 4096 doubles): the block's entries as (re, im) pairs; not
 * written for a phase run.
 * (Introspection: no counterpart in the paper.) */
qs_status qs_plan_op_get(qs_plan_t p, int64_t i, int32_t* type, int32_t* qubits, int32_t* nq,
                         int32_t* gate_index, double* mat);
/* Self-check of the blocks rebuilt on the device from theta: resolves theta,
 * builds them on the device, copies them back and returns the largest
 * difference to the host's FP64 ordered products (W images compared as bf16
 * values) and the number of such blocks. Synchronises; no state is touched.
 * (Self-check: no counterpart in the paper.) */
qs_status qs_plan_check_device_blocks(qs_plan_t p, qs_state_t s, const double* theta, size_t ntheta,
                                      double* max_abs_diff, int64_t* nblocks);
/* Tile qubits of pass i (ascending, capacity 14; a phase pass lists the qubits
 * of its run, capacity n) and its op range [op_begin, op_end).
 * (Introspection: no counterpart in the paper.) */
qs_status qs_plan_pass_get(qs_plan_t p, int64_t i, int32_t* tile_qubits, int32_t* m,
                           int64_t* op_begin, int64_t* op_end);
/* Terms of phase-run op i (type 4): the run multiplies amplitude x by
 * prod_j exp(i alpha_j (-1)^popcount(masks[j] & x)), alpha_j = alpha0[j] +
 * coef[j] * theta[param_index[j]] (param_index[j] >= 0) or alpha0[j]. The
 * phase polynomial of the run's gates: with b_q the bit of qubit q,
 * RZ(a) = exp(-i a/2 (-1)^b), P(a) = exp(i a b) and a CNOT adds the control's
 * parity to the target's. Writes min(cap, count) terms; *nterms = count.
 * QS_ERR_ARG when op i is not a phase run.
 * (The phase polynomial of a diagonal run: no counterpart in the paper.) */
qs_status qs_plan_phase_terms(qs_plan_t p, int64_t i, uint64_t* masks, int32_t* param_index, double* alpha0,
                              double* coef, int64_t cap, int64_t* nterms);

/* ---------------- host-resident states (Section 3.2, batched processing) ----------------
 * A state larger than device memory stays in host memory (on Grace, the CPU's
 * memory reached over NVLink-C2C). The high n - batch_qubits qubits index
 * batches of 2^batch_qubits contiguous amplitudes (Section 3.2: the batch
 * index is the high qubits). The circuit is cut into streamed passes, each
 * touching at most pass_qubits batch-index qubits: the tile-pass scheduler with
 * the batch_qubits low qubits always present, so gates move ahead of gates they
 * commute with (disjoint qubits, or diagonal on the shared ones). For each
 * pass, every group of 2^(qubits it selects) batches is copied into
 * one of three device buffers, the pass's gates run there as a plan over
 * batch_qubits + selected qubits (planned with opts, so tile, tensor-core and
 * phase passes all apply), and the group is copied back; copies in, compute
 * and copies out run on three streams, so one group loads while another is
 * computed and a third is stored (the multi-buffering of Tab. 2). */
typedef struct {
  int64_t passes;        /* streamed passes: the state crosses the host link twice per pass */
  int64_t groups;        /* buffer loads over all passes */
  int64_t copies;        /* host <-> device copies issued */
  double bytes_h2d, bytes_d2h;
  double device_bytes;   /* device memory held by the three buffers */
  int64_t reserved[4];
} qs_stream_info;

/* Applies the circuit to host_psi (2^n amplitudes of dtype, interleaved (re, im);
 * page-locked memory for overlapped copies, e.g. cudaHostAlloc or a pinned
 * torch tensor), in place. 1 <= batch_qubits <= n, 0 <= pass_qubits <= n -
 * batch_qubits, batch_qubits + pass_qubits <= 40; every gate may touch at
 * most pass_qubits qubits >= batch_qubits (QS_ERR_ARG otherwise). Device
 * memory: 3 x 2^(batch_qubits + pass_qubits) amplitudes. Blocks until the
 * state is back in host memory. info may be NULL.
 * Section 3.2: batches of 2^batch_qubits contiguous amplitudes, the high
 * qubits as batch index, multi-buffered copies (Tab. 2). */
qs_status qs_stream_apply(void* host_psi, int n, qs_dtype dtype, const qs_gate* gates, size_t ngates,
                          const double* theta, size_t ntheta, const qs_plan_opts* opts, int batch_qubits,
                          int pass_qubits, qs_stream_info* info);
/* Host only: the streamed passes qs_stream_apply would run. high_masks[i] = the
 * batch-index qubits pass i touches, pass_end[i] = the end of its gates in
 * order (both capacity cap, may be NULL); order (capacity ngates, may be NULL)
 * = the gate indices in execution order.
 * (Section 3.2's batch passes, planned on the host.) */
qs_status qs_stream_plan(int n, const qs_gate* gates, size_t ngates, int batch_qubits, int pass_qubits,
                         int64_t* npasses, uint64_t* high_masks, int64_t* pass_end, int64_t cap,
                         int32_t* order);

/* ---------------- measurement (no counterpart in the paper) ----------------
 * With timing enabled, every kernel launch issued by qs_plan_execute is
 * bracketed by two CUDA events on the state's stream. qs_plan_timing_read
 * waits for the recorded events, returns the summed device time of the
 * bracketed launches (ms) and their number, and starts a new interval. */
qs_status qs_plan_set_timing(qs_plan_t p, int enable);
qs_status qs_plan_timing_read(qs_plan_t p, double* total_ms, int64_t* launches);
/* Same, split by launch kind: [0] = tile passes or per-gate kernels, [1] =
 * tensor-core passes (arrays of 2, may be NULL).
 * (Measurement: no counterpart in the paper.) */
qs_status qs_plan_timing_read_kinds(qs_plan_t p, double* total_ms, int64_t* launches, double* kind_ms,
                                    int64_t* kind_launches);

/* Bounded waits of the tensor-core passes and of bulk-staged tile passes
 * (reserved[5] = 2): every wait of their pipelines
 * (a landing slot, an operand, an accumulator) polls an mbarrier at most
 * `polls` times (0 = the default bound, 2^26 polls that may each suspend the
 * thread briefly; below 64, immediate non-blocking checks) before the pass
 * records a timeout, stops, lets its copies and MMAs in flight complete
 * (under the default bound), frees its tensor memory and returns; the
 * execution then fails with QS_ERR_TIMEOUT and the state is left partly
 * updated. A small limit makes the waits run out on purpose (a test of that
 * path); the plan keeps the limit until it is set again.
 * (Failure detection: no counterpart in the paper.) */
qs_status qs_plan_set_wait_limit(qs_plan_t p, uint32_t polls);

/* ---------------- diagnostics (no counterpart in the paper) ---------------- */

const char* qs_last_error(void);
/* Number of library kernel launches issued by this process so far.
 * (Diagnostics: no counterpart in the paper.) */
int64_t qs_launch_count(void);
/* Number of device allocations (cudaMalloc) the library has made in this
 * process so far: states, plan tables, scratch buffers. A call that should not
 * allocate leaves it unchanged. (Diagnostics: no counterpart in the paper.) */
int64_t qs_device_alloc_count(void);
const char* qs_version(void);

#ifdef __cplusplus
}
#endif
#endif
