/*
 * qsim.h -- C ABI of the GB300 state-vector simulator.
 *
 * The library applies sequences of elementary gates to the 2^n complex
 * amplitudes of an n-qubit register held in GPU memory, the operation that
 * Sec. III.A of De Raedt et al., "Massive parallel quantum computer simulator"
 * (quant-ph/0608239) reduces every quantum algorithm to (Eqs. NUM2-NUM8).
 *
 * Conventions for every entry point:
 *  - Qubit q is bit q of the amplitude index, qubit 0 the least significant
 *    bit (Sec. II.A, Eq. STAT2).  Amplitudes are interleaved (re, im): float2
 *    for QSIM_C64, double2 for QSIM_C128.
 *  - Qubit arguments are LOGICAL qubits.  The library may keep the amplitudes
 *    under a permutation sigma of the index bits (the qubit-to-bit map of
 *    Sec. III.B); every reader (qsim_get_state, qsim_probs, qsim_qubit_probs,
 *    qsim_sample) undoes it, so callers always see logical order.
 *  - Gate matrices arrive as IEEE double (re, im) pairs, row-major, and are
 *    rounded to the state's precision on entry.  Unitarity is not checked.
 *  - Calls that only enqueue GPU work are asynchronous and stream-ordered on
 *    the handle's stream.  Calls that return values to host memory
 *    (qsim_norm, qsim_probs, qsim_qubit_probs, qsim_get_state, qsim_sample)
 *    synchronise that stream before returning.
 *  - All buffers passed in are owned by the caller and are not retained after
 *    the call returns.  A handle owns its device memory unless it was made by
 *    qsim_attach.
 *  - No call aborts the process.  A failed call returns a non-zero
 *    qsim_status, leaves the state unchanged when the failure is detected on
 *    the host (bad argument), and records a message for qsim_last_error().
 *  - Handles are not thread-safe; distinct handles may be used from distinct
 *    host threads.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QSIM_API __attribute__((visibility("default")))
#else
#define QSIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QSIM_OK = 0,
    QSIM_EINVAL = 1,        /* bad argument; nothing was changed */
    QSIM_ENOMEM = 2,        /* device or pinned host allocation failed */
    QSIM_ECUDA = 3,         /* a CUDA call failed; see qsim_last_error() */
    QSIM_ETIMEOUT = 4,      /* a bounded device-side wait expired */
    QSIM_EUNSUPPORTED = 5   /* valid request the library cannot serve */
} qsim_status;

typedef enum {
    QSIM_C64 = 0,           /* complex64: float2 amplitudes, FP32 arithmetic */
    QSIM_C128 = 1           /* complex128: double2 amplitudes (IEEE FP64 in memory).
                               Per-gate sweeps and tile passes compute in
                               double-float (an unevaluated sum of two FP32
                               values, about 48 significand bits; magnitudes
                               below 2^-126 flush to zero).  Dense 5-qubit
                               blocks run on the tensor cores as exact bf16
                               digit-slice products summed in double-float
                               (an output's error below 2^-43.7 of its group's
                               largest magnitude); other dense blocks in FP64
                               on the CUDA cores.  Sec. III.A asks for 13-15
                               significant digits; double-float keeps ~14.4. */
} qsim_dtype;

typedef struct qsim_state *qsim_handle;

/* Gate kinds of qsim_gate.kind (Sec. II). */
enum {
    QSIM_GATE_H = 0,    /* Hadamard, Eq. Hadamard */
    QSIM_GATE_X = 1,    /* pi/2 rotation about x, e^{i pi S^x/2}, Eq. Xoperation */
    QSIM_GATE_Y = 2,    /* pi/2 rotation about y, e^{i pi S^y/2}, Eq. Yoperation */
    QSIM_GATE_XB = 3,   /* inverse of X */
    QSIM_GATE_YB = 4,   /* inverse of Y */
    QSIM_GATE_NOT = 5,  /* bit flip: CNOT with one control (Eq. NUM6), Toffoli with two (Eq. NUM8) */
    QSIM_GATE_R = 6,    /* phase shift R(phi) = diag(1, e^{i phi}), Eq. singlephase; param[0] = phi */
    QSIM_GATE_V = 7,    /* V(phi) of Eq. COMM4; param[0] = phi */
    QSIM_GATE_SU2 = 8,  /* [[a+ib, c+id], [-c+id, a-ib]], param[0..3] = (a, b, c, d) */
    QSIM_GATE_U = 9,    /* explicit 2x2 matrix, param[0..7] = row-major (re, im) */
    QSIM_GATE_SWAP = 10 /* quantum SWAP gate of target and target2 */
};

/* One gate of a circuit.  Any gate may carry controls: it then acts only on
 * the amplitudes whose control bits are all 1 (Eqs. NUM6-NUM8). */
typedef struct {
    int32_t kind;       /* QSIM_GATE_* */
    int32_t target;     /* logical target qubit */
    int32_t target2;    /* second target (QSIM_GATE_SWAP), else ignored */
    int32_t reserved;   /* must be 0 */
    uint64_t ctrl_mask; /* logical control qubits, bit q = qubit q; must not contain a target */
    double param[8];    /* kind-specific parameters (see above) */
} qsim_gate;

/* How qsim_run_circuit executes a gate list. */
enum {
    QSIM_MODE_PERGATE = 0, /* one sweep of the state per gate (Sec. III.A) */
    QSIM_MODE_FUSED = 1,   /* planner: shared-memory tile passes, qubit
                              interchanges and dense fused blocks */
    QSIM_MODE_AUTO = 2     /* plans: one candidate per tile size and per
                              tensor-core fusion width (complex64: 4, 5, 6;
                              complex128: 5);
                              the plan's first runs time each candidate with
                              CUDA events on the handle's stream, every later
                              run uses the fastest.  Every run applies the
                              whole circuit.  qsim_run_circuit treats AUTO as
                              FUSED with the default sizes. */
};

typedef struct {
    int32_t mode;       /* QSIM_MODE_* */
    int32_t tile_bits;  /* T, qubits held per shared-memory tile; 0 = default */
    int32_t fuse_k;     /* > 0: apply the circuit as dense blocks of at most fuse_k qubits
                           (1..6), each the FP64 product of its gates: complex64 with
                           k = 4 or 5 on the tensor cores (3xTF32) and k = 6 (bf16 in
                           three slices, six products), complex128 with
                           k = 5 on the tensor cores (exact bf16 digit slices), other
                           widths on the CUDA cores (FP64 for complex128).  A block may take a
                           gate past earlier gates on other qubits (they commute).
                           On the complex64 tensor-core plans, a long run of commuting
                           phase shifts (diag(1, e^{i phi}), at most one control: the
                           controlled phases between the registers of a QFT adder)
                           becomes one phase pass instead of spreading over blocks,
                           where that gives fewer passes.
                           QSIM_EINVAL if a gate acts on more than fuse_k qubits
                           (controls included).  0 or -1: tile passes */
    int32_t max_swap;   /* most bit pairs exchanged per interchange pass; 0 = default */
    int32_t wait_budget_us; /* batches: longest device-side wait between passes
                               before QSIM_ETIMEOUT; 0 = about 2 s */
    int32_t reserved[3];
} qsim_opts;

/* Fill opts with the defaults (QSIM_MODE_FUSED, automatic sizes). */
QSIM_API void qsim_default_opts(qsim_opts *opts);

/* ---- state lifetime ------------------------------------------------------
 * qsim_alloc: allocate an n-qubit state (1 <= n <= 34) on the current CUDA
 * device and set it to |0...0>.  Memory is 2^n * 8 bytes (C64) or 2^n * 16
 * bytes (C128) (Sec. III.A: the state needs 2^(n+4) bytes in double).
 * Errors: EINVAL (n out of range, out == NULL), ENOMEM, ECUDA. */
QSIM_API qsim_status qsim_alloc(int n, qsim_dtype dt, qsim_handle *out);

/* qsim_attach: wrap caller-owned device memory dev_ptr (2^n amplitudes of dt,
 * 16-byte aligned) and a CUDA stream (cudaStream_t, or NULL for the legacy
 * default stream).  The contents are left as they are and read in logical
 * order.  qsim_free releases only the handle. */
QSIM_API qsim_status qsim_attach(void *dev_ptr, int n, qsim_dtype dt, void *stream, qsim_handle *out);

/* qsim_free: release the handle (and its memory, unless attached).  NULL is a
 * no-op.  Waits for the handle's pending work. */
QSIM_API qsim_status qsim_free(qsim_handle h);

/* Set the stream later work is enqueued on (cudaStream_t or NULL). */
QSIM_API qsim_status qsim_set_stream(qsim_handle h, void *cuda_stream);

/* Query size, dtype and device pointer. */
QSIM_API qsim_status qsim_info(qsim_handle h, int *n, qsim_dtype *dt, void **dev_ptr);

/* ---- initial states -------------------------------------------------------
 * qsim_set_basis: INITIAL STATE x (App. A): a_x = 1, all others 0; resets the
 * qubit-to-bit map to the identity.  EINVAL if x >= 2^n. */
QSIM_API qsim_status qsim_set_basis(qsim_handle h, uint64_t x);

/* qsim_set_shor_state: the state of Eq. Shor2 (Sec. V.B) after the
 * modular exponentiation: with the x-register on qubits 0..X-1 and the
 * f-register on qubits X..n-1,
 *     a_{x + 2^X f(x)} = 2^(-X/2),  f(x) = y^x mod G,  x = 0 .. 2^X - 1,
 * all other amplitudes 0.  The paper gives no gate network for the modular
 * exponentiation, so the state is written directly (one device kernel).
 * Resets the qubit-to-bit map to the identity.  EINVAL unless 1 <= X < n,
 * 2 <= G <= 2^(n - X), G < 2^32 and 1 <= y < G. */
QSIM_API qsim_status qsim_set_shor_state(qsim_handle h, int X, uint64_t y, uint64_t G);

/* qsim_set_state: copy 2^n amplitudes (logical order, the state's dtype) from
 * host memory; resets the map to the identity.  bytes must equal the state
 * size. */
QSIM_API qsim_status qsim_set_state(qsim_handle h, const void *host_in, size_t bytes);

/* ---- gates ----------------------------------------------------------------
 * qsim_apply_1q: a'0 = U00 a0 + U01 a1, a'1 = U10 a0 + U11 a1 on every pair
 * of amplitudes (a0, a1) whose indices differ only in bit t (Eqs. NUM2-NUM5
 * for a general 2x2 U).  U = 8 doubles, row-major (re, im).  EINVAL if t is
 * not in [0, n) or U is NULL. */
QSIM_API qsim_status qsim_apply_1q(qsim_handle h, int t, const double U[8]);

/* qsim_apply_ctrl: as qsim_apply_1q but only on pairs whose control qubits
 * (ctrl_mask, logical) are all 1: CNOT (Eq. NUM6), controlled phase
 * (Eq. COMM5), controlled-V (Eq. NUM7), Toffoli (Eq. NUM8) and any
 * multi-controlled U.  EINVAL if ctrl_mask contains t or a bit >= n. */
QSIM_API qsim_status qsim_apply_ctrl(qsim_handle h, uint64_t ctrl_mask, int t, const double U[8]);

/* qsim_apply_gate: one qsim_gate (any kind, with controls). */
QSIM_API qsim_status qsim_apply_gate(qsim_handle h, const qsim_gate *g);

/* qsim_apply_fused: dense 2^k x 2^k unitary U (row-major, 2 * 4^k doubles
 * (re, im)) on the k distinct logical qubits qubits[0..k-1]: qubits[j] is bit
 * j of U's row/column index; for every group of 2^k amplitudes that differ
 * only in those qubits, a'_r = sum_c U_rc a_c.  1 <= k <= min(6, n), else
 * EINVAL.  A product of
 * the paper's gates on k qubits, built on the host in FP64, applied in one
 * pass of the state: on the tensor cores for complex64 with k = 4, 5, 6 and for
 * complex128 with k = 5 when every entry of U lies in (-2, 2) (n >= k + 7),
 * otherwise on the CUDA cores. */
QSIM_API qsim_status qsim_apply_fused(qsim_handle h, int k, const int *qubits, const double *U);

/* qsim_swap_qubits: the SWAP command of App. A (Sec. III.B): interchange the
 * index-bit positions that hold logical qubits a[i] and b[i], i < K, moving
 * the amplitudes in one pass (Eqs. onequbitchange, twoqubitchange0-5 and the
 * K-pair generalisation) and updating the qubit-to-bit map.  The logical state
 * is unchanged; only its layout in memory changes.  1 <= K <= min(8, n/2),
 * all 2K qubits distinct.  K = 1: one sweep over the half of the state whose
 * two bits differ.  K >= 2: one pass reading and writing the state once
 * (tiles of 2^11 complex64 or 2^10 complex128 amplitudes holding all 2K bits
 * in shared memory); when the 2K bits do not fit one tile the pairs are
 * exchanged in groups, one pass per group. */
QSIM_API qsim_status qsim_swap_qubits(qsim_handle h, int K, const int *a, const int *b);

/* qsim_permute_bits: the raw data movement of an interchange: exchange the
 * PHYSICAL index bits l[i] <-> h[i], i < K, of the stored amplitudes without
 * touching the map (so the logical state changes).  For tests of the layout
 * tables of Sec. III.B and for callers managing their own layout. */
QSIM_API qsim_status qsim_permute_bits(qsim_handle h, int K, const int *l, const int *hbits);

/* qsim_get_layout: phys[q] = index bit currently holding logical qubit q. */
QSIM_API qsim_status qsim_get_layout(qsim_handle h, int *phys);

/* qsim_run_circuit: apply ng gates in order, as opts->mode says (NULL =
 * defaults).  The gate list is read during the call only.  On EINVAL (a bad
 * gate) nothing has been applied.  After any other error (ECUDA, ETIMEOUT)
 * the state is unspecified: a complex128 run keeps the amplitudes in an
 * internal double-float form between its first and last tile pass, and a
 * run stopped in between leaves them so. */
QSIM_API qsim_status qsim_run_circuit(qsim_handle h, const qsim_gate *gates, size_t ng, const qsim_opts *opts);

/* ---- plans: a circuit planned and uploaded once, run many times ------------
 * qsim_plan_create validates and plans gates for handle h (its n, dtype and
 * current qubit-to-bit map) and uploads the tile programs to device memory,
 * so that qsim_plan_run only enqueues kernels.  A plan may be run on any
 * handle with the same n, dtype and map; EINVAL otherwise.  qsim_plan_run
 * leaves the map unchanged; after an error (ECUDA, ETIMEOUT) the state is
 * unspecified, as for qsim_run_circuit. */
typedef struct qsim_plan_s *qsim_plan;

typedef struct {
    int32_t passes;      /* shared-memory tile passes per run */
    int32_t sweeps;      /* whole-state per-gate sweeps per run */
    int32_t ops;         /* gate operations in all tile programs */
    int32_t tile_bits;   /* T of the tile passes (0 if none) */
    int32_t phases;      /* register phases over all passes (complex64 register kernel) */
    int32_t reserved;
    double gates;        /* logical gates of the circuit */
    double alg_bytes;    /* algorithmic bytes of one run: 2 * amplitude size * amplitudes
                            each pass or sweep must read and write */
    double alg_flops;    /* algorithmic real floating-point operations of one run:
                            14 per amplitude for a dense 2x2 gate, 6 for a diagonal
                            or anti-diagonal one, 0 for a pure exchange, scaled by
                            the fraction of amplitudes the gate's controls select */
    int32_t mode;        /* mode of the plan the figures above describe */
    int32_t fuse_k;      /* its dense-block width (0: tile passes) */
    int32_t candidates;  /* QSIM_MODE_AUTO: number of candidate plans, else 0 */
    int32_t chosen;      /* QSIM_MODE_AUTO: the candidate in use, -1 while tuning */
    int32_t cand_tile_bits[8];  /* per candidate: tile size ... */
    int32_t cand_fuse_k[8];     /* ... fusion width (0: tile passes) ... */
    double cand_ms[8];          /* ... and its measured run time (0 until timed) */
} qsim_plan_stats;

QSIM_API qsim_status qsim_plan_create(qsim_handle h, const qsim_gate *gates, size_t ng, const qsim_opts *opts,
                                      qsim_plan *out);
QSIM_API qsim_status qsim_plan_run(qsim_handle h, qsim_plan p);
QSIM_API qsim_status qsim_plan_get_stats(qsim_plan p, qsim_plan_stats *out);
QSIM_API qsim_status qsim_plan_free(qsim_plan p);

/* qsim_fuse_blocks: the dense blocks a plan with fuse_k = k applies, computed
 * on the host (no state, no device work), for inspecting a fusion before
 * running it.  Gates are read in order on qubits 0..n-1 (identity map).  The
 * blocks are the circuit's gates grouped into products on at most k qubits
 * (Sec. II.B gates; a block may take a gate past earlier gates on other
 * qubits, with which it commutes); applied in order they equal the circuit.
 * Sets *nblocks to their number and, for blocks b < max_blocks, writes
 * pos[b * k + j] = the qubit of bit j of block b's index and, if U is not
 * NULL, U[b * 2 * 4^k ...] = its 2^k x 2^k unitary (FP64, row-major (re, im)
 * pairs).  pos and U may be NULL (count only); both are caller-owned.
 * QSIM_EINVAL: a bad gate, k outside [1, min(6, n)], or a gate on more than
 * k qubits (controls included). */
QSIM_API qsim_status qsim_fuse_blocks(int n, const qsim_gate *gates, size_t ng, int k, int32_t *pos, double *U,
                                      size_t max_blocks, size_t *nblocks);

/* ---- instrumentation --------------------------------------------------------
 * qsim_profile_enable(h, 1): from now on every kernel launch made for h is
 * bracketed by CUDA events recorded on h's stream.  qsim_profile_read waits
 * for the stream, aggregates the event timings per kernel family and resets
 * the record: out[i] for i < *count (at most max entries). */
typedef struct {
    char name[32];       /* kernel family, e.g. "tile_pass", "pair_sweep" */
    uint64_t launches;
    double total_ms;     /* sum of event-timed durations */
    double alg_bytes;    /* algorithmic bytes of those launches */
    double alg_flops;    /* algorithmic floating-point operations of those launches */
} qsim_kernel_time;

QSIM_API qsim_status qsim_profile_enable(qsim_handle h, int on);
QSIM_API qsim_status qsim_profile_read(qsim_handle h, qsim_kernel_time *out, int max, int *count);

/* Running totals since the handle was created: kernel launches made for it
 * and bytes it copied host->device (inputs: states, gate programs, uniforms)
 * and device->host (results). */
typedef struct {
    uint64_t launches;
    uint64_t h2d_bytes;
    uint64_t d2h_bytes;
} qsim_counters;

QSIM_API qsim_status qsim_get_counters(qsim_handle h, qsim_counters *out);

/* ---- batches of independent circuits -------------------------------------
 * One circuit of a batch: the state hs (C64, made by qsim_alloc or
 * qsim_attach) is set to |x0> and the gates are applied. */
typedef struct {
    qsim_handle state;
    uint64_t x0;
    const qsim_gate *gates;
    size_t ng;
} qsim_circuit;

/* qsim_run_batch: run nc independent circuits (complex64 states of up to 24
 * qubits, on one device) on the stream of cs[0].state; every state is set to
 * its |x0> (in the identity qubit layout) and its gates applied.  Circuits of
 * fewer than 20 qubits run as tile passes in one persistent launch; circuits
 * of 20 qubits or more, which carry nearly all the bytes of a mixed batch,
 * run after it as dense blocks on the tensor cores (6 qubits, or opts->fuse_k
 * = 4 or 5; opts->fuse_k = -1 keeps them in the persistent launch, as does a
 * gate wider than the block).  Waits for completion.  ETIMEOUT if a
 * device-side wait expired (the states are then undefined); opts->
 * wait_budget_us bounds the waits between passes of the persistent launch.
 * Equivalent to qsim_batch_create + one qsim_batch_run + qsim_batch_free,
 * without the graph capture (its launches are enqueued directly). */
QSIM_API qsim_status qsim_run_batch(const qsim_circuit *cs, size_t nc, const qsim_opts *opts);

/* A planned batch: the circuits' tile programs, the ordered work list and the
 * dense blocks are uploaded once and the runs' launches are captured in a
 * CUDA graph, so every qsim_batch_run is one graph launch.  The circuits'
 * states must stay alive. */
typedef struct qsim_batch_s *qsim_batch;

typedef struct {
    int64_t circuits;
    int64_t gates;
    int64_t passes;      /* tile passes over all circuits */
    int64_t items;       /* (circuit, pass, tile) work items of one run */
    int32_t graph;       /* 1 if runs replay a captured CUDA graph */
    int32_t fused;       /* circuits on the tensor-core lane (dense blocks) */
    double alg_bytes;    /* algorithmic bytes of one run: each pass or block reads and writes its state once */
    double alg_flops;    /* algorithmic real flops of one run (same count as the plan statistics) */
    int64_t blocks;      /* dense blocks of the tensor-core lane */
    int64_t kernels;     /* kernel launches of one run */
} qsim_batch_stats;

QSIM_API qsim_status qsim_batch_create(const qsim_circuit *cs, size_t nc, const qsim_opts *opts, qsim_batch *out);
/* Enqueue one run on the batch's stream (asynchronous). */
QSIM_API qsim_status qsim_batch_run(qsim_batch b);
/* Wait for the batch's runs; ETIMEOUT if a device-side wait expired. */
QSIM_API qsim_status qsim_batch_sync(qsim_batch b);
QSIM_API qsim_status qsim_batch_get_stats(qsim_batch b, qsim_batch_stats *out);
QSIM_API qsim_status qsim_batch_free(qsim_batch b);

/* ---- measurement ------------------------------------------------------------
 * qsim_norm: sum_i |a_i|^2 (Eq. STAT1), accumulated in FP64. */
QSIM_API qsim_status qsim_norm(qsim_handle h, double *out);

/* qsim_probs: out[i] = |a_i|^2 for the 2^n logical basis states, FP64;
 * len must equal 2^n. */
QSIM_API qsim_status qsim_probs(qsim_handle h, double *out, size_t len);

/* qsim_qubit_probs: out[q] = <Q_q> = probability that logical qubit q is 1
 * (Eq. Shor7; DO MEASUREMENT of App. A, no collapse), FP64, n values.  For
 * n >= 13 the sums run in double-float (about 48 bits) over groups of 8192
 * amplitudes and in FP64 across groups; complex128 squares carry a relative
 * error below 2^-44, and magnitudes of 2^64 or more are outside the float
 * range these sums use. */
QSIM_API qsim_status qsim_qubit_probs(qsim_handle h, double *out);

/* qsim_qubit_probs_noalloc: the per-qubit marginals of qsim_qubit_probs for
 * callers that must not allocate device memory (a framework that owns the
 * device through its own pool, a latency-bound loop that cannot take the
 * implicit synchronisation of cudaMalloc/cudaFree, an embedder that forbids
 * allocation after start-up).  The paper has no counterpart: this is an
 * interface variant only.
 *
 * amp: device pointer to 2^n amplitudes of dt (16-byte aligned), read in
 * PHYSICAL index order (no handle, no qubit map).  dev_out: caller-owned
 * device memory for n doubles; dev_out[b] = P(index bit b = 1), accumulated in
 * FP64.  stream: cudaStream_t (NULL = legacy default stream); the call only
 * enqueues work and returns.  1 <= n <= 34, else EINVAL.
 *
 * No device memory is allocated or freed: the block partial sums go to one
 * static device array of 608 x 34 doubles (161.5 KiB) that every GPU loading
 * the library holds until the process exits.  Every call looks the array's
 * address up (cudaGetSymbolAddress) on the current device; the first call on
 * a device may load the library's device code there, so make it before any
 * stream capture.  All calls on a device share
 * the array, so calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and corrupt each other's results; serialise
 * them.  The array keeps the last call's partial sums, which no later call
 * reads before overwriting them. */
QSIM_API qsim_status qsim_qubit_probs_noalloc(const void *amp, int n, qsim_dtype dt, void *stream, double *dev_out);

/* qsim_sample: draw ns basis states with probability |a_x|^2 / norm
 * (Sec. V.B).  u[j] in [0, 1) are the caller's uniform numbers; sample j is
 * the smallest logical index x with u[j] * norm < P(0) + ... + P(x) (FP64
 * cumulative sums).  out receives ns indices. */
QSIM_API qsim_status qsim_sample(qsim_handle h, const double *u, size_t ns, uint64_t *out);

/* qsim_get_state: copy the 2^n amplitudes in logical order to host memory;
 * bytes must equal the state size. */
QSIM_API qsim_status qsim_get_state(qsim_handle h, void *host_out, size_t bytes);

/* Wait for the handle's pending work. */
QSIM_API qsim_status qsim_sync(qsim_handle h);

/* Message of the last failed call on this host thread ("" if none). */
QSIM_API const char *qsim_last_error(void);

/* Library version string. */
QSIM_API const char *qsim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
