/*
 * rcs.h -- C ABI of the GB300 random-circuit-sampling state-vector library.
 *
 * The library implements, on one GPU, the three stages of the hybrid pipeline
 * of Wold & Kasirajan, "Revisiting Quantum Supremacy: Simulating Sycamore-Class
 * Circuits Using Hybrid CPU/GPU HPC Workloads" (Section 3.2, items 1, 3, 4):
 * quantum state construction from a circuit, measurement sampling of many
 * shots, and the linear cross-entropy benchmark (XEB) of the samples. The paper
 * runs the first stage on a GPU and the other two as CPU jobs; here all three
 * are CUDA kernels on a dense complex64 state vector held in HBM.
 *
 * Conventions (the paper fixes none of them):
 *  - qubit q is bit q of the basis index (qubit 0 = least significant bit);
 *  - the state is 2^n complex64 amplitudes, interleaved (re, im), 8 bytes each;
 *  - a gate on targets (t0, t1) uses local index j = bit(t0) + 2 bit(t1);
 *  - bitstrings are uint64 basis indices (bit q = qubit q), n <= 34.
 *
 * Errors: every int-returning call returns RCS_OK (0) or a negative RCS_ERR_*
 * code and never aborts the process; rcs_last_error() gives a message. A call
 * that fails argument validation leaves the state unchanged.
 *
 * Ownership: every pointer argument is owned by the caller. Host arrays are
 * read (or written) only during the call. Pointers documented as DEVICE must
 * be device memory of the context's GPU. The device state is owned by the
 * context and freed by rcs_destroy().
 *
 * Streams: all device work of a context is issued on its stream (rcs_opts.stream,
 * a cudaStream_t; 0 = the legacy default stream). Calls taking or returning HOST
 * data synchronise that stream before returning; calls on DEVICE pointers only
 * enqueue work and return.
 */
#ifndef RCS_H
#define RCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define RCS_OK 0
#define RCS_ERR_ARG (-1)         /* malformed argument (null pointer, bad size, non-unitary matrix) */
#define RCS_ERR_QUBIT (-2)       /* qubit index out of range, or repeated within a gate */
#define RCS_ERR_OOM (-3)         /* device allocation failed */
#define RCS_ERR_CUDA (-4)        /* a CUDA runtime call failed (message has the CUDA error) */
#define RCS_ERR_TIMEOUT (-5)     /* a bounded device-side wait ran out; the kernel returned early */
#define RCS_ERR_UNSUPPORTED (-6) /* valid request this build cannot serve (e.g. no sm_103 GPU) */

/* ---- gate kinds (the Sycamore-class gate set; matrices below) */
#define RCS_GATE_SQRT_X 0 /* ((1+i) I + (1-i) X) / 2 */
#define RCS_GATE_SQRT_Y 1 /* ((1+i) I + (1-i) Y) / 2 */
#define RCS_GATE_SQRT_W 2 /* ((1+i) I + (1-i) W) / 2, W = (X + Y) / sqrt(2) */
#define RCS_GATE_FSIM 3   /* [[1,0,0,0],[0,c,-is,0],[0,-is,c,0],[0,0,0,e^{-i phi}]], c = cos theta, s = sin theta */
#define RCS_GATE_U1 4     /* caller's 2x2 unitary in rcs_gate.u */
#define RCS_GATE_U2 5     /* caller's 4x4 unitary in rcs_gate.u (local index j = bit(q[0]) + 2 bit(q[1])) */

#define RCS_FLAG_ADJOINT 1 /* apply the conjugate transpose of the gate */

/* ---- numerical paths for the state update */
#define RCS_PREC_FP32_PLAIN 0 /* one kernel launch per gate, FP32 SIMT (the baseline path) */
#define RCS_PREC_FP32_FUSED 1 /* gates fused into k-qubit unitaries (k <= k_max <= 7), FP32 SIMT */
#define RCS_PREC_BF16X3 2     /* fused 6-qubit unitaries on tcgen05 tensor cores, BF16 hi/lo split, 3 products, FP32 accumulate */
#define RCS_PREC_TF32X3 3     /* the same passes with a TF32 hi/lo split (3 products, FP32 accumulate): about
                               * 2^-21 relative error per product instead of 2^-17, at half the tensor rate */

typedef struct rcs_ctx rcs_ctx;
typedef struct rcs_plan rcs_plan;

/* Grid of qubits: rows x cols cells, minus `n_removed` cells whose row-major ids
 * are in `removed`. Only the qubit count n = rows*cols - n_removed matters to the
 * simulator; the circuit's gates name qubits by index. */
typedef struct {
    int32_t rows, cols, n_removed;
    const int32_t *removed;
} rcs_grid;

/* One gate. nq = 1 or 2 (must match kind). q[1] is ignored when nq = 1. theta and
 * phi are used by RCS_GATE_FSIM only. u (U1/U2 only) points to 2^nq x 2^nq
 * complex128 entries, row-major, interleaved (re, im); it must be unitary to
 * 1e-6. 40 bytes, naturally aligned. */
typedef struct {
    uint8_t kind, nq, flags, reserved;
    int32_t q[2];
    double theta, phi;
    const double *u;
} rcs_gate;

/* Options. precision: RCS_PREC_*. k_max: largest fused block (FP32_FUSED: 2..7,
 * default 4; widths 5 to 7 multiply tiles of slices by U in shared memory and are
 * bound by the FP32 FMA pipe, at 16 to 64 flop per byte; BF16X3 and TF32X3: 6).
 * autotune: 1 = for FP32_FUSED, rcs_apply_circuit chooses
 * k_max in 2..5 minimising (passes at width k) x (measured time of a width-k pass
 * on this state), by timed trial passes on the first call for this qubit count on
 * this device (cached for the process; the trials leave the state bit-identical).
 * flags: RCS_OPT_* bits (0 = defaults). stream: cudaStream_t for all device work. */
typedef struct {
    int32_t precision;
    int32_t k_max;
    int32_t autotune;
    int32_t flags;
    uint64_t stream;
} rcs_opts;

/* Opt-in for BF16X3 plans on 13 or more qubits: apply two consecutive 6-qubit passes in
 * one round trip of the state through HBM (the pair kernel: each 2^13-amplitude tile is
 * read once, both unitaries are applied on the tensor cores, and it is written once).
 * The arithmetic of each unitary is the same as in a single pass (BF16 hi/lo split of
 * the FP32 input, three products, FP32 accumulation); only the order of the FP32
 * accumulation differs. Off by default: on GB300 a pair launch currently takes longer
 * than the two single passes it replaces (its regrouping step and tensor-memory
 * traffic lengthen the per-tile pipeline), so the default plans keep one round trip
 * per pass. */
#define RCS_OPT_PAIR_PASSES 1

/* Description of a built plan (rcs_plan_info). */
typedef struct {
    int32_t n_qubits;
    int32_t precision;
    int64_t n_gates;
    int64_t n_passes;
    int32_t k_max;        /* largest block width used */
    int32_t pair_passes;  /* two-unitary round trips of a run from |0...0> (RCS_OPT_PAIR_PASSES) */
    double hbm_bytes;     /* algorithmic HBM bytes: 16 * 2^n per pass */
    double flops;         /* algorithmic real flops of all passes (x3 for the split-precision path) */
    int64_t prefix_passes; /* leading passes a run from |0...0> does on compact sub-states (0: none) */
    int32_t prefix_qubits; /* qubits of the widest (last) sub-state */
    int32_t prefix_stages; /* sub-states, nested and growing, each expanded into the next; the first
                              full pass reads the last one directly where its kernel allows, else it
                              is expanded into the full state */
    double zero_hbm_bytes; /* algorithmic HBM bytes of rcs_plan_run from |0...0>: each round trip (a
                              pass, or a pair of passes) at the size of the state it runs on, the zero
                              fill, the expansions */
} rcs_plan_stats;

/* ------------------------------------------------------------------ context */

/* Creates a context for n = rows*cols - n_removed qubits (1 <= n <= 34) on the
 * current CUDA device and sets the state to |0...0> (Section 3.2 item 1 starts
 * from the all-zero state of the circuit's qubits). Allocates 8 * 2^n bytes of
 * state plus the sampler's block sums and prefix (2^n / 1024 * 16 bytes). opts may be NULL
 * (FP32_FUSED, k_max 4, legacy stream). Returns RCS_ERR_OOM if the state does
 * not fit in device memory. */
int rcs_create(const rcs_grid *grid, const rcs_opts *opts, rcs_ctx **out);

/* Releases the context and its device memory. NULL is a no-op. */
void rcs_destroy(rcs_ctx *ctx);

/* Last error message for ctx, or for the calling thread when ctx is NULL. */
const char *rcs_last_error(const rcs_ctx *ctx);

/* Number of qubits of the context. */
int rcs_num_qubits(const rcs_ctx *ctx);

/* Changes the stream used for the context's device work (cudaStream_t). */
int rcs_set_stream(rcs_ctx *ctx, uint64_t stream);

/* Resets the state to |0...0>. Lazy: no kernel runs now. A tensor-core or fused
 * circuit started from |0...0> runs its leading passes on compact sub-states (the
 * qubits they have not touched yet are still |0>): the planner picks up to two
 * nested stages, each expanded into the next, and the first full pass reads the
 * last sub-state itself, writing the whole state. Any other first use fills the
 * state with |0...0> first. */
int rcs_reset(rcs_ctx *ctx);

/* ------------------------------------------------------------------ state construction (Section 3.2 item 1) */

/* Applies the n_gates host gates, in order, to the current state (psi <- U_G ... U_1 psi).
 * The gate list is validated (kinds, qubit range, distinct targets, unitarity of
 * U1/U2), fused by the planner of the context's precision into passes, uploaded
 * and launched. The gate array may be freed when the call returns; the launches
 * are asynchronous on the context's stream.
 *
 * Qubit layout: on a fresh state (after rcs_create or rcs_reset, which |0...0> makes
 * layout-free) the fused paths may store the circuit's qubits in a permuted bit
 * order, chosen so that no fused pass targets two of the five lowest index bits
 * (such passes cannot stream memory at full rate). This is invisible to the caller:
 * samples, amplitudes and XEB use the circuit's own qubit numbering, later circuits
 * follow the layout, and rcs_state_read/write/device first restore the identity
 * layout (at most five exact swap passes). rcs_qubit_layout reports it. */
int rcs_apply_circuit(rcs_ctx *ctx, const rcs_gate *gates, size_t n_gates);

/* Applies one dense k-qubit unitary (1 <= k <= 7) to targets[0..k-1] (distinct,
 * local index j = sum_i bit(targets[i]) 2^i); u_re_im holds 2^k x 2^k complex128
 * entries, row-major, interleaved, unitary to 1e-6. k = 6 with the BF16X3 or TF32X3
 * precision on n >= 13 runs the tensor-core kernel; every other k runs the FP32
 * fused kernels (k = 6, 7: U in shared memory). Asynchronous. */
int rcs_apply_unitary(rcs_ctx *ctx, int k, const int32_t *targets, const double *u_re_im);

/* Applies count dense unitaries in order (psi <- U_{count-1} ... U_0 psi), each as
 * rcs_apply_unitary would: unitary i has k[i] targets (1..7), listed in targets at
 * offset k[0] + ... + k[i-1], and its 2^k x 2^k complex128 matrix (row-major,
 * interleaved) at u_re_im[i]. All are validated before anything runs (a rejected
 * list leaves the state unchanged). With BF16X3 on n >= 13 qubits and
 * RCS_OPT_PAIR_PASSES in the context's flags, consecutive 6-qubit unitaries share one
 * round trip of the state (the pair kernel). Asynchronous. */
int rcs_apply_unitaries(rcs_ctx *ctx, size_t count, const int32_t *k, const int32_t *targets,
                        const double *const *u_re_im);

/* Host-only planning (no GPU needed): fuses the gates into passes for an n-qubit
 * state with the given options (NULL = FP32_FUSED, k_max 4). The plan keeps its
 * own copy of everything it needs. */
int rcs_plan_build(int n_qubits, const rcs_gate *gates, size_t n_gates, const rcs_opts *opts, rcs_plan **out);

/* Layout a plan stores its circuit in: phys_of[q] = index bit of circuit qubit q
 * (n_qubits entries; the identity unless the planner chose one, see
 * rcs_apply_circuit). A plan with a non-identity layout runs only on a fresh state. */
int rcs_plan_layout(const rcs_plan *plan, int32_t *phys_of);

/* Statistics of a plan. */
int rcs_plan_info(const rcs_plan *plan, rcs_plan_stats *out);

/* Pass i of a plan: *k targets written to targets[0..k-1] (ascending; local index
 * j = sum_i bit(targets[i]) 2^i) and, if u_re_im is not NULL, its 2^k x 2^k matrix
 * (row-major complex128, interleaved) as planned in FP64. targets must hold 8 ints,
 * u_re_im 2 * 4^k doubles. */
int rcs_plan_pass(const rcs_plan *plan, size_t i, int32_t *k, int32_t *targets, double *u_re_im);

/* Device time (ms) of the full-state passes of the last rcs_apply_circuit or
 * rcs_plan_run on this context (CUDA events around them on the context's stream;
 * the sub-state prefix and expansion are not included), and how many kernel
 * launches they took (a two-unitary round trip is one launch). Waits for those
 * passes to finish. */
int rcs_last_pass_timing(rcs_ctx *ctx, float *ms, int64_t *full_passes);

/* Uploads the plan's pass table and matrices to the device of ctx (once per plan
 * and context; later calls are no-ops). */
int rcs_plan_upload(rcs_ctx *ctx, rcs_plan *plan);

/* Launches every pass of an uploaded plan on the current state (asynchronous). A
 * plan with its own layout needs a fresh state (else RCS_ERR_ARG). */
int rcs_plan_run(rcs_ctx *ctx, rcs_plan *plan);

/* Frees a plan and its device copies. NULL is a no-op. */
void rcs_plan_destroy(rcs_plan *plan);

/* ------------------------------------------------------------------ readout */

/* Gathers amplitudes psi[bits[i]] into out_re_im[2i], out_re_im[2i+1] (complex64
 * promoted exactly to complex128). Section 3.2 item 3: each sampling job logs the
 * measurement amplitudes of its shots; this is that read-out of the built state
 * for any list of bitstrings. Synchronous. bits[i] < 2^n or RCS_ERR_ARG. */
int rcs_amplitudes(rcs_ctx *ctx, const uint64_t *bits, size_t n, double *out_re_im);

/* Current qubit layout of the context: phys_of[q] = index bit where circuit qubit q
 * is stored (n entries). */
int rcs_qubit_layout(const rcs_ctx *ctx, int32_t *phys_of);

/* Copies amplitudes [first, first+count) of the state to host floats (interleaved
 * re, im; 2*count floats), in the circuit's qubit numbering. Synchronous. */
int rcs_state_read(rcs_ctx *ctx, uint64_t first, uint64_t count, float *out_re_im);

/* Overwrites amplitudes [first, first+count) from host floats. Synchronous. */
int rcs_state_write(rcs_ctx *ctx, uint64_t first, uint64_t count, const float *in_re_im);

/* Device address of the state (2^n complex64, interleaved). The context keeps
 * ownership; writes through it must be followed by no other call of this API
 * until they are complete on the context's stream. */
int rcs_state_device(rcs_ctx *ctx, void **d_state);

/* Synchronises the context's stream and reports device-side errors raised by
 * earlier asynchronous calls (RCS_ERR_TIMEOUT for a bounded wait that ran out,
 * RCS_ERR_ARG for an out-of-range bitstring or an unusable state), then clears them. */
int rcs_sync(rcs_ctx *ctx);

/* Test hook for the bounded waits of the tensor-core kernels (single passes and pair
 * passes), process-wide: while skip_tile >= 0, every tensor-core launch has its first CTA
 * skip the MMAs of its tile number skip_tile (it issues and commits nothing for that
 * tile), so the waits for that tile run out after wait_limit_s seconds of SM clock; the
 * kernel then stops, waits for its own MMAs and copies in flight, frees its tensor memory
 * and raises the error that rcs_sync reports as RCS_ERR_TIMEOUT (the state is then
 * partly updated). skip_tile = -1 restores normal operation; wait_limit_s <= 0 restores
 * the default limit (about one second). The limit converts to cycles at the current
 * device's clock rate. No GPU fault is involved. */
int rcs_tc_test_fault(int64_t skip_tile, double wait_limit_s);

/* T = sum_i |psi_i|^2, reduced exactly in 2^-62 fixed point and returned as double.
 * This is the normalisation that the sampler's cumulative distribution (Section 3.2
 * item 3) and the linear XEB (Section 3.2 item 4, scored in Section 5.1) divide by.
 * Synchronous. */
int rcs_norm(rcs_ctx *ctx, double *out);

/* ------------------------------------------------------------------ sampling (Section 3.2 item 3) */

/* Draws `shots` samples x_s = smallest i with C_i > u_s * T, where C_i = sum_{j<=i}
 * |psi_j|^2, T = C_{2^n-1} (prefix sums exact in 2^-62 fixed point), and u_s is
 * word (s mod 4) of Philox4x64-10(counter = (s div 4, 0, 0, 0), key = (seed, 0))
 * mapped to [0,1) as (x >> 11) 2^-53. Zero-probability indices are never drawn.
 * Writes shots uint64 indices to HOST out_bits. Synchronous. The state must
 * have norm < 3.9 (unitary circuits keep it at 1); a state of norm 0 gives
 * 2^64 - 1 for every shot. */
int rcs_sample(rcs_ctx *ctx, uint64_t shots, uint64_t seed, uint64_t *out_bits);

/* As rcs_sample, writing to DEVICE memory d_out_bits; asynchronous (a call with
 * more shots than any before it on this context first grows a device scratch of
 * 8 bytes per shot, which synchronizes the context's stream). */
int rcs_sample_device(rcs_ctx *ctx, uint64_t shots, uint64_t seed, uint64_t *d_out_bits);

/* Shots first_shot .. first_shot + shots - 1 of the same stream (shot s always uses
 * uniform u_s): sampling a state in pieces, in one process or in several that loaded
 * the same saved state, gives exactly the draws of one rcs_sample call. HOST out_bits.
 * Synchronous. RCS_ERR_ARG if the range overflows 64 bits. */
int rcs_sample_range(rcs_ctx *ctx, uint64_t first_shot, uint64_t shots, uint64_t seed, uint64_t *out_bits);

/* ------------------------------------------------------------------ persistence (Section 3.2 items 2-3)

 * The paper writes the built state to a shared filesystem and reloads it in many
 * sampling jobs. rcs_state_save writes the context's state to `path`: a 280-byte
 * header (magic "RCSSTATE", version 1, n, the stored layout of each qubit, 2^n),
 * then 2^n complex64 amplitudes in stored order (8 x 2^n bytes; 128 GiB at 34
 * qubits), streamed through a 64 MiB pinned buffer. rcs_state_load reads such a file
 * into a context of the same qubit count, layout included, so samples, amplitudes
 * and XEB stay in the circuit's own numbering. Both synchronous. Errors: RCS_ERR_ARG
 * for a file that cannot be opened, written or read in full, a wrong header or qubit
 * count (the state is untouched when the header is rejected; a truncated file
 * leaves it undefined), RCS_ERR_OOM / RCS_ERR_CUDA for the staging copies. */
int rcs_state_save(rcs_ctx *ctx, const char *path);
int rcs_state_load(rcs_ctx *ctx, const char *path);

/* ------------------------------------------------------------------ scoring (Section 3.2 item 4) */

/* Linear XEB of the samples against the current state:
 * F = 2^n * (1/N) sum_s |psi_{x_s}|^2 / T - 1, reduced in FP64. HOST samples,
 * HOST result. Synchronous. A sample >= 2^n gives RCS_ERR_ARG. */
int rcs_xeb(rcs_ctx *ctx, const uint64_t *samples, size_t n, double *out_xeb);

/* As rcs_xeb with DEVICE samples and a DEVICE double result; asynchronous.
 * An out-of-range sample makes the result NaN. */
int rcs_xeb_device(rcs_ctx *ctx, const uint64_t *d_samples, size_t n, double *d_out_xeb);

/* ------------------------------------------------------------------ batched circuits */

/* Many independent circuits (different qubit counts and depths) run together: one
 * persistent kernel applies every fused pass of every circuit, then each circuit is
 * sampled and scored; the whole sequence is one captured CUDA graph, replayed by
 * rcs_batch_launch. This is the many-instance form of Section 3.2 items 1, 3, 4 (the
 * paper's jobs, Section 4.3). */
typedef struct rcs_batch rcs_batch;

/* One circuit of a batch: n_qubits (2..30), its host gate list (validated and
 * copied at creation), the shots to draw (0..2^26) and the sampling seed. */
typedef struct {
    int32_t n_qubits;
    int32_t reserved;
    const rcs_gate *gates;
    size_t n_gates;
    uint64_t shots;
    uint64_t seed;
} rcs_batch_item;

/* Builds a batch: allocates every state and sampler buffer, plans every circuit,
 * uploads what the kernels need and captures the graph. Synchronous.
 * Engine, by opts->precision:
 *   FP32_FUSED (or FP32_PLAIN, or opts NULL): every pass of every circuit is an item
 *     list of one persistent kernel launch. The passes are FP32 fused; opts->k_max in
 *     2..5 fixes the fusion width, while 0 or opts->autotune = 1 lets timed trials of
 *     the batched kernel choose it per qubit count, cached for the process.
 *   BF16X3 or TF32X3: every circuit is planned like rcs_apply_circuit on a fresh
 *     state (fused 6-qubit tensor-core passes, its own qubit layout and sub-state
 *     prefix). Every pass of every circuit of 13 or more qubits is a work item of one
 *     cooperative persistent tensor-core launch; the tiles per work item are chosen by
 *     timed launches of that kernel on the batch at creation (rcs_batch_tuning).
 *     Circuits under 13 qubits (FP32 fused passes), or with no gates, run as launch
 *     chains of their own before it. opts->k_max must be 0 or 6.
 * Samples, XEB and rcs_batch_state_read use each circuit's own qubit numbering in
 * either engine. */
int rcs_batch_create(const rcs_batch_item *items, size_t n_items, const rcs_opts *opts, rcs_batch **out);

/* Launches the batch's graph on `stream` (cudaStream_t): reset every state to
 * |0...0>, apply all circuits, sample, score. Asynchronous. */
int rcs_batch_launch(rcs_batch *batch, uint64_t stream);

/* Synchronises `stream` and reports device-side errors of the last launch:
 * RCS_ERR_TIMEOUT if a pass waited past its limit for the passes before it (the
 * kernel then stops taking work and returns), then clears them. */
int rcs_batch_wait(rcs_batch *batch, uint64_t stream);

/* Number of circuits; per circuit its qubit count, chosen fusion width and pass count. */
int rcs_batch_size(const rcs_batch *batch);
int rcs_batch_info(const rcs_batch *batch, size_t i, int32_t *n_qubits, int32_t *k, int64_t *n_passes);

/* Tensor-core engine: the work-item size of the persistent kernel (tiles of 128 slices
 * per item) that the timed trials at creation chose, and each candidate's trial time
 * (ms per launch of the kernel alone, HOST doubles, candidates 2, 4, 8, 16 and 32 tiles
 * in that order; 0 for a candidate not tried). Either pointer may be NULL.
 * RCS_ERR_UNSUPPORTED when no circuit of the batch runs in the persistent kernel (the
 * FP32 engine, or only circuits under 13 qubits). */
int rcs_batch_tuning(const rcs_batch *batch, uint32_t *tiles_per_item, double *trial_ms);

/* Copies circuit i's samples (shots uint64, HOST) and XEB (HOST double) of the last
 * completed launch; either pointer may be NULL. Synchronous. */
int rcs_batch_result(rcs_batch *batch, size_t i, uint64_t *out_bits, double *out_xeb);

/* Copies amplitudes [first, first+count) of circuit i's state to host floats. */
int rcs_batch_state_read(rcs_batch *batch, size_t i, uint64_t first, uint64_t count, float *out_re_im);

/* Test hook for the bounded waits of either persistent engine: work item skip_item
 * (>= 0; the FP32 kernel's items, or the persistent tensor-core kernel's) never
 * publishes its completion, so the passes after it wait until wait_limit_s and the
 * launch ends with RCS_ERR_TIMEOUT; skip_item = -1 restores normal operation (limit
 * ~2 s by default). Everything the item issued still completes. Recaptures the graph.
 * RCS_ERR_UNSUPPORTED for a tensor-core batch none of whose circuits runs in the
 * persistent kernel. */
int rcs_batch_set_fault(rcs_batch *batch, int64_t skip_item, double wait_limit_s);

/* Last error message of the batch. */
const char *rcs_batch_last_error(const rcs_batch *batch);

/* Frees the batch (synchronises the device first). NULL is a no-op. */
void rcs_batch_destroy(rcs_batch *batch);

/* The whole batch in one synchronous call: circuit i has grids[i] (its qubit count
 * rows*cols - n_removed, 2..30), the host gate list gates[i][0 .. n_gates[i]-1],
 * shots[i] shots and sampling seed seeds[i]. Creates a batch with opts (engine as in
 * rcs_batch_create; NULL = the persistent FP32 engine), runs it once on opts->stream,
 * copies circuit i's samples to out_bits[i] (shots[i] uint64, HOST) and its XEB to
 * out_xeb[i] (HOST), and frees everything. out_bits, any out_bits[i], or out_xeb may
 * be NULL to skip that output. Errors as the calls it is made of; the message is in
 * rcs_last_error(NULL). */
int rcs_batch_run(const rcs_grid *grids, const rcs_gate *const *gates, const size_t *n_gates, size_t n_inst,
                  const uint64_t *shots, const uint64_t *seeds, uint64_t **out_bits, double *out_xeb,
                  const rcs_opts *opts);

/* ------------------------------------------------------------------ allocation-free scoring */

/* Linear XEB, as rcs_xeb_device, for callers that cannot allocate device memory:
 * no context is needed and no cudaMalloc, cudaFree or allocating library routine
 * is called. (The paper has no counterpart; this serves callers such as hosts
 * whose device memory comes only from their own arena, or that forbid device
 * allocations after start-up.)
 *
 * d_state: DEVICE, 2^n_qubits complex64 amplitudes (interleaved re, im), 16-byte
 * aligned; d_samples: DEVICE, count uint64 basis indices, 8-byte aligned;
 * d_out_xeb: DEVICE, one double, 8-byte aligned (a misaligned pointer gives
 * RCS_ERR_ARG before anything is launched);
 * stream: cudaStream_t (0 = legacy default stream). Work is enqueued on the
 * stream and the call returns; an index >= 2^n or an unusable state makes the
 * result NaN.
 *
 * Scratch lives in one fixed 192 KiB device array inside this library, which
 * every GPU that loads the library holds until the process exits. Hence:
 * count <= 67108864 (2^26) and 1 <= n_qubits <= 34, else RCS_ERR_ARG with a
 * message for rcs_last_error(NULL). The first call on a device looks up the
 * array's device address (with that device current). The address is kept for
 * the process: after a cudaDeviceReset() of a device, do not call this entry
 * point on that device again. Devices with ordinals >= 64 get
 * RCS_ERR_UNSUPPORTED. Every call shares the array: calls whose work overlaps on
 * the GPU (other streams, other host threads) race and must be serialised by the
 * caller. */
int rcs_xeb_static(const void *d_state, int n_qubits, const uint64_t *d_samples, size_t count, double *d_out_xeb,
                   uint64_t stream);

#ifdef __cplusplus
}
#endif
#endif /* RCS_H */
