// Internal declarations shared by the library's own translation units.
#pragma once

#include <complex>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/rcs.h"

namespace rcs {

using cd = std::complex<double>;

constexpr int kMaxQubits = 34;
constexpr int kSampleBlockLog2 = 10;  // sampler block = 1024 amplitudes
constexpr int kTcK = 6;               // width of the tensor-core fused pass
constexpr int kSimtParamK = 4;        // widest FP32 fused pass with U in the kernel parameters
constexpr int kSimtKMax = 7;          // widest FP32 fused pass (U from a device image above 4)

// Records msg as the calling thread's last error (rcs_last_error(NULL)); returns code.
int set_thread_error(int code, const std::string &msg);

// Text of the last failed kernel launch on this thread (cleared by the call).
std::string take_launch_error();

// Runs f(0) .. f(count - 1) on the library's persistent host worker threads (the calling
// thread takes part) and returns when all are done; f must be safe to run concurrently.
void host_parallel_for(size_t count, const std::function<void(size_t)> &f);

// ---- gates (gates.cpp)
struct HostGate {
    int nq;
    int q[2];
    cd m[16];  // 2^nq x 2^nq row-major, local index j = bit(q[0]) + 2 bit(q[1])
};

// Validates one ABI gate against an n-qubit register and writes its matrix.
// Returns RCS_OK or an RCS_ERR_* code with a message in *why.
int gate_to_host(const rcs_gate &g, int n, HostGate *out, std::string *why);

// ---- plan (planner.cpp)
enum PassKind : int32_t {
    PASS_1Q = 0,    // plain per-gate, one qubit
    PASS_2Q = 1,    // plain per-gate, two qubits
    PASS_SIMT = 2,  // fused k-qubit unitary, FP32 SIMT
    PASS_TC = 3,    // fused 6-qubit unitary, tcgen05 split precision (BF16x3 or TF32x3, per plan)
};

struct Pass {
    PassKind kind;
    int k;
    int t[8];               // ascending targets
    std::vector<cd> U;      // 2^k x 2^k, local index over ascending targets
};

struct Plan {
    int n = 0;
    std::vector<int> phys_of;  // stored position of each circuit qubit; empty = identity
    int precision = RCS_PREC_FP32_FUSED;
    int k_max = 4;
    int64_t n_gates = 0;
    std::vector<Pass> passes;
    std::vector<int> stage_spans;  // sub-state widths of a run from |0...0> (empty: one of n - 4)
    bool pairs = false;  // consecutive tensor-core passes run as one two-unitary round trip (BF16X3)
    // device copies, per context device (uploaded lazily)
    int dev = -1;
    void *d_tc_ops = nullptr;   // hi/lo operand images of PASS_TC passes
    std::vector<int64_t> tc_offset;  // byte offset of each pass's image (-1 if none): the split
                                     // images of PASS_TC passes, the FP32 U of wide PASS_SIMT ones
    std::vector<int64_t> pair_offset;  // byte offset of each pass's pair-kernel image (-1 if none)
};

// Fuses gates into passes. k_max: largest block; pad_to: 0, or a width every
// block is padded to with identity qubits (the tensor-core path needs k = 6).
void plan_fuse(int n, const std::vector<HostGate> &gates, int k_max, int pad_to, std::vector<Pass> *out);

// The same in two steps: the blocking (which gates form each pass; independent of
// how the qubits are labelled), then the passes for a gate list with those blocks.
struct Blocking {
    std::vector<std::vector<int>> gates;  // gate indices of each block, in application order
    // Run from |0...0>: stage s holds blocks [stage_end[s-1], stage_end[s]) and runs on a
    // sub-state of at most spans[s] qubits (nested, growing); padding keeps its blocks off
    // avoid[s], the qubits outside that sub-state. Empty: the default single stage (n - 4).
    std::vector<int> spans;
    std::vector<uint64_t> avoid;
    std::vector<int> stage_end;
};
// from_zero: the blocks will run from |0...0>, so they are chosen by cost with the
// sub-state prefix counted (see planner.cpp); otherwise by fewest blocks.
Blocking plan_blocks(int n, const std::vector<HostGate> &gates, int k_max, bool from_zero);
void make_passes(int n, const std::vector<HostGate> &gates, const Blocking &b, int pad_to, std::vector<Pass> *out);

// Physical position of every logical qubit for a blocking (phys_of[logical]): up
// to five qubits that never share a block trade places with qubits on bits 0..4
// (so no pass targets two of the lowest qubits); at most five transpositions.
// Identity when n < 12. Returns whether the layout differs from the identity.
bool choose_layout(int n, const std::vector<HostGate> &gates, const Blocking &b, int *phys_of);

// Bit permutation of basis indices: bit i of the input moves to bit to[i].
struct BitMap {
    uint8_t to[64];
    int32_t n;
    int32_t identity;
};
BitMap identity_map(int n);

// Plain per-gate plan: one PASS_1Q / PASS_2Q per gate (targets canonicalised ascending).
void plan_plain(int n, const std::vector<HostGate> &gates, std::vector<Pass> *out);

// Device error bits (the context's error word).
constexpr int kErrBadAmplitude = 1;  // |amplitude component| >= 2, Inf or NaN met by a reduction
constexpr int kErrNormOverflow = 2;  // fixed-point total >= 4 (state norm too large to sample)
constexpr int kErrBadIndex = 4;      // bitstring >= 2^n met by a gather
constexpr int kErrTimeout = 8;       // a bounded wait inside a kernel ran out

// ---- kernels (launchers; all asynchronous on `stream`)

int launch_init_zero(void *psi, int n, void *stream);
int launch_expand(void *psi, int n, const void *sub, uint64_t tmask, void *stream);

// Leading passes of a fused plan that a run from |0...0> can do on compact
// sub-states. Stage s takes the longest following run of passes whose targets, with
// those of the earlier stages, span at most plan.stage_spans[s] qubits (n - 4 when no
// spans are set), widened with untouched qubits to the size the kernels need. Stage
// masks are nested. Returns the number of sub-state passes (0: not worth it).
struct SubStage {
    int first = 0, count = 0;  // passes [first, first + count)
    uint64_t tmask = 0;        // qubits of the sub-state (cumulative over the stages)
};
int plan_stages(const Plan &plan, std::vector<SubStage> *stages);
// Device bytes of the sub-state buffers of the stages (one after another).
size_t substage_bytes(const std::vector<SubStage> &stages);
// Runs the stages of a plan from |0...0> into psi (2^n amplitudes): reset of the first
// sub-state, its passes, an expansion into the next sub-state, ..., and either an
// expansion into psi or, when the next pass can read a sub-state, that pass taking the
// last sub-state as input (*fused = 1: the caller resumes one pass later). `sub` holds
// substage_bytes(stages). Asynchronous; launch error text kept.
int run_substages(const Plan &plan, const std::vector<SubStage> &stages, void *psi, void *sub,
                  const uint8_t *d_ops, int *d_err, void *stream, int *fused);
// Launches one pass of a plan on a 2^n-amplitude state (ops: its operand image, if any).
int launch_plan_pass(void *psi, int n, const Pass &p, const uint8_t *ops, int *d_err, void *stream, bool tf32);
int launch_pass_plain(void *psi, int n, const Pass &p, void *stream);
// Fused FP32 SIMT pass of width p.k = 1..kSimtKMax. Widths up to kSimtParamK carry U in
// the kernel parameters (ops unused); wider ones read it from ops, the device copy of
// simt_build_ops(p) (16-byte aligned), and give RCS_ERR_ARG without it.
int launch_pass_simt(void *psi, int n, const Pass &p, const uint8_t *ops, void *stream);
// Bytes of a SIMT pass's device image (0 for widths up to kSimtParamK) and its builder.
size_t simt_ops_bytes(int k);
void simt_build_ops(const Pass &p, uint8_t *out);
// Sets the fused SIMT kernels' shared-memory attribute on the current device (once);
// launch_pass_simt calls it, and a caller about to capture a graph calls it first.
int simt_prepare_device();
// Sets the tensor-core kernels' shared-memory attribute on the current device (once);
// launch_pass_tc calls it, and a caller about to capture a graph calls it first.
int tc_prepare_device();
// tf32: the TF32x3 kernel (operand image from tc_build_ops(p, img, true)), else BF16x3.
int launch_pass_tc(void *psi, int n, const Pass &p, const void *d_ops, int *d_err, void *stream, bool tf32);
// The same pass reading its input from a sub-state instead of psi: the state is |0> on
// the qubits outside tmask, and sub holds its amplitudes with those qubits at 0 at their
// compact index; the pass writes the whole 2^n state to psi (an expansion and a pass in
// one). tc_pass_takes_substate says whether a pass can run this way (slice-order kernel).
bool tc_pass_takes_substate(const Pass &p, int n);
int launch_pass_tc_from_sub(void *psi, int n, const Pass &p, const void *d_ops, int *d_err, void *stream, bool tf32,
                            const void *sub, uint64_t tmask);

// Test hook of the tensor-core kernels' bounded waits (process-wide): the wait limit and
// the tile (of CTA 0) whose MMAs are skipped, as every launch reads them, and the setter.
void tc_test_fault(long long *wait_cycles, int *skip_tile);
void tc_set_test_fault(int skip_tile, long long wait_cycles);

// Persistent tensor-core kernel of the batched engine (k_batch_tc.cu): every pass of
// many circuits in one cooperative launch. A step is one 6-qubit tensor-core pass on a
// state of m qubits (13..30) at dst; its input is dst itself, or a sub-state src whose
// qubits are tmask (in dst's numbering; the state is |0> on the others), or, with
// from_zero, the state |0...0>. ops is the pass's operand image (tc_build_ops).
struct BtcStep {
    void *dst = nullptr;
    int m = 0;
    const void *src = nullptr;
    int src_m = 0;          // qubits of src (popcount of tmask)
    uint64_t tmask = 0;
    bool from_zero = false;
    const void *ops = nullptr;
    Pass p;
};
struct BtcPlan;
// Builds the pass and item tables (each pass cut into items of tiles_per_item tiles of
// 128 slices) on the current device and sets the kernel's shared-memory attribute.
// Steps of one circuit run in order; circuits are independent. Synchronous.
int btc_create(const std::vector<std::vector<BtcStep>> &circuits, bool tf32, uint32_t tiles_per_item,
               BtcPlan **out);
uint32_t btc_items(const BtcPlan *p);
// Clears the completion counters and launches the kernel on `stream` (capturable).
// d_err[0] receives kErrTimeout if a wait ran out; d_err[1] is the launch-wide abort
// word (0 on entry). skip_item >= 0: that item never publishes its completion (test).
int btc_launch(const BtcPlan *p, int *d_err, long long wait_cycles, long long skip_item, void *stream);
void btc_destroy(BtcPlan *p);

// Size in bytes of the operand image of one 6-qubit pass (BF16x3: 64 KB, TF32x3:
// 96 KB), and its builder.
size_t tc_ops_bytes(bool tf32);
void tc_build_ops(const Pass &p, void *host_image, bool tf32);

// Two consecutive 6-qubit passes in one round trip of a 2^n state (k_pair.cu, BF16x3):
// whether two passes can run this way, the size and builder of one pass's image for
// it (48 KB, complex block form), and the launcher.
bool pair_fits(const Pass &p1, const Pass &p2, int n);
size_t pair_ops_bytes();
void pair_build_ops(const Pass &p, void *host_image);
int launch_pair_tc(void *psi, int n, const Pass &p1, const Pass &p2, const void *d_ops1, const void *d_ops2, int *d_err,
                   void *stream);
// Whether passes i and i+1 (< end) of a plan run as one two-unitary round trip.
bool plan_pairs_at(const Plan &plan, size_t i, size_t end, int n);
// Launches passes [first, end) of a plan on the 2^n-amplitude state psi, their targets
// renumbered into the sub-state of mask T when T != 0; consecutive tensor-core passes
// share a round trip where plan_pairs_at says so. *launches counts kernel launches.
int launch_pass_range(const Plan &plan, void *psi, int n, size_t first, size_t end, uint64_t T, const uint8_t *d_ops,
                      int *d_err, void *stream, int64_t *launches);

// Sampler / readout (k_sample.cu)
// to_stored: caller basis index -> stored index (the state's qubit layout). Blocks are
// 1024 consecutive caller indices in every layout.
int launch_block_sums(const void *psi, int n, uint64_t *bsum, int *d_err, const BitMap &to_stored, void *stream);
size_t scan_chunks(int n);
int launch_block_scan(const uint64_t *bsum, uint64_t *bpre, uint64_t *chunk_tot, uint64_t *total, int n, int *d_err,
                      void *stream);
// to_stored / in_map take the caller's basis index to the stored one. The sampler
// draws the caller index x = min{i : C_i > u T} with C in the caller's order, from
// block sums made with the same map.
// Shots first .. first + shots - 1 of the seed's stream (shot g uses uniform g).
// Needs the block prefix bpre and total T of launch_block_scan; hist (2^(n-10) entries,
// the block sums' array: overwritten), chunk (scan_chunks(n) + 1 entries) and order
// (shots entries) are scratch.
int launch_sample(const void *psi, int n, uint64_t *hist, const uint64_t *bpre, const uint64_t *total, uint64_t *chunk,
                  uint64_t first, uint64_t shots, uint64_t seed, uint64_t *d_out, uint64_t *order, int *d_err,
                  const BitMap &to_stored, void *stream);
int launch_gather(const void *psi, int n, const uint64_t *d_bits, size_t count, double *d_out_re_im, int *d_err,
                  const BitMap &in_map, void *stream);
int launch_xeb(const void *psi, int n, const uint64_t *d_samples, size_t count, const uint64_t *total,
               double *d_partials, double *d_out, const BitMap &in_map, void *stream);
size_t xeb_partials_count(size_t count);

// ---- planning shared by single circuits and batches (api.cu)
// Plans a circuit for a fresh n-qubit state with the given options (a qubit layout
// allowed) and builds the operand images of its tensor-core passes; thread error on failure.
int plan_fresh_circuit(int n, const std::vector<HostGate> &gates, const rcs_opts &o, Plan *plan,
                       std::vector<uint8_t> *images);
// A pass of the plan's sub-state prefix, its targets renumbered into the sub-state of mask T.
Pass substate_pass(const Pass &p, uint64_t T);
// Bit map of a plan's layout: caller basis index -> stored index.
BitMap plan_to_stored(const Plan &plan);

}  // namespace rcs
