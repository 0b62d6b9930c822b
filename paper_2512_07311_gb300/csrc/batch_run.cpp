// The one-call form of the batched engine (rcs_batch_run): builds a batch from
// per-circuit grids, gate lists, shot counts and seeds, runs it once, copies the
// samples and XEB values out and frees it, through the batch calls of the C ABI.
#include <string>
#include <vector>

#include "internal.h"
#include "rcs.h"

using namespace rcs;

extern "C" {

int rcs_batch_run(const rcs_grid *grids, const rcs_gate *const *gates, const size_t *n_gates, size_t n_inst,
                  const uint64_t *shots, const uint64_t *seeds, uint64_t **out_bits, double *out_xeb,
                  const rcs_opts *opts) {
    if (n_inst == 0) return set_thread_error(RCS_ERR_ARG, "empty batch");
    if (!grids || !gates || !n_gates || !shots || !seeds) return set_thread_error(RCS_ERR_ARG, "null argument");
    std::vector<rcs_batch_item> items(n_inst);
    for (size_t i = 0; i < n_inst; ++i) {
        const rcs_grid &g = grids[i];
        if (g.rows < 1 || g.cols < 1 || g.n_removed < 0 || g.n_removed >= g.rows * g.cols ||
            (g.n_removed > 0 && !g.removed))
            return set_thread_error(RCS_ERR_ARG, "bad grid of circuit " + std::to_string(i));
        items[i].n_qubits = g.rows * g.cols - g.n_removed;
        items[i].reserved = 0;
        items[i].gates = gates[i];
        items[i].n_gates = n_gates[i];
        items[i].shots = shots[i];
        items[i].seed = seeds[i];
    }
    rcs_batch *b = nullptr;
    int rc = rcs_batch_create(items.data(), n_inst, opts, &b);
    if (rc != RCS_OK) return rc;
    const uint64_t stream = opts ? opts->stream : 0;
    if ((rc = rcs_batch_launch(b, stream)) == RCS_OK && (rc = rcs_batch_wait(b, stream)) == RCS_OK)
        for (size_t i = 0; i < n_inst && rc == RCS_OK; ++i)
            rc = rcs_batch_result(b, i, out_bits ? out_bits[i] : nullptr, out_xeb ? out_xeb + i : nullptr);
    if (rc != RCS_OK) set_thread_error(rc, rcs_batch_last_error(b));
    rcs_batch_destroy(b);
    return rc;
}

}  // extern "C"
