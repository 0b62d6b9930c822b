// Gate-fusion planner: merges runs of 1- and 2-qubit gates into dense k-qubit
// unitaries (one state pass each). The paper's engine is closed and describes no
// fusion; this is the standard greedy frontier construction on the gate DAG.
//
// A block is grown from the current frontier (gates whose predecessors on every
// one of their qubits are already placed). Among the frontier gates whose qubits
// keep the block within k_max qubits, the planner takes the one adding the fewest
// new qubits, earliest in circuit order on ties, until none fits. Every gate in a
// block has all its predecessors in earlier blocks or in the block itself, and
// gates left out either follow it on a block qubit or act on other qubits, so the
// product of the blocks in emission order equals the circuit.
#include <algorithm>
#include <bit>
#include <cstring>

#include "internal.h"

namespace rcs {

// Multiplies U (2^k x 2^k, row-major) on the left by gate g embedded on local
// qubit positions pos[0..nq-1].
static void left_multiply(std::vector<cd> &U, int k, const HostGate &g, const int *pos) {
    const int d = 1 << k;
    const int gd = 1 << g.nq;
    uint32_t gmask = 0;
    for (int i = 0; i < g.nq; ++i) gmask |= 1u << pos[i];
    for (int col = 0; col < d; ++col) {
        for (int r0 = 0; r0 < d; ++r0) {
            if (r0 & gmask) continue;
            int rows[4];
            cd v[4];
            for (int j = 0; j < gd; ++j) {
                int r = r0;
                for (int i = 0; i < g.nq; ++i)
                    if ((j >> i) & 1) r |= 1 << pos[i];
                rows[j] = r;
                v[j] = U[size_t(r) * d + col];
            }
            for (int j = 0; j < gd; ++j) {
                cd s = 0.0;
                for (int l = 0; l < gd; ++l) s += g.m[j * gd + l] * v[l];
                U[size_t(rows[j]) * d + col] = s;
            }
        }
    }
}

static Pass make_pass(PassKind kind, uint64_t qmask, const std::vector<const HostGate *> &blk) {
    Pass p;
    p.kind = kind;
    p.k = std::popcount(qmask);
    int i = 0;
    for (int q = 0; q < 64; ++q)
        if ((qmask >> q) & 1) p.t[i++] = q;
    for (; i < 8; ++i) p.t[i] = -1;
    const int d = 1 << p.k;
    p.U.assign(size_t(d) * d, cd(0.0));
    for (int r = 0; r < d; ++r) p.U[size_t(r) * d + r] = 1.0;
    for (const HostGate *g : blk) {
        int pos[2];
        for (int a = 0; a < g->nq; ++a) pos[a] = int(std::find(p.t, p.t + p.k, g->q[a]) - p.t);
        left_multiply(p.U, p.k, *g, pos);
    }
    return p;
}

void plan_fuse(int n, const std::vector<HostGate> &gates, int k_max, int pad_to, std::vector<Pass> *out) {
    out->clear();
    const size_t G = gates.size();
    k_max = std::max(2, std::min(k_max, n));
    std::vector<std::vector<int>> queue(n);
    for (size_t g = 0; g < G; ++g)
        for (int a = 0; a < gates[g].nq; ++a) queue[gates[g].q[a]].push_back(int(g));
    std::vector<size_t> head(n, 0);
    std::vector<uint64_t> gmask(G);
    for (size_t g = 0; g < G; ++g) {
        uint64_t m = 0;
        for (int a = 0; a < gates[g].nq; ++a) m |= 1ull << gates[g].q[a];
        gmask[g] = m;
    }
    auto ready = [&](int g) {
        for (int a = 0; a < gates[g].nq; ++a) {
            int q = gates[g].q[a];
            if (head[q] >= queue[q].size() || queue[q][head[q]] != g) return false;
        }
        return true;
    };
    size_t placed = 0;
    while (placed < G) {
        uint64_t Q = 0;
        std::vector<const HostGate *> blk;
        for (;;) {
            int best = -1, best_new = 1 << 30;
            for (int q = 0; q < n; ++q) {
                if (head[q] >= queue[q].size()) continue;
                int g = queue[q][head[q]];
                if (!ready(g)) continue;
                uint64_t nm = Q | gmask[g];
                if (std::popcount(nm) > k_max) continue;
                int nnew = std::popcount(gmask[g] & ~Q);
                if (nnew < best_new || (nnew == best_new && g < best)) {
                    best = g;
                    best_new = nnew;
                }
            }
            if (best < 0) break;
            Q |= gmask[best];
            blk.push_back(&gates[best]);
            for (int a = 0; a < gates[best].nq; ++a) head[gates[best].q[a]]++;
            ++placed;
        }
        // pad with the highest free qubits (identity on them)
        for (int q = n - 1; q >= 0 && std::popcount(Q) < pad_to; --q) Q |= 1ull << q;
        out->push_back(make_pass(pad_to > 0 ? PASS_TC : PASS_SIMT, Q, blk));
    }
}

void plan_plain(int n, const std::vector<HostGate> &gates, std::vector<Pass> *out) {
    (void)n;
    out->clear();
    out->reserve(gates.size());
    for (const HostGate &g : gates) {
        uint64_t m = 0;
        for (int a = 0; a < g.nq; ++a) m |= 1ull << g.q[a];
        std::vector<const HostGate *> one{&g};
        out->push_back(make_pass(g.nq == 1 ? PASS_1Q : PASS_2Q, m, one));
    }
}

}  // namespace rcs
