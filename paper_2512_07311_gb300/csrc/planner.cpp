// Gate-fusion planner: merges runs of 1- and 2-qubit gates into dense k-qubit
// unitaries (one state pass each). The paper's engine is closed and describes no
// fusion; this is a greedy frontier construction on the gate DAG.
//
// A block is grown from the current frontier (gates whose predecessors on every
// one of their qubits are already placed), adding frontier gates while the block
// stays within k_max qubits. Every gate in a block has all its predecessors in
// earlier blocks or in the block itself, and gates left out either follow it on a
// block qubit or act on other qubits, so the product of the blocks in emission
// order equals the circuit.
#include <algorithm>
#include <bit>
#include <cmath>
#include <cstring>
#include <array>
#include <mutex>
#include <memory>
#include <functional>
#include <condition_variable>
#include <atomic>
#include <unordered_set>
#include <thread>

#include "internal.h"

namespace rcs {

// Multiplies U (2^k x 2^k, row-major) on the left by gate g embedded on local
// qubit positions pos[0..nq-1].
static void left_multiply(std::vector<cd> &U, int k, const HostGate &g, const int *pos) {
    const int d = 1 << k;
    const int gd = 1 << g.nq;
    uint32_t gmask = 0;
    for (int i = 0; i < g.nq; ++i) gmask |= 1u << pos[i];
    double mr[16], mi[16];
    for (int e = 0; e < gd * gd; ++e) {
        mr[e] = g.m[e].real();
        mi[e] = g.m[e].imag();
    }
    double *u = reinterpret_cast<double *>(U.data());  // interleaved (re, im), row-major
    for (int r0 = 0; r0 < d; ++r0) {
        if (r0 & gmask) continue;
        double *row[4];
        for (int j = 0; j < gd; ++j) {
            int r = r0;
            for (int i = 0; i < g.nq; ++i)
                if ((j >> i) & 1) r |= 1 << pos[i];
            row[j] = u + size_t(r) * 2 * d;
        }
        for (int col = 0; col < d; ++col) {  // rows are contiguous: the inner loop streams them
            double vr[4], vi[4];
            for (int l = 0; l < gd; ++l) {
                vr[l] = row[l][2 * col];
                vi[l] = row[l][2 * col + 1];
            }
            for (int j = 0; j < gd; ++j) {
                double sr = 0.0, si = 0.0;
                for (int l = 0; l < gd; ++l) {
                    sr += mr[j * gd + l] * vr[l] - mi[j * gd + l] * vi[l];
                    si += mr[j * gd + l] * vi[l] + mi[j * gd + l] * vr[l];
                }
                row[j][2 * col] = sr;
                row[j][2 * col + 1] = si;
            }
        }
    }
}

// A persistent pool of host threads (up to 15 workers, started on first use). A job is a
// range of indices; the calling thread works on its own job as well, so nested jobs (a
// beam search inside a task) always make progress even when every worker is busy.
class TaskPool {
  public:
    static TaskPool &get() {
        static TaskPool *pool = new TaskPool;  // never destroyed: workers sleep until exit
        return *pool;
    }
    void run(size_t count, const std::function<void(size_t)> &f) {
        if (count == 0) return;
        auto job = std::make_shared<Job>(f, count);
        {
            std::lock_guard<std::mutex> lk(mu_);
            jobs_.push_back(job);
        }
        cv_.notify_all();
        work_on(*job);
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return job->done.load() == count; });
        jobs_.erase(std::find(jobs_.begin(), jobs_.end(), job));
    }
    size_t workers() const { return threads_; }

  private:
    struct Job {
        Job(const std::function<void(size_t)> &fn, size_t c) : f(fn), count(c) {}
        std::function<void(size_t)> f;
        size_t count;
        std::atomic<size_t> next{0}, done{0};
    };
    TaskPool() {
        threads_ = std::min<size_t>(15, std::max(1u, std::thread::hardware_concurrency()) - 1);
        for (size_t t = 0; t < threads_; ++t) std::thread([this] { worker(); }).detach();
    }
    void work_on(Job &j) {
        for (;;) {
            const size_t i = j.next.fetch_add(1);
            if (i >= j.count) return;
            j.f(i);
            if (j.done.fetch_add(1) + 1 == j.count) {
                std::lock_guard<std::mutex> lk(mu_);
                done_cv_.notify_all();
            }
        }
    }
    void worker() {
        for (;;) {
            std::shared_ptr<Job> j;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] {
                    for (const auto &x : jobs_)
                        if (x->next.load() < x->count) return true;
                    return false;
                });
                for (const auto &x : jobs_)
                    if (x->next.load() < x->count) {
                        j = x;
                        break;
                    }
            }
            if (j) work_on(*j);
        }
    }
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::vector<std::shared_ptr<Job>> jobs_;
    size_t threads_ = 0;
};

// Runs f(0 .. count-1) on the task pool (each index once; f must only write its own
// slot), or inline when there is no parallelism to gain.
template <class F>
static void parallel_for(size_t count, F f) {
    if (count <= 1 || TaskPool::get().workers() == 0) {
        for (size_t i = 0; i < count; ++i) f(i);
        return;
    }
    TaskPool::get().run(count, std::function<void(size_t)>(f));
}

void host_parallel_for(size_t count, const std::function<void(size_t)> &f) { parallel_for(count, f); }

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

namespace {

// The gate DAG as per-qubit queues; a gate is ready when it heads the queue of each
// of its qubits.
struct Dag {
    int n;
    const std::vector<HostGate> *g;
    std::vector<std::vector<int>> queue;
    std::vector<uint64_t> mask;
    std::vector<std::array<size_t, 2>> qpos;  // position of gate g in the queue of its qubit a

    // placed under frontier `head`: every one of its qubits has moved past it
    bool placed(size_t gi, const std::vector<size_t> &head) const {
        const HostGate &x = (*g)[gi];
        for (int a = 0; a < x.nq; ++a)
            if (qpos[gi][size_t(a)] >= head[x.q[a]]) return false;
        return true;
    }

    bool ready(int gi, const std::vector<size_t> &head) const {
        const HostGate &x = (*g)[gi];
        for (int a = 0; a < x.nq; ++a) {
            const int q = x.q[a];
            if (head[q] >= queue[q].size() || queue[q][head[q]] != gi) return false;
        }
        return true;
    }
    // Ready gates in order of their lowest qubit (each visited once, from that qubit).
    void ready_gates(const std::vector<size_t> &head, std::vector<int> *out) const {
        out->clear();
        for (int q = 0; q < n; ++q) {
            if (head[q] >= queue[q].size()) continue;
            const int gi = queue[q][head[q]];
            if (std::countr_zero(mask[size_t(gi)]) == q && ready(gi, head)) out->push_back(gi);
        }
    }
    void take(int gi, std::vector<size_t> &head) const {
        const HostGate &x = (*g)[gi];
        for (int a = 0; a < x.nq; ++a) head[x.q[a]]++;
    }
};

struct Block {
    std::vector<int> gates;  // in application order
    uint64_t Q = 0;
};

// Grows one block from the current frontier. Each step takes, among the ready gates
// that keep the block within k_max qubits, the one adding the fewest new qubits;
// ties go to the gate after which most of the next `window` gates on its new qubits
// would fit in the block (window > 0), then to the earliest gate. A seed >= 0 is
// taken first.
Block grow(const Dag &d, std::vector<size_t> &head, int k_max, int window, int seed, uint64_t allow = ~0ull) {
    Block b;
    thread_local std::vector<int> ready;
    if (seed >= 0) {
        b.gates.push_back(seed);
        b.Q |= d.mask[seed];
        d.take(seed, head);
    }
    // The ready set is kept up to date as gates are taken (taking a gate can only make the
    // gates now at the heads of its own qubits ready); the choice below does not depend on
    // the set's order (ties go to the lowest gate index).
    d.ready_gates(head, &ready);
    for (;;) {
        int best = -1, best_new = 1 << 30, best_aff = -1;
        for (int gi : ready) {
            if (d.mask[gi] & ~allow) continue;
            const uint64_t nm = b.Q | d.mask[gi];
            if (std::popcount(nm) > k_max) continue;
            const int nnew = std::popcount(d.mask[gi] & ~b.Q);
            int aff = 0;
            if (window > 0) {
                uint64_t fresh = d.mask[gi] & ~b.Q;
                while (fresh) {
                    const int q = std::countr_zero(fresh);
                    fresh &= fresh - 1;
                    for (size_t p = head[q] + 1; p < d.queue[q].size() && p <= head[q] + size_t(window); ++p) {
                        if ((d.mask[d.queue[q][p]] & ~nm) != 0) break;
                        ++aff;
                    }
                }
            }
            if (nnew < best_new || (nnew == best_new && (aff > best_aff || (aff == best_aff && gi < best)))) {
                best = gi;
                best_new = nnew;
                best_aff = aff;
            }
        }
        if (best < 0) break;
        b.gates.push_back(best);
        b.Q |= d.mask[best];
        d.take(best, head);
        for (size_t i = 0; i < ready.size(); ++i)
            if (ready[i] == best) {
                ready[i] = ready.back();
                ready.pop_back();
                break;
            }
        const HostGate &x = (*d.g)[size_t(best)];
        int added = -1;  // a gate at the head of both of best's qubits is added once
        for (int a = 0; a < x.nq; ++a) {
            const int q = x.q[a];
            if (head[q] >= d.queue[q].size()) continue;
            const int gi = d.queue[q][head[q]];
            if (gi != added && d.ready(gi, head)) {
                ready.push_back(gi);
                added = gi;
            }
        }
    }
    return b;
}

// One complete blocking of the circuit. seed_search: start every block from the ready
// gate whose grown block holds the most gates (earliest seed on ties). With `allow`
// (a qubit mask) only gates inside it are placed, and the blocking ends when none is
// ready; `head`/`placed` give the start and receive the end.
std::vector<Block> blocking_from(const Dag &d, size_t G, int k_max, int window, bool seed_search, uint64_t allow,
                                 std::vector<size_t> &head, size_t &placed) {
    std::vector<Block> blocks;
    std::vector<int> seeds;
    while (placed < G) {
        if (!seed_search) {
            Block b = grow(d, head, k_max, window, -1, allow);
            if (b.gates.empty()) break;
            blocks.push_back(std::move(b));
        } else {
            d.ready_gates(head, &seeds);
            Block best;
            std::vector<size_t> best_head;
            int best_first = 1 << 30;
            for (int sd : seeds) {
                if (d.mask[sd] & ~allow) continue;
                std::vector<size_t> h = head;
                Block b = grow(d, h, k_max, window, sd, allow);
                if (b.gates.size() > best.gates.size() || (b.gates.size() == best.gates.size() && sd < best_first)) {
                    best = std::move(b);
                    best_head = std::move(h);
                    best_first = sd;
                }
            }
            if (best.gates.empty()) break;
            head = std::move(best_head);
            blocks.push_back(std::move(best));
        }
        placed += blocks.back().gates.size();
    }
    return blocks;
}

std::vector<Block> blocking(const Dag &d, size_t G, int k_max, int window, bool seed_search) {
    std::vector<size_t> head(size_t(d.n), 0);
    size_t placed = 0;
    return blocking_from(d, G, k_max, window, seed_search, ~0ull, head, placed);
}

// Beam search over blockings. A state is the frontier (queue heads) after some blocks;
// the number of gates placed follows from it. Each step grows, from every state, the
// block seeded by each ready gate (the same growth rule as above), keeps the
// `expand` largest per state, merges equal frontiers, and keeps the `width` states
// with the most gates placed. The first state to place every gate ends the search;
// its blocks are read back through the parent links. The expansions of a step run on
// host threads, each state writing its own slot, and the merge walks the slots in
// order, so the result does not depend on thread timing.
std::vector<Block> beam_blocking(const Dag &d, size_t G, int k_max, int window, int width, int expand,
                                 const std::vector<size_t> &head0, size_t placed0, unsigned max_threads = 16) {
    struct Node {
        int parent;
        std::vector<int> gates;  // the block that led here
    };
    struct State {
        std::vector<size_t> head;
        size_t placed;
        int node;  // index into this step's nodes
    };
    struct Cand {
        size_t placed;
        int seed;
        std::vector<size_t> head;
        Block b;
    };
    std::vector<std::vector<Node>> steps;
    std::vector<State> states{State{head0, placed0, -1}};
    while (true) {
        for (const State &st : states)
            if (st.placed == G) {
                std::vector<Block> out(steps.size());
                int node = st.node;
                for (size_t k = steps.size(); k-- > 0;) {
                    out[k].gates = steps[k][size_t(node)].gates;
                    node = steps[k][size_t(node)].parent;
                }
                return out;
            }
        std::vector<std::vector<Cand>> slot(states.size());
        auto work = [&](size_t i) {
            std::vector<int> seeds;
            d.ready_gates(states[i].head, &seeds);
            std::vector<Cand> cs;
            cs.reserve(seeds.size());
            for (int sd : seeds) {
                Cand c;
                c.head = states[i].head;
                c.b = grow(d, c.head, k_max, window, sd);
                c.placed = states[i].placed + c.b.gates.size();
                c.seed = sd;
                cs.push_back(std::move(c));
            }
            std::stable_sort(cs.begin(), cs.end(), [](const Cand &x, const Cand &y) {
                return x.placed != y.placed ? x.placed > y.placed : x.seed < y.seed;
            });
            if (cs.size() > size_t(expand)) cs.resize(size_t(expand));
            slot[i] = std::move(cs);
        };
        if (max_threads <= 1) {
            for (size_t i = 0; i < states.size(); ++i) work(i);
        } else {
            parallel_for(states.size(), work);
        }
        // merge equal frontiers (first occurrence in state order wins ties), keep the best `width`
        struct HeadHash {
            size_t operator()(const std::vector<size_t> *h) const {
                uint64_t x = 1469598103934665603ull;  // FNV-1a over the queue positions
                for (size_t v : *h) x = (x ^ uint64_t(v)) * 1099511628211ull;
                return size_t(x);
            }
        };
        struct HeadEq {
            bool operator()(const std::vector<size_t> *a, const std::vector<size_t> *b) const { return *a == *b; }
        };
        std::unordered_set<const std::vector<size_t> *, HeadHash, HeadEq> seen;
        std::vector<std::pair<size_t, size_t>> order;
        for (size_t i = 0; i < slot.size(); ++i)
            for (size_t j = 0; j < slot[i].size(); ++j)
                if (seen.insert(&slot[i][j].head).second) order.emplace_back(i, j);
        if (order.empty()) return {};
        std::stable_sort(order.begin(), order.end(), [&](const auto &x, const auto &y) {
            return slot[x.first][x.second].placed > slot[y.first][y.second].placed;
        });
        if (order.size() > size_t(width)) order.resize(size_t(width));
        std::vector<Node> nodes;
        std::vector<State> next;
        for (const auto &o : order) {
            Cand &c = slot[o.first][o.second];
            nodes.push_back(Node{states[o.first].node, std::move(c.b.gates)});
            next.push_back(State{std::move(c.head), c.placed, int(nodes.size() - 1)});
        }
        steps.push_back(std::move(nodes));
        states = std::move(next);
    }
}

}  // namespace

constexpr int kBeamWidth = 32;  // states kept per step of the beam search
constexpr int kBeamExpand = 8;  // blocks grown per state and step
constexpr int kSmallBeamWidth = 8;  // the beam that ranks the staged candidates
constexpr int kSmallBeamExpand = 4;

namespace {

// Gates not yet placed under frontier `head` that can run before any gate touching a
// qubit outside W: one scan in circuit order (a gate is in iff it lies in W and none
// of its qubits has met an unplaced gate that is out). Returns their number.
size_t closure_size(const Dag &d, const std::vector<size_t> &head, uint64_t W) {
    uint64_t blocked = 0;
    size_t in = 0;
    for (size_t gi = 0; gi < d.mask.size(); ++gi) {
        if (d.placed(gi, head)) continue;
        const uint64_t m = d.mask[gi];
        if ((m & ~W) == 0 && (m & blocked) == 0) ++in;
        else blocked |= m;
    }
    return in;
}

// Greedily picks k qubits of `pool` to leave out of the sub-state: each time the one
// whose exclusion keeps the closure from `head` largest (lowest qubit on ties).
uint64_t choose_excluded(const Dag &d, const std::vector<size_t> &head, int k, uint64_t pool, uint64_t full) {
    uint64_t X = 0;
    for (int r = 0; r < k; ++r) {
        size_t bsize = 0;
        int bq = -1;
        for (int q = 0; q < d.n; ++q) {
            if (!((pool >> q) & 1) || ((X >> q) & 1)) continue;
            const size_t c = closure_size(d, head, full & ~(X | (1ull << q)));
            if (bq < 0 || c > bsize) {
                bsize = c;
                bq = q;
            }
        }
        if (bq < 0) break;
        X |= 1ull << bq;
    }
    return X;
}

// Cost of a blocking run from |0...0>, in full-state passes: the leading blocks whose
// qubits span at most `span` qubits run on a 2^span sub-state (2^(span-n) each).
double zero_cost(const Dag &d, const std::vector<Block> &b, int n, int span) {
    uint64_t U = 0;
    size_t p = 0;
    for (const Block &blk : b) {
        uint64_t m = 0;
        for (int gi : blk.gates) m |= d.mask[size_t(gi)];
        if (std::popcount(U | m) > span) break;
        U |= m;
        ++p;
    }
    if (p < 2) p = 0;
    return double(b.size() - p) + double(p) * std::ldexp(1.0, span - n);
}

}  // namespace

// Fuses the gates into blocks of at most k_max qubits. Several greedy blockings are
// built -- the plain frontier rule, best-seed growth with affinity windows of 0, 1, 2,
// 3 and 6 next gates, and a beam search -- and the one with the fewest blocks is kept.
// For a run from |0...0> (from_zero) the choice is by cost instead (full passes plus
// sub-state passes x 2^(width - n)), and staged candidates are added. For a single
// stage of k = 2..5 excluded qubits, or two nested stages (k1 then k2 < k1 excluded),
// the excluded qubits are chosen greedily to keep the largest closure (the gates that
// precede every gate on them). Each stage's closure is blocked inside its sub-state,
// and the rest of the circuit after it (by a small beam search to pick the candidate,
// then by the full one). On the 34-qubit 20-cycle workload at k = 6 this takes the full-state passes
// from 37 (45 passes, 8 of them on a 30-qubit sub-state) to 27.
Blocking plan_blocks(int n, const std::vector<HostGate> &gates, int k_max, bool from_zero) {
    const size_t G = gates.size();
    k_max = std::max(2, std::min(k_max, n));
    Dag d;
    d.n = n;
    d.g = &gates;
    d.queue.assign(n, {});
    d.mask.resize(G);
    d.qpos.resize(G);
    for (size_t g = 0; g < G; ++g) {
        uint64_t m = 0;
        for (int a = 0; a < gates[g].nq; ++a) {
            d.qpos[g][size_t(a)] = d.queue[gates[g].q[a]].size();
            d.queue[gates[g].q[a]].push_back(int(g));
            m |= 1ull << gates[g].q[a];
        }
        d.mask[g] = m;
    }
    const int default_span = n - 4;
    const uint64_t full = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    // staged candidates: k excluded qubits per stage, nested and shrinking
    struct Cand {
        double est = 1e300;  // greedy rest + sub-state cost
        double sub_cost = 0.0;
        std::vector<int> ks;
        std::vector<uint64_t> X;
        std::vector<int> stage_end;
        std::vector<Block> pre;
        std::vector<size_t> head;
        size_t placed = 0;
    };
    std::vector<std::vector<int>> configs;
    if (from_zero && G > 0) {
        const int min_sub = std::max(kTcK + 7, k_max);
        for (int k = 2; k <= 5; ++k)
            if (n - k >= min_sub) configs.push_back({k});
        const int pairs[][2] = {{4, 2}, {5, 2}, {6, 2}, {4, 3}, {5, 3}, {6, 3}, {7, 3}, {6, 4}, {7, 4}};
        for (const auto &pr : pairs)
            if (n - pr[0] >= min_sub) configs.push_back({pr[0], pr[1]});
    }
    // the greedy portfolio (the plain rule, then best-seed growth with affinity windows)
    // and the staged candidates run as one set of host tasks
    const std::pair<int, bool> variants[] = {{0, false}, {0, true}, {1, true}, {2, true}, {3, true}, {6, true}};
    const size_t nport = G ? std::size(variants) : 1;
    std::vector<std::vector<Block>> port(nport);
    std::vector<Cand> cands(configs.size());
    // the staged candidates (each about 10 ms of beam search) are handed out first, the short
    // greedy portfolio runs (a few ms each) fill in behind them
    parallel_for(nport + cands.size(), [&](size_t t) {
        if (t >= cands.size()) {
            const size_t task = t - cands.size();
            port[task] = blocking(d, G, k_max, variants[task].first, variants[task].second);
            return;
        }
        const size_t task = t + nport;
        const std::vector<int> &ks = configs[task - nport];
        Cand c;
        c.ks = ks;
        c.head.assign(size_t(n), 0);
        uint64_t pool = full;
        double sub_cost = 0.0;
        for (size_t si = 0; si < ks.size(); ++si) {
            const uint64_t X = choose_excluded(d, c.head, ks[si], pool, full);
            std::vector<Block> b = blocking_from(d, G, k_max, 2, true, full & ~X, c.head, c.placed);
            sub_cost += double(b.size()) * std::ldexp(1.0, -ks[si]);
            if (si > 0) sub_cost += 0.5 * std::ldexp(1.0, -ks[si]);  // expansion into this sub-state
            for (Block &x : b) c.pre.push_back(std::move(x));
            c.stage_end.push_back(int(c.pre.size()));
            c.X.push_back(X);
            pool = X;
        }
        // the rest estimated by a small single-threaded beam (greedy growth alone cannot tell
        // the candidates apart: on the 34-qubit workload it gives 30 for all, the beam 28-34)
        const std::vector<Block> rest =
            beam_blocking(d, G, k_max, 0, kSmallBeamWidth, kSmallBeamExpand, c.head, c.placed, 1);
        c.sub_cost = sub_cost;
        c.est = double(rest.size()) + sub_cost;
        cands[task - nport] = std::move(c);
    });
    std::vector<Block> best = std::move(port[0]);
    for (size_t i = 1; i < port.size(); ++i) {
        const bool better = from_zero ? zero_cost(d, port[i], n, default_span) < zero_cost(d, best, n, default_span)
                                      : port[i].size() < best.size();
        if (better) best = std::move(port[i]);
    }
    Blocking out;
    if (!from_zero) {
        if (G > 0) {
            std::vector<std::vector<Block>> beams(2);
            parallel_for(2, [&](size_t i) {
                beams[i] = beam_blocking(d, G, k_max, i == 0 ? 0 : 2, kBeamWidth, kBeamExpand,
                                         std::vector<size_t>(size_t(d.n), 0), 0);
            });
            for (std::vector<Block> &b : beams)
                if (!b.empty() && b.size() < best.size()) best = std::move(b);
        }
    } else if (!cands.empty()) {
        const double best_cost = zero_cost(d, best, n, default_span);
        size_t pi = 0;
        for (size_t i = 1; i < cands.size(); ++i)
            if (cands[i].est < cands[pi].est) pi = i;
        Cand &pick = cands[pi];
        std::vector<Block> rest_best;
        {
            std::vector<size_t> h = pick.head;
            size_t pl = pick.placed;
            rest_best = blocking_from(d, G, k_max, 2, true, ~0ull, h, pl);
        }
        std::vector<std::vector<Block>> beams(2);
        parallel_for(2, [&](size_t i) {
            beams[i] = beam_blocking(d, G, k_max, i == 0 ? 0 : 2, kBeamWidth, kBeamExpand, pick.head, pick.placed);
        });
        for (std::vector<Block> &r : beams)
            if ((!r.empty() || pick.placed == G) && r.size() < rest_best.size()) rest_best = std::move(r);
        const double cost = pick.sub_cost + double(rest_best.size());
        if (cost < best_cost) {
            best = std::move(pick.pre);
            for (Block &b : rest_best) best.push_back(std::move(b));
            for (size_t si = 0; si < pick.ks.size(); ++si) {
                out.spans.push_back(n - pick.ks[si]);
                out.avoid.push_back(pick.X[si]);
                out.stage_end.push_back(pick.stage_end[si]);
            }
        }
    }
    out.gates.reserve(best.size());
    for (Block &b : best) out.gates.push_back(std::move(b.gates));
    return out;
}

// Passes for the blocks, each padded to pad_to qubits with the highest qubits it
// does not use (identity on them).
void make_passes(int n, const std::vector<HostGate> &gates, const Blocking &b, int pad_to, std::vector<Pass> *out) {
    out->assign(b.gates.size(), Pass{});
    parallel_for(b.gates.size(), [&](size_t bi) {
        const std::vector<int> &blk_gates = b.gates[bi];
        uint64_t Q = 0;
        std::vector<const HostGate *> blk;
        blk.reserve(blk_gates.size());
        for (int gi : blk_gates) {
            blk.push_back(&gates[gi]);
            for (int a = 0; a < gates[gi].nq; ++a) Q |= 1ull << gates[gi].q[a];
        }
        uint64_t avoid = 0;  // padding stays inside the block's sub-state
        for (size_t si = 0; si < b.stage_end.size(); ++si)
            if (bi < size_t(b.stage_end[si])) {
                avoid = b.avoid[si];
                break;
            }
        for (int q = n - 1; q >= 0 && std::popcount(Q) < pad_to; --q)
            if (!((avoid >> q) & 1)) Q |= 1ull << q;
        for (int q = n - 1; q >= 0 && std::popcount(Q) < pad_to; --q) Q |= 1ull << q;
        (*out)[bi] = make_pass(pad_to > 0 ? PASS_TC : PASS_SIMT, Q, blk);
    });
}

void plan_fuse(int n, const std::vector<HostGate> &gates, int k_max, int pad_to, std::vector<Pass> *out) {
    make_passes(n, gates, plan_blocks(n, gates, k_max, false), pad_to, out);
}

// Five qubits are placed on bits 0..4, each swapping places with the qubit that sat
// there: five that share no block (fewest memberships), else the five of the 16 least
// used that the fewest blocks target twice or more. The state kernels give a warp 32 neighbouring
// slices, which are side by side in memory only while the lowest bits are not targets;
// with this layout a pass targets as few of bits 0..4 as the blocking allows (at most
// one on the benchmark workloads).
bool choose_layout(int n, const std::vector<HostGate> &gates, const Blocking &b, int *phys_of) {
    for (int q = 0; q < n; ++q) phys_of[q] = q;
    if (n < 12) return false;
    std::vector<uint64_t> masks;
    masks.reserve(b.gates.size());
    std::vector<int> count(n, 0);
    for (const std::vector<int> &blk : b.gates) {
        uint64_t m = 0;
        for (int gi : blk)
            for (int a = 0; a < gates[gi].nq; ++a) m |= 1ull << gates[gi].q[a];
        masks.push_back(m);
        for (int q = 0; q < n; ++q) count[q] += int((m >> q) & 1);
    }
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return count[x] < count[y]; });
    // Five qubits that share no block, with the fewest memberships: a depth-first search
    // over the qubits in membership order, pruned by the count so far. If no such five
    // exist, the five of the 16 least-used qubits that the fewest blocks target twice or
    // more (then the fewest memberships; every subset tried, at most C(16, 5) = 4368).
    const int want = std::min(5, n);
    std::vector<uint64_t> share(size_t(n), 0);  // qubits that share a block with q
    for (uint64_t m : masks)
        for (uint64_t r = m; r; r &= r - 1) share[size_t(std::countr_zero(r))] |= m;
    uint64_t chosen = 0;
    long best_cnt = -1;
    {
        uint64_t S = 0;
        auto dfs = [&](auto &&self, int from, int left, long cnt) -> void {
            if (left == 0) {
                if (best_cnt < 0 || cnt < best_cnt) {
                    best_cnt = cnt;
                    chosen = S;
                }
                return;
            }
            for (int i = from; i <= n - left; ++i) {
                const int q = order[size_t(i)];
                // order is by count: the cheapest completion adds left x count[q]
                if (best_cnt >= 0 && cnt + long(left) * count[size_t(q)] >= best_cnt) return;
                if (share[size_t(q)] & S) continue;
                S |= 1ull << q;
                self(self, i + 1, left - 1, cnt + count[size_t(q)]);
                S &= ~(1ull << q);
            }
        };
        dfs(dfs, 0, want, 0);
    }
    if (best_cnt < 0) {
        const int pool = std::min(n, 16);
        long best_conf = -1;
        std::vector<int> idx(static_cast<size_t>(want));
        for (int i = 0; i < want; ++i) idx[size_t(i)] = i;
        while (true) {
            uint64_t S = 0;
            long cnt = 0;
            for (int i : idx) {
                S |= 1ull << order[size_t(i)];
                cnt += count[size_t(order[size_t(i)])];
            }
            long conf = 0;
            for (uint64_t m : masks) conf += std::max(0, std::popcount(m & S) - 1);
            if (best_conf < 0 || conf < best_conf || (conf == best_conf && cnt < best_cnt)) {
                best_conf = conf;
                best_cnt = cnt;
                chosen = S;
            }
            int k = want - 1;  // next subset in lexicographic order
            while (k >= 0 && idx[size_t(k)] == pool - want + k) --k;
            if (k < 0) break;
            ++idx[size_t(k)];
            for (int r = k + 1; r < want; ++r) idx[size_t(r)] = idx[size_t(r - 1)] + 1;
        }
    }
    const int picked = std::popcount(chosen);
    // pair the chosen qubits above bit `picked-1` with the unchosen qubits below it: at most
    // five transpositions, so restoring the identity layout takes at most five swaps
    std::vector<int> up, down;
    for (int q = 0; q < n; ++q) {
        const bool c = (chosen >> q) & 1;
        if (c && q >= picked) up.push_back(q);
        if (!c && q < picked) down.push_back(q);
    }
    for (size_t i = 0; i < up.size(); ++i) {
        phys_of[up[i]] = down[i];
        phys_of[down[i]] = up[i];
    }
    return !up.empty();
}

int plan_stages(const Plan &plan, std::vector<SubStage> *stages) {
    stages->clear();
    const int n = plan.n;
    std::vector<int> spans = plan.stage_spans;
    if (spans.empty()) spans.push_back(n - 4);
    uint64_t T = 0;
    size_t p = 0;
    int need = 0, total = 0;
    for (const int span : spans) {
        if (span >= n) break;
        SubStage st;
        st.first = int(p);
        while (p < plan.passes.size()) {
            const Pass &q = plan.passes[p];
            if (q.kind != PASS_TC && q.kind != PASS_SIMT) break;
            uint64_t Tn = T;
            for (int i = 0; i < q.k; ++i) Tn |= 1ull << q.t[i];
            if (std::popcount(Tn) > span) break;
            T = Tn;
            need = std::max(need, q.kind == PASS_TC ? kTcK + 7 : q.k);
            ++p;
        }
        // widened, after its passes, with idle |0> qubits to the size the kernels need
        for (int b = 0; b < n && std::popcount(T) < need; ++b) T |= 1ull << b;
        if (std::popcount(T) >= n) {
            stages->clear();
            return 0;
        }
        st.count = int(p) - st.first;
        st.tmask = T;
        if (st.count > 0) {
            stages->push_back(st);
            total += st.count;
        }
    }
    if (total < 2) {
        stages->clear();
        return 0;
    }
    return total;
}

size_t substage_bytes(const std::vector<SubStage> &stages) {
    size_t b = 0;
    for (const SubStage &s : stages) b += size_t(8) << std::popcount(s.tmask);
    return b;
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
