// Gate-fusion planner: merges runs of 1- and 2-qubit gates into dense k-qubit
// unitaries (one state pass each). The paper's engine is closed and describes no
// fusion; this is a search over frontier constructions on the gate DAG: greedy
// growth, beam searches over grown blocks, and a beam search over closures of
// connected qubit sets.
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
#include <map>
#include <set>
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

// Beam search whose moves are closures. From a frontier, the closure of a qubit set T is
// every unplaced gate that can run before any gate touching a qubit outside T: the gates
// whose support -- the qubits of the gate and of all its unplaced ancestors -- lies in T.
// One scan in circuit order gives every support, so a candidate set's closure size is the
// number of gates whose support it contains. The candidate sets are the connected
// k_max-qubit sets of the circuit's coupling graph inside `allow`, plus the block grown
// from every ready seed (as in beam_blocking, so that qubits without couplings progress
// too). Each step keeps the `expand` largest moves per state and the `width` states with
// the most gates placed, merging equal frontiers. The first state with `target` gates
// placed ends the search. Returns false (no blocking) when there are more than max_sets
// candidate sets, as on densely coupled circuits. Ties go to the lower set, then the
// earlier state, so the result does not depend on thread timing.
bool closure_beam(const Dag &d, size_t G, int k_max, int width, int expand, const std::vector<size_t> &head0,
                  size_t placed0, uint64_t allow, size_t target, std::vector<Block> *result,
                  size_t max_sets = 20000) {
    result->clear();
    const int n = d.n;
    std::vector<uint64_t> adj(size_t(n), 0);
    for (size_t g = 0; g < G; ++g)
        if (std::popcount(d.mask[g]) == 2) {
            const int a = std::countr_zero(d.mask[g]);
            const int b = 63 - std::countl_zero(d.mask[g]);
            adj[size_t(a)] |= 1ull << b;
            adj[size_t(b)] |= 1ull << a;
        }
    std::vector<uint64_t> sets;
    {
        std::unordered_set<uint64_t> cur;
        for (int q = 0; q < n; ++q)
            if ((allow >> q) & 1) cur.insert(1ull << q);
        for (int s = 1; s < k_max; ++s) {
            std::unordered_set<uint64_t> nx;
            for (uint64_t m : cur) {
                uint64_t nb = 0;
                for (uint64_t r = m; r; r &= r - 1) nb |= adj[size_t(std::countr_zero(r))];
                nb &= ~m & allow;
                for (; nb; nb &= nb - 1) nx.insert(m | (1ull << std::countr_zero(nb)));
            }
            if (nx.size() > max_sets) return false;
            if (nx.empty()) break;
            cur = std::move(nx);
        }
        sets.assign(cur.begin(), cur.end());
        std::sort(sets.begin(), sets.end());
    }
    std::vector<std::vector<uint32_t>> sets_with;  // the candidate sets holding qubit q
    sets_with.resize(size_t(n));
    for (size_t i = 0; i < sets.size(); ++i)
        for (uint64_t r = sets[i]; r; r &= r - 1) sets_with[size_t(std::countr_zero(r))].push_back(uint32_t(i));

    // Supports of the unplaced gates under `head` that fit a candidate set, merged by value
    // as (support, gates). Supports only widen along a qubit's gates, so the scan stops once
    // every qubit's latest support is too wide or its gates are done.
    auto supports = [&](const std::vector<size_t> &head, std::vector<std::pair<uint64_t, uint32_t>> *out) {
        uint64_t last[64] = {};
        size_t rem[64] = {};
        uint64_t live = 0;
        size_t first = G;
        for (int q = 0; q < n; ++q) {
            rem[q] = d.queue[size_t(q)].size() - head[size_t(q)];
            if (rem[q] && ((allow >> q) & 1)) live |= 1ull << q;
            if (rem[q]) first = std::min(first, size_t(d.queue[size_t(q)][head[size_t(q)]]));
        }
        out->clear();
        for (size_t gi = first; gi < G && live; ++gi) {
            if (d.placed(gi, head)) continue;
            const uint64_t m = d.mask[gi];
            uint64_t s = m;
            for (uint64_t r = m; r; r &= r - 1) s |= last[std::countr_zero(r)];
            for (uint64_t r = m; r; r &= r - 1) {
                const int q = std::countr_zero(r);
                last[q] = s;
                if (--rem[q] == 0) live &= ~(1ull << q);
            }
            if (std::popcount(s) <= k_max && (s & ~allow) == 0) out->emplace_back(s, 1u);
            else live &= ~m;
        }
        std::sort(out->begin(), out->end());
        size_t w = 0;
        for (size_t i = 0; i < out->size(); ++i) {
            if (w > 0 && (*out)[w - 1].first == (*out)[i].first) (*out)[w - 1].second += (*out)[i].second;
            else (*out)[w++] = (*out)[i];
        }
        out->resize(w);
    };
    // Takes the closure of T as a block (circuit order is an application order).
    auto take_closure = [&](std::vector<size_t> &head, uint64_t T, Block *b) {
        uint64_t last[64] = {};
        std::vector<int> in;
        size_t first = G;
        for (int q = 0; q < n; ++q)
            if (head[size_t(q)] < d.queue[size_t(q)].size())
                first = std::min(first, size_t(d.queue[size_t(q)][head[size_t(q)]]));
        for (size_t gi = first; gi < G; ++gi) {
            if (d.placed(gi, head)) continue;
            const uint64_t m = d.mask[gi];
            uint64_t s = m;
            for (uint64_t r = m; r; r &= r - 1) s |= last[std::countr_zero(r)];
            for (uint64_t r = m; r; r &= r - 1) last[std::countr_zero(r)] = s;
            if ((s & ~T) == 0) in.push_back(int(gi));
        }
        for (int gi : in) {
            d.take(gi, head);
            b->gates.push_back(gi);
            b->Q |= d.mask[size_t(gi)];
        }
    };

    struct Node {
        int parent;
        std::vector<int> gates;
    };
    struct State {
        std::vector<size_t> head;
        size_t placed;
        int node;
    };
    struct Move {
        size_t placed;
        uint64_t T;  // closure of T, or (seed >= 0) the block grown from seed
        int seed;
    };
    std::vector<std::vector<Node>> steps;
    std::vector<State> states{State{head0, placed0, -1}};
    while (true) {
        for (const State &st : states)
            if (st.placed >= target) {
                result->resize(steps.size());
                int node = st.node;
                for (size_t k = steps.size(); k-- > 0;) {
                    (*result)[k].gates = steps[k][size_t(node)].gates;
                    node = steps[k][size_t(node)].parent;
                }
                return true;
            }
        std::vector<std::vector<Move>> slot(states.size());
        parallel_for(states.size(), [&](size_t i) {
            std::vector<std::pair<uint64_t, uint32_t>> sup;
            supports(states[i].head, &sup);
            std::vector<uint32_t> cnt(sets.size(), 0);
            for (const auto &s : sup)
                for (uint32_t si : sets_with[size_t(std::countr_zero(s.first))])
                    if ((s.first & ~sets[si]) == 0) cnt[si] += s.second;
            std::vector<Move> ms;
            for (size_t si = 0; si < sets.size(); ++si)
                if (cnt[si]) ms.push_back(Move{states[i].placed + cnt[si], sets[si], -1});
            std::vector<int> seeds;
            d.ready_gates(states[i].head, &seeds);
            for (int sd : seeds) {
                if (d.mask[size_t(sd)] & ~allow) continue;
                std::vector<size_t> h = states[i].head;
                const Block b = grow(d, h, k_max, 0, sd, allow);
                ms.push_back(Move{states[i].placed + b.gates.size(), 0, sd});
            }
            // the `expand` largest, earlier moves first on ties
            const size_t keep = std::min(ms.size(), size_t(expand));
            std::vector<uint32_t> idx(ms.size());
            for (size_t j = 0; j < idx.size(); ++j) idx[j] = uint32_t(j);
            std::partial_sort(idx.begin(), idx.begin() + std::ptrdiff_t(keep), idx.end(), [&](uint32_t x, uint32_t y) {
                return ms[x].placed != ms[y].placed ? ms[x].placed > ms[y].placed : x < y;
            });
            slot[i].clear();
            for (size_t j = 0; j < keep; ++j) slot[i].push_back(ms[idx[j]]);
        });
        std::vector<std::pair<size_t, size_t>> order;
        for (size_t i = 0; i < slot.size(); ++i)
            for (size_t j = 0; j < slot[i].size(); ++j) order.emplace_back(i, j);
        std::stable_sort(order.begin(), order.end(), [&](const auto &x, const auto &y) {
            return slot[x.first][x.second].placed > slot[y.first][y.second].placed;
        });
        std::set<std::vector<size_t>> seen;
        std::vector<Node> nodes;
        std::vector<State> next;
        for (const auto &o : order) {
            if (int(next.size()) >= width) break;
            const Move &mv = slot[o.first][o.second];
            std::vector<size_t> h = states[o.first].head;
            Block b;
            if (mv.seed >= 0) b = grow(d, h, k_max, 0, mv.seed, allow);
            else take_closure(h, mv.T, &b);
            if (!seen.insert(h).second) continue;
            nodes.push_back(Node{states[o.first].node, std::move(b.gates)});
            next.push_back(State{std::move(h), mv.placed, int(nodes.size() - 1)});
        }
        if (next.empty()) return false;
        steps.push_back(std::move(nodes));
        states = std::move(next);
    }
}

}  // namespace

constexpr int kBeamWidth = 32;  // states kept per step of the beam search
constexpr int kBeamExpand = 8;  // blocks grown per state and step
constexpr int kSmallBeamWidth = 8;  // the beam that ranks the staged candidates
constexpr int kSmallBeamExpand = 4;
constexpr int kClosureWidth = 16;       // states kept per step of the closure search
constexpr int kClosureExpand = 16;      // moves kept per state and step
constexpr int kStageClosureWidth = 8;   // the closure search inside a sub-state stage
constexpr int kStageClosureExpand = 8;
constexpr int kFinalists = 3;           // staged candidates whose rest gets the full searches

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
// 3 and 6 next gates, two beam searches over grown blocks and a beam search over
// closures of connected qubit sets -- and the one with the fewest blocks is kept.
// For a run from |0...0> (from_zero) the choice is by cost instead (full passes plus
// sub-state passes x 2^(width - n)), and staged candidates are added: one to three
// nested stages, each leaving k qubits out of its sub-state (a subset of those the
// stage before it left out). The excluded qubits are chosen greedily to keep the
// largest closure (the gates that precede every gate on them). Each stage's closure is
// blocked inside its sub-state (greedy growth or the closure search, whichever needs
// fewer blocks; stages shared by several candidates are blocked once), and the rest of
// the circuit after it is estimated by a small beam search. The best few candidates by
// that estimate get the full searches for their rest. On the 34-qubit 20-cycle
// workload at k = 6 this takes the full-state passes from 37 (45 passes, 8 of them on
// a 30-qubit sub-state) to 26, after 17 passes on sub-states of 28, 30 and 32 qubits.
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
    std::vector<std::vector<int>> configs;
    if (from_zero && G > 0) {
        const int min_sub = std::max(kTcK + 7, k_max);
        for (int k = 2; k <= 5; ++k)
            if (n - k >= min_sub) configs.push_back({k});
        const int pairs[][2] = {{4, 2}, {5, 2}, {6, 2}, {4, 3}, {5, 3}, {6, 3}, {7, 3}, {6, 4}, {7, 4}};
        for (const auto &pr : pairs)
            if (n - pr[0] >= min_sub) configs.push_back({pr[0], pr[1]});
        const int triples[][3] = {{6, 4, 2}, {7, 4, 2}, {8, 4, 2}, {5, 3, 2}, {6, 3, 2}, {7, 5, 2}, {8, 5, 2}};
        for (const auto &tr : triples)
            if (n - tr[0] >= min_sub) configs.push_back({tr[0], tr[1], tr[2]});
    }
    // Every distinct stage prefix of the candidates, parents before children: the stage's
    // excluded qubits, its blocks, the frontier after it and the sub-state cost so far.
    struct Stage {
        std::vector<int> ks;
        int parent = -1;
        uint64_t X = 0;
        std::vector<Block> blocks;
        std::vector<size_t> head;
        size_t placed = 0;
        double cost = 0.0;
    };
    std::vector<Stage> stages;
    std::map<std::vector<int>, int> stage_of;
    auto block_stage = [&](Stage &s) {
        const Stage *par = s.parent >= 0 ? &stages[size_t(s.parent)] : nullptr;
        const int k = s.ks.back();
        const std::vector<size_t> head0 = par ? par->head : std::vector<size_t>(size_t(n), 0);
        const size_t placed0 = par ? par->placed : 0;
        s.X = choose_excluded(d, head0, k, par ? par->X : full, full);
        const uint64_t allow = full & ~s.X;
        s.head = head0;
        s.placed = placed0;
        s.blocks = blocking_from(d, G, k_max, 2, true, allow, s.head, s.placed);
        // both searches place the same gates (the stage's closure), so the frontier is the same
        std::vector<Block> cl;
        if (closure_beam(d, G, k_max, kStageClosureWidth, kStageClosureExpand, head0, placed0, allow, s.placed, &cl) &&
            cl.size() < s.blocks.size())
            s.blocks = std::move(cl);
        s.cost = (par ? par->cost + 0.5 * std::ldexp(1.0, -k) : 0.0) + double(s.blocks.size()) * std::ldexp(1.0, -k);
    };
    size_t depth_max = 0;
    for (const std::vector<int> &c : configs) depth_max = std::max(depth_max, c.size());
    // the greedy portfolio (the plain rule, then best-seed growth with affinity windows)
    // runs as host tasks beside the first stages
    const std::pair<int, bool> variants[] = {{0, false}, {0, true}, {1, true}, {2, true}, {3, true}, {6, true}};
    const size_t nport = G ? std::size(variants) : 1;
    std::vector<std::vector<Block>> port(nport);
    for (size_t depth = 1; depth <= std::max<size_t>(depth_max, 1); ++depth) {
        const size_t lo = stages.size();
        for (const std::vector<int> &c : configs) {
            if (c.size() < depth) continue;
            std::vector<int> pre(c.begin(), c.begin() + std::ptrdiff_t(depth));
            if (stage_of.count(pre)) continue;
            Stage s;
            s.ks = pre;
            if (depth > 1) s.parent = stage_of.at(std::vector<int>(pre.begin(), pre.end() - 1));
            stage_of[pre] = int(stages.size());
            stages.push_back(std::move(s));
        }
        const size_t extra = depth == 1 ? nport : 0;
        parallel_for(stages.size() - lo + extra, [&](size_t t) {
            if (t < stages.size() - lo) {
                block_stage(stages[lo + t]);
            } else {
                const size_t task = t - (stages.size() - lo);
                port[task] = blocking(d, G, k_max, variants[task].first, variants[task].second);
            }
        });
    }
    // each candidate's rest estimated by a small single-threaded beam (greedy growth alone
    // cannot tell the candidates apart: on the 34-qubit workload it gives 30 for all, the
    // beam 26-34)
    struct Cand {
        double est = 1e300;
        int stage = -1;  // its last stage
    };
    std::vector<Cand> cands(configs.size());
    parallel_for(cands.size(), [&](size_t i) {
        const Stage &s = stages[size_t(stage_of.at(configs[i]))];
        const std::vector<Block> rest =
            beam_blocking(d, G, k_max, 0, kSmallBeamWidth, kSmallBeamExpand, s.head, s.placed, 1);
        cands[i].stage = stage_of.at(configs[i]);
        cands[i].est = (rest.empty() && s.placed < G ? 1e300 : double(rest.size())) + s.cost;
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
            std::vector<std::vector<Block>> searches(3);
            std::vector<char> ok(3, 0);
            parallel_for(3, [&](size_t i) {
                if (i < 2) {
                    searches[i] = beam_blocking(d, G, k_max, i == 0 ? 0 : 2, kBeamWidth, kBeamExpand,
                                                std::vector<size_t>(size_t(d.n), 0), 0);
                    ok[i] = !searches[i].empty();
                } else {
                    ok[i] = closure_beam(d, G, k_max, kClosureWidth, kClosureExpand,
                                         std::vector<size_t>(size_t(d.n), 0), 0, full, G, &searches[i]);
                }
            });
            for (size_t i = 0; i < searches.size(); ++i)
                if (ok[i] && searches[i].size() < best.size()) best = std::move(searches[i]);
        }
    } else if (!cands.empty()) {
        const double best_cost = zero_cost(d, best, n, default_span);
        // the finalists: the best estimates (the earlier candidate on ties)
        std::vector<size_t> rank(cands.size());
        for (size_t i = 0; i < rank.size(); ++i) rank[i] = i;
        std::stable_sort(rank.begin(), rank.end(), [&](size_t x, size_t y) { return cands[x].est < cands[y].est; });
        rank.resize(std::min(rank.size(), size_t(kFinalists)));
        // each finalist's rest: greedy best-seed growth and the closure search, or, where the
        // closure search does not apply (too many candidate sets), the two beams over grown blocks
        constexpr size_t kSearches = 4;
        std::vector<std::vector<Block>> rests(rank.size() * kSearches);
        std::vector<char> ok(rests.size(), 0);
        parallel_for(rank.size() * 2, [&](size_t u) {
            const Stage &s = stages[size_t(cands[rank[u / 2]].stage)];
            const size_t t = (u / 2) * kSearches;
            if (u % 2 == 0) {
                std::vector<size_t> h = s.head;
                size_t pl = s.placed;
                rests[t] = blocking_from(d, G, k_max, 2, true, ~0ull, h, pl);
                ok[t] = pl == G;
                return;
            }
            ok[t + 3] = closure_beam(d, G, k_max, kClosureWidth, kClosureExpand, s.head, s.placed, full, G, &rests[t + 3]);
            if (ok[t + 3]) return;
            for (size_t which = 1; which < 3; ++which) {
                rests[t + which] =
                    beam_blocking(d, G, k_max, which == 1 ? 0 : 2, kBeamWidth, kBeamExpand, s.head, s.placed);
                ok[t + which] = !rests[t + which].empty() || s.placed == G;
            }
        });
        size_t pick = rests.size();
        double pick_cost = 1e300;
        for (size_t t = 0; t < rests.size(); ++t) {
            if (!ok[t]) continue;
            const double cost = stages[size_t(cands[rank[t / kSearches]].stage)].cost + double(rests[t].size());
            if (cost < pick_cost) {
                pick_cost = cost;
                pick = t;
            }
        }
        if (pick < rests.size() && pick_cost < best_cost) {
            // the stages of the pick, first to last
            std::vector<int> chain;
            for (int si = cands[rank[pick / kSearches]].stage; si >= 0; si = stages[size_t(si)].parent)
                chain.push_back(si);
            std::reverse(chain.begin(), chain.end());
            best.clear();
            for (int si : chain) {
                Stage &s = stages[size_t(si)];
                for (Block &b : s.blocks) best.push_back(std::move(b));
                out.spans.push_back(n - s.ks.back());
                out.avoid.push_back(s.X);
                out.stage_end.push_back(int(best.size()));
            }
            for (Block &b : rests[pick]) best.push_back(std::move(b));
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
