// Multilevel graph bisection for the column-preserving partitioner (Sec. 4.2).
//
// The paper clusters the lines of an extruded mesh with a graph partitioner
// (METIS / Zoltan) when no structured layout is known, and names a partition
// taken from the matrix alone as the way to use the solver as a black box
// (Sec. 6).  This file is that partitioner for one bisection: the vertices
// are the vertical lines found in the matrix, an edge joins two lines that
// share a nonzero, and its weight is the sum of |a_ij| over those nonzeros.
//
//   coarsening   heavy-edge matching in a seeded random vertex order, a pair
//                matched only below a weight cap, until about 80 vertices remain or
//                a round shrinks the graph by less than 5 %;
//   initial cut  graph growing from twelve seeds on the coarsest graph (the
//                first a pseudo-peripheral vertex), each refined, the
//                smallest cut kept;
//   refinement   on every level back up: a move of the heaviest-gain
//                vertices off an overweight part, then boundary
//                Fiduccia-Mattheyses passes (each vertex moves at most once
//                per pass, the pass is rolled back to its best balanced
//                prefix) while a pass improves the cut.
//
// On the finest level every vertex weighs one line and the balance window is
// empty: part 0 ends with exactly `na` vertices.  The result depends only on
// the input graph (no thread count, no clock, no global random state).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <memory>
#include <numeric>
#include <queue>
#include <vector>

#include "hs_internal.h"

namespace {

struct WGraph {
    int n = 0;
    std::vector<int> ptr, adj, vw;
    std::vector<double> w;
    int maxvw = 1;
    std::vector<int> cmap;  // vertex -> vertex of the next coarser graph
};

// 32-bit integer mixer (the "lowbias32" constants of C. Wellons' hash
// prospector); it drives the matching order and picks the growing seeds.
uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Heavy-edge matching, vertices visited in a seeded random order: an unmatched vertex
// takes its unmatched neighbour of largest edge weight (ties: smaller index)
// whose combined vertex weight stays <= cap, else stays single.  Coarse
// vertices are numbered in the order of their smallest member.  Returns
// false (and builds nothing) when the graph would shrink by less than 5 %.
bool coarsen(WGraph& g, WGraph& c, int cap, uint32_t seed) {
    const int n = g.n;
    std::vector<int> order(n), match(n, -1);
    // visiting order: a Fisher-Yates shuffle driven by mix32 of (seed, step)
    std::iota(order.begin(), order.end(), 0);
    for (int i = n - 1; i > 0; i--) std::swap(order[i], order[mix32(seed + (uint32_t)i) % (uint32_t)(i + 1)]);
    for (int u : order) {
        if (match[u] >= 0) continue;
        int best = u;
        double bw = -1.0;
        for (int e = g.ptr[u]; e < g.ptr[u + 1]; e++) {
            const int v = g.adj[e];
            if (match[v] >= 0 || g.vw[u] + g.vw[v] > cap) continue;
            if (g.w[e] > bw || (g.w[e] == bw && v < best)) {
                best = v;
                bw = g.w[e];
            }
        }
        match[u] = best;
        match[best] = u;
    }
    g.cmap.assign(n, -1);
    int nc = 0;
    for (int u = 0; u < n; u++)
        if (g.cmap[u] < 0) {
            g.cmap[u] = nc;
            g.cmap[match[u]] = nc;
            nc++;
        }
    if ((double)nc > 0.95 * n) {
        g.cmap.clear();
        return false;
    }
    c.n = nc;
    c.vw.assign(nc, 0);
    c.ptr.assign(nc + 1, 0);
    c.adj.clear();
    c.w.clear();
    c.adj.reserve(g.adj.size());
    c.w.reserve(g.adj.size());
    std::vector<int> rep(nc), pos(nc, -1);
    for (int u = 0; u < n; u++)
        if (u <= match[u]) rep[g.cmap[u]] = u;
    for (int cu = 0; cu < nc; cu++) {
        const int start = (int)c.adj.size();
        const int m0 = rep[cu], m1 = match[m0];
        for (int k = 0; k < (m1 == m0 ? 1 : 2); k++) {
            const int m = k ? m1 : m0;
            c.vw[cu] += g.vw[m];
            for (int e = g.ptr[m]; e < g.ptr[m + 1]; e++) {
                const int cv = g.cmap[g.adj[e]];
                if (cv == cu) continue;
                if (pos[cv] >= start) {
                    c.w[pos[cv]] += g.w[e];
                } else {
                    pos[cv] = (int)c.adj.size();
                    c.adj.push_back(cv);
                    c.w.push_back(g.w[e]);
                }
            }
        }
        c.ptr[cu + 1] = (int)c.adj.size();
    }
    c.maxvw = *std::max_element(c.vw.begin(), c.vw.end());
    return true;
}

struct Cand {
    double g;
    int v;
    bool operator<(const Cand& o) const { return g < o.g || (g == o.g && v > o.v); }  // max gain, then min index
};

// Binary max-heap on a vector that keeps its capacity between uses.
struct Heap {
    std::vector<Cand> v;
    void clear() { v.clear(); }
    bool empty() const { return v.empty(); }
    const Cand& top() const { return v.front(); }
    void push(Cand c) {
        v.push_back(c);
        std::push_heap(v.begin(), v.end());
    }
    void pop() {
        std::pop_heap(v.begin(), v.end());
        v.pop_back();
    }
};

// Buffers of one bisection, kept per thread so that the many small
// bisections deep in the recursion allocate nothing.
struct Work {
    std::vector<char> side, locked, seen, best;
    std::vector<double> gain;
    std::vector<int> nbnd, moves, queue;
    Heap h[2];
};

// A two-way partition of one level with incrementally kept gains:
// gain[v] = (weight of v's edges to the other part) - (to its own part), the
// decrease of the cut when v changes part; nbnd[v] = its neighbours in the
// other part (v is on the boundary when nbnd[v] > 0).
struct State {
    const WGraph& g;
    Work& wk;
    std::vector<char>& side;
    std::vector<double>& gain;
    std::vector<int>& nbnd;
    double cut = 0.0;
    int64_t wa = 0;  // weight of part 0

    State(const WGraph& gr, Work& w) : g(gr), wk(w), side(w.side), gain(w.gain), nbnd(w.nbnd) {}

    void init() {
        gain.assign(g.n, 0.0);
        nbnd.assign(g.n, 0);
        cut = 0.0;
        wa = 0;
        for (int v = 0; v < g.n; v++) {
            if (side[v] == 0) wa += g.vw[v];
            for (int e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
                if (side[g.adj[e]] != side[v]) {
                    gain[v] += g.w[e];
                    nbnd[v]++;
                    if (v < g.adj[e]) cut += g.w[e];
                } else {
                    gain[v] -= g.w[e];
                }
            }
        }
    }

    void move(int v) {
        const char from = side[v];
        side[v] = (char)(1 - from);
        wa += from == 0 ? -(int64_t)g.vw[v] : (int64_t)g.vw[v];
        cut -= gain[v];
        gain[v] = -gain[v];
        nbnd[v] = (g.ptr[v + 1] - g.ptr[v]) - nbnd[v];
        for (int e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
            const int u = g.adj[e];
            if (side[u] == from) {  // the edge is now cut
                gain[u] += 2.0 * g.w[e];
                nbnd[u]++;
            } else {  // the edge is now inside part side[v]
                gain[u] -= 2.0 * g.w[e];
                nbnd[u]--;
            }
        }
    }

    // top candidate of a lazily kept heap for part s (stale entries dropped)
    bool top(Heap& h, int s, bool use_locks, Cand& out) {
        while (!h.empty()) {
            const Cand c = h.top();
            if (side[c.v] == s && gain[c.v] == c.g && !(use_locks && wk.locked[c.v])) {
                out = c;
                return true;
            }
            h.pop();
        }
        return false;
    }
};

// Moves vertices off the overweight part, largest gain first, until
// lo <= wa <= hi; a vertex whose move would overshoot the other bound is
// passed over.  Stops early only when nothing movable is left.
void rebalance(State& s, int64_t lo, int64_t hi) {
    if (s.wa >= lo && s.wa <= hi) return;
    const int from = s.wa > hi ? 0 : 1;
    Heap& h = s.wk.h[0];
    h.clear();
    for (int v = 0; v < s.g.n; v++)
        if (s.side[v] == from) h.push({s.gain[v], v});
    Cand c;
    while ((from == 0 ? s.wa > hi : s.wa < lo) && s.top(h, from, false, c)) {
        h.pop();
        const int64_t nwa = from == 0 ? s.wa - s.g.vw[c.v] : s.wa + s.g.vw[c.v];
        if (from == 0 ? nwa < lo : nwa > hi) continue;
        s.move(c.v);
        for (int e = s.g.ptr[c.v]; e < s.g.ptr[c.v + 1]; e++) {
            const int u = s.g.adj[e];
            if (s.side[u] == from) h.push({s.gain[u], u});
        }
    }
}

// One boundary FM pass.  Moves stay inside the window ta +- slack; the best
// prefix is the one with the smallest cut among states with |wa - ta| <= tol
// (ties: the smaller deviation, then the shorter prefix).  Returns whether
// the pass kept any move.
bool fm_pass(State& s, int64_t ta, int64_t tol, int64_t slack, double eps) {
    const WGraph& g = s.g;
    Work& wk = s.wk;
    wk.locked.assign(g.n, 0);
    Heap* h = wk.h;
    h[0].clear();
    h[1].clear();
    for (int v = 0; v < g.n; v++)
        if (s.nbnd[v] > 0) h[(int)s.side[v]].push({s.gain[v], v});
    std::vector<int>& moves = wk.moves;
    moves.clear();
    double best_cut = s.cut;
    int64_t best_dev = std::llabs(s.wa - ta);
    size_t best_len = 0;
    const int limit = std::max(50, g.n / 50);
    int since = 0;
    for (;;) {
        Cand c[2];
        bool ok[2];
        for (int p = 0; p < 2; p++) {
            for (;;) {
                ok[p] = s.top(h[p], p, true, c[p]);
                if (!ok[p]) break;
                const int64_t nwa = p == 0 ? s.wa - g.vw[c[p].v] : s.wa + g.vw[c[p].v];
                if (std::llabs(nwa - ta) <= slack) break;
                h[p].pop();  // would leave the window: skipped for this pass
            }
        }
        int p;
        if (ok[0] && ok[1]) {
            if (c[0].g != c[1].g) {
                p = c[0].g > c[1].g ? 0 : 1;
            } else {
                const int64_t d0 = std::llabs(s.wa - g.vw[c[0].v] - ta), d1 = std::llabs(s.wa + g.vw[c[1].v] - ta);
                p = d0 != d1 ? (d0 < d1 ? 0 : 1) : (c[0].v < c[1].v ? 0 : 1);
            }
        } else if (ok[0] || ok[1]) {
            p = ok[0] ? 0 : 1;
        } else {
            break;
        }
        const int v = c[p].v;
        h[p].pop();
        s.move(v);
        wk.locked[v] = 1;
        moves.push_back(v);
        for (int e = g.ptr[v]; e < g.ptr[v + 1]; e++) {
            const int u = g.adj[e];
            if (!wk.locked[u] && s.nbnd[u] > 0) h[(int)s.side[u]].push({s.gain[u], u});
        }
        const int64_t dev = std::llabs(s.wa - ta);
        if (dev <= tol && (s.cut < best_cut - eps || (s.cut <= best_cut + eps && dev < best_dev))) {
            best_cut = s.cut;
            best_dev = dev;
            best_len = moves.size();
            since = 0;
        } else if (++since > limit) {
            break;
        }
    }
    for (size_t i = moves.size(); i > best_len; i--) s.move(moves[i - 1]);
    return best_len > 0;
}

void refine(State& s, int64_t ta, int64_t tol, int64_t slack, double eps) {
    rebalance(s, ta - tol, ta + tol);
    for (int pass = 0; pass < 8; pass++)
        if (!fm_pass(s, ta, tol, slack, eps)) break;
}

// Last vertex of a BFS from `start` (within start's component).
int bfs_last(const WGraph& g, int start, Work& wk) {
    wk.seen.assign(g.n, 0);
    std::vector<int>& q = wk.queue;
    q.assign(1, start);
    wk.seen[start] = 1;
    for (size_t i = 0; i < q.size(); i++)
        for (int e = g.ptr[q[i]]; e < g.ptr[q[i] + 1]; e++)
            if (!wk.seen[g.adj[e]]) {
                wk.seen[g.adj[e]] = 1;
                q.push_back(g.adj[e]);
            }
    return q.back();
}

// Graph growing: part 0 starts as {seed} and takes, while it is below the
// target, the boundary vertex of part 1 with the largest gain that fits
// (the smallest-index vertex that fits when no boundary vertex does).
void grow(State& s, int seed, int64_t ta, int64_t tol) {
    const WGraph& g = s.g;
    s.side.assign(g.n, 1);
    s.init();
    s.move(seed);
    Heap& h = s.wk.h[1];
    h.clear();
    auto push_nb = [&](int v) {
        for (int e = g.ptr[v]; e < g.ptr[v + 1]; e++)
            if (s.side[g.adj[e]] == 1) h.push({s.gain[g.adj[e]], g.adj[e]});
    };
    push_nb(seed);
    int scan = 0;
    while (s.wa < ta) {
        Cand c;
        int v = -1;
        while (s.top(h, 1, false, c)) {
            h.pop();
            if (s.wa + g.vw[c.v] <= ta + tol) {
                v = c.v;
                break;
            }
        }
        if (v < 0) {
            for (; scan < g.n; scan++)
                if (s.side[scan] == 1 && s.wa + g.vw[scan] <= ta + tol) break;
            if (scan == g.n) break;
            v = scan;
        }
        s.move(v);
        push_nb(v);
    }
}

thread_local Work tl_work;

}  // namespace

void hs::ml_bisect(int n, const int* ptr, const int* adj, const double* w, int na, std::vector<char>& part) {
    part.assign(n, 1);
    if (n == 0 || na <= 0) return;
    if (na >= n) {
        part.assign(n, 0);
        return;
    }
    constexpr int kCoarsenTo = 80, kSeeds = 12;
    Work& wk = tl_work;
    std::vector<std::unique_ptr<WGraph>> G;
    G.emplace_back(new WGraph);
    {
        WGraph& g0 = *G[0];
        g0.n = n;
        g0.ptr.assign(ptr, ptr + n + 1);
        g0.adj.assign(adj + ptr[0], adj + ptr[n]);
        g0.w.assign(w + ptr[0], w + ptr[n]);
        if (ptr[0] != 0)
            for (int& p : g0.ptr) p -= ptr[0];
        g0.vw.assign(n, 1);
        g0.maxvw = 1;
    }
    double total = 0.0;
    for (double x : G[0]->w) total += x;
    const double eps = 1e-12 * total;
    const int cap = std::max(1, (int)(1.5 * n / kCoarsenTo));
    while (G.back()->n > kCoarsenTo && G.size() < 48) {
        std::unique_ptr<WGraph> c(new WGraph);
        if (!coarsen(*G.back(), *c, cap, (uint32_t)G.size() * 0x9e3779b9u)) break;
        G.push_back(std::move(c));
    }
    const int64_t ta = na;
    auto tol_of = [&](size_t l) -> int64_t { return l == 0 ? 0 : G[l]->maxvw; };
    auto slack_of = [&](size_t l) -> int64_t { return std::max<int64_t>(tol_of(l), G[l]->maxvw); };

    // initial bisection of the coarsest graph: the best of the grown parts
    const size_t top = G.size() - 1;
    const WGraph& gc = *G[top];
    int seeds[kSeeds];
    int nseeds = 0;
    seeds[nseeds++] = bfs_last(gc, bfs_last(gc, 0, wk), wk);
    for (uint32_t i = 1; nseeds < kSeeds && i < 256; i++) {
        const int s = (int)(mix32(i * 0x632be5abu) % (uint32_t)gc.n);
        if (std::find(seeds, seeds + nseeds, s) == seeds + nseeds) seeds[nseeds++] = s;
    }
    std::vector<char>& best = wk.best;
    best.clear();
    double best_cut = 0.0;
    int64_t best_dev = 0;
    for (int k = 0; k < nseeds; k++) {
        State s(gc, wk);
        grow(s, seeds[k], ta, tol_of(top));
        refine(s, ta, tol_of(top), slack_of(top), eps);
        const int64_t dev = std::llabs(s.wa - ta);
        if (best.empty() || s.cut < best_cut - eps || (s.cut <= best_cut + eps && dev < best_dev)) {
            best = s.side;
            best_cut = s.cut;
            best_dev = dev;
        }
    }
    // projection and refinement level by level
    std::vector<char> coarse;
    coarse.swap(best);
    for (size_t l = top; l-- > 0;) {
        const WGraph& g = *G[l];
        State s(g, wk);
        s.side.resize(g.n);
        for (int v = 0; v < g.n; v++) s.side[v] = coarse[g.cmap[v]];
        s.init();
        refine(s, ta, tol_of(l), slack_of(l), eps);
        coarse.assign(s.side.begin(), s.side.end());
        G[l + 1].reset();
    }
    part.assign(coarse.begin(), coarse.end());
    best.swap(coarse);  // keep the capacity for the next call
}
