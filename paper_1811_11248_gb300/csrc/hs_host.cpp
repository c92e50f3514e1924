// hs_host.cpp -- host side of the hierarchical solver: column-preserving
// partition (Sec. 4.2), per-level symbolic planning (phases, neighbour / fill
// lists, block pattern with fill, Schur targets), the level-by-level driver of
// Algorithm 1, the solve phase of Algorithm 2 (captured once as a CUDA graph),
// PCG / GMRES (Sec. 5) and the C-ABI of include/hsolve.h.
//
// The phase rule (the paper leaves the cluster order of Algorithm 1 open):
// repeatedly take the greedy maximal independent set, in ascending cluster
// index, of the unprocessed clusters in the current block graph; that set is
// one phase.  Clusters of a phase share no block, so eliminating them together
// equals eliminating them one after another, up to the summation order of
// their additive Schur updates, which is fixed (ascending cluster index).
// Structure: the neighbours of a cluster are the blocks present in the level's
// input; eliminating a cluster's fine part creates a block between every pair
// of its neighbours; a cluster with no fill block has rank 0 and leaves.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <exception>
#include <mutex>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <unistd.h>
#include <unordered_map>
#include <vector>

#include "../../include/hsolve.h"
#include "hs_internal.h"

using namespace hs;

namespace {

// ---------------------------------------------------------------------------
// small utilities
// ---------------------------------------------------------------------------
struct HsError {
    int code;
};

#define CK(x)                                                                        \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            if (e_ == cudaErrorMemoryAllocation) throw HsError{HS_ERR_OOM};          \
            std::fprintf(stderr, "hsolve: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                  \
            throw HsError{HS_ERR_CUDA};                                              \
        }                                                                            \
    } while (0)

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Stream on which DBuf allocations and frees are ordered (set by every C-ABI
// entry point that allocates).  Allocations come from the device's default
// memory pool, which keeps freed blocks for reuse by the next setup.
thread_local cudaStream_t g_alloc_stream = nullptr;

void prepare_pool() {
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

struct Trace {
    bool on = std::getenv("HS_TRACE") != nullptr;
    double t = now_s();
    void mark(const char* what) {
        if (!on) return;
        const double n = now_s();
        std::fprintf(stderr, "hs_trace %-28s %8.3f ms\n", what, (n - t) * 1e3);
        t = n;
    }
};

// Device buffer owned by a handle.
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, g_alloc_stream);
        p = nullptr;
        bytes = 0;
    }
    void ensure(size_t b) {
        if (p && bytes >= b) return;
        alloc(b);
    }
    void alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        CK(cudaMallocAsync(&p, b, g_alloc_stream));
        bytes = b;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Pinned host staging for host<->device copies (copies from pageable memory
// are staged synchronously by the driver).  Data is appended; the area is
// reused only after every stream with copies pending from it has drained.
struct PinnedStage {
    char* p = nullptr;
    size_t cap = 0, used = 0;
    std::vector<cudaStream_t> pending;
    ~PinnedStage() {
        if (p) cudaFreeHost(p);
    }
    void drain() {
        for (cudaStream_t s : pending) cudaStreamSynchronize(s);
        pending.clear();
        used = 0;
    }
    // space for `bytes` that the caller fills, then copies on stream st
    char* take(size_t bytes, cudaStream_t st) {
        const size_t need = (bytes + 255) & ~(size_t)255;
        if (used + need > cap) {
            drain();
            if (need > cap) {
                if (p) cudaFreeHost(p);
                p = nullptr;
                cap = std::max(need, (size_t)16 << 20);
                CK(cudaHostAlloc(reinterpret_cast<void**>(&p), cap, cudaHostAllocDefault));
            }
        }
        char* d = p + used;
        used += need;
        if (std::find(pending.begin(), pending.end(), st) == pending.end()) pending.push_back(st);
        return d;
    }
    // the caller has synchronised st: the area is free if st was the only user
    void synced(cudaStream_t st) {
        if (pending.size() == 1 && pending[0] == st) {
            pending.clear();
            used = 0;
        }
    }
};
thread_local PinnedStage g_stage;
thread_local PinnedStage g_pattern_stage;  // the pattern read back by a setup with device inputs

template <class T>
void upload(DBuf& d, const std::vector<T>& h, cudaStream_t st) {
    d.alloc(sizeof(T) * std::max<size_t>(h.size(), 1));
    if (h.empty()) return;
    char* pin = g_stage.take(sizeof(T) * h.size(), st);
    std::memcpy(pin, h.data(), sizeof(T) * h.size());
    CK(cudaMemcpyAsync(d.p, pin, sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
}

// device -> host through the staging area; synchronises st
template <class T>
void download(std::vector<T>& h, const void* d, size_t count, cudaStream_t st) {
    h.resize(count);
    if (count == 0) return;
    char* pin = g_stage.take(sizeof(T) * count, st);
    CK(cudaMemcpyAsync(pin, d, sizeof(T) * count, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::memcpy(h.data(), pin, sizeof(T) * count);
    g_stage.synced(st);
}

void sorted_insert(std::vector<int>& v, int x) {
    auto it = std::lower_bound(v.begin(), v.end(), x);
    if (it == v.end() || *it != x) v.insert(it, x);
}
void sorted_erase(std::vector<int>& v, int x) {
    auto it = std::lower_bound(v.begin(), v.end(), x);
    if (it != v.end() && *it == x) v.erase(it);
}
bool sorted_has(const std::vector<int>& v, int x) { return std::binary_search(v.begin(), v.end(), x); }

// Run f(lo, hi, t) over [0, n) split into contiguous ranges on up to
// hs_threads() host threads (the results never depend on the split).
// Default: up to 16, leaving two of the machine's cores to other threads
// (the workers poll between jobs, and a polling worker that shares a core
// with the caller or a driver thread would slow them).
int hs_threads() {
    static const int t = [] {
        const unsigned h = std::thread::hardware_concurrency();
        const char* e = std::getenv("HS_THREADS");
        int v = e ? std::atoi(e) : (int)std::min(16u, h > 3 ? h - 2 : 1u);
        return std::max(1, v);
    }();
    return t;
}

// set on the worker threads of a batched partition: nested work stays serial
thread_local bool tl_serial = false;

// Persistent worker threads for the host planner (created on first use):
// run(T, fn) runs fn(0) .. fn(T-1), fn(0) on the caller, the rest on whichever
// thread (worker or caller) takes them first, and returns when all are done.
// A call from a worker, or while another call is running, runs serially on
// its thread.  Between jobs a worker polls for the next one for a while
// (HS_SPIN_US microseconds, default 2000) before it sleeps: the planner's
// parallel loops come in bursts a few hundred microseconds apart, and waking a
// sleeping thread costs tens of microseconds per job.
thread_local bool tl_in_pool = false;

class Pool {
  public:
    static Pool& get() {
        static Pool p(hs_threads() - 1);
        return p;
    }
    int workers() const { return (int)th_.size(); }
    // Starts the workers polling (they find no task) so that the next job
    // does not wait for them to wake: for a caller about to run a burst of
    // parallel loops.
    void wake() {
        if (getpid() != pid_ || th_.empty()) return;
        std::unique_lock<std::mutex> busy(run_mu_, std::try_to_lock);
        if (!busy.owns_lock()) return;
        {
            std::unique_lock<std::mutex> lk(mu_);
            if (inside_.load(std::memory_order_acquire) > 0) return;
            job_ = nullptr;
            njob_ = 0;
            next_.store(1, std::memory_order_relaxed);
            pending_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
    }
    bool try_run(int T, const std::function<void(int)>& fn) {
        if (getpid() != pid_) return false;  // a forked child has no workers
        std::unique_lock<std::mutex> busy(run_mu_, std::try_to_lock);
        if (!busy.owns_lock()) return false;
        {
            // workers join a job under mu_; a worker still inside the
            // previous job (it took no task, or its last one) leaves first
            std::unique_lock<std::mutex> lk(mu_);
            while (inside_.load(std::memory_order_acquire) > 0) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            }
            job_ = &fn;
            njob_ = T;
            next_.store(1, std::memory_order_relaxed);
            pending_.store(T - 1, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        fn(0);
        for (;;) {  // the caller takes tasks no worker has taken yet
            const int t = next_.fetch_add(1, std::memory_order_acq_rel);
            if (t >= T) break;
            fn(t);
            pending_.fetch_sub(1, std::memory_order_acq_rel);
        }
        for (int k = 0; pending_.load(std::memory_order_acquire) != 0; k++)
            if (k > 4096) std::this_thread::yield();
        return true;
    }
    ~Pool() {
        if (getpid() != pid_) {  // forked child: the threads are not ours
            for (auto& t : th_) t.detach();
            return;
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }

  private:
    explicit Pool(int n) : pid_(getpid()) {
        const char* e = std::getenv("HS_SPIN_US");
        spin_us_ = e ? std::max(0, std::atoi(e)) : 2000;
        for (int i = 0; i < n; i++) th_.emplace_back([this] { loop(); });
    }
    void loop() {
        tl_in_pool = true;
        unsigned seen = gen_.load(std::memory_order_acquire);
        for (;;) {
            // poll for the next job (the clock read every 64 polls, the core
            // offered to other threads every 256), then sleep
            const auto t0 = std::chrono::steady_clock::now();
            for (int k = 1; gen_.load(std::memory_order_acquire) == seen; k++) {
                if ((k & 255) == 0) std::this_thread::yield();
                if ((k & 63) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(spin_us_)) {
                    std::unique_lock<std::mutex> lk(mu_);
                    cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
                    break;
                }
            }
            const std::function<void(int)>* f;
            int n;
            {
                std::lock_guard<std::mutex> lk(mu_);
                if (stop_) return;
                seen = gen_.load(std::memory_order_acquire);
                f = job_;
                n = njob_;
                inside_.fetch_add(1, std::memory_order_acq_rel);
            }
            for (;;) {
                const int t = next_.fetch_add(1, std::memory_order_acq_rel);
                if (t >= n) break;
                (*f)(t);
                pending_.fetch_sub(1, std::memory_order_acq_rel);
            }
            inside_.fetch_sub(1, std::memory_order_acq_rel);
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_, run_mu_;
    std::condition_variable cv_;
    std::atomic<unsigned> gen_{0};
    std::atomic<int> next_{0}, pending_{0}, inside_{0};
    const std::function<void(int)>* job_ = nullptr;
    int njob_ = 0;
    int spin_us_ = 2000;
    bool stop_ = false;
    pid_t pid_;
};

// Runs fn(t) for t < T (t = 0 on the calling thread; the others on the
// pool's workers) and rethrows the first exception any of them raised.
template <class F>
void run_threads(int T, F&& fn) {
    std::exception_ptr err;
    std::mutex mu;
    std::function<void(int)> wrap = [&](int t) {
        try {
            fn(t);
        } catch (...) {
            std::lock_guard<std::mutex> g(mu);
            if (!err) err = std::current_exception();
        }
    };
    T = std::max(1, std::min(T, Pool::get().workers() + 1));
    if (T <= 1 || tl_in_pool || !Pool::get().try_run(T, wrap))
        for (int t = 0; t < T; t++) wrap(t);
    if (err) std::rethrow_exception(err);
}

template <class F>
void parallel_ranges(int64_t n, int64_t grain, F&& f) {
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(hs_threads(), n / std::max<int64_t>(grain, 1)));
    if (T <= 1 || tl_serial) {
        f((int64_t)0, n, 0);
        return;
    }
    run_threads(T, [&](int t) { f(n * t / T, n * (t + 1) / T, t); });
}

// out = f(0) ++ f(1) ++ ... ++ f(n-1), items appended by f(i, out) in
// parallel chunks and concatenated in index order.
template <class T, class F>
std::vector<T> parallel_collect(int64_t n, int64_t grain, F&& f) {
    const int NT = (int)std::max<int64_t>(1, std::min<int64_t>(hs_threads(), n / std::max<int64_t>(grain, 1)));
    std::vector<std::vector<T>> part(NT);
    parallel_ranges(n, grain, [&](int64_t lo, int64_t hi, int t) {
        for (int64_t i = lo; i < hi; i++) f(i, part[t]);
    });
    std::vector<T> out;
    size_t tot = 0;
    for (auto& v : part) tot += v.size();
    out.reserve(tot);
    for (auto& v : part) out.insert(out.end(), v.begin(), v.end());
    return out;
}

// ---------------------------------------------------------------------------
// Partition (Sec. 4.2)
// ---------------------------------------------------------------------------
struct Partitioner {
    int nl = 0;
    std::vector<double> lx, ly;
    bool have_coords = false;
    bool multilevel = false;
    std::vector<int> gptr, gadj;
    std::vector<double> gw;       // line-graph edge weights (multilevel only)
    std::vector<int> own, loc;    // per line: its set at the current depth and its place there
    int L = 0;
    std::vector<int> leaf_of;
    int next_leaf = 0;
    std::vector<char> state;

    // BFS inside `set` from `start`; new components start at the lowest unvisited line.
    std::vector<int> bfs(const std::vector<int>& set, int start) {
        std::vector<int> out;
        out.reserve(set.size());
        for (int x : set) state[x] = 1;
        std::vector<int> queue;
        queue.reserve(set.size());
        int root = start;
        while (out.size() < set.size()) {
            if (state[root] != 1) {
                root = -1;
                for (int x : set)
                    if (state[x] == 1 && (root < 0 || x < root)) root = x;
            }
            state[root] = 2;
            queue.clear();
            queue.push_back(root);
            for (size_t h = 0; h < queue.size(); h++) {
                const int u = queue[h];
                out.push_back(u);
                for (int e = gptr[u]; e < gptr[u + 1]; e++) {
                    const int w = gadj[e];
                    if (state[w] == 1) {
                        state[w] = 2;
                        queue.push_back(w);
                    }
                }
            }
        }
        for (int x : set) state[x] = 0;
        return out;
    }

    // One bisection of `set` (ascending) without coordinates: the first
    // ceil(k/2) lines of a BFS order started from a pseudo-peripheral line;
    // both parts come out ascending.  The BFS reads the marks of neighbouring
    // lines, which may belong to another set, so it runs on one set at a
    // time.  The multilevel rule bisects the weighted subgraph induced by
    // `set` (its lines carry own == sid) into ceil(k/2) and floor(k/2) lines.
    // With coordinates, bisect_coords below.
    void bisect(const std::vector<int>& set, std::vector<int>& a, std::vector<int>& b, int sid = -1) {
        const size_t k = set.size(), left = (k + 1) / 2;
        a.clear();
        b.clear();
        if (multilevel) {
            std::vector<int> sp(k + 1, 0), sa;
            std::vector<double> sw;
            for (size_t i = 0; i < k; i++) {
                const int x = set[i];
                for (int e = gptr[x]; e < gptr[x + 1]; e++)
                    if (own[gadj[e]] == sid) {
                        sa.push_back(loc[gadj[e]]);
                        sw.push_back(gw[e]);
                    }
                sp[i + 1] = (int)sa.size();
            }
            std::vector<char> part;
            ml_bisect((int)k, sp.data(), sa.data(), sw.data(), (int)left, part);
            a.reserve(left);
            b.reserve(k - left);
            for (size_t i = 0; i < k; i++) (part[i] == 0 ? a : b).push_back(set[i]);
        } else {
            const int lo = *std::min_element(set.begin(), set.end());
            std::vector<int> first = bfs(set, lo);
            std::vector<int> order = bfs(set, first.back());
            a.assign(order.begin(), order.begin() + left);
            b.assign(order.begin() + left, order.end());
            std::sort(a.begin(), a.end());
            std::sort(b.begin(), b.end());
        }
    }

    // Leaf ids follow the depth-first order: the left half of the set below
    // leaf offset `base` at depth d keeps `base`, the right half starts
    // 2^(L-d-1) further.  Depth-first recursion (the BFS rule).
    void split(std::vector<int> set, int depth, int base) {
        if (depth == L) {
            for (int x : set) leaf_of[x] = base;
            return;
        }
        std::vector<int> a, b;
        bisect(set, a, b);
        std::vector<int>().swap(set);
        const int half = 1 << (L - depth - 1);
        split(std::move(a), depth + 1, base);
        split(std::move(b), depth + 1, base + half);
    }

    // The coordinate rule on v[0, k) (ascending) in place: the left part is
    // the ceil(k/2) smallest lines in (coordinate, index) order along the
    // longer extent; the pivot is selected by nth_element on a copy in tmp
    // (at least k ints), then both parts are written back ascending.
    void bisect_coords(int* v, int k, int* tmp) {
        const int left = (k + 1) / 2;
        double x0 = lx[v[0]], x1 = x0, y0 = ly[v[0]], y1 = y0;
        for (int i = 0; i < k; i++) {
            const int x = v[i];
            x0 = std::min(x0, lx[x]); x1 = std::max(x1, lx[x]);
            y0 = std::min(y0, ly[x]); y1 = std::max(y1, ly[x]);
        }
        const std::vector<double>& key = (x1 - x0 >= y1 - y0) ? lx : ly;
        auto less = [&](int u, int w) { return key[u] < key[w] || (key[u] == key[w] && u < w); };
        std::copy(v, v + k, tmp);
        std::nth_element(tmp, tmp + (left - 1), tmp + k, less);
        const int piv = tmp[left - 1];
        int na = 0, nb = 0;
        for (int i = 0; i < k; i++) {
            const int x = v[i];
            if (less(x, piv) || x == piv) v[na++] = x;
            else tmp[nb++] = x;
        }
        std::copy(tmp, tmp + nb, v + na);
    }
    void split_coords(int* v, int k, int depth, int base, int* tmp) {
        if (depth == L || k <= 0) {
            for (int i = 0; i < k; i++) leaf_of[v[i]] = base;
            return;
        }
        bisect_coords(v, k, tmp);
        const int left = (k + 1) / 2, half = 1 << (L - depth - 1);
        if (depth < 3 && k > 4096 && !tl_serial) {  // the two halves' scratch is disjoint too
            run_threads(2, [&](int t) {
                if (t == 1) split_coords(v, left, depth + 1, base, tmp);
                else split_coords(v + left, k - left, depth + 1, base + half, tmp + left);
            });
        } else {
            split_coords(v, left, depth + 1, base, tmp);
            split_coords(v + left, k - left, depth + 1, base + half, tmp);
        }
    }

    // The same leaves; with coordinates in place on one array (for many
    // lines in L rounds, the sets of a round bisected in parallel), for the
    // multilevel rule in L rounds of parallel bisections.
    void split_all(std::vector<int> all) {
        if (have_coords && !multilevel) {
            const int k = (int)all.size();
            std::vector<int> tmp(std::max(k, 1));  // scratch: a set's copy sits at the set's offset
            if (nl <= (1 << 15) || tl_serial) {
                split_coords(all.data(), k, 0, 0, tmp.data());
                return;
            }
            // sets of a round: (offset, size, leaf base), contiguous in `all`
            std::vector<std::array<int, 3>> sets{{0, k, 0}}, next;
            for (int depth = 0; depth < L; depth++) {
                const int half = 1 << (L - depth - 1);
                parallel_ranges((int64_t)sets.size(), 1, [&](int64_t lo, int64_t hi, int) {
                    for (int64_t i = lo; i < hi; i++)
                        if (sets[i][1] > 0)
                            bisect_coords(all.data() + sets[i][0], sets[i][1], tmp.data() + sets[i][0]);
                });
                next.clear();
                for (const auto& st : sets) {
                    const int left = (st[1] + 1) / 2;
                    next.push_back({st[0], left, st[2]});
                    next.push_back({st[0] + left, st[1] - left, st[2] + half});
                }
                sets.swap(next);
            }
            parallel_ranges((int64_t)sets.size(), 64, [&](int64_t lo, int64_t hi, int) {
                for (int64_t i = lo; i < hi; i++)
                    for (int j = 0; j < sets[i][1]; j++) leaf_of[all[sets[i][0] + j]] = sets[i][2];
            });
            return;
        }
        if (!multilevel) {
            split(std::move(all), 0, 0);
            return;
        }
        std::vector<std::vector<int>> sets(1), next;
        sets[0] = std::move(all);
        std::vector<int> base(1, 0), nbase;
        for (int depth = 0; depth < L; depth++) {
            const int ns = (int)sets.size(), half = 1 << (L - depth - 1);
            next.assign(2 * (size_t)ns, {});
            nbase.assign(2 * (size_t)ns, 0);
            // each line learns its set at this depth before any set is bisected
            parallel_ranges(ns, 1, [&](int64_t lo, int64_t hi, int) {
                for (int64_t i = lo; i < hi; i++)
                    for (size_t j = 0; j < sets[i].size(); j++) {
                        own[sets[i][j]] = (int)i;
                        loc[sets[i][j]] = (int)j;
                    }
            });
            parallel_ranges(ns, 1, [&](int64_t lo, int64_t hi, int) {
                for (int64_t i = lo; i < hi; i++) {
                    bisect(sets[i], next[2 * i], next[2 * i + 1], (int)i);
                    nbase[2 * i] = base[i];
                    nbase[2 * i + 1] = base[i] + half;
                    std::vector<int>().swap(sets[i]);
                }
            });
            sets.swap(next);
            base.swap(nbase);
        }
        parallel_ranges((int64_t)sets.size(), 64, [&](int64_t lo, int64_t hi, int) {
            for (int64_t i = lo; i < hi; i++)
                for (int x : sets[i]) leaf_of[x] = base[i];
        });
    }
};

int partition_impl(int64_t n64, const int64_t* rowptr, const int32_t* col, const double* val, const double* coords,
                   int leaf_lines, double theta, std::vector<int32_t>& perm, std::vector<int32_t>& leaf_ptr,
                   int method = kPartAuto) {
    const int n = (int)n64;
    Trace tr;
    // strongly coupled lines: union-find over |a_ij| >= theta * max_{k != i} |a_ik|.
    // Strong edges are found and linked in parallel: a root is only ever
    // linked (by compare-and-swap) under a smaller root, so every component
    // ends with its smallest DOF as root whatever the order of the links.
    std::vector<std::atomic<int>> root(n);
    parallel_ranges(n, 1 << 16, [&](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; i++) root[i].store((int)i, std::memory_order_relaxed);
    });
    auto find = [&](int x) {
        for (;;) {
            int p = root[x].load(std::memory_order_relaxed);
            if (p == x) return x;
            const int gp = root[p].load(std::memory_order_relaxed);
            // path halving (links only point to smaller indices, so a value
            // read here is always an ancestor; a failed exchange is harmless)
            if (gp != p) root[x].compare_exchange_weak(p, gp, std::memory_order_relaxed);
            x = gp;
        }
    };
    auto unite = [&](int a, int b) {
        for (;;) {
            a = find(a);
            b = find(b);
            if (a == b) return;
            if (a < b) std::swap(a, b);  // link the larger root under the smaller
            int expect = a;
            if (root[a].compare_exchange_strong(expect, b, std::memory_order_relaxed)) return;
        }
    };
    parallel_ranges(n, 4096, [&](int64_t lo, int64_t hi, int) {
        for (int64_t i = lo; i < hi; i++) {
            double m = 0.0;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
                if (col[e] != i) m = std::max(m, std::fabs(val[e]));
            if (m <= 0.0) continue;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
                const int j = col[e];
                if (j != i && std::fabs(val[e]) >= theta * m) unite((int)i, j);
            }
        }
    });
    tr.mark("  partition: union-find");
    Partitioner P;
    std::vector<int> line_of(n), first;
    if (n <= (1 << 18) || tl_serial) {
        std::vector<int> id(n, -1);
        for (int i = 0; i < n; i++) {
            const int r = find(i);  // roots are final: no link is running
            if (id[r] < 0) { id[r] = (int)first.size(); first.push_back(i); }
            line_of[i] = id[r];
        }
    } else {
        // every root is the smallest DOF of its line, so numbering the roots
        // in ascending order numbers the lines by their first DOF: chunk
        // counts of roots, a prefix sum, then the ids (roots are final)
        constexpr int nchunk = 64;
        std::vector<int> rc(nchunk + 1, 0);
        auto is_root = [&](int64_t i) { return root[i].load(std::memory_order_relaxed) == (int)i; };
        parallel_ranges(nchunk, 1, [&](int64_t lo, int64_t hi, int) {
            for (int64_t ch = lo; ch < hi; ch++) {
                int k = 0;
                for (int64_t i = n * ch / nchunk; i < n * (ch + 1) / nchunk; i++) k += is_root(i);
                rc[ch + 1] = k;
            }
        });
        for (int ch = 0; ch < nchunk; ch++) rc[ch + 1] += rc[ch];
        first.resize(rc[nchunk]);
        parallel_ranges(nchunk, 1, [&](int64_t lo, int64_t hi, int) {
            for (int64_t ch = lo; ch < hi; ch++) {
                int id = rc[ch];
                for (int64_t i = n * ch / nchunk; i < n * (ch + 1) / nchunk; i++)
                    if (is_root(i)) {
                        first[id] = (int)i;
                        line_of[i] = id++;
                    }
            }
        });
        parallel_ranges(n, 1 << 16, [&](int64_t lo, int64_t hi, int) {
            for (int64_t i = lo; i < hi; i++) {
                const int r = find((int)i);
                if (r != i) line_of[i] = line_of[r];
            }
        });
    }
    P.nl = (int)first.size();
    tr.mark("  partition: line ids");
    // DOFs grouped by line (counting sort), ascending within a line
    std::vector<int> lptr(P.nl + 1, 0), ldof(n);
    for (int i = 0; i < n; i++) lptr[line_of[i] + 1]++;
    for (int l = 0; l < P.nl; l++) lptr[l + 1] += lptr[l];
    {
        std::vector<int> pos(lptr.begin(), lptr.end() - 1);
        for (int i = 0; i < n; i++) ldof[pos[line_of[i]]++] = i;
    }
    {
        // each line's neighbour lines collected with a visit stamp and sorted
        const int nl = P.nl;
        // neighbour lines of each line, ranges of lines on separate threads
        const int T = hs_threads();
        std::vector<std::vector<int>> adj(T), cnt(T);
        std::vector<int64_t> lo_of(T + 1, 0);
        parallel_ranges(nl, 256, [&](int64_t lo, int64_t hi, int t) {
            std::vector<int> stamp(nl, -1);
            auto& a = adj[t];
            auto& k = cnt[t];
            lo_of[t] = lo;
            for (int64_t l = lo; l < hi; l++) {
                const size_t b = a.size();
                for (int q = lptr[l]; q < lptr[l + 1]; q++) {
                    const int i = ldof[q];
                    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
                        const int lj = line_of[col[e]];
                        if (lj != l && stamp[lj] != (int)l) {
                            stamp[lj] = (int)l;
                            a.push_back(lj);
                        }
                    }
                }
                std::sort(a.begin() + b, a.end());
                k.push_back((int)(a.size() - b));
            }
        });
        P.gptr.assign(nl + 1, 0);
        P.gadj.clear();
        int64_t total = 0;
        for (int t = 0; t < T; t++) total += (int64_t)adj[t].size();
        P.gadj.reserve(total);
        int l = 0;
        for (int t = 0; t < T; t++) {
            for (int k : cnt[t]) {
                P.gptr[l + 1] = P.gptr[l] + k;
                l++;
            }
            P.gadj.insert(P.gadj.end(), adj[t].begin(), adj[t].end());
        }
    }
    tr.mark("  partition: line graph");
    if (method == kPartMultilevel) {
        // edge weight between two lines: sum of |a_ij| over the nonzeros
        // joining them (summed in DOF order, then CSR order)
        P.multilevel = true;
        P.gw.assign(P.gadj.size(), 0.0);
        const int nl = P.nl;
        parallel_ranges(nl, 256, [&](int64_t lo, int64_t hi, int) {
            std::vector<double> acc(nl, 0.0);
            for (int64_t l = lo; l < hi; l++) {
                for (int q = lptr[l]; q < lptr[l + 1]; q++) {
                    const int i = ldof[q];
                    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
                        const int lj = line_of[col[e]];
                        if (lj != l) acc[lj] += std::fabs(val[e]);
                    }
                }
                for (int e = P.gptr[l]; e < P.gptr[l + 1]; e++) {
                    P.gw[e] = acc[P.gadj[e]];
                    acc[P.gadj[e]] = 0.0;
                }
            }
        });
        P.own.assign(nl, -1);
        P.loc.assign(nl, 0);
        coords = nullptr;
        tr.mark("  partition: edge weights");
    }
    if (coords) {
        P.have_coords = true;
        P.lx.resize(P.nl);
        P.ly.resize(P.nl);
        for (int l = 0; l < P.nl; l++) {
            P.lx[l] = coords[2 * (int64_t)first[l]];
            P.ly[l] = coords[2 * (int64_t)first[l] + 1];
        }
    }
    int L = 0;
    while (((int64_t)P.nl + (1LL << L) - 1) / (1LL << L) > leaf_lines && (1LL << (L + 1)) <= P.nl) L++;
    P.L = L;
    P.leaf_of.assign(P.nl, -1);
    P.state.assign(P.nl, 0);
    std::vector<int> all(P.nl);
    for (int l = 0; l < P.nl; l++) all[l] = l;
    P.split_all(std::move(all));
    tr.mark("  partition: bisection");
    // DOFs grouped by leaf, ascending within a leaf (a counting sort; for
    // many DOFs over contiguous chunks: counts per leaf and chunk, offsets
    // leaf by leaf with the chunks in order, then every chunk places its DOFs)
    const int nleaf = 1 << L;
    const int nch = tl_serial ? 1 : (int)std::max<int64_t>(1, std::min<int64_t>(hs_threads(), n / 8192));
    leaf_ptr.assign(nleaf + 1, 0);
    perm.assign(n, 0);
    if (nch == 1) {
        for (int i = 0; i < n; i++) leaf_ptr[P.leaf_of[line_of[i]] + 1]++;
        for (int c = 0; c < nleaf; c++) leaf_ptr[c + 1] += leaf_ptr[c];
        std::vector<int32_t> pos(leaf_ptr.begin(), leaf_ptr.end() - 1);
        for (int i = 0; i < n; i++) perm[pos[P.leaf_of[line_of[i]]]++] = i;
    } else {
        std::vector<int> leaf_dof(n);
        std::vector<int32_t> cnt((size_t)nleaf * nch, 0);  // [leaf][chunk]
        parallel_ranges(nch, 1, [&](int64_t lo, int64_t hi, int) {
            for (int64_t ch = lo; ch < hi; ch++)
                for (int64_t i = (int64_t)n * ch / nch; i < (int64_t)n * (ch + 1) / nch; i++) {
                    leaf_dof[i] = P.leaf_of[line_of[i]];
                    cnt[(size_t)leaf_dof[i] * nch + ch]++;
                }
        });
        int32_t run = 0;
        for (int c = 0; c < nleaf; c++) {
            for (int ch = 0; ch < nch; ch++) {
                const int32_t k = cnt[(size_t)c * nch + ch];
                cnt[(size_t)c * nch + ch] = run;
                run += k;
            }
            leaf_ptr[c + 1] = run;
        }
        parallel_ranges(nch, 1, [&](int64_t lo, int64_t hi, int) {
            for (int64_t ch = lo; ch < hi; ch++)
                for (int64_t i = (int64_t)n * ch / nch; i < (int64_t)n * (ch + 1) / nch; i++)
                    perm[cnt[(size_t)leaf_dof[i] * nch + ch]++] = (int32_t)i;
        });
    }
    tr.mark("  partition: permutation");
    return HS_OK;
}

// ---------------------------------------------------------------------------
// Symbolic plan of one level
// ---------------------------------------------------------------------------
// Per-cluster sorted index lists in one flat array (CSR): list c is
// idx[ptr[c] .. ptr[c + 1]).  One allocation per kind of list, not one per
// cluster (small allocations dominated the planning of small levels).
struct ListSet {
    std::vector<int64_t> ptr = std::vector<int64_t>(1, 0);
    std::vector<int32_t> idx;
    struct View {
        const int32_t *b, *e;
        const int32_t* begin() const { return b; }
        const int32_t* end() const { return e; }
        size_t size() const { return (size_t)(e - b); }
        bool empty() const { return b == e; }
        int32_t operator[](size_t i) const { return b[i]; }
    };
    View operator[](int64_t c) const { return View{idx.data() + ptr[c], idx.data() + ptr[c + 1]}; }
};

// ListSet of n lists, list i made by f(i, out, t) appending to out (t: the
// chunk, for per-chunk scratch; at most hs_threads() chunks); contiguous
// chunks of lists on separate threads, concatenated in order.
template <class F>
ListSet build_lists(int64_t n, int64_t grain, F&& f) {
    ListSet L;
    L.ptr.assign(n + 1, 0);
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(hs_threads(), n / std::max<int64_t>(grain, 1)));
    std::vector<std::vector<int32_t>> part(T);
    auto chunk = [&](int t) {
        const int64_t lo = n * t / T, hi = n * (t + 1) / T;
        for (int64_t i = lo; i < hi; i++) {
            const size_t before = part[t].size();
            f(i, part[t], t);
            L.ptr[i + 1] = (int64_t)(part[t].size() - before);
        }
    };
    if (T == 1 || tl_serial) for (int t = 0; t < T; t++) chunk(t);
    else run_threads(T, chunk);
    for (int64_t i = 0; i < n; i++) L.ptr[i + 1] += L.ptr[i];
    L.idx.resize((size_t)L.ptr[n]);
    size_t o = 0;
    for (auto& v : part) {
        std::copy(v.begin(), v.end(), L.idx.begin() + o);
        o += v.size();
    }
    return L;
}

struct LevelPlan {
    int nc = 0;
    std::vector<int> size0;
    ListSet adj0;                        // level input pattern (no diagonal)
    std::vector<int> phase;              // -1: empty cluster
    std::vector<std::vector<int>> phases;
    ListSet nl, wl;                      // n / w blocks of each cluster when it is eliminated
    ListSet all;                         // every block that exists during the level (with diagonal)
    ListSet endp;                        // blocks at level end (with diagonal of kept clusters)
    std::vector<char> vanished;
    // the list planner's per-cluster working lists, kept until the plan is
    // released (then freed on all threads)
    std::vector<std::vector<std::vector<int>>> scratch;
};

// The lists a planner makes for the clusters lo .. hi of one range, in
// cluster order: for each kind (n, w, all, end) the concatenated entries and
// every cluster's count.
enum { LS_NL = 0, LS_WL = 1, LS_ALL = 2, LS_END = 3, LS_N = 4 };
struct RangeLists {
    std::vector<int32_t> data[LS_N];
    std::vector<int32_t> cnt[LS_N];
};

// Phase rule and fill pattern (Sec. 3.2, Sec. 4.2) of the clusters lo .. hi,
// which share no block with any other cluster: phases are rounds of a greedy
// maximal independent set in ascending cluster order on the current block
// graph; eliminating c couples every pair of its neighbours.  The selection
// is sequential; the eliminations of one phase are applied in parallel: the
// selected clusters are pairwise non-adjacent, so each one's neighbour lists
// are final when the phase starts, and a neighbour p that several of them
// share receives the union of their couplings (set unions, so the order in
// which they land does not matter).
struct PlanLists {  // the list planner's per-cluster lists (indexed by cluster)
    std::vector<std::vector<int>> nl, wl, all, endp;
};

void plan_range(LevelPlan& P, PlanLists& Q, std::vector<std::vector<int>>& cur, int lo, int hi,
                std::vector<std::vector<int>>& phases) {
    std::vector<char> done(hi - lo, 0), insel(hi - lo, 0), target(hi - lo, 0), blocked(hi - lo, 0);
    auto D = [&](int c) -> char& { return done[c - lo]; };
    auto S = [&](int c) -> char& { return insel[c - lo]; };
    auto B = [&](int c) -> char& { return blocked[c - lo]; };  // has a selected neighbour
    auto T = [&](int c) -> char& { return target[c - lo]; };   // gains couplings in this phase
    std::vector<int> tg, scratch, tgi(hi - lo, 0);
    std::vector<std::vector<int>> src;  // per target of the phase: its selected neighbours
    int remaining = 0;
    for (int c = lo; c < hi; c++) {
        if (P.size0[c] > 0) remaining++;
        else D(c) = 1;
    }
    int first = lo;  // clusters below `first` are all done
    // v <- v u (add \ {p}), both sorted, in place: count the new entries,
    // grow v by that much and merge from the back (no temporary list)
    auto merge_into = [](std::vector<int>& v, const std::vector<int>& add, int p) {
        size_t i = 0, nnew = 0;
        for (int x : add) {
            if (x == p) continue;  // p does not gain itself
            while (i < v.size() && v[i] < x) i++;
            if (i == v.size() || v[i] != x) nnew++;
        }
        if (nnew == 0) return;
        const size_t a = v.size();
        v.resize(a + nnew);
        ptrdiff_t ia = (ptrdiff_t)a - 1, ib = (ptrdiff_t)add.size() - 1, o = (ptrdiff_t)(a + nnew) - 1;
        while (ib >= 0) {
            const int x = add[ib];
            if (x == p) { ib--; continue; }
            if (ia >= 0 && v[ia] >= x) {
                if (v[ia] == x) ib--;  // present already: kept once
                v[o--] = v[ia--];
            } else {
                v[o--] = x;
                ib--;
            }
        }
    };
    while (remaining > 0) {
        std::vector<int> sel;
        while (first < hi && D(first)) first++;
        // each selected cluster: neighbours in the level's input pattern (n)
        // and fill neighbours (w), and without fill it vanishes from the
        // graph; tg: the clusters that gain couplings, each listed once
        tg.clear();
        int64_t work = 0;  // size of the list merges ahead, roughly
        for (int c = first; c < hi; c++) {
            if (D(c) || B(c)) continue;
            S(c) = 1;
            sel.push_back(c);
            const auto& a0 = P.adj0[c];
            Q.nl[c].reserve(std::min(cur[c].size(), a0.size()));
            Q.wl[c].reserve(cur[c].size());
            size_t k = 0;  // merge-walk of cur[c] against adj0[c] (both sorted)
            for (int q : cur[c]) {
                B(q) = 1;  // the block graph is symmetric
                while (k < a0.size() && a0[k] < q) k++;
                if (k < a0.size() && a0[k] == q) {
                    Q.nl[c].push_back(q);
                    if (!T(q)) {
                        T(q) = 1;
                        tgi[q - lo] = (int)tg.size();
                        if (tg.size() == src.size()) src.emplace_back();
                        src[tg.size()].clear();
                        tg.push_back(q);
                    }
                    src[tgi[q - lo]].push_back(c);
                } else {
                    Q.wl[c].push_back(q);
                }
            }
            if (Q.wl[c].empty()) P.vanished[c] = 1;
            work += (int64_t)Q.nl[c].size() * (int64_t)cur[c].size();
        }
        const int ph = (int)phases.size();
        const int64_t ns = (int64_t)sel.size();
        // every target: the union of what its selected neighbours bring,
        // merged once into each of its lists; then the neighbours that left
        // the graph are dropped from it
        auto update = [&](int64_t a, int64_t b, std::vector<int>& add) {
            for (int64_t i = a; i < b; i++) {
                const int p = tg[i];
                const auto& sp = src[i];
                const std::vector<int>* u = &Q.nl[sp[0]];
                int skip = p;
                if (sp.size() > 1) {
                    add.clear();
                    for (int c : sp) merge_into(add, Q.nl[c], p);
                    u = &add;
                    skip = -1;
                }
                merge_into(cur[p], *u, skip);
                for (int c : sp)
                    if (P.vanished[c]) {
                        sorted_erase(cur[p], c);
                        Q.all[p].push_back(c);  // the block existed during the level
                    }
                target[p - lo] = 0;
            }
        };
        if (work < (1 << 17) || tl_serial || tl_in_pool) {
            update(0, (int64_t)tg.size(), scratch);
        } else {
            parallel_ranges((int64_t)tg.size(), 256, [&](int64_t a, int64_t b, int) {
                std::vector<int> add;
                update(a, b, add);
            });
        }
        for (int c : sel) {
            for (int q : cur[c]) B(q) = 0;
            if (P.vanished[c]) {
                Q.all[c].insert(Q.all[c].end(), cur[c].begin(), cur[c].end());
                cur[c].clear();
            }
            D(c) = 1;
            S(c) = 0;
            P.phase[c] = ph;
        }
        remaining -= (int)ns;
        phases.push_back(std::move(sel));
    }
    // every block that existed during the level: the lists' final state, the
    // blocks to clusters that left (recorded as they left) and the diagonal
    auto finish = [&](int64_t a, int64_t b) {
        for (int64_t c = a; c < b; c++) {
            auto& al = Q.all[c];
            al.reserve(al.size() + cur[c].size() + 1);
            al.insert(al.end(), cur[c].begin(), cur[c].end());
            if (P.size0[c] > 0) al.push_back((int)c);
            std::sort(al.begin(), al.end());
            al.erase(std::unique(al.begin(), al.end()), al.end());
            Q.endp[c] = std::move(cur[c]);
            if (P.size0[c] > 0 && !P.vanished[c]) sorted_insert(Q.endp[c], (int)c);
        }
    };
    if (tl_serial || tl_in_pool) finish(lo, hi);
    else parallel_ranges(hi - lo, 2048, [&](int64_t a, int64_t b, int) { finish(lo + a, lo + b); });
}

// The same phase rule and fill pattern as plan_range for a range of at most
// kBitsMax clusters, with the block graph held as one bit row per cluster:
// selecting a cluster marks its row as blocked, the n / w split is the row
// with / without the level's input pattern, and the fill of a phase is an OR
// of the selected clusters' n rows into their neighbours' rows (unions, so
// the order does not matter), after which the clusters that vanished are
// cleared from them.  Lists come out sorted, as plan_range writes them.
constexpr int kBitsMax = 2048;

void plan_range_bits(LevelPlan& P, int lo, int hi, std::vector<std::vector<int>>& phases, RangeLists& out) {
    const int m = hi - lo, W = (m + 63) / 64;
    // the three bit matrices in one buffer kept by the thread (a fresh
    // allocation of this size costs more in page faults than the planning)
    static thread_local std::vector<uint64_t> bits;
    const size_t mw = (size_t)m * W;
    if (bits.size() < 3 * mw) bits.resize(3 * mw);
    std::memset(bits.data(), 0, sizeof(uint64_t) * 3 * mw);
    uint64_t* const cur = bits.data();
    uint64_t* const in = cur + mw;
    uint64_t* const gone = in + mw;
    std::vector<uint64_t> blocked(W), nlb((size_t)W);
    auto row = [&](uint64_t* b, int c) { return b + (size_t)(c - lo) * W; };
    auto set = [&](uint64_t* r, int q) { r[(q - lo) >> 6] |= 1ull << ((q - lo) & 63); };
    auto has = [&](const uint64_t* r, int q) { return (r[(q - lo) >> 6] >> ((q - lo) & 63)) & 1ull; };
    // appends the set bits of r, ascending; returns their number
    auto to_list = [&](const uint64_t* r, std::vector<int32_t>& o) {
        const size_t b0 = o.size();
        for (int w = 0; w < W; w++)
            for (uint64_t x = r[w]; x; x &= x - 1) o.push_back(lo + 64 * w + __builtin_ctzll(x));
        return (int32_t)(o.size() - b0);
    };
    // n and w lists in elimination order (offsets per cluster), put in
    // cluster order at the end
    std::vector<int32_t> nw;
    std::vector<int64_t> off_n(m, 0), off_w(m, 0);
    std::vector<int32_t> cnt_n(m, 0), cnt_w(m, 0);
    std::vector<char> done(m, 0);
    int remaining = 0;
    for (int c = lo; c < hi; c++) {
        for (int q : P.adj0[c]) {
            set(row(cur, c), q);
            set(row(in, c), q);
        }
        if (P.size0[c] > 0) remaining++;
        else done[c - lo] = 1;
    }
    int first = lo;
    std::vector<int> sel;
    while (remaining > 0) {
        sel.clear();
        std::fill(blocked.begin(), blocked.end(), 0);
        while (first < hi && done[first - lo]) first++;
        for (int c = first; c < hi; c++) {
            if (done[c - lo] || has(blocked.data(), c)) continue;
            sel.push_back(c);
            const uint64_t* r = row(cur, c);
            for (int w = 0; w < W; w++) blocked[w] |= r[w];
        }
        const int ph = (int)phases.size();
        // n / w lists; the fill: every n-neighbour p gains the others
        for (int c : sel) {
            const uint64_t *r = row(cur, c), *a = row(in, c);
            bool fill = false;
            for (int w = 0; w < W; w++) {
                nlb[w] = r[w] & ~a[w];
                fill |= nlb[w] != 0;
            }
            off_w[c - lo] = (int64_t)nw.size();
            cnt_w[c - lo] = to_list(nlb.data(), nw);
            for (int w = 0; w < W; w++) nlb[w] = r[w] & a[w];
            off_n[c - lo] = (int64_t)nw.size();
            cnt_n[c - lo] = to_list(nlb.data(), nw);
            if (!fill) P.vanished[c] = 1;
            for (int32_t e = 0; e < cnt_n[c - lo]; e++) {
                const int p2 = nw[off_n[c - lo] + e];
                uint64_t* rp = row(cur, p2);
                for (int w = 0; w < W; w++) rp[w] |= nlb[w];
                rp[(p2 - lo) >> 6] &= ~(1ull << ((p2 - lo) & 63));
            }
        }
        // clusters without fill leave the graph (their blocks existed during
        // the level); every selected cluster is done
        for (int c : sel) {
            if (P.vanished[c]) {
                const uint64_t bit = 1ull << ((c - lo) & 63);
                for (int32_t e = 0; e < cnt_n[c - lo]; e++) {
                    const int p2 = nw[off_n[c - lo] + e];
                    row(cur, p2)[(c - lo) >> 6] &= ~bit;
                    row(gone, p2)[(c - lo) >> 6] |= bit;
                }
                uint64_t *rc = row(cur, c), *gc = row(gone, c);
                for (int w = 0; w < W; w++) {
                    gc[w] |= rc[w];
                    rc[w] = 0;
                }
            }
            done[c - lo] = 1;
            P.phase[c] = ph;
        }
        remaining -= (int)sel.size();
        phases.push_back(sel);
    }
    for (int k = 0; k < LS_N; k++) out.cnt[k].assign(m, 0);
    {
        // exact sizes of the four lists first, so that none of them grows
        size_t tot_all = 0, tot_end = 0;
        for (int c = lo; c < hi; c++) {
            const uint64_t *rc = row(cur, c), *gc = row(gone, c);
            size_t a = 0, e = 0;
            for (int w = 0; w < W; w++) {
                a += (size_t)__builtin_popcountll(gc[w] | rc[w]);
                e += (size_t)__builtin_popcountll(rc[w]);
            }
            tot_all += a + 1;
            tot_end += e + 1;
        }
        out.data[LS_NL].reserve(out.data[LS_NL].size() + nw.size());
        out.data[LS_WL].reserve(out.data[LS_WL].size() + nw.size());
        out.data[LS_ALL].reserve(out.data[LS_ALL].size() + tot_all);
        out.data[LS_END].reserve(out.data[LS_END].size() + tot_end);
    }
    for (int c = lo; c < hi; c++) {
        const int i = c - lo;
        out.cnt[LS_NL][i] = cnt_n[i];
        out.data[LS_NL].insert(out.data[LS_NL].end(), nw.begin() + off_n[i], nw.begin() + off_n[i] + cnt_n[i]);
        out.cnt[LS_WL][i] = cnt_w[i];
        out.data[LS_WL].insert(out.data[LS_WL].end(), nw.begin() + off_w[i], nw.begin() + off_w[i] + cnt_w[i]);
        uint64_t *rc = row(cur, c), *gc = row(gone, c);
        for (int w = 0; w < W; w++) gc[w] |= rc[w];
        if (P.size0[c] > 0) set(gc, c);
        out.cnt[LS_ALL][i] = to_list(gc, out.data[LS_ALL]);
        if (P.size0[c] > 0 && !P.vanished[c]) set(rc, c);
        out.cnt[LS_END][i] = to_list(rc, out.data[LS_END]);
    }
}

// The list planner's lists of the clusters lo .. hi into out (copied on all
// threads when `parallel`); with `release` the lists are freed by the
// calling thread (otherwise they stay with the plan until it is released).
void take_lists(PlanLists& Q, int lo, int hi, RangeLists& out, bool parallel, bool release_here) {
    std::vector<std::vector<int>>* src[LS_N] = {&Q.nl, &Q.wl, &Q.all, &Q.endp};
    std::vector<int64_t> off(hi - lo + 1);
    for (int k = 0; k < LS_N; k++) {
        auto& v = *src[k];
        out.cnt[k].assign(hi - lo, 0);
        off[0] = 0;
        for (int c = lo; c < hi; c++) {
            out.cnt[k][c - lo] = (int32_t)v[c].size();
            off[c - lo + 1] = off[c - lo] + (int64_t)v[c].size();
        }
        out.data[k].resize((size_t)off[hi - lo]);
        auto copy = [&](int64_t a, int64_t b) {
            for (int64_t c = a; c < b; c++) std::copy(v[c].begin(), v[c].end(), out.data[k].begin() + off[c - lo]);
        };
        if (parallel) parallel_ranges(hi - lo, 4096, [&](int64_t a, int64_t b, int) { copy(lo + a, lo + b); });
        else copy(lo, hi);
    }
    if (release_here)
        for (int c = lo; c < hi; c++)
            for (auto* v : src) std::vector<int>().swap((*v)[c]);
}

// Frees a plan; the list planner's working lists on all threads (they were
// allocated by the planning threads, and freeing hundreds of thousands of
// them from one thread costs milliseconds).
void release_plan(LevelPlan& P) {
    for (auto& v : P.scratch) {
        const int64_t n = (int64_t)v.size();
        parallel_ranges(n, 2048, [&](int64_t lo, int64_t hi, int) {
            for (int64_t c = lo; c < hi; c++) std::vector<int>().swap(v[c]);
        });
    }
    P = LevelPlan{};
}

// ranges: cluster ranges that share no block (independent problems); each
// is planned on its own thread and phase k of the level is the union of the
// ranges' phase k (identical to planning all clusters at once).  Ranges of
// at most kBitsMax clusters run the bit-row planner, larger ones the list
// planner.
void plan_level(LevelPlan& P, const std::vector<std::pair<int, int>>& ranges = {}) {
    const int nc = P.nc;
    Trace tr;
    P.phase.assign(nc, -1);
    P.vanished.assign(nc, 0);
    P.phases.clear();
    std::vector<std::pair<int, int>> rg = ranges;
    if (rg.empty()) rg.push_back({0, nc});
    const int nr = (int)rg.size();
    std::vector<std::vector<std::vector<int>>> ph(nr);
    std::vector<RangeLists> out(nr);
    auto small = [&](int k) { return rg[k].second - rg[k].first <= kBitsMax; };
    bool any_large = false;
    for (int k = 0; k < nr; k++) any_large |= !small(k);
    // the list planner's working lists start as the input pattern, made by
    // the thread that plans them (one range: by all threads), with room for
    // the fill to come so that the phases seldom reallocate
    PlanLists Q;
    std::vector<std::vector<int>> cur;
    if (any_large) {
        cur.resize(nc);
        Q.nl.resize(nc);
        Q.wl.resize(nc);
        Q.all.resize(nc);
        Q.endp.resize(nc);
    }
    auto init = [&](int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; c++) {
            const auto a0 = P.adj0[c];
            cur[c].reserve(4 * a0.size() + 4);
            cur[c].assign(a0.begin(), a0.end());
        }
    };
    if (nr == 1 && !small(0)) parallel_ranges(nc, 1024, [&](int64_t lo, int64_t hi, int) { init(lo, hi); });
    tr.mark("    plan: working lists");
    std::atomic<int> next{0};
    auto work = [&] {
        for (int k = next++; k < nr; k = next++) {
            if (small(k)) {
                plan_range_bits(P, rg[k].first, rg[k].second, ph[k], out[k]);
                continue;
            }
            if (nr > 1) init(rg[k].first, rg[k].second);
            plan_range(P, Q, cur, rg[k].first, rg[k].second, ph[k]);
            if (nr == 1) tr.mark("    plan: list planner");
            take_lists(Q, rg[k].first, rg[k].second, out[k], nr == 1, nr > 1);
        }
    };
    run_threads(std::min<int>(hs_threads(), nr), [&](int) { work(); });
    tr.mark("    plan: phases and lists");
    if (any_large && nr == 1)  // freed with the plan
        for (auto* v : {&Q.nl, &Q.wl, &Q.all, &Q.endp}) P.scratch.push_back(std::move(*v));
    size_t nph = 0;
    for (auto& v : ph) nph = std::max(nph, v.size());
    P.phases.assign(nph, {});
    for (size_t k = 0; k < nph; k++)
        for (auto& v : ph)
            if (k < v.size()) P.phases[k].insert(P.phases[k].end(), v[k].begin(), v[k].end());
    // the ranges' lists, concatenated in range (= cluster) order
    ListSet* dst[LS_N] = {&P.nl, &P.wl, &P.all, &P.endp};
    for (int t = 0; t < LS_N; t++) {
        ListSet& L = *dst[t];
        L.ptr.assign(nc + 1, 0);
        std::vector<int64_t> base(nr + 1, 0);
        for (int k = 0; k < nr; k++) {
            const int lo = rg[k].first;
            for (int i = 0; i < rg[k].second - lo; i++) L.ptr[lo + i + 1] = out[k].cnt[t][i];
            base[k + 1] = base[k] + (int64_t)out[k].data[t].size();
        }
        for (int c = 0; c < nc; c++) L.ptr[c + 1] += L.ptr[c];
        if (nr == 1) {  // one range: its entries are the list set's
            L.idx = std::move(out[0].data[t]);
            continue;
        }
        L.idx.resize((size_t)base[nr]);
        auto copy = [&](int64_t a, int64_t b) {
            for (int64_t k = a; k < b; k++)
                std::copy(out[k].data[t].begin(), out[k].data[t].end(), L.idx.begin() + base[k]);
        };
        if (nr > 64) parallel_ranges(nr, 16, [&](int64_t a, int64_t b, int) { copy(a, b); });
        else copy(0, nr);
    }
    tr.mark("    plan: list sets");
}

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
// kernel classes of the profile: the per-phase factor kernel (level-wise
// launches), Schur updates, assembly, dense tops, preconditioner applies,
// Krylov vector kernels, the fused coarse-level factor kernel and the SpMV
enum {
    KC_FACTOR = 0, KC_SCHUR = 1, KC_ASSEMBLY = 2, KC_TOP = 3, KC_APPLY = 4, KC_KRYLOV = 5, KC_FACTOR_FUSED = 6,
    KC_SPMV = 7, KC_N = 8
};

struct Level {
    int nc = 0;
    std::vector<int> size0, fin, phase;
    std::vector<int64_t> slot;  // vector slot offsets (size nc + 1)
    int nphases = 0;
    std::vector<int> ph_task, ph_target;  // per-phase ranges (size nphases + 1)
    int smax = 0, wmax = 0, lmax = 0, nmax = 0;
    std::vector<TaskDev> tasks;
    std::vector<ListDev> lists;
    // solve phase: (task, k) lists of the updates each cluster receives from
    // tasks of earlier phases (early) / later phases (late)
    // (CSR over clusters: entries ptr[c] .. ptr[c+1], ascending task order)
    std::vector<int32_t> early_ptr, late_ptr;
    std::vector<std::pair<int, int>> early, late;
    std::vector<int64_t> stg;          // stage offset of every task
    std::vector<int32_t> hmeta;        // rank and n-column layout of every task
    DBuf d_feat;                       // rank-predictor features per task (record_ranks)
    std::vector<int> task_rank;        // filled after the level
    std::vector<ApPull> ap_pulls;      // early pulls of the tasks, then the late pulls
    int64_t work_max_phase = 0;        // largest sum over a stage of s^2 + f * ncols
    int nstages = 0;                   // solve stages of the level
    std::vector<int> ap_stage;         // stage ranges in the solve task array
    DBuf d_tasks, d_lists, d_meta, d_fac, d_slot, d_vcopy, d_y, d_stage;
    DBuf d_ap_tasks, d_ap_pulls, d_ap_nbs, d_ap_fins, d_ph;
    int nvcopy = 0, nfin = 0;
    bool fused = false;                // factored by the fused coarse-level kernel
    int64_t fac_doubles = 0;
    // algorithmic work of the level (filled after it ran)
    double flops_factor = 0, flops_compress = 0, flops_schur = 0;
};

struct Prof {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[KC_N];
    size_t used[KC_N] = {0};
    int64_t launches[KC_N] = {0};
    double ms[KC_N] = {0};
    void begin(int k, cudaStream_t st) {
        launches[k]++;
        if (!on) return;
        if (used[k] == ev[k].size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            ev[k].push_back({a, b});
        }
        cudaEventRecord(ev[k][used[k]].first, st);
    }
    void end(int k, cudaStream_t st) {
        if (!on) return;
        cudaEventRecord(ev[k][used[k]].second, st);
        used[k]++;
    }
    void collect() {
        if (!on) return;
        for (int k = 0; k < KC_N; k++) {
            for (size_t i = 0; i < used[k]; i++) {
                float t = 0.f;
                cudaEventSynchronize(ev[k][i].second);
                cudaEventElapsedTime(&t, ev[k][i].first, ev[k][i].second);
                ms[k] += t;
            }
            used[k] = 0;
        }
    }
    void reset() {
        for (int k = 0; k < KC_N; k++) { ms[k] = 0; launches[k] = 0; used[k] = 0; }
    }
    ~Prof() {
        for (int k = 0; k < KC_N; k++)
            for (auto& e : ev[k]) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    }
};

}  // namespace

struct hs_factor_s {
    struct Group {  // one independent problem of the handle
        int64_t leaf_lo, leaf_hi, dof_lo, dof_hi;
        int depth;
    };
    int64_t n = 0, nnz = 0;
    double apply_bytes = 0;  // algorithmic bytes of one preconditioner apply
    std::vector<Group> groups;
    std::vector<int64_t> prob_ptr;  // DOF offsets of the problems (original order)
    DBuf d_model;                   // rank predictor (options.rank_model), device copy
    int64_t prob_maxlen = 0;
    DBuf d_pp;
    std::vector<DBuf> top_bufs;  // dense tops, one buffer per level at which problems end
    std::vector<TopDev> tops;    // per problem
    DBuf d_tops;
    double* top_L = nullptr;     // the single problem's top (chain and dense coarse operator)
    int device = 0;
    cudaStream_t st = nullptr;
    hs_options opt{};
    std::vector<int32_t> perm;
    int depth = 0;
    std::vector<std::unique_ptr<Level>> lev;
    int ntop = 0;
    DBuf d_perm, d_rowptr, d_col, d_val, d_top, d_ytop;
    // Krylov workspace
    DBuf d_kv, d_part, d_scal, d_V, d_Z, d_h;
    int64_t factor_bytes = 0;
    cudaGraphExec_t apply_graph = nullptr;
    int64_t graph_kernels = 0;
    int fp32 = 0;          // factor stored and applied in FP32 (mixed-precision form)
    int first_coarse = 0;  // first level of the single-CTA chain (or of the dense operator)
    bool coarse_dense = false;
    int ncoarse = 0;       // size of the dense coarse operator
    DBuf d_aplevels, d_coarse, d_ycout;
    double* apply_out = nullptr;  // level-0 vector holding the result of the graph
    Prof prof;
    double work_flops[KC_N] = {0};    // FP64 flops
    double work_flops32[KC_N] = {0};  // FP32 flops (the mixed form's compression and Schur products)
    double work_bytes[KC_N] = {0};
    ~hs_factor_s() {
        if (apply_graph) cudaGraphExecDestroy(apply_graph);
    }
};

namespace {

// Raises the error a status word (status, level, cluster) read back from the
// kernels stands for.
void raise_status(hs_factor_s* h, const int32_t* st, hs_info* info) {
    if (st[0] == ST_NOT_SPD) {
        if (info) {
            // a dense top fails as (depth of its problem, problem index)
            const bool top = st[1] < 0;
            const int g = top && st[2] >= 0 && st[2] < (int)h->tops.size() ? h->tops[st[2]].pad : 0;
            info->fail_level = top ? h->groups[g].depth : st[1];
            info->fail_cluster = top ? g : st[2];
        }
        throw HsError{HS_ERR_NOT_SPD};
    }
    if (st[0] == ST_TIMEOUT) throw HsError{HS_ERR_TIMEOUT};
    if (st[0] != ST_OK) throw HsError{HS_ERR_UNSUPPORTED};
}

void check_status(hs_factor_s* h, DBuf& d_status, hs_info* info) {
    std::vector<int32_t> st;
    download(st, d_status.p, 3, h->st);
    raise_status(h, st.data(), info);
}

// Block table of a level: CSR over clusters of the blocks in `all`.
struct BlockTable {
    std::vector<int32_t> ptr, col, ld;
    std::vector<int32_t> tpos;  // tpos[b]: index of the transposed block (q, p) of block b = (p, q)
    std::vector<int64_t> off;
    int64_t total = 0;
    int find(int p, int q) const {
        auto b = col.begin() + ptr[p], e = col.begin() + ptr[p + 1];
        auto it = std::lower_bound(b, e, q);
        if (it == e || *it != q) throw HsError{HS_ERR_ARG};  // planner invariant broken
        return (int)(it - col.begin());
    }
    // find(p, q) for lookups of ascending q in one row: `cur` (the previous
    // result, or any value) is a hint; a short forward scan from it, else a
    // binary search.  Same result as find.
    int find_from(int p, int q, int& cur) const {
        const int b = ptr[p], e = ptr[p + 1];
        int k = (cur >= b && cur < e && col[cur] <= q) ? cur : b;
        for (int step = 0; step < 8 && k < e && col[k] < q; step++) k++;
        if (k < e && col[k] < q) k = (int)(std::lower_bound(col.begin() + k, col.begin() + e, q) - col.begin());
        if (k >= e || col[k] != q) throw HsError{HS_ERR_ARG};  // planner invariant broken
        cur = k;
        return k;
    }
};

BlockTable make_table(const LevelPlan& P) {
    // row starts and byte offsets by prefix sums, then the rows in parallel
    BlockTable T;
    const int nc = P.nc;
    T.ptr.assign(nc + 1, 0);
    std::vector<int64_t> rowsz(nc + 1, 0);
    for (int c = 0; c < nc; c++) {
        T.ptr[c + 1] = T.ptr[c] + (int)P.all[c].size();
        int64_t w = 0;
        for (int q : P.all[c]) w += P.size0[q];
        rowsz[c + 1] = rowsz[c] + (int64_t)P.size0[c] * w;
    }
    const int nb = T.ptr[nc];
    T.col.resize(nb);
    T.off.resize(nb);
    T.ld.resize(nb);
    parallel_ranges(nc, 256, [&](int64_t lo, int64_t hi, int) {
        for (int64_t c = lo; c < hi; c++) {
            int64_t o = rowsz[c];
            int b = T.ptr[c];
            for (int q : P.all[c]) {
                T.col[b] = q;
                T.off[b] = o;
                T.ld[b] = P.size0[q];
                o += (int64_t)P.size0[c] * P.size0[q];
                b++;
            }
        }
    });
    T.total = rowsz[nc];
    // transposed positions (the block pattern is symmetric): small tables by
    // one sweep of row cursors (row q lists its p in ascending order), large
    // ones by parallel lookups; checked either way
    T.tpos.resize(nb);
    if (nb < (1 << 17)) {
        std::vector<int32_t> cursor(T.ptr.begin(), T.ptr.end() - 1);
        for (int p = 0; p < nc; p++)
            for (int b = T.ptr[p]; b < T.ptr[p + 1]; b++) {
                const int q = T.col[b];
                const int t = cursor[q]++;
                if (t >= T.ptr[q + 1] || T.col[t] != p) throw HsError{HS_ERR_ARG};  // planner invariant broken
                T.tpos[b] = t;
            }
    } else {
        std::atomic<int> bad{0};
        parallel_ranges(nc, 256, [&](int64_t lo, int64_t hi, int) {
            for (int64_t p = lo; p < hi; p++)
                for (int b = T.ptr[p]; b < T.ptr[p + 1]; b++) {
                    const int q = T.col[b];
                    auto e = T.col.begin() + T.ptr[q + 1];
                    auto it = std::lower_bound(T.col.begin() + T.ptr[q], e, (int32_t)p);
                    if (it == e || *it != p) bad = 1;
                    else T.tpos[b] = (int32_t)(it - T.col.begin());
                }
        });
        if (bad) throw HsError{HS_ERR_ARG};
    }
    return T;
}

// Factor one level: plan, device records, phases.  `blocks` holds the level's
// assembled matrix (layout T).  Returns the final sizes.
void factor_level(hs_factor_s* h, int l, LevelPlan& P, const BlockTable& T, DBuf& blocks, DBuf& d_cur,
                  DBuf& d_status, hs_info* info, const std::vector<std::pair<int, int>>& ranges,
                  const std::function<void()>& overlap) {
    Level& L = *h->lev[l];
    cudaStream_t st = h->st;
    Trace tr0;
    L.nc = P.nc;
    L.size0 = P.size0;
    L.phase = P.phase;
    L.nphases = (int)P.phases.size();
    L.slot.assign(P.nc + 1, 0);
    for (int c = 0; c < P.nc; c++) L.slot[c + 1] = L.slot[c] + P.size0[c];

    // tasks in phase order
    std::vector<int> task_of(P.nc, -1);
    int64_t fac = 0, ws_phase_max = 0, stage = 0;
    int32_t meta = 0;
    L.ph_task.assign(1, 0);
    L.ph_target.assign(1, 0);
    DBuf d_targets, d_contribs;
    L.smax = 1; L.wmax = 1; L.lmax = 1; L.nmax = 1;
    // task ti = the ti-th cluster in phase order; sizes first (parallel),
    // then prefix offsets, then the records (parallel)
    std::vector<int> order;
    for (int ph = 0; ph < L.nphases; ph++) {
        order.insert(order.end(), P.phases[ph].begin(), P.phases[ph].end());
        L.ph_task.push_back((int)order.size());
    }
    const int nt = (int)order.size();
    std::vector<int32_t> t_ncap(nt), t_wcap(nt);
    parallel_ranges(nt, 256, [&](int64_t lo, int64_t hi, int) {
        for (int64_t ti = lo; ti < hi; ti++) {
            const int c = (int)order[ti];
            int ncap = 0, wcap = 0;
            for (int q : P.nl[c]) ncap += P.size0[q];
            wcap = ncap;
            for (int q : P.wl[c]) wcap += P.size0[q];
            t_ncap[ti] = ncap;
            t_wcap[ti] = wcap;
        }
    });
    L.tasks.resize(nt);
    L.stg.resize(nt);
    std::vector<int32_t> list_off(nt + 1, 0);
    for (int ph = 0; ph < L.nphases; ph++) {
        int64_t ws = 0;
        for (int ti = L.ph_task[ph]; ti < L.ph_task[ph + 1]; ti++) {
            const int c = order[ti];
            TaskDev& t = L.tasks[ti];
            t.c = c;
            t.s = P.size0[c];
            t.nn = (int)P.nl[c].size();
            t.nw = (int)P.wl[c].size();
            t.list = list_off[ti];
            list_off[ti + 1] = list_off[ti] + t.nn + t.nw;
            t.ncap = (t_ncap[ti] + 3) & ~3;  // ld of C: rows of whole float4 / double2 groups
            t.wcap = t_wcap[ti];
            t.meta = meta;
            meta += 1 + 2 * t.nn;
            L.stg[ti] = stage;
            stage += std::max(t.ncap, 1);
            // W and C start on 4-element boundaries (vector loads in the solve phase)
            fac = (fac + 3) & ~(int64_t)3;
            t.w_off = fac; fac += (int64_t)t.s * t.s;
            fac = (fac + 3) & ~(int64_t)3;
            t.c_off = fac; fac += (int64_t)t.s * std::max(t.ncap, 1);
            t.m_off = ws; ws += (int64_t)t.s * (t.wcap + t.s);
            L.smax = std::max(L.smax, t.s);
            L.wmax = std::max(L.wmax, t.wcap);
            L.lmax = std::max(L.lmax, t.nn + t.nw);
            L.nmax = std::max(L.nmax, t.ncap);
            task_of[c] = ti;
        }
        ws_phase_max = std::max(ws_phase_max, ws);
    }
    tr0.mark("  tasks: sizes and offsets");
    L.lists.resize(list_off[nt]);
    parallel_ranges(nt, 128, [&](int64_t lo, int64_t hi, int) {
        for (int64_t ti = lo; ti < hi; ti++) {
            TaskDev& t = L.tasks[ti];
            const int c = t.c;
            t.diag_blk = T.find(c, c);
            int cur = -1;
            for (int k = 0; k < t.nn + t.nw; k++) {
                const int q = k < t.nn ? P.nl[c][k] : P.wl[c][k - t.nn];
                ListDev& le = L.lists[t.list + k];
                le = ListDev{};
                le.q = q;
                le.blk_cq = T.find_from(c, q, cur);
                le.blk_qc = T.tpos[le.blk_cq];
            }
        }
    });
    tr0.mark("  tasks: lists");
    // Schur targets of every phase (built before the launch of a fused
    // level; with per-phase launches, while the first phase runs)
    auto build_targets = [&] {
        // Schur targets of every phase: (p, q), p <= q, contributions in
        // ascending task order (sort by target, stable in task order).  The
        // independent cluster ranges are handled on their own threads and
        // concatenated (targets of a range lie in that range).
        {
            struct TC {
                int p, q;
                ContribDev c;
            };
            const int nr = std::max<int>(1, (int)ranges.size());
            std::vector<std::vector<std::vector<TargetDev>>> rt(nr, std::vector<std::vector<TargetDev>>(L.nphases));
            std::vector<std::vector<std::vector<ContribDev>>> rc(nr, std::vector<std::vector<ContribDev>>(L.nphases));
            std::atomic<int> next{0};
            // work items: (range, phase) pairs, independent of each other
            const int nitems = nr * L.nphases;
            auto work = [&] {
                std::vector<TC> tcs, tmp;
                std::vector<int> cntv;
                for (int item = next++; item < nitems; item = next++) {
                    const int k = item / L.nphases;
                    const int lo = ranges.empty() ? 0 : ranges[k].first, hi = ranges.empty() ? P.nc : ranges[k].second;
                    {
                        const int ph = item % L.nphases;
                        const auto& cs = P.phases[ph];
                        auto b0 = std::lower_bound(cs.begin(), cs.end(), lo), b1 = std::lower_bound(cs.begin(), cs.end(), hi);
                        tcs.clear();
                        for (auto it = b0; it != b1; ++it) {
                            const int c = *it, ti = task_of[c];
                            const auto& nlc = P.nl[c];
                            for (int a = 0; a < (int)nlc.size(); a++)
                                for (int b = 0; b < (int)nlc.size(); b++)
                                    if (nlc[a] <= nlc[b]) tcs.push_back(TC{nlc[a], nlc[b], ContribDev{ti, a, b}});
                        }
                        // stable order by (p, q): counting sort on q, then on p
                        // (keys are cluster ids in [lo, hi))
                        if (!tcs.empty()) {
                            const int span = hi - lo;
                            cntv.assign(span + 1, 0);
                            tmp.resize(tcs.size());
                            for (const TC& x : tcs) cntv[x.q - lo + 1]++;
                            for (int u = 0; u < span; u++) cntv[u + 1] += cntv[u];
                            for (const TC& x : tcs) tmp[cntv[x.q - lo]++] = x;
                            cntv.assign(span + 1, 0);
                            for (const TC& x : tmp) cntv[x.p - lo + 1]++;
                            for (int u = 0; u < span; u++) cntv[u + 1] += cntv[u];
                            for (const TC& x : tmp) tcs[cntv[x.p - lo]++] = x;
                        }
                        auto& tg = rt[k][ph];
                        auto& ct = rc[k][ph];
                        int cur = -1;  // targets come in (p, q) order
                        for (size_t i = 0; i < tcs.size();) {
                            size_t j = i;
                            TargetDev g{};
                            g.p = tcs[i].p;
                            g.q = tcs[i].q;
                            g.blk_pq = T.find_from(g.p, g.q, cur);
                            g.blk_qp = T.tpos[g.blk_pq];
                            g.c_begin = (int)ct.size();
                            while (j < tcs.size() && tcs[j].p == g.p && tcs[j].q == g.q) ct.push_back(tcs[j++].c);
                            g.c_end = (int)ct.size();
                            tg.push_back(g);
                            i = j;
                        }
                    }
                }
            };
            // threads only when there are enough pairs to pay for waking them
            int64_t npairs = 0;
            for (int ti = 0; ti < nt; ti++) npairs += (int64_t)L.tasks[ti].nn * L.tasks[ti].nn;
            run_threads(npairs < (1 << 11) ? 1 : std::min<int>(hs_threads(), std::max(nitems, 1)), [&](int) { work(); });
            tr0.mark("  targets: pairs");
            // concatenation in (phase, range) order: offsets first, then the
            // copies item by item in parallel
            std::vector<int64_t> toff(nitems + 1, 0), coff(nitems + 1, 0);
            for (int ph = 0, it = 0; ph < L.nphases; ph++) {
                for (int k = 0; k < nr; k++, it++) {
                    toff[it + 1] = toff[it] + (int64_t)rt[k][ph].size();
                    coff[it + 1] = coff[it] + (int64_t)rc[k][ph].size();
                }
                L.ph_target.push_back((int)toff[it]);
            }
            // written straight into pinned staging (one area for both) and
            // copied to the device from there
            const size_t tb = sizeof(TargetDev) * (size_t)toff[nitems], cb = sizeof(ContribDev) * (size_t)coff[nitems];
            const size_t tb_al = (tb + 255) & ~(size_t)255;
            char* pin = g_stage.take(tb_al + cb, st);
            TargetDev* targets = reinterpret_cast<TargetDev*>(pin);
            ContribDev* contribs = reinterpret_cast<ContribDev*>(pin + tb_al);
            parallel_ranges(nitems, 2, [&](int64_t lo, int64_t hi, int) {
                for (int64_t it = lo; it < hi; it++) {
                    const int ph = (int)(it / nr), k = (int)(it % nr);
                    const int base = (int)coff[it];
                    int64_t o = toff[it];
                    for (TargetDev g : rt[k][ph]) {
                        g.c_begin += base;
                        g.c_end += base;
                        targets[o++] = g;
                    }
                    std::copy(rc[k][ph].begin(), rc[k][ph].end(), contribs + coff[it]);
                    // freed here, in parallel (a worker allocated them)
                    std::vector<TargetDev>().swap(rt[k][ph]);
                    std::vector<ContribDev>().swap(rc[k][ph]);
                }
            });
            d_targets.alloc(std::max<size_t>(tb, 16));
            d_contribs.alloc(std::max<size_t>(cb, 16));
            if (tb) CK(cudaMemcpyAsync(d_targets.p, targets, tb, cudaMemcpyHostToDevice, st));
            if (cb) CK(cudaMemcpyAsync(d_contribs.p, contribs, cb, cudaMemcpyHostToDevice, st));
        }
        tr0.mark("  targets");
    };
    L.wmax = std::max(L.wmax, 64);  // the fused kernel's Schur step stages 32 x 4 int64 in the column table
    const bool nodc = h->opt.no_dc != 0;
    if ((nodc ? factor_nodc_smem_bytes(L.smax, L.wmax, L.lmax) : factor_smem_bytes(L.smax, L.wmax, L.lmax)) >
        (size_t)kFactorMaxSmem)
        throw HsError{HS_ERR_UNSUPPORTED};
    Trace tr;
    tr.mark("  records");

    upload(L.d_tasks, L.tasks, st);
    upload(L.d_lists, L.lists, st);
    DBuf d_ws;
    tr.mark("  uploads: records");
    L.d_meta.alloc(sizeof(int32_t) * std::max<int32_t>(meta, 1));
    L.d_fac.alloc((h->fp32 ? sizeof(float) : sizeof(double)) * std::max<int64_t>(fac, 1));
    L.fac_doubles = fac;
    L.d_stage.alloc(sizeof(double) * std::max<int64_t>(stage, 1));
    d_ws.alloc(sizeof(double) * std::max<int64_t>(ws_phase_max, 1));
    upload(L.d_slot, L.slot, st);

    std::vector<int32_t> ld(T.ld.begin(), T.ld.end());
    DBuf d_off, d_ld;
    upload(d_off, T.off, st);
    upload(d_ld, ld, st);
    const double eps2 = h->opt.tol * h->opt.tol;
    float* feat = nullptr;
    if (h->opt.record_ranks) {
        L.d_feat.alloc(sizeof(float) * kFeat * std::max(nt, 1));
        feat = L.d_feat.as<float>();
    }
    tr.mark("  uploads");
    int64_t mcap = 0;  // largest block row (with the identity columns)
    for (const TaskDev& t : L.tasks) mcap = std::max<int64_t>(mcap, (int64_t)t.s * (t.wcap + t.s));
    const bool fused = !nodc && h->opt.fused_levels && L.smax <= kFusedSmax &&
                       fused_smem_bytes(L.smax, L.wmax, L.lmax, mcap) <= (size_t)kFactorMaxSmem;
    if (fused) build_targets();
    if (fused && nt > 0) {
        DBuf d_pht, d_phg, d_bar;
        upload(d_pht, L.ph_task, st);
        upload(d_phg, L.ph_target, st);
        d_bar.alloc(2 * sizeof(unsigned));
        int max_items = 1, max_tasks = 0;
        int64_t target_rounds = 0;
        for (int ph = 0; ph < L.nphases; ph++) {
            const int ntk = L.ph_task[ph + 1] - L.ph_task[ph], ntg = L.ph_target[ph + 1] - L.ph_target[ph];
            max_items = std::max({max_items, ntk, ntg});
            max_tasks = std::max(max_tasks, ntk);
            target_rounds += (ntg + kClusterWarps - 1) / kClusterWarps;
        }
        // one cluster when the tasks of every phase fit its warps at once and
        // the Schur targets take few rounds
        const int cluster_ok = max_tasks <= kClusterWarps && target_rounds <= (int64_t)kClusterTargetRounds * L.nphases;
        h->prof.begin(KC_FACTOR_FUSED, st);
        CK(launch_factor_level_fused(st, L.d_tasks.as<TaskDev>(), d_pht.as<int32_t>(), d_targets.as<TargetDev>(),
                                     d_phg.as<int32_t>(), d_contribs.as<ContribDev>(), L.nphases,
                                     L.d_lists.as<ListDev>(), blocks.as<double>(), d_off.as<int64_t>(),
                                     d_ld.as<int32_t>(), d_cur.as<int32_t>(), L.d_fac.p, h->fp32,
                                     L.d_meta.as<int32_t>(), d_ws.as<double>(), eps2, d_status.as<int32_t>(), l,
                                     L.smax, L.wmax, L.lmax, mcap, max_items, d_bar.as<unsigned>(), feat,
                                     h->d_model.as<float>(), h->opt.wait_polls, cluster_ok));
        h->prof.end(KC_FACTOR_FUSED, st);
    }
    for (int ph = 0; ph < (fused ? 0 : L.nphases); ph++) {
        const int t0 = L.ph_task[ph], nt = L.ph_task[ph + 1] - t0;
        h->prof.begin(KC_FACTOR, st);
        if (nodc)
            CK(launch_factor_nodc(st, L.d_tasks.as<TaskDev>(), t0, nt, L.smax, L.wmax, L.lmax,
                                  L.d_lists.as<ListDev>(), blocks.as<double>(), d_off.as<int64_t>(),
                                  d_ld.as<int32_t>(), d_cur.as<int32_t>(), L.d_fac.p, h->fp32,
                                  L.d_meta.as<int32_t>(), d_ws.as<double>(), eps2, d_status.as<int32_t>(), l));
        else
            CK(launch_factor_phase(st, L.d_tasks.as<TaskDev>(), t0, nt, L.smax, L.wmax, L.lmax,
                                   L.d_lists.as<ListDev>(), blocks.as<double>(), d_off.as<int64_t>(),
                                   d_ld.as<int32_t>(), d_cur.as<int32_t>(), L.d_fac.p, h->fp32,
                                   L.d_meta.as<int32_t>(), d_ws.as<double>(), eps2, d_status.as<int32_t>(), l, feat,
                                   h->d_model.as<float>()));
        h->prof.end(KC_FACTOR, st);
        if (ph == 0) build_targets();
        const int g0 = L.ph_target[ph], ng = L.ph_target[ph + 1] - g0;
        if (ng > 0) {
            h->prof.begin(KC_SCHUR, st);
            CK(launch_schur_phase(st, d_targets.as<TargetDev>(), g0, ng, d_contribs.as<ContribDev>(),
                                  L.d_tasks.as<TaskDev>(), L.d_fac.p, L.d_meta.as<int32_t>(),
                                  blocks.as<double>(), d_off.as<int64_t>(), d_ld.as<int32_t>(),
                                  d_cur.as<int32_t>(), h->fp32, h->opt.schur_products));
            h->prof.end(KC_SCHUR, st);
        }
    }
    if (!fused && L.nphases == 0) build_targets();
    tr.mark("  launches");
    // solve-phase updates: neighbour q of task t receives C_t(:, q)^T y_t(fine)
    // before its own transform (q in a later phase) or at level end (earlier)
    {
        L.early_ptr.assign(P.nc + 1, 0);
        L.late_ptr.assign(P.nc + 1, 0);
        for (int ti = 0; ti < nt; ti++) {
            const TaskDev& t = L.tasks[ti];
            for (int k = 0; k < t.nn; k++) {
                const int q = L.lists[t.list + k].q;
                (P.phase[q] > P.phase[t.c] ? L.early_ptr : L.late_ptr)[q + 1]++;
            }
        }
        for (int q = 0; q < P.nc; q++) {
            L.early_ptr[q + 1] += L.early_ptr[q];
            L.late_ptr[q + 1] += L.late_ptr[q];
        }
        L.early.resize(L.early_ptr[P.nc]);
        L.late.resize(L.late_ptr[P.nc]);
        std::vector<int32_t> fe(L.early_ptr.begin(), L.early_ptr.end() - 1), fl(L.late_ptr.begin(), L.late_ptr.end() - 1);
        for (int ti = 0; ti < nt; ti++) {
            const TaskDev& t = L.tasks[ti];
            for (int k = 0; k < t.nn; k++) {
                const int q = L.lists[t.list + k].q;
                if (P.phase[q] > P.phase[t.c]) L.early[fe[q]++] = {ti, k};
                else L.late[fl[q]++] = {ti, k};
            }
        }
    }
    overlap();  // host work of earlier levels while these kernels run
    L.fused = fused;
    // the level's results in one read-back: status word, final cluster sizes
    // and the tasks' rank / column layout
    std::vector<int32_t> hmeta(meta);
    if (nt == 0) {
        // nothing to eliminate (every cluster empty): no kernel ran, sizes stay
        L.fin.assign(P.size0.begin(), P.size0.end());
    } else {
        const size_t b_st = sizeof(int32_t) * 3, b_fin = sizeof(int32_t) * P.nc, b_meta = sizeof(int32_t) * meta;
        const size_t o_fin = 256, o_meta = o_fin + ((b_fin + 255) & ~(size_t)255);
        char* pin = g_stage.take(o_meta + b_meta, st);
        CK(cudaMemcpyAsync(pin, d_status.p, b_st, cudaMemcpyDeviceToHost, st));
        if (b_fin) CK(cudaMemcpyAsync(pin + o_fin, d_cur.p, b_fin, cudaMemcpyDeviceToHost, st));
        if (b_meta) CK(cudaMemcpyAsync(pin + o_meta, L.d_meta.p, b_meta, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        tr.mark("  kernels (sync)");
        raise_status(h, reinterpret_cast<const int32_t*>(pin), info);
        const int32_t* fin = reinterpret_cast<const int32_t*>(pin + o_fin);
        L.fin.assign(fin, fin + P.nc);
        if (b_meta) std::memcpy(hmeta.data(), pin + o_meta, b_meta);
        g_stage.synced(st);
    }
    tr.mark("  downloads");
    L.hmeta = std::move(hmeta);
}

// The level's solve-phase records (tasks, pulls, neighbour records, stages)
// and its algorithmic work, from its readback; run by the setup while the
// next level's kernels execute.
void level_records(hs_factor_s* h, int l) {
    Level& L = *h->lev[l];
    cudaStream_t st = h->st;
    Trace tr;
    const int nt = (int)L.tasks.size();
    const bool fused = L.fused, nodc = h->opt.no_dc != 0;
    const std::vector<int32_t>& hmeta = L.hmeta;
    // solve-phase records with resolved offsets
    {
        std::vector<ApTask> at(nt);
        // pulls (early updates) and neighbour records: offsets first, then
        // every task's records in parallel
        const int pull_base = (int)L.ap_pulls.size();
        std::vector<int32_t> nb_off(nt + 1, 0);
        for (int ti = 0; ti < nt; ti++) nb_off[ti + 1] = nb_off[ti] + L.tasks[ti].nn;
        std::vector<ApNb> nbs(nb_off[nt]);
        L.ap_pulls.resize(pull_base + L.early.size());
        std::vector<int32_t> pull_off(nt + 1, pull_base);
        for (int ti = 0; ti < nt; ti++) {
            const int c = L.tasks[ti].c;
            pull_off[ti + 1] = pull_off[ti] + (L.early_ptr[c + 1] - L.early_ptr[c]);
        }
        parallel_ranges(nt, 256, [&](int64_t lo, int64_t hi, int) {
            for (int64_t ti = lo; ti < hi; ti++) {
                const TaskDev& t = L.tasks[ti];
                const int32_t* mt = hmeta.data() + t.meta;
                ApTask a{};
                a.y = L.slot[t.c];
                a.w = t.w_off;
                a.cm = t.c_off;
                a.stg = L.stg[ti];
                a.s = t.s;
                a.r = mt[0];
                a.ncols = t.nn > 0 ? mt[1 + 2 * (t.nn - 1)] + mt[2 + 2 * (t.nn - 1)] : 0;
                a.ncap = t.ncap;
                a.pull0 = pull_off[ti];
                int o = pull_off[ti];
                for (int e = L.early_ptr[t.c]; e < L.early_ptr[t.c + 1]; e++) {
                    const auto& pk = L.early[e];
                    L.ap_pulls[o++] = ApPull{L.stg[pk.first] + hmeta[L.tasks[pk.first].meta + 1 + 2 * pk.second]};
                }
                a.pull1 = o;
                a.nb0 = nb_off[ti];
                for (int e = 0; e < t.nn; e++) {
                    ApNb nb{};
                    nb.y = L.slot[L.lists[t.list + e].q];
                    nb.col = mt[1 + 2 * e];
                    nb.m = mt[2 + 2 * e];
                    nbs[nb_off[ti] + e] = nb;
                }
                a.nb1 = nb_off[ti + 1];
                at[ti] = a;
            }
        });
        // Solve stages: a task depends only on the tasks whose staged update
        // it subtracts (fill couplings were compressed away), so stage =
        // longest chain of such dependencies; the backward runs the stages in
        // reverse.  Tasks of a stage are independent.
        std::vector<int> stage_of(nt, 0);
        for (int ti = 0; ti < nt; ti++) {
            const int c = L.tasks[ti].c;
            for (int e = L.early_ptr[c]; e < L.early_ptr[c + 1]; e++)
                stage_of[ti] = std::max(stage_of[ti], stage_of[L.early[e].first] + 1);
        }
        int nst = 0;
        for (int v : stage_of) nst = std::max(nst, v + 1);
        std::vector<int> order(L.tasks.size());
        for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return stage_of[a] < stage_of[b]; });
        std::vector<ApTask> ats(at.size());
        L.ap_stage.assign(1, 0);
        std::vector<int64_t> swork(nst, 0);
        for (size_t i = 0; i < order.size(); i++) {
            ats[i] = at[order[i]];
            const ApTask& a = ats[i];
            swork[stage_of[order[i]]] += (int64_t)a.s * a.s + (int64_t)(a.s - a.r) * a.ncols;
            if (i + 1 == order.size() || stage_of[order[i + 1]] != stage_of[order[i]])
                L.ap_stage.push_back((int)i + 1);
        }
        L.nstages = nst;
        L.work_max_phase = 0;
        for (auto w : swork) L.work_max_phase = std::max(L.work_max_phase, w);
        upload(L.d_ap_tasks, ats, st);
        upload(L.d_ap_nbs, nbs, st);
        upload(L.d_ph, L.ap_stage, st);
        L.early.clear();
        L.early_ptr.clear();
    }
    tr.mark("  solve records");
    // algorithmic work: POTRF s^3/3, TRSM s^2 (n + w), CPQR sum_k 4 (s-k)(w-k) + 4 s r n, Schur n^2 f
    L.task_rank.resize(L.tasks.size());
    for (size_t ti = 0; ti < L.tasks.size(); ti++) {
        const TaskDev& t = L.tasks[ti];
        const int r = L.hmeta[t.meta];
        L.task_rank[ti] = r;
        double ncol = 0, wcol = 0;
        for (int k = 0; k < t.nn + t.nw; k++) {
            const int q = L.lists[t.list + k].q;
            const int w = (L.phase[q] >= 0 && L.phase[q] < L.phase[t.c]) ? L.fin[q] : L.size0[q];
            (k < t.nn ? ncol : wcol) += w;
        }
        const double s = t.s;
        // Cholesky + scaling (FP64 in both forms); compression and
        // sparsification (FP32 in the mixed form)
        L.flops_factor += s * s * s / 3.0 + s * s * (ncol + wcol);
        double fq = 4.0 * s * r * ncol;
        for (int k = 0; k < r; k++) fq += 4.0 * (s - k) * (wcol - k);
        L.flops_compress += fq;
        L.flops_schur += ncol * ncol * (s - r);  // symmetric half, FMA = 2
    }
    const int kc = fused ? KC_FACTOR_FUSED : KC_FACTOR;
    h->work_flops[kc] += L.flops_factor;
    (h->fp32 && !nodc ? h->work_flops32 : h->work_flops)[kc] += L.flops_compress;
    (h->fp32 ? h->work_flops32 : h->work_flops)[KC_SCHUR] += L.flops_schur;
}

// Coarse-vector copies from level l to the next level / the top: the
// backward scatter (vcopy) and the forward end-of-level records (late
// updates + gather); uploads the level's update list.
void make_vcopies(hs_factor_s* h, Level& L, const std::vector<int64_t>& dst_of, const std::vector<char>& to_top) {
    std::vector<VCopyDev> v;
    std::vector<ApFin> fins;
    for (int c = 0; c < L.nc; c++) {
        if (L.fin[c] <= 0) continue;
        VCopyDev x{};
        x.src = L.slot[c];
        x.dst = dst_of[c];
        x.len = L.fin[c];
        x.to_top = to_top[c];
        v.push_back(x);
        ApFin f{};
        f.y = L.slot[c];
        f.dst = x.dst;
        f.len = L.fin[c];
        f.to_top = to_top[c];
        f.pull0 = (int)L.ap_pulls.size();
        for (int e = L.late_ptr[c]; e < L.late_ptr[c + 1]; e++) {
            const auto& pk = L.late[e];
            L.ap_pulls.push_back(ApPull{L.stg[pk.first] + L.hmeta[L.tasks[pk.first].meta + 1 + 2 * pk.second]});
        }
        f.pull1 = (int)L.ap_pulls.size();
        fins.push_back(f);
    }
    L.nvcopy = (int)v.size();
    L.nfin = (int)fins.size();
    upload(L.d_vcopy, v, h->st);
    upload(L.d_ap_fins, fins, h->st);
    upload(L.d_ap_pulls, L.ap_pulls, h->st);
    L.late.clear();
    L.late.shrink_to_fit();
    L.late_ptr.clear();
}

// Block copies from level-l blocks (table T, final sizes fin, end pattern
// endp) into the parents: cluster a goes to parent par[a] at row offset
// poff[a] (next level, table Tn, sizes nsize), or, when par[a] < 0, into its
// problem's dense top at row tpos[a] of the matrix at tmat[a] (order tn[a]).
std::vector<CopyDev> make_assembly(const LevelPlan& P, const std::vector<int>& fin, const BlockTable& T,
                                   const BlockTable* Tn, const std::vector<int>& nsize, const std::vector<int>& par,
                                   const std::vector<int>& poff, const std::vector<int64_t>& tmat,
                                   const std::vector<int64_t>& tpos, const std::vector<int>& tn, bool to_tops) {
    return parallel_collect<CopyDev>(P.nc, 128, [&](int64_t a, std::vector<CopyDev>& cps) {
        if (fin[a] <= 0) return;
        if ((par[a] < 0) != to_tops) return;
        int cur = -1, curn = -1;
        for (int b : P.endp[a]) {
            if (fin[b] <= 0) continue;
            CopyDev c{};
            const int sb = T.find_from((int)a, b, cur);
            c.src = T.off[sb];
            c.src_ld = T.ld[sb];
            if (!to_tops) {
                const int db = Tn->find_from(par[a], par[b], curn);
                c.dst = Tn->off[db] + (int64_t)poff[a] * nsize[par[b]] + poff[b];
                c.dst_ld = nsize[par[b]];
            } else {
                c.dst = tmat[a] + tpos[a] * (int64_t)tn[a] + tpos[b];
                c.dst_ld = tn[a];
            }
            c.rows = fin[a];
            c.cols = fin[b];
            cps.push_back(c);
        }
    });
}

void build_apply_graph(hs_factor_s* h);
double apply_work_bytes(const hs_factor_s* h);

// Partitions every problem of a block-diagonal batch on its own (Sec. 4.2)
// and concatenates the trees: problem p's leaves follow problem p-1's.
void partition_batched(hs_factor_s* h, const int64_t* rp, const int32_t* cl, const double* vl,
                       std::vector<int32_t>& leaf_ptr) {
    const int np = (int)h->prob_ptr.size() - 1;
    const int64_t* pp = h->prob_ptr.data();
    std::vector<std::vector<int32_t>> perm(np), lp(np);
    std::atomic<int> next{0}, bad{0};
    auto work = [&] {
        struct Serial {  // nested parallel loops of this thread stay serial
            Serial() { tl_serial = true; }
            ~Serial() { tl_serial = false; }
        } serial;
        std::vector<int64_t> srp;
        std::vector<int32_t> scol;
        for (int p = next++; p < np; p = next++) {
            const int64_t lo = pp[p], hi = pp[p + 1], m = hi - lo;
            srp.assign(m + 1, 0);
            scol.clear();
            for (int64_t i = lo; i < hi; i++) {
                for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
                    if (cl[e] < lo || cl[e] >= hi) { bad = 1; break; }
                    scol.push_back((int32_t)(cl[e] - lo));
                }
                srp[i - lo + 1] = (int64_t)scol.size();
            }
            if (bad) return;
            partition_impl(m, srp.data(), scol.data(), vl + rp[lo], h->opt.coords ? h->opt.coords + 2 * lo : nullptr,
                           h->opt.leaf_lines, h->opt.theta, perm[p], lp[p], h->opt.partitioner);
        }
    };
    run_threads(std::min(hs_threads(), np), [&](int) { work(); });
    if (bad) throw HsError{HS_ERR_ARG};  // an entry couples two problems
    h->perm.resize(h->n);
    leaf_ptr.assign(1, 0);
    h->groups.clear();
    for (int p = 0; p < np; p++) {
        const int nleaf = (int)lp[p].size() - 1;
        int depth = h->opt.depth;
        if (depth < 0) {
            int Lg = 0;
            while ((1 << (Lg + 1)) <= nleaf) Lg++;
            depth = std::max(nleaf >= 2 ? 1 : 0, Lg - 2);
        }
        // every problem needs one level at least: a lone leaf has none
        if (depth < 1 || depth > 30 || nleaf % (1 << depth) != 0) throw HsError{HS_ERR_ARG};
        hs_factor_s::Group G{(int64_t)leaf_ptr.size() - 1, 0, pp[p], pp[p + 1], depth};
        for (int64_t k = 0; k < pp[p + 1] - pp[p]; k++) h->perm[pp[p] + k] = (int32_t)(perm[p][k] + pp[p]);
        for (int c = 0; c < nleaf; c++) leaf_ptr.push_back((int32_t)(pp[p] + lp[p][c + 1]));
        G.leaf_hi = (int64_t)leaf_ptr.size() - 1;
        h->groups.push_back(G);
    }
}

void setup_impl(hs_factor_s* h, const int64_t* rowptr, const int32_t* col, const double* val,
                const hs_tree* tree_in, hs_info* info) {
    cudaStream_t st = h->st;
    if (!tl_in_pool && !tl_serial) Pool::get().wake();  // the planner's loops follow
    const int64_t n = h->n;
    Trace tr;
    // host copy of the pattern (the symbolic analysis runs on the host)
    const int64_t* rp = rowptr;
    const int32_t* cl = col;
    const double* vl = val;
    if (h->opt.mem == HS_MEM_DEVICE) {
        // the pattern (and values, for the partitioner) are read on the host
        int64_t nnz0 = 0;
        CK(cudaMemcpyAsync(&nnz0, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (nnz0 < 0) throw HsError{HS_ERR_ARG};
        // into a pinned area of their own, used in place for the whole setup
        // (kept between calls: later setups of the same size reuse it)
        g_pattern_stage.drain();
        const size_t b_rp = sizeof(int64_t) * (n + 1), b_col = sizeof(int32_t) * nnz0;
        const size_t b_val = tree_in ? 0 : sizeof(double) * nnz0;
        const size_t o_col = (b_rp + 255) & ~(size_t)255, o_val = o_col + ((b_col + 255) & ~(size_t)255);
        const size_t o_flag = o_val + ((b_val + 255) & ~(size_t)255);
        char* pin = g_pattern_stage.take(o_flag + 256, st);
        int64_t* prp = reinterpret_cast<int64_t*>(pin);
        int32_t* pcol = reinterpret_cast<int32_t*>(pin + o_col);
        double* pval = reinterpret_cast<double*>(pin + o_val);
        int32_t* pbad = reinterpret_cast<int32_t*>(pin + o_flag);
        // the pattern is validated where it lies, by a kernel, while it is
        // copied down (the flag comes back with it)
        DBuf d_bad;
        d_bad.alloc(sizeof(int32_t));
        CK(cudaMemsetAsync(d_bad.p, 0, sizeof(int32_t), st));
        CK(launch_check_csr(st, n, nnz0, rowptr, col, d_bad.as<int32_t>()));
        CK(cudaMemcpyAsync(prp, rowptr, b_rp, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(pcol, col, b_col, cudaMemcpyDeviceToHost, st));
        if (b_val) CK(cudaMemcpyAsync(pval, val, b_val, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(pbad, d_bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (*pbad != 0 || prp[n] != nnz0) throw HsError{HS_ERR_ARG};
        rp = prp;
        cl = pcol;
        vl = b_val ? pval : nullptr;
        tr.mark("  pattern download");
    }
    const int64_t nnz = rp[n];
    h->nnz = nnz;
    if (h->opt.mem != HS_MEM_DEVICE) {
        std::atomic<int> bad{0};
        parallel_ranges(n, 1 << 16, [&](int64_t lo, int64_t hi, int) {
            for (int64_t i = lo; i < hi; i++)
                if (rp[i + 1] < rp[i]) bad = 1;
        });
        if (bad || rp[0] != 0) throw HsError{HS_ERR_ARG};
        parallel_ranges(nnz, 1 << 18, [&](int64_t lo, int64_t hi, int) {
            for (int64_t e = lo; e < hi; e++)
                if (cl[e] < 0 || cl[e] >= n) bad = 1;
        });
        if (bad) throw HsError{HS_ERR_ARG};
    }
    tr.mark("  pattern checks");
    // device copies of A (SpMV), in flight during the partition
    h->d_rowptr.alloc(sizeof(int64_t) * (n + 1));
    h->d_col.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    h->d_val.alloc(sizeof(double) * std::max<int64_t>(nnz, 1));
    {
        const cudaMemcpyKind kind = h->opt.mem == HS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(h->d_rowptr.p, rowptr, sizeof(int64_t) * (n + 1), kind, st));
        if (nnz) {
            CK(cudaMemcpyAsync(h->d_col.p, col, sizeof(int32_t) * nnz, kind, st));
            CK(cudaMemcpyAsync(h->d_val.p, val, sizeof(double) * nnz, kind, st));
        }
    }

    // partition tree
    std::vector<int32_t> leaf_ptr;
    int depth;
    const bool batched = !h->prob_ptr.empty();
    if (batched) {
        partition_batched(h, rp, cl, vl, leaf_ptr);
        depth = 0;
        for (const auto& G : h->groups) depth = std::max(depth, G.depth);
    } else if (tree_in) {
        if (!tree_in->perm || !tree_in->leaf_ptr || tree_in->n_leaf <= 0) throw HsError{HS_ERR_ARG};
        h->perm.assign(tree_in->perm, tree_in->perm + n);
        leaf_ptr.assign(tree_in->leaf_ptr, tree_in->leaf_ptr + tree_in->n_leaf + 1);
        depth = tree_in->depth;
    } else {
        partition_impl(n, rp, cl, vl, h->opt.coords, h->opt.leaf_lines, h->opt.theta, h->perm, leaf_ptr,
                       h->opt.partitioner);
        depth = h->opt.depth;
    }
    const int nleaf = (int)leaf_ptr.size() - 1;
    if (depth < 0) {
        int Lg = 0;
        while ((1 << (Lg + 1)) <= nleaf) Lg++;
        depth = std::max(nleaf >= 2 ? 1 : 0, Lg - 2);
    }
    if (leaf_ptr[0] != 0 || leaf_ptr[nleaf] != n) throw HsError{HS_ERR_ARG};
    if (!batched && depth > 0 && (depth > 30 || nleaf % (1 << depth) != 0)) throw HsError{HS_ERR_ARG};
    if (!batched) h->groups.assign(1, hs_factor_s::Group{0, nleaf, 0, n, depth});
    if (tree_in) {  // a caller's permutation (the partitioner's are valid by construction)
        std::vector<char> seen(n, 0);
        for (int64_t i = 0; i < n; i++) {
            const int32_t p = h->perm[i];
            if (p < 0 || p >= n || seen[p]) throw HsError{HS_ERR_ARG};
            seen[p] = 1;
        }
    }
    h->depth = depth;
    tr.mark("pattern+partition");

    if (h->opt.rank_model) {
        // the caller's layout, then W2 transposed for the factor kernel
        std::vector<float> mdl(h->opt.rank_model, h->opt.rank_model + kModelFloats);
        const float* W2 = h->opt.rank_model + 2 * kMlpIn + kMlpHidden * kMlpIn + kMlpHidden;
        for (int k = 0; k < kMlpHidden; k++)
            for (int j = 0; j < kMlpHidden; j++) mdl.push_back(W2[j * kMlpHidden + k]);
        upload(h->d_model, mdl, st);
    }
    // device copy of the permutation
    upload(h->d_perm, h->perm, st);

    // level 0 pattern
    std::vector<int32_t> dof_cluster(n), dof_local(n);
    parallel_ranges(nleaf, 64, [&](int64_t lo, int64_t hi, int) {
        for (int64_t c = lo; c < hi; c++)
            for (int k = leaf_ptr[c]; k < leaf_ptr[c + 1]; k++) {
                dof_cluster[h->perm[k]] = (int32_t)c;
                dof_local[h->perm[k]] = k - leaf_ptr[c];
            }
    });
    LevelPlan P;
    P.nc = nleaf;
    P.size0.resize(nleaf);
    for (int c = 0; c < nleaf; c++) P.size0[c] = leaf_ptr[c + 1] - leaf_ptr[c];
    {
        // block pattern of level 0, kept symmetric even if the CSR pattern is not
        std::vector<std::vector<int>> stamp(hs_threads());
        P.adj0 = build_lists(nleaf, 64, [&](int64_t c, std::vector<int32_t>& out, int t) {
            auto& st = stamp[t];
            if (st.empty()) st.assign(nleaf, -1);
            const size_t b0 = out.size();
            for (int k = leaf_ptr[c]; k < leaf_ptr[c + 1]; k++) {
                const int i = h->perm[k];
                for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
                    const int q = dof_cluster[cl[e]];
                    if (q != c && st[q] != c) {
                        st[q] = (int)c;
                        out.push_back(q);
                    }
                }
            }
            std::sort(out.begin() + b0, out.end());
        });
        std::vector<std::vector<int>> missing(nleaf);  // q gains c where c -> q but not q -> c
        bool any = false;
        for (int c = 0; c < nleaf; c++)
            for (int q : P.adj0[c]) {
                const auto r = P.adj0[q];
                if (!std::binary_search(r.begin(), r.end(), c)) {
                    missing[q].push_back(c);
                    any = true;
                }
            }
        if (any) {
            ListSet old = std::move(P.adj0);
            P.adj0 = build_lists(nleaf, 1 << 30, [&](int64_t c, std::vector<int32_t>& out, int) {
                const size_t b0 = out.size();
                out.insert(out.end(), old[c].begin(), old[c].end());
                out.insert(out.end(), missing[c].begin(), missing[c].end());
                std::sort(out.begin() + b0, out.end());
                out.erase(std::unique(out.begin() + b0, out.end()), out.end());
            });
        }
    }

    DBuf d_status;
    d_status.alloc(sizeof(int32_t) * 4);
    CK(cudaMemsetAsync(d_status.p, 0, sizeof(int32_t) * 4, st));

    tr.mark("upload A, level-0 pattern");
    std::vector<std::pair<int, int>> ranges;
    for (const auto& G : h->groups) ranges.push_back({(int)G.leaf_lo, (int)G.leaf_hi});
    plan_level(P, ranges);
    BlockTable T = make_table(P);
    tr.mark("level-0 plan");
    DBuf blocks;
    blocks.alloc(sizeof(double) * std::max<int64_t>(T.total, 1));
    CK(cudaMemsetAsync(blocks.p, 0, sizeof(double) * std::max<int64_t>(T.total, 1), st));
    {
        DBuf d_dc, d_dl, d_bp, d_bc, d_bo, d_bl;
        upload(d_dc, dof_cluster, st);
        upload(d_dl, dof_local, st);
        upload(d_bp, T.ptr, st);
        upload(d_bc, T.col, st);
        upload(d_bo, T.off, st);
        upload(d_bl, T.ld, st);
        h->prof.begin(KC_ASSEMBLY, st);
        CK(launch_scatter_csr(st, n, h->d_rowptr.as<int64_t>(), h->d_col.as<int32_t>(), h->d_val.as<double>(),
                              d_dc.as<int32_t>(), d_dl.as<int32_t>(), d_bp.as<int32_t>(), d_bc.as<int32_t>(),
                              d_bo.as<int64_t>(), d_bl.as<int32_t>(), blocks.as<double>()));
        h->prof.end(KC_ASSEMBLY, st);
    }
    h->work_bytes[KC_ASSEMBLY] += 20.0 * nnz;
    tr.mark("level-0 scatter");

    h->lev.clear();
    h->tops.clear();
    h->top_bufs.clear();
    int64_t ntop_total = 0;
    // clusters of the current level: one contiguous range per problem still active
    struct Active {
        int g, lo, hi;
    };
    std::vector<Active> act;
    {
        int64_t base = 0;
        for (int g = 0; g < (int)h->groups.size(); g++) {
            const auto& G = h->groups[g];
            if (G.depth >= 1) act.push_back(Active{g, (int)G.leaf_lo, (int)G.leaf_hi});
            base += G.leaf_hi - G.leaf_lo;
        }
    }
    if (act.empty()) {
        // a single problem without levels: its level-0 matrix is the dense top
        std::vector<int64_t> toff(P.nc + 1, 0);
        for (int a = 0; a < P.nc; a++) toff[a + 1] = toff[a] + P.size0[a];
        const int nt = (int)toff[P.nc];
        h->top_bufs.emplace_back();
        h->top_bufs.back().alloc(sizeof(double) * std::max<int64_t>((int64_t)nt * nt, 1));
        CK(cudaMemsetAsync(h->top_bufs.back().p, 0, sizeof(double) * std::max<int64_t>((int64_t)nt * nt, 1), st));
        std::vector<CopyDev> cps;
        for (int a = 0; a < P.nc; a++)
            for (int b : P.all[a]) {
                CopyDev cp{};
                const int sb = T.find(a, b);
                cp.src = T.off[sb];
                cp.src_ld = T.ld[sb];
                cp.dst = toff[a] * (int64_t)nt + toff[b];
                cp.dst_ld = nt;
                cp.rows = P.size0[a];
                cp.cols = P.size0[b];
                cps.push_back(cp);
            }
        DBuf d_cps;
        upload(d_cps, cps, st);
        CK(launch_copy_blocks(st, d_cps.as<CopyDev>(), (int)cps.size(), blocks.as<double>(),
                              h->top_bufs.back().as<double>()));
        h->tops.push_back(TopDev{h->top_bufs.back().as<double>(), 0, nt, 0});
        ntop_total = nt;
    }
    // the previous level's solve records and vector copies, built while
    // the next level's kernels run
    std::function<void()> deferred;
    auto run_deferred = [&] {
        if (deferred) {
            auto f = std::move(deferred);
            deferred = nullptr;
            f();
        }
    };
    for (int l = 0; !act.empty(); l++) {
        h->lev.emplace_back(new Level());
        DBuf d_cur;
        upload(d_cur, P.size0, st);
        ranges.clear();
        for (const Active& a : act) ranges.push_back({a.lo, a.hi});
        factor_level(h, l, P, T, blocks, d_cur, d_status, info, ranges, run_deferred);
        tr.mark("level factor (records+kernels)");
        Level& L = *h->lev[l];
        const std::vector<int>& fin = L.fin;
        // parents: problems that go on get their sibling pairs merged at the
        // next level; problems whose last level this was get a dense top
        const int nc = P.nc;
        std::vector<int> par(nc, -1), poff(nc, 0), tn(nc, 0);
        std::vector<int64_t> tmat(nc, 0), tpos(nc, 0), dst(nc, 0);
        std::vector<char> to_top(nc, 0);
        std::vector<Active> nact;
        std::vector<int> nsize;
        struct Fin {
            int g, lo, hi;
            std::vector<int64_t> toff;
            int n;
            int64_t mat, vec;
        };
        std::vector<Fin> ending;
        int64_t mat_total = 0;
        for (const Active& a : act) {
            const int cnt = a.hi - a.lo;
            for (int cc = a.lo; cc < a.hi; cc++) poff[cc] = ((cc - a.lo) & 1) ? fin[cc - 1] : 0;
            if (h->groups[a.g].depth > l + 1) {
                const int nlo = (int)nsize.size();
                for (int k = 0; k < cnt / 2; k++) nsize.push_back(fin[a.lo + 2 * k] + fin[a.lo + 2 * k + 1]);
                for (int cc = a.lo; cc < a.hi; cc++) par[cc] = nlo + (cc - a.lo) / 2;
                nact.push_back(Active{a.g, nlo, nlo + cnt / 2});
            } else {
                Fin f{a.g, a.lo, a.hi, std::vector<int64_t>(cnt / 2 + 1, 0), 0, 0, 0};
                for (int k = 0; k < cnt / 2; k++)
                    f.toff[k + 1] = f.toff[k] + fin[a.lo + 2 * k] + fin[a.lo + 2 * k + 1];
                f.n = (int)f.toff[cnt / 2];
                f.mat = mat_total;
                mat_total += (int64_t)f.n * f.n;
                f.vec = ntop_total;
                ntop_total += f.n;
                for (int cc = a.lo; cc < a.hi; cc++) {
                    to_top[cc] = 1;
                    tn[cc] = f.n;
                    tmat[cc] = f.mat;
                    tpos[cc] = f.toff[(cc - a.lo) / 2] + poff[cc];
                    dst[cc] = f.vec + tpos[cc];
                }
                ending.push_back(std::move(f));
            }
        }
        const int nn = (int)nsize.size();
        std::vector<int64_t> nslot(nn + 1, 0);
        for (int k = 0; k < nn; k++) nslot[k + 1] = nslot[k] + nsize[k];
        for (int cc = 0; cc < nc; cc++)
            if (par[cc] >= 0) dst[cc] = nslot[par[cc]] + poff[cc];
        deferred = [h, l, dst = std::move(dst), to_top = std::move(to_top)] {
            level_records(h, l);
            make_vcopies(h, *h->lev[l], dst, to_top);
        };
        if (!ending.empty()) {
            // dense tops of the problems that end here
            h->top_bufs.emplace_back();
            DBuf& tb = h->top_bufs.back();
            tb.alloc(sizeof(double) * std::max<int64_t>(mat_total, 1));
            CK(cudaMemsetAsync(tb.p, 0, sizeof(double) * std::max<int64_t>(mat_total, 1), st));
            std::vector<CopyDev> cps = make_assembly(P, fin, T, nullptr, nsize, par, poff, tmat, tpos, tn, true);
            DBuf d_cps;
            upload(d_cps, cps, st);
            h->prof.begin(KC_TOP, st);
            CK(launch_copy_blocks(st, d_cps.as<CopyDev>(), (int)cps.size(), blocks.as<double>(), tb.as<double>()));
            h->prof.end(KC_TOP, st);
            for (const Fin& f : ending) h->tops.push_back(TopDev{tb.as<double>() + f.mat, f.vec, f.n, f.g});
        }
        if (nn > 0) {
            LevelPlan Pn;
            Pn.nc = nn;
            Pn.size0 = nsize;
            std::vector<int> kid0(nn, -1);  // first child of every parent (children are consecutive)
            for (int a = nc - 1; a >= 0; a--)
                if (par[a] >= 0) kid0[par[a]] = a;
            Pn.adj0 = build_lists(nn, 128, [&](int64_t k, std::vector<int32_t>& v, int) {
                const size_t b0 = v.size();
                for (int a = kid0[k]; a < nc && par[a] == k; a++) {
                    if (fin[a] <= 0) continue;
                    for (int b : P.endp[a])
                        if (fin[b] > 0 && par[b] != k) v.push_back(par[b]);
                }
                std::sort(v.begin() + b0, v.end());
                v.erase(std::unique(v.begin() + b0, v.end()), v.end());
            });
            tr.mark("next-level adjacency");
            ranges.clear();
            for (const Active& a : nact) ranges.push_back({a.lo, a.hi});
            plan_level(Pn, ranges);
            tr.mark("next-level plan_level");
            BlockTable Tn = make_table(Pn);
            tr.mark("  make_table");
            DBuf nblocks;
            nblocks.alloc(sizeof(double) * std::max<int64_t>(Tn.total, 1));
            CK(cudaMemsetAsync(nblocks.p, 0, sizeof(double) * std::max<int64_t>(Tn.total, 1), st));
            std::vector<CopyDev> cps = make_assembly(P, fin, T, &Tn, nsize, par, poff, tmat, tpos, tn, false);
            tr.mark("  make_assembly");
            DBuf d_cps;
            upload(d_cps, cps, st);
            h->prof.begin(KC_ASSEMBLY, st);
            CK(launch_copy_blocks(st, d_cps.as<CopyDev>(), (int)cps.size(), blocks.as<double>(),
                                  nblocks.as<double>()));
            h->prof.end(KC_ASSEMBLY, st);
            tr.mark("  assembly kernels");
            blocks = std::move(nblocks);
            release_plan(P);
            P = std::move(Pn);
            T = std::move(Tn);
        }
        act = std::move(nact);
        tr.mark("next-level plan+assembly");
    }
    run_deferred();
    // factor every dense top (one CTA per problem)
    h->ntop = (int)ntop_total;
    h->d_ytop.alloc(sizeof(double) * std::max<int64_t>(ntop_total, 1));
    upload(h->d_tops, h->tops, st);
    h->top_L = h->tops.empty() ? nullptr : h->tops[0].L;
    if (h->groups.size() == 1 && !h->tops.empty()) h->ntop = h->tops[0].n;
    if (ntop_total > 0) {
        h->prof.begin(KC_TOP, st);
        if (h->tops.size() == 1)
            CK(launch_dense_cholesky(st, h->tops[0].n, h->tops[0].L, d_status.as<int32_t>()));
        else
            CK(launch_tops_cholesky(st, h->d_tops.as<TopDev>(), (int)h->tops.size(), d_status.as<int32_t>()));
        h->prof.end(KC_TOP, st);
    }
    blocks.release();
    // level vectors for the solve phase
    int64_t fb = 0;
    for (const TopDev& tp : h->tops) fb += (int64_t)tp.n * tp.n * 8;
    for (auto& Lp : h->lev) {
        Lp->d_y.alloc(sizeof(double) * std::max<int64_t>(Lp->slot[Lp->nc], 1));
        fb += Lp->fac_doubles * (h->fp32 ? 4 : 8);
    }
    h->factor_bytes = fb;
    tr.mark("top");
    // the dense coarse operator is formed and the solve graph captured while
    // the tops' Cholesky runs; then one synchronisation reads the status of
    // both (and of everything the setup enqueued)
    build_apply_graph(h);
    h->apply_bytes = apply_work_bytes(h);
    check_status(h, d_status, info);
    tr.mark("apply graph");
}

// Algorithmic bytes of one apply (Algorithm 2): every stored factor entry
// (W = U^T G^-1 and the n-columns of C per cluster) is read once forward and
// once backward; per level the vector is read and written in each direction
// plus the staged neighbour updates (three vectors); the dense coarse
// operator (or the top's lower triangle twice) once; the two permutations.
double apply_work_bytes(const hs_factor_s* h) {
    const double elt = h->fp32 ? 4.0 : 8.0;
    const int D = (int)h->lev.size();
    const int lc = (h->groups.size() > 1) ? D : h->first_coarse;
    double bytes = 40.0 * (double)h->n;
    for (int l = 0; l < D; l++) {
        const Level& L = *h->lev[l];
        if (l >= lc && h->coarse_dense) break;  // folded into the dense operator
        double fac = 0.0;
        for (size_t ti = 0; ti < L.tasks.size(); ti++) {
            const TaskDev& t = L.tasks[ti];
            const int32_t* mt = L.hmeta.data() + t.meta;
            const int ncols = t.nn > 0 ? mt[1 + 2 * (t.nn - 1)] + mt[2 + 2 * (t.nn - 1)] : 0;
            fac += (double)t.s * t.s + (double)(t.s - mt[0]) * ncols;
        }
        bytes += 2.0 * elt * fac + 3.0 * 8.0 * (double)L.slot[L.nc];
    }
    if (h->coarse_dense) bytes += 8.0 * (double)h->ncoarse * h->ncoarse + 16.0 * h->ncoarse;
    else for (const TopDev& t : h->tops) bytes += 8.0 * (double)t.n * t.n;
    return bytes;
}

// First level handled by the single-CTA coarse kernel: every level from there
// on has clusters of at most kCoarseSmax DOFs and little work per phase.
int first_coarse_level(const hs_factor_s* h) {
    int lc = (int)h->lev.size();
    for (int l = (int)h->lev.size() - 1; l >= 0; l--) {
        const Level& L = *h->lev[l];
        if (L.smax > kCoarseSmax || L.nmax > kCoarseNmax || L.work_max_phase > (int64_t)1 << 16) break;
        lc = l;
    }
    return lc;
}

// Algorithm 2 on the internal level vectors (y0 holds r in partition order).
void enqueue_apply(hs_factor_s* h) {
    cudaStream_t st = h->st;
    const int D = (int)h->lev.size();
    const int lc = h->first_coarse;
    auto vec_of = [&](int l) { return l < D ? h->lev[l]->d_y.as<double>() : h->d_ytop.as<double>(); };
    // forward writes level l+1's vector; in dense mode the backward reads the
    // dense operator's output for the first coarse level
    auto next_of = [&](int l) { return vec_of(l + 1); };
    auto back_of = [&](int l) {
        return (h->coarse_dense && l + 1 == lc) ? h->d_ycout.as<double>() : vec_of(l + 1);
    };
    for (int l = 0; l < lc; l++) {
        Level& L = *h->lev[l];
        for (int k = 0; k < L.nstages; k++) {
            const int t0 = L.ap_stage[k], nt = L.ap_stage[k + 1] - t0;
            CK(launch_ap_fwd(st, L.d_ap_tasks.as<ApTask>(), t0, nt, L.smax, L.d_ap_pulls.as<ApPull>(), L.d_fac.p,
                             h->fp32, L.d_stage.as<double>(), L.d_y.as<double>()));
        }
        CK(launch_ap_fin(st, L.d_ap_fins.as<ApFin>(), L.nfin, L.d_ap_pulls.as<ApPull>(), L.d_stage.as<double>(),
                         L.d_y.as<double>(), next_of(l), h->d_ytop.as<double>()));
    }
    if (h->groups.size() > 1)  // every problem's dense top, one CTA each
        CK(launch_tops_solve(st, h->d_tops.as<TopDev>(), (int)h->tops.size(), h->d_ytop.as<double>()));
    else if (h->coarse_dense)
        CK(launch_dense_gemv(st, h->ncoarse, h->d_coarse.as<double>(), vec_of(lc), h->d_ycout.as<double>()));
    else
        CK(launch_ap_coarse(st, h->d_aplevels.as<ApLevel>(), D - lc, h->ntop, h->top_L,
                            h->d_ytop.as<double>(), h->fp32));
    for (int l = lc - 1; l >= 0; l--) {
        Level& L = *h->lev[l];
        // one problem: its top's solution sits where back_of points (the
        // dense coarse operator's output, or the top vector)
        CK(launch_vcopy(st, L.d_vcopy.as<VCopyDev>(), L.nvcopy, back_of(l), L.d_y.as<double>(), 1,
                        h->groups.size() > 1 ? h->d_ytop.as<double>() : back_of(l)));
        for (int k = L.nstages - 1; k >= 0; k--) {
            const int t0 = L.ap_stage[k], nt = L.ap_stage[k + 1] - t0;
            CK(launch_ap_bwd(st, L.d_ap_tasks.as<ApTask>(), t0, nt, L.smax, L.nmax, L.d_ap_nbs.as<ApNb>(), L.d_fac.p,
                             h->fp32, L.d_y.as<double>()));
        }
    }
}

void build_apply_graph(hs_factor_s* h) {
    if (h->apply_graph) { cudaGraphExecDestroy(h->apply_graph); h->apply_graph = nullptr; }
    if (h->lev.empty() && h->ntop == 0) return;
    const int D = (int)h->lev.size();
    const int lc0 = first_coarse_level(h);
    auto level_len = [&](int l) -> int64_t { return l < D ? h->lev[l]->slot[h->lev[l]->nc] : h->ntop; };
    // dense coarse operator: among the levels (>= lc0) with at most
    // coarse_dense DOFs, the one with the smallest modelled cost of building
    // it (a single-CTA pass over the remaining stages per unit vector: the
    // larger of a per-(vector x stage) cost and one chain's latency) plus
    // kModelApplies applies (the levels above it as stage kernels, and the
    // dense product).  Constants measured on GB300.
    int ld = -1;
    if (h->opt.coarse_dense > 0) {
        constexpr double kVecStageUs = 0.012, kChainStageUs = 2.4, kLaunchUs = 5.0, kModelApplies = 10.0,
                         kGemvBytesPerUs = 4e6;
        auto stages = [&](int l) { return l < D ? 2.0 * h->lev[l]->nstages + 2.0 : 2.0; };
        double best = 0.0;
        for (int l = lc0; l <= D; l++) {
            const int64_t n = level_len(l);
            if (n > h->opt.coarse_dense) continue;
            int64_t stride = 0;  // the batched build needs one workspace per unit vector
            for (int k = l; k <= D; k++) stride += std::max<int64_t>(level_len(k), 1);
            for (int k = l; k < D; k++) stride += (int64_t)(h->lev[k]->d_stage.bytes / sizeof(double));
            if ((double)stride * n * 8.0 > 2e9) continue;
            double chain = 0.0, above = 0.0;
            for (int k = l; k <= D; k++) chain += stages(k);
            for (int k = lc0; k < l; k++) above += stages(k);
            const double build = std::max((double)n * chain * kVecStageUs, chain * kChainStageUs);
            const double cost = build + kModelApplies * (above * kLaunchUs + 8.0 * (double)n * n / kGemvBytesPerUs);
            if (std::getenv("HS_TRACE"))
                std::fprintf(stderr, "hs_trace dense candidate level %d: n %lld, modelled cost %.1f us\n", l,
                             (long long)n, cost);
            if (ld < 0 || cost < best) { ld = l; best = cost; }
        }
    }
    h->coarse_dense = ld >= 0;
    h->first_coarse = h->coarse_dense ? ld : lc0;
    if (h->groups.size() > 1) {  // several problems: fine-level kernels down to the tops
        h->coarse_dense = false;
        h->first_coarse = D;
    }
    if (std::getenv("HS_TRACE")) {
        for (size_t l = 0; l < h->lev.size(); l++)
            std::fprintf(stderr, "hs_trace level %zu: %d clusters, %d phases, %d solve stages, smax %d, ncap %d%s\n", l,
                         h->lev[l]->nc, h->lev[l]->nphases, h->lev[l]->nstages, h->lev[l]->smax, h->lev[l]->nmax,
                         (int)l >= h->first_coarse ? (h->coarse_dense ? " (dense coarse operator)" : " (coarse kernel)")
                                                   : "");
    }
    // ApLevel records of the coarse levels; in dense mode their vectors and
    // stage arrays live in a per-right-hand-side workspace (stride apart)
    auto make_levels = [&](double* ws_base, int64_t* stride_out, double** yin0, double** ytop0) {
        std::vector<ApLevel> al;
        std::vector<int64_t> yoff, soff;
        int64_t o = 0;
        for (int l = h->first_coarse; l <= D; l++) { yoff.push_back(o); o += std::max<int64_t>(level_len(l), 1); }
        for (int l = h->first_coarse; l < D; l++) {
            soff.push_back(o);
            o += std::max<int64_t>(h->lev[l]->d_stage.bytes / sizeof(double), 1);
        }
        if (stride_out) *stride_out = o;
        for (int l = h->first_coarse; l < D; l++) {
            Level& L = *h->lev[l];
            const int k = l - h->first_coarse;
            ApLevel a{};
            a.tasks = L.d_ap_tasks.as<ApTask>();
            a.ph = L.d_ph.as<int32_t>();
            a.pulls = L.d_ap_pulls.as<ApPull>();
            a.nbs = L.d_ap_nbs.as<ApNb>();
            a.fins = L.d_ap_fins.as<ApFin>();
            a.vcopy = L.d_vcopy.as<VCopyDev>();
            a.fac = L.d_fac.p;
            if (ws_base) {
                a.stage = ws_base + soff[k];
                a.y = ws_base + yoff[k];
                a.ynext = ws_base + yoff[k + 1];
            } else {
                a.stage = L.d_stage.as<double>();
                a.y = L.d_y.as<double>();
                a.ynext = (l + 1 < D) ? h->lev[l + 1]->d_y.as<double>() : h->d_ytop.as<double>();
            }
            a.nph = L.nstages;
            a.nfin = L.nfin;
            a.nvcopy = L.nvcopy;
            al.push_back(a);
        }
        if (yin0) *yin0 = ws_base + yoff[0];
        if (ytop0) *ytop0 = ws_base + yoff.back();
        return al;
    };
    if (h->coarse_dense) {
        const int n = (int)level_len(ld);
        h->ncoarse = n;
        h->d_coarse.alloc(sizeof(double) * std::max<int64_t>((int64_t)n * n, 1));
        h->d_ycout.alloc(sizeof(double) * std::max(n, 1));
        int64_t stride = 0;
        make_levels(nullptr, &stride, nullptr, nullptr);
        DBuf ws;
        ws.alloc(sizeof(double) * std::max<int64_t>(stride * std::max(n, 1), 1));
        double *yin0 = nullptr, *ytop0 = nullptr;
        std::vector<ApLevel> al = make_levels(ws.as<double>(), nullptr, &yin0, &ytop0);
        DBuf d_al;
        upload(d_al, al, h->st);
        h->prof.begin(KC_TOP, h->st);
        CK(launch_ap_coarse_batch(h->st, d_al.as<ApLevel>(), (int)al.size(), h->ntop, h->top_L, ytop0,
                                  yin0, n, stride, h->d_coarse.as<double>(), h->fp32));
        h->prof.end(KC_TOP, h->st);
    } else {
        std::vector<ApLevel> al = make_levels(nullptr, nullptr, nullptr, nullptr);
        upload(h->d_aplevels, al, h->st);
    }
    h->apply_out = (h->coarse_dense && ld == 0) ? h->d_ycout.as<double>() : nullptr;
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = h->st;
    h->st = cap;
    cudaGraph_t g = nullptr;
    try {
        const int64_t before = launch_count();
        CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        enqueue_apply(h);
        CK(cudaStreamEndCapture(cap, &g));
        h->graph_kernels = launch_count() - before;
        launch_count_add(-h->graph_kernels);  // captured, not executed
        CK(cudaGraphInstantiate(&h->apply_graph, g, 0));
    } catch (...) {
        h->st = saved;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        throw;
    }
    h->st = saved;
    cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
}

// z = M^-1 r (device vectors, original ordering)
void apply_impl(hs_factor_s* h, const double* r, double* z) {
    cudaStream_t st = h->st;
    double* y0 = h->lev.empty() ? h->d_ytop.as<double>() : h->lev[0]->d_y.as<double>();
    h->prof.begin(KC_APPLY, st);
    h->work_bytes[KC_APPLY] += h->apply_bytes;
    CK(launch_permute(st, h->n, h->d_perm.as<int32_t>(), r, y0, 0));
    if (h->apply_graph) {
        CK(cudaGraphLaunch(h->apply_graph, st));
        launch_count_add(h->graph_kernels);
    }
    CK(launch_permute(st, h->n, h->d_perm.as<int32_t>(), h->apply_out ? h->apply_out : y0, z, 1));
    h->prof.end(KC_APPLY, st);
}

// one device double read back through the pinned staging area (a copy to
// pageable memory would be staged by the driver); synchronises the stream
double read_scalar(hs_factor_s* h, const double* d) {
    double* pin = reinterpret_cast<double*>(g_stage.take(sizeof(double), h->st));
    CK(cudaMemcpyAsync(pin, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const double v = *pin;
    g_stage.synced(h->st);
    return v;
}

// the same into a stack variable (no staging area, which may allocate): for
// the allocation-free PCG
double read_scalar_stack(hs_factor_s* h, const double* d) {
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return v;
}

// y = A x with the handle's CSR copy (profiled as its own class; algorithmic
// bytes 12 nnz + 24 n: values and column indices once, row pointers, x and y)
void spmv_prof(hs_factor_s* h, const double* x, double* y) {
    const int64_t n = h->n;
    h->prof.begin(KC_SPMV, h->st);
    CK(launch_spmv(h->st, n, h->d_rowptr.as<int64_t>(), h->d_col.as<int32_t>(), h->d_val.as<double>(), x, y));
    h->prof.end(KC_SPMV, h->st);
    h->work_bytes[KC_SPMV] += 12.0 * (double)h->nnz + 24.0 * (double)n;
}

int pcg_impl(hs_factor_s* h, const double* b, double* x, hs_info* info) {
    cudaStream_t st = h->st;
    const int64_t n = h->n;
    h->d_kv.ensure(sizeof(double) * 4 * n);
    double* r = h->d_kv.as<double>();
    double* z = r + n;
    double* p = z + n;
    double* q = p + n;
    // block partials, then the fused kernels' arrival counter
    h->d_part.ensure(sizeof(double) * (kDotParts + 2));
    h->d_scal.ensure(sizeof(double) * 8);
    double* part = h->d_part.as<double>();
    unsigned* cnt = reinterpret_cast<unsigned*>(part + kDotParts);
    double* sc = h->d_scal.as<double>();  // 0, 2: rz (alternating), 1 pq, 3 rr, 4 bb
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned), st));
    auto spmv = [&](const double* xx, double* yy) { spmv_prof(h, xx, yy); };
    auto dot = [&](const double* a, const double* bb, double* out) {
        h->prof.begin(KC_KRYLOV, st);
        CK(launch_dot_fused(st, n, a, bb, part, cnt, out));
        h->prof.end(KC_KRYLOV, st);
    };
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    dot(b, b, sc + 4);
    const double bn = std::sqrt(read_scalar(h, sc + 4));
    if (bn == 0.0) {
        info->iters = 0;
        info->rel_resid = 0.0;
        return HS_OK;
    }
    int rz = 0;  // slot of the current r^T z; the next one goes to the other
    apply_impl(h, r, z);
    CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    dot(r, z, sc + rz);
    int it = 0;
    double rn = bn;
    int rc = HS_ERR_NOCONV;
    while (it < h->opt.maxit) {
        // q = A p with pq = p^T q; then x, r and rr = r^T r (one pass each)
        h->prof.begin(KC_SPMV, st);
        CK(launch_spmv_dot(st, n, h->d_rowptr.as<int64_t>(), h->d_col.as<int32_t>(), h->d_val.as<double>(), p, q,
                           part, cnt, sc + 1));
        h->prof.end(KC_SPMV, st);
        h->work_bytes[KC_SPMV] += 12.0 * (double)h->nnz + 32.0 * (double)n;
        h->prof.begin(KC_KRYLOV, st);
        CK(launch_pcg_xr_dot(st, n, sc + rz, sc + 1, p, q, x, r, part, cnt, sc + 3));
        h->prof.end(KC_KRYLOV, st);
        it++;
        rn = std::sqrt(read_scalar(h, sc + 3));
        if (rn / bn <= h->opt.rtol) {
            spmv(x, q);
            h->prof.begin(KC_KRYLOV, st);
            CK(launch_axpby(st, n, 1.0, b, -1.0, q));
            h->prof.end(KC_KRYLOV, st);
            dot(q, q, sc + 3);
            rn = std::sqrt(read_scalar(h, sc + 3));
            if (rn / bn <= h->opt.rtol) { rc = HS_OK; break; }
            CK(cudaMemcpyAsync(r, q, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            apply_impl(h, r, z);
            CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            dot(r, z, sc + rz);
            continue;
        }
        apply_impl(h, r, z);
        const int rzn = 2 - rz;
        dot(r, z, sc + rzn);
        h->prof.begin(KC_KRYLOV, st);
        CK(launch_pcg_update_p(st, n, sc + rzn, sc + rz, z, p));
        h->prof.end(KC_KRYLOV, st);
        rz = rzn;
    }
    info->iters = it;
    info->rel_resid = rn / bn;
    return rc;
}

// PCG on every problem of a batched handle at once: one preconditioner apply
// and one SpMV per iteration serve all problems; scalars, stopping test and
// true-residual restarts are per problem (each follows the single-problem
// PCG above step for step).  iters / rel: host arrays, one entry per problem.
int pcg_batched_impl(hs_factor_s* h, const double* b, double* x, int32_t* iters, double* rel, hs_info* info) {
    cudaStream_t st = h->st;
    const int64_t n = h->n;
    const int np = (int)h->prob_ptr.size() - 1;
    const int64_t ml = h->prob_maxlen;
    const int64_t* pp = h->d_pp.as<int64_t>();
    h->d_kv.ensure(sizeof(double) * 4 * n);
    double* r = h->d_kv.as<double>();
    double* z = r + n;
    double* p = z + n;
    double* q = p + n;
    h->d_scal.ensure(sizeof(double) * kBScal * np + sizeof(int32_t) * (kBFlag * np + 4));
    double* sc = h->d_scal.as<double>();
    int32_t* fl = reinterpret_cast<int32_t*>(sc + (int64_t)kBScal * np);
    int32_t* cnt = fl + (int64_t)kBFlag * np;
    const double rtol = h->opt.rtol;
    auto kr = [&](cudaError_t e) {
        CK(e);
    };
    auto counts = [&]() {
        int32_t v[2];
        CK(cudaMemcpyAsync(v, cnt, sizeof(v), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return std::make_pair(v[0], v[1]);
    };
    h->prof.begin(KC_KRYLOV, st);
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    kr(launch_seg_dot(st, np, pp, b, b, sc, BS_BB));
    kr(launch_bpcg_book(st, np, 0, rtol, sc, fl, cnt));
    h->prof.end(KC_KRYLOV, st);
    int active = counts().second;
    int it = 0;
    while (active > 0) {
        apply_impl(h, r, z);
        h->prof.begin(KC_KRYLOV, st);
        kr(launch_seg_dot(st, np, pp, r, z, sc, BS_RZN));
        kr(launch_bpcg_vec(st, 1, np, ml, pp, sc, fl, z, nullptr, p, nullptr));
        kr(launch_bpcg_book(st, np, 1, rtol, sc, fl, cnt));
        h->prof.end(KC_KRYLOV, st);
        if (it >= h->opt.maxit) break;
        spmv_prof(h, p, q);
        h->prof.begin(KC_KRYLOV, st);
        kr(launch_seg_dot(st, np, pp, p, q, sc, BS_PQ));
        kr(launch_bpcg_vec(st, 0, np, ml, pp, sc, fl, p, q, x, r));
        kr(launch_seg_dot(st, np, pp, r, r, sc, BS_RR));
        kr(launch_bpcg_book(st, np, 2, rtol, sc, fl, cnt));
        h->prof.end(KC_KRYLOV, st);
        it++;
        if (counts().first > 0) {
            // true residual b - A x of every problem; the candidates stop or restart
            spmv_prof(h, x, q);
            h->prof.begin(KC_KRYLOV, st);
            kr(launch_axpby(st, n, 1.0, b, -1.0, q));
            kr(launch_seg_dot(st, np, pp, q, q, sc, BS_RRT));
            kr(launch_bpcg_book(st, np, 3, rtol, sc, fl, cnt));
            kr(launch_bpcg_vec(st, 2, np, ml, pp, sc, fl, q, nullptr, r, nullptr));
            h->prof.end(KC_KRYLOV, st);
            active = counts().second;
        }
    }
    std::vector<double> hs((size_t)kBScal * np);
    std::vector<int32_t> hf((size_t)kBFlag * np);
    CK(cudaMemcpyAsync(hs.data(), sc, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hf.data(), fl, sizeof(int32_t) * hf.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    info->iters = 0;
    info->rel_resid = 0.0;
    bool all = true;
    for (int k = 0; k < np; k++) {
        const int32_t itk = hf[(size_t)k * kBFlag + BF_ITERS];
        const double rk = hs[(size_t)k * kBScal + BS_REL];
        if (iters) iters[k] = itk;
        if (rel) rel[k] = rk;
        info->iters = std::max(info->iters, itk);
        info->rel_resid = std::max(info->rel_resid, rk);
        if (hf[(size_t)k * kBFlag + BF_ACTIVE]) all = false;
    }
    return all ? HS_OK : HS_ERR_NOCONV;
}

int gmres_impl(hs_factor_s* h, const double* b, double* x, hs_info* info) {
    cudaStream_t st = h->st;
    const int64_t n = h->n;
    const int m = std::max(1, h->opt.restart);
    h->d_V.ensure(sizeof(double) * (size_t)(m + 1) * n);
    h->d_Z.ensure(sizeof(double) * (size_t)m * n);
    h->d_kv.ensure(sizeof(double) * n);
    h->d_part.ensure(sizeof(double) * 256 * (m + 2));
    h->d_h.ensure(sizeof(double) * 2 * (m + 2));
    h->d_scal.ensure(sizeof(double) * 8);
    double* V = h->d_V.as<double>();
    double* Z = h->d_Z.as<double>();
    double* w = h->d_kv.as<double>();
    double* part = h->d_part.as<double>();
    double* dh = h->d_h.as<double>();
    double* sc = h->d_scal.as<double>();
    CK(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)(m + 1) * n, st));
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    auto norm = [&](const double* a) {
        h->prof.begin(KC_KRYLOV, st);
        CK(launch_dot(st, n, a, a, part, sc));
        h->prof.end(KC_KRYLOV, st);
        return std::sqrt(read_scalar(h, sc));
    };
    const double bn = norm(b);
    if (bn == 0.0) {
        info->iters = 0;
        info->rel_resid = 0.0;
        return HS_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yv(m), hh(m + 1), hh2(m + 1);
    int it = 0, rc = HS_ERR_NOCONV;
    double rn = bn;
    for (;;) {
        // true residual (iterative refinement restart)
        spmv_prof(h, x, w);
        CK(launch_axpby(st, n, 1.0, b, -1.0, w));
        const double beta = norm(w);
        rn = beta;
        if (beta / bn <= h->opt.rtol) { rc = HS_OK; break; }
        if (it >= h->opt.maxit) break;
        CK(launch_axpby(st, n, 1.0 / beta, w, 0.0, V));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int kk = 0;
        for (int j = 0; j < m && it < h->opt.maxit; j++) {
            apply_impl(h, V + (size_t)j * n, Z + (size_t)j * n);
            spmv_prof(h, Z + (size_t)j * n, w);
            h->prof.begin(KC_KRYLOV, st);
            // classical Gram-Schmidt, twice
            CK(launch_gemv_t(st, n, j + 1, V, n, w, part, dh));
            CK(launch_gmres_update(st, n, j + 1, dh, V, n, w, -1.0));
            CK(launch_gemv_t(st, n, j + 1, V, n, w, part, dh + m + 1));
            CK(launch_gmres_update(st, n, j + 1, dh + m + 1, V, n, w, -1.0));
            h->prof.end(KC_KRYLOV, st);
            CK(cudaMemcpyAsync(hh.data(), dh, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hh2.data(), dh + m + 1, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
            const double hn = norm(w);
            for (int k = 0; k <= j; k++) H[(size_t)k * m + j] = hh[k] + hh2[k];
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0) CK(launch_axpby(st, n, 1.0 / hn, w, 0.0, V + (size_t)(j + 1) * n));
            for (int k = 0; k < j; k++) {
                const double a = H[(size_t)k * m + j], c2 = H[(size_t)(k + 1) * m + j];
                H[(size_t)k * m + j] = cs[k] * a + sn[k] * c2;
                H[(size_t)(k + 1) * m + j] = -sn[k] * a + cs[k] * c2;
            }
            const double a = H[(size_t)j * m + j], c2 = H[(size_t)(j + 1) * m + j];
            const double d = std::sqrt(a * a + c2 * c2);
            cs[j] = d > 0 ? a / d : 1.0;
            sn[j] = d > 0 ? c2 / d : 0.0;
            H[(size_t)j * m + j] = d;
            H[(size_t)(j + 1) * m + j] = 0.0;
            const double t = g[j];
            g[j] = cs[j] * t;
            g[j + 1] = -sn[j] * t;
            it++;
            kk = j + 1;
            if (std::fabs(g[j + 1]) / bn <= h->opt.rtol || hn == 0.0) break;
        }
        for (int k = kk - 1; k >= 0; k--) {
            double t = g[k];
            for (int j = k + 1; j < kk; j++) t -= H[(size_t)k * m + j] * yv[j];
            yv[k] = t / H[(size_t)k * m + k];
        }
        CK(cudaMemcpyAsync(dh, yv.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, st));
        CK(launch_gmres_update(st, n, kk, dh, Z, n, x, 1.0));
    }
    info->iters = it;
    info->rel_resid = rn / bn;
    return rc;
}

// PCG of hs_krylov_noalloc: the same iteration as pcg_impl, with every work
// vector in the library's static device scratch and no profiling, so that no
// device memory is allocated.
int pcg_noalloc(hs_factor_s* h, const double* b, double* x, double* scratch, hs_info* info) {
    cudaStream_t st = h->st;
    const int64_t n = h->n;
    double* r = scratch;
    double* z = r + kNoAllocMaxN;
    double* p = z + kNoAllocMaxN;
    double* q = p + kNoAllocMaxN;
    double* part = q + kNoAllocMaxN;
    double* sc = part + kDotParts;  // 0 rz, 1 pq, 2 rz_new, 3 rr, 4 bb
    double* y0 = h->lev.empty() ? h->d_ytop.as<double>() : h->lev[0]->d_y.as<double>();
    auto apply = [&](const double* rr, double* zz) {
        CK(launch_permute(st, n, h->d_perm.as<int32_t>(), rr, y0, 0));
        if (h->apply_graph) {
            CK(cudaGraphLaunch(h->apply_graph, st));
            launch_count_add(h->graph_kernels);
        }
        CK(launch_permute(st, n, h->d_perm.as<int32_t>(), h->apply_out ? h->apply_out : y0, zz, 1));
    };
    auto spmv = [&](const double* xx, double* yy) {
        CK(launch_spmv(st, n, h->d_rowptr.as<int64_t>(), h->d_col.as<int32_t>(), h->d_val.as<double>(), xx, yy));
    };
    auto dot = [&](const double* a, const double* bb, double* out) { CK(launch_dot(st, n, a, bb, part, out)); };
    // the scratch keeps the previous call's contents: everything read below is
    // written first in this call (x is zeroed, r copied from b, scalars set by dot)
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    dot(b, b, sc + 4);
    const double bn = std::sqrt(read_scalar_stack(h, sc + 4));
    if (bn == 0.0) {
        info->iters = 0;
        info->rel_resid = 0.0;
        return HS_OK;
    }
    apply(r, z);
    CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    dot(r, z, sc + 0);
    int it = 0;
    double rn = bn;
    int rc = HS_ERR_NOCONV;
    while (it < h->opt.maxit) {
        spmv(p, q);
        dot(p, q, sc + 1);
        CK(launch_pcg_update_xr(st, n, sc + 0, sc + 1, p, q, x, r));
        it++;
        dot(r, r, sc + 3);
        rn = std::sqrt(read_scalar_stack(h, sc + 3));
        if (rn / bn <= h->opt.rtol) {
            spmv(x, q);
            CK(launch_axpby(st, n, 1.0, b, -1.0, q));
            dot(q, q, sc + 3);
            rn = std::sqrt(read_scalar_stack(h, sc + 3));
            if (rn / bn <= h->opt.rtol) { rc = HS_OK; break; }
            CK(cudaMemcpyAsync(r, q, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            apply(r, z);
            CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            dot(r, z, sc + 0);
            continue;
        }
        apply(r, z);
        dot(r, z, sc + 2);
        CK(launch_pcg_update_p(st, n, sc + 2, sc + 0, z, p));
        CK(cudaMemcpyAsync(sc + 0, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    info->iters = it;
    info->rel_resid = rn / bn;
    return rc;
}

template <class F>
int run_guarded(F&& f) {
    try {
        f();
        return HS_OK;
    } catch (const HsError& e) {
        return e.code;
    } catch (const std::bad_alloc&) {
        return HS_ERR_OOM;
    } catch (...) {
        return HS_ERR_CUDA;
    }
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

int hs_default_options(hs_options* opt) {
    if (!opt) return HS_ERR_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->tol = 1e-2;
    opt->schur_products = HS_PRODUCTS_TF32X3;
    opt->depth = -1;
    opt->leaf_lines = 4;
    opt->theta = 0.5;
    opt->precision = HS_PREC_FP64;
    opt->krylov = HS_KRYLOV_PCG;
    opt->restart = 50;
    opt->rtol = 1e-8;
    opt->maxit = 1000;
    opt->mem = HS_MEM_HOST;
    opt->stream = nullptr;
    opt->coords = nullptr;
    opt->coarse_dense = 4096;
    opt->fused_levels = 1;
    opt->record_ranks = 0;
    opt->rank_model = nullptr;
    return HS_OK;
}

static int partition_entry(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                           const double* coords, int32_t leaf_lines, double theta, int method, hs_tree* out) {
    if (!out) return HS_ERR_ARG;
    out->n_leaf = 0;
    out->perm = nullptr;
    out->leaf_ptr = nullptr;
    out->depth = 0;
    if (n <= 0 || n > INT32_MAX || !rowptr || !col || !val || leaf_lines <= 0) return HS_ERR_ARG;
    return run_guarded([&] {
        std::vector<int32_t> perm, lp;
        partition_impl(n, rowptr, col, val, coords, leaf_lines, theta, perm, lp, method);
        const int nleaf = (int)lp.size() - 1;
        out->perm = static_cast<int32_t*>(std::malloc(sizeof(int32_t) * n));
        out->leaf_ptr = static_cast<int32_t*>(std::malloc(sizeof(int32_t) * (nleaf + 1)));
        if (!out->perm || !out->leaf_ptr) {
            std::free(out->perm);
            std::free(out->leaf_ptr);
            out->perm = nullptr;
            out->leaf_ptr = nullptr;
            throw HsError{HS_ERR_OOM};
        }
        std::memcpy(out->perm, perm.data(), sizeof(int32_t) * n);
        std::memcpy(out->leaf_ptr, lp.data(), sizeof(int32_t) * (nleaf + 1));
        out->n_leaf = nleaf;
        int Lg = 0;
        while ((1 << (Lg + 1)) <= nleaf) Lg++;
        out->depth = std::max(nleaf >= 2 ? 1 : 0, Lg - 2);
    });
}

int hs_partition_extruded(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                          const double* coords, int32_t leaf_lines, double theta, hs_tree* out) {
    return partition_entry(n, rowptr, col, val, coords, leaf_lines, theta, kPartAuto, out);
}

int hs_partition_multilevel(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                            int32_t leaf_lines, double theta, hs_tree* out) {
    return partition_entry(n, rowptr, col, val, nullptr, leaf_lines, theta, kPartMultilevel, out);
}

int hs_tree_free(hs_tree* t) {
    if (!t) return HS_ERR_ARG;
    std::free(t->perm);
    std::free(t->leaf_ptr);
    t->perm = nullptr;
    t->leaf_ptr = nullptr;
    t->n_leaf = 0;
    return HS_OK;
}

int hs_plan_level(int32_t nc, const int64_t* adj_ptr, const int32_t* adj, const int32_t* size0, int32_t nranges,
                  const int32_t* ranges, int32_t* phase, int32_t* vanished, int64_t* end_ptr, int32_t* end_adj,
                  int64_t end_cap, int64_t* all_ptr, int32_t* all_adj, int64_t all_cap) {
    if (nc < 0 || !adj_ptr || !size0 || !phase || !vanished || !end_ptr || !all_ptr || nranges < 0)
        return HS_ERR_ARG;
    if (nranges > 0 && !ranges) return HS_ERR_ARG;
    return run_guarded([&] {
        if (adj_ptr[0] != 0) throw HsError{HS_ERR_ARG};
        for (int32_t c = 0; c < nc; c++)
            if (adj_ptr[c + 1] < adj_ptr[c] || size0[c] < 0) throw HsError{HS_ERR_ARG};
        if (adj_ptr[nc] > 0 && !adj) throw HsError{HS_ERR_ARG};
        LevelPlan P;
        P.nc = nc;
        P.size0.assign(size0, size0 + nc);
        for (int32_t c = 0; c < nc; c++) {
            // sorted, no self loop, in range
            for (int64_t e = adj_ptr[c]; e < adj_ptr[c + 1]; e++) {
                const int32_t q = adj[e];
                if (q < 0 || q >= nc || q == c || (e > adj_ptr[c] && adj[e - 1] >= q)) throw HsError{HS_ERR_ARG};
                // a cluster without DOFs has no blocks
                if (size0[c] == 0 || size0[q] == 0) throw HsError{HS_ERR_ARG};
            }
        }
        P.adj0.ptr.assign(adj_ptr, adj_ptr + nc + 1);
        P.adj0.idx.assign(adj, adj + adj_ptr[nc]);
        for (int32_t c = 0; c < nc; c++)  // symmetric
            for (int q : P.adj0[c]) {
                const auto r = P.adj0[q];
                if (!std::binary_search(r.begin(), r.end(), c)) throw HsError{HS_ERR_ARG};
            }
        std::vector<std::pair<int, int>> rg;
        if (nranges > 0) {
            // consecutive, covering [0, nc), no block between two ranges
            std::vector<int> range_of(nc, -1);
            int next = 0;
            for (int32_t k = 0; k < nranges; k++) {
                const int lo = ranges[2 * k], hi = ranges[2 * k + 1];
                if (lo != next || hi < lo || hi > nc) throw HsError{HS_ERR_ARG};
                for (int c2 = lo; c2 < hi; c2++) range_of[c2] = k;
                rg.push_back({lo, hi});
                next = hi;
            }
            if (next != nc) throw HsError{HS_ERR_ARG};
            for (int32_t c = 0; c < nc; c++)
                for (int q : P.adj0[c])
                    if (range_of[q] != range_of[c]) throw HsError{HS_ERR_ARG};
        }
        plan_level(P, rg);
        int64_t tot = 0, tota = 0;
        end_ptr[0] = 0;
        all_ptr[0] = 0;
        for (int32_t c = 0; c < nc; c++) {
            phase[c] = P.phase[c];
            vanished[c] = P.vanished[c] ? 1 : 0;
            tot += (int64_t)P.endp[c].size();
            end_ptr[c + 1] = tot;
            tota += (int64_t)P.all[c].size();
            all_ptr[c + 1] = tota;
        }
        if (end_adj) {
            if (end_cap < tot) throw HsError{HS_ERR_ARG};
            for (int32_t c = 0; c < nc; c++)
                std::copy(P.endp[c].begin(), P.endp[c].end(), end_adj + end_ptr[c]);
        }
        if (all_adj) {
            if (all_cap < tota) throw HsError{HS_ERR_ARG};
            for (int32_t c = 0; c < nc; c++)
                std::copy(P.all[c].begin(), P.all[c].end(), all_adj + all_ptr[c]);
        }
        release_plan(P);
    });
}

// the no-DC elimination serves neither the rank predictor nor its records
static int nodc_options_check(const hs_options* opt) {
    if (opt->no_dc != 0 && opt->no_dc != 1) return HS_ERR_ARG;
    if (opt->schur_products < 0 || opt->schur_products > 3) return HS_ERR_ARG;
    if (opt->partitioner != HS_PART_AUTO && opt->partitioner != HS_PART_MULTILEVEL) return HS_ERR_ARG;
    if (opt->no_dc && (opt->rank_model || opt->record_ranks)) return HS_ERR_UNSUPPORTED;
    return HS_OK;
}

int hs_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const hs_tree* tree,
             const hs_options* opt, hs_handle* out, hs_info* info) {
    if (!out) return HS_ERR_ARG;
    *out = nullptr;
    if (info) { std::memset(info, 0, sizeof(*info)); info->fail_level = -1; info->fail_cluster = -1; }
    if (n <= 0 || n > INT32_MAX || !rowptr || !col || !val || !opt) return HS_ERR_ARG;
    if (!(opt->tol >= 0.0) || opt->leaf_lines <= 0 || (opt->mem != HS_MEM_HOST && opt->mem != HS_MEM_DEVICE) ||
        (opt->precision != HS_PREC_FP64 && opt->precision != HS_PREC_MIXED))
        return HS_ERR_ARG;
    if (const int rc0 = nodc_options_check(opt)) return rc0;
    hs_factor_s* h = new (std::nothrow) hs_factor_s();
    if (!h) return HS_ERR_OOM;
    h->n = n;
    h->opt = *opt;
    h->st = static_cast<cudaStream_t>(opt->stream);
    h->prof.on = opt->profile != 0;
    h->fp32 = opt->precision == HS_PREC_MIXED ? 1 : 0;
    const double t0 = now_s();
    g_alloc_stream = h->st;
    prepare_pool();
    const int rc = run_guarded([&] {
        CK(cudaGetDevice(&h->device));
        setup_impl(h, rowptr, col, val, tree, info);
        h->prof.collect();
    });
    if (rc != HS_OK) {
        delete h;
        return rc;
    }
    if (info) {
        info->setup_s = now_s() - t0;
        info->factor_bytes = h->factor_bytes;
    }
    *out = h;
    return HS_OK;
}

int hs_setup_batched(int32_t nprob, const int64_t* prob_ptr, int64_t n, const int64_t* rowptr, const int32_t* col,
                     const double* val, const hs_options* opt, hs_handle* out, hs_info* info) {
    if (!out) return HS_ERR_ARG;
    *out = nullptr;
    if (info) { std::memset(info, 0, sizeof(*info)); info->fail_level = -1; info->fail_cluster = -1; }
    if (nprob <= 0 || nprob > 65535 || !prob_ptr || n <= 0 || n > INT32_MAX || !rowptr || !col || !val || !opt)
        return HS_ERR_ARG;
    if (prob_ptr[0] != 0 || prob_ptr[nprob] != n) return HS_ERR_ARG;
    for (int p = 0; p < nprob; p++)
        if (prob_ptr[p + 1] <= prob_ptr[p]) return HS_ERR_ARG;
    if (!(opt->tol >= 0.0) || opt->leaf_lines <= 0 || (opt->mem != HS_MEM_HOST && opt->mem != HS_MEM_DEVICE) ||
        (opt->precision != HS_PREC_FP64 && opt->precision != HS_PREC_MIXED))
        return HS_ERR_ARG;
    if (const int rc0 = nodc_options_check(opt)) return rc0;
    hs_factor_s* h = new (std::nothrow) hs_factor_s();
    if (!h) return HS_ERR_OOM;
    h->n = n;
    h->opt = *opt;
    h->st = static_cast<cudaStream_t>(opt->stream);
    h->prof.on = opt->profile != 0;
    h->fp32 = opt->precision == HS_PREC_MIXED ? 1 : 0;
    h->prob_ptr.assign(prob_ptr, prob_ptr + nprob + 1);
    for (int p = 0; p < nprob; p++) h->prob_maxlen = std::max(h->prob_maxlen, prob_ptr[p + 1] - prob_ptr[p]);
    const double t0 = now_s();
    g_alloc_stream = h->st;
    prepare_pool();
    const int rc = run_guarded([&] {
        CK(cudaGetDevice(&h->device));
        upload(h->d_pp, h->prob_ptr, h->st);
        setup_impl(h, rowptr, col, val, nullptr, info);
        h->prof.collect();
    });
    if (rc != HS_OK) {
        delete h;
        return rc;
    }
    if (info) {
        info->setup_s = now_s() - t0;
        info->factor_bytes = h->factor_bytes;
    }
    *out = h;
    return HS_OK;
}

int hs_krylov_batched(hs_handle h, const double* b, double* x, int32_t* iters, double* rel_resid, hs_info* info) {
    if (!h || !b || !x) return HS_ERR_ARG;
    if (h->prob_ptr.empty()) return HS_ERR_UNSUPPORTED;
    if (h->opt.krylov != HS_KRYLOV_PCG) return HS_ERR_UNSUPPORTED;
    hs_info tmp{};
    hs_info* inf = info ? info : &tmp;
    const double t0 = now_s();
    int krc = HS_OK;
    g_alloc_stream = h->st;
    const int rc = run_guarded([&] {
        krc = pcg_batched_impl(h, b, x, iters, rel_resid, inf);
        CK(cudaStreamSynchronize(h->st));
        h->prof.collect();
    });
    inf->solve_s = now_s() - t0;
    return rc != HS_OK ? rc : krc;
}

int hs_num_problems(hs_handle h, int32_t* nprob) {
    if (!h || !nprob) return HS_ERR_ARG;
    *nprob = h->prob_ptr.empty() ? 1 : (int32_t)h->prob_ptr.size() - 1;
    return HS_OK;
}

int hs_problem_info(hs_handle h, int32_t prob, int32_t* leaf_lo, int32_t* leaf_hi, int32_t* depth, int32_t* ntop) {
    if (!h || prob < 0 || prob >= (int32_t)h->groups.size()) return HS_ERR_ARG;
    const auto& G = h->groups[prob];
    if (leaf_lo) *leaf_lo = (int32_t)G.leaf_lo;
    if (leaf_hi) *leaf_hi = (int32_t)G.leaf_hi;
    if (depth) *depth = G.depth;
    if (ntop) {
        *ntop = 0;
        for (const TopDev& t : h->tops)
            if (t.pad == prob) *ntop = t.n;
    }
    return HS_OK;
}

int hs_apply(hs_handle h, const double* r, double* z) {
    if (!h || !r || !z || r == z) return HS_ERR_ARG;
    return run_guarded([&] { apply_impl(h, r, z); });
}

int hs_krylov(hs_handle h, const double* b, double* x, hs_info* info) {
    if (!h || !b || !x) return HS_ERR_ARG;
    hs_info tmp{};
    hs_info* inf = info ? info : &tmp;
    const double t0 = now_s();
    int krc = HS_OK;
    g_alloc_stream = h->st;
    const int rc = run_guarded([&] {
        if (!h->prob_ptr.empty())
            krc = h->opt.krylov == HS_KRYLOV_PCG ? pcg_batched_impl(h, b, x, nullptr, nullptr, inf)
                                                 : (int)HS_ERR_UNSUPPORTED;
        else
            krc = h->opt.krylov == HS_KRYLOV_GMRES ? gmres_impl(h, b, x, inf) : pcg_impl(h, b, x, inf);
        CK(cudaStreamSynchronize(h->st));
        h->prof.collect();
    });
    inf->solve_s = now_s() - t0;
    return rc != HS_OK ? rc : krc;
}

int hs_krylov_noalloc(hs_handle h, const double* b, double* x, hs_info* info) {
    if (!h || !b || !x) return HS_ERR_ARG;
    if (h->n > kNoAllocMaxN) return HS_ERR_ARG;               // beyond the fixed scratch
    // one PCG over one operator: GMRES handles and batched handles (whose
    // problems stop one by one) are not served
    if (h->opt.krylov != HS_KRYLOV_PCG || !h->prob_ptr.empty()) return HS_ERR_UNSUPPORTED;
    {
        // the scratch address is looked up on the current device, which must
        // be the one the handle's factor and stream live on
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) return HS_ERR_ARG;
    }
    hs_info tmp{};
    hs_info* inf = info ? info : &tmp;
    const double t0 = now_s();
    int krc = HS_OK;
    const int rc = run_guarded([&] {
        double* scratch = nullptr;
        CK(noalloc_scratch(&scratch));
        krc = pcg_noalloc(h, b, x, scratch, inf);
        CK(cudaStreamSynchronize(h->st));
    });
    inf->solve_s = now_s() - t0;
    return rc != HS_OK ? rc : krc;
}

int hs_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* b, double* x,
             const hs_options* opt, hs_info* info) {
    if (!opt || !b || !x) return HS_ERR_ARG;
    hs_info tmp{};
    hs_info* inf = info ? info : &tmp;
    hs_handle h = nullptr;
    int rc = hs_setup(n, rowptr, col, val, nullptr, opt, &h, inf);
    if (rc != HS_OK) return rc;
    const double t0 = now_s();
    rc = run_guarded([&] {
        cudaStream_t st = h->st;
        if (opt->mem == HS_MEM_DEVICE) {
            const int krc = hs_krylov(h, b, x, inf);
            if (krc != HS_OK) throw HsError{krc};
        } else {
            g_alloc_stream = h->st;
            DBuf db, dx;
            db.alloc(sizeof(double) * n);
            dx.alloc(sizeof(double) * n);
            CK(cudaMemcpyAsync(db.p, b, sizeof(double) * n, cudaMemcpyHostToDevice, st));
            const int krc = hs_krylov(h, db.as<double>(), dx.as<double>(), inf);
            CK(cudaMemcpyAsync(x, dx.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (krc != HS_OK) throw HsError{krc};
        }
    });
    inf->solve_s = now_s() - t0;
    hs_destroy(h);
    return rc;
}

int hs_destroy(hs_handle h) {
    if (!h) return HS_OK;
    g_alloc_stream = h->st;
    cudaStreamSynchronize(h->st);  // no pending apply may still use the graph
    delete h;                      // frees are ordered on the handle's stream
    return HS_OK;
}

int hs_num_levels(hs_handle h, int32_t* levels) {
    if (!h || !levels) return HS_ERR_ARG;
    *levels = (int32_t)h->lev.size();
    return HS_OK;
}

int hs_level_clusters(hs_handle h, int32_t level, int32_t* nc) {
    if (!h || !nc || level < 0 || level >= (int32_t)h->lev.size()) return HS_ERR_ARG;
    *nc = h->lev[level]->nc;
    return HS_OK;
}

int hs_level_info(hs_handle h, int32_t level, int32_t* size0, int32_t* final_size, int32_t* phase) {
    if (!h || level < 0 || level >= (int32_t)h->lev.size()) return HS_ERR_ARG;
    const Level& L = *h->lev[level];
    for (int c = 0; c < L.nc; c++) {
        if (size0) size0[c] = L.size0[c];
        if (final_size) final_size[c] = L.fin[c];
        if (phase) phase[c] = L.phase[c];
    }
    return HS_OK;
}

int hs_top_size(hs_handle h, int32_t* ntop) {
    if (!h || !ntop) return HS_ERR_ARG;
    *ntop = h->ntop;
    return HS_OK;
}

int hs_kernel_stats(hs_handle h, int32_t nclasses, double* times_ms, int64_t* launches, double* flops64,
                    double* flops32, double* bytes) {
    if (!h || nclasses < 0) return HS_ERR_ARG;
    for (int k = 0; k < nclasses; k++) {
        const bool ok = k < KC_N;
        if (times_ms) times_ms[k] = ok ? h->prof.ms[k] : 0.0;
        if (launches) launches[k] = ok ? h->prof.launches[k] : 0;
        if (flops64) flops64[k] = ok ? h->work_flops[k] : 0.0;
        if (flops32) flops32[k] = ok ? h->work_flops32[k] : 0.0;
        if (bytes) bytes[k] = ok ? h->work_bytes[k] : 0.0;
    }
    return HS_OK;
}

int hs_reset_kernel_stats(hs_handle h) {
    if (!h) return HS_ERR_ARG;
    h->prof.reset();
    return HS_OK;
}

int hs_rank_samples(hs_handle h, float* feat, int32_t* rank, int32_t* size, int64_t* count) {
    if (!h || !count) return HS_ERR_ARG;
    int64_t k = 0;
    for (auto& Lp : h->lev) k += (int64_t)Lp->tasks.size();
    if (!feat) {
        *count = h->opt.record_ranks ? k : 0;
        return HS_OK;
    }
    if (!h->opt.record_ranks || !rank || !size) return HS_ERR_ARG;
    return run_guarded([&] {
        g_alloc_stream = h->st;
        int64_t o = 0;
        for (auto& Lp : h->lev) {
            const Level& L = *Lp;
            const int nt = (int)L.tasks.size();
            if (nt == 0) continue;
            CK(cudaMemcpyAsync(feat + o * kFeat, L.d_feat.p, sizeof(float) * kFeat * nt, cudaMemcpyDeviceToHost, h->st));
            for (int ti = 0; ti < nt; ti++) {
                rank[o + ti] = L.task_rank[ti];
                size[o + ti] = L.tasks[ti].s;
            }
            o += nt;
        }
        CK(cudaStreamSynchronize(h->st));
        *count = o;
    });
}

int hs_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream) {
    if (!params || n < 0 || (n > 0 && (!x || !y))) return HS_ERR_ARG;
    return run_guarded([&] { CK(launch_mlp_forward(static_cast<cudaStream_t>(stream), params, x, n, y)); });
}

int hs_mlp_grad(const float* params, const float* x, const float* t, const int32_t* idx, int32_t batch,
                float* grad, float* loss, void* stream) {
    if (!params || !x || !t || !grad || !loss || batch < 1 || batch > kMlpMaxBatch) return HS_ERR_ARG;
    return run_guarded(
        [&] { CK(launch_mlp_grad(static_cast<cudaStream_t>(stream), params, x, t, idx, batch, grad, loss)); });
}

int hs_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr, void* stream) {
    if (!params || !grad || !m || !v || step < 1) return HS_ERR_ARG;
    return run_guarded([&] { CK(launch_mlp_adam(static_cast<cudaStream_t>(stream), params, grad, m, v, step, lr)); });
}

int hs_mlp_train(float* params, const float* x, const float* t, int64_t n, const int32_t* order, int64_t nsteps,
                 int32_t batch, float lr, float* losses, void* stream) {
    if (!params || !x || !t || n <= 0 || !order || nsteps < 0 || batch < 1 || batch > kMlpMaxBatch)
        return HS_ERR_ARG;
    for (int64_t i = 0; i < nsteps * batch; i++)
        if (order[i] < 0 || order[i] >= n) return HS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return run_guarded([&] {
        g_alloc_stream = st;
        DBuf d_th, d_x, d_t, d_ord, d_g, d_m, d_v, d_loss;
        d_th.alloc(sizeof(float) * kMlpParams);
        d_x.alloc(sizeof(float) * n * kMlpIn);
        d_t.alloc(sizeof(float) * n);
        d_ord.alloc(sizeof(int32_t) * std::max<int64_t>(nsteps * batch, 1));
        d_g.alloc(sizeof(float) * kMlpParams);
        d_m.alloc(sizeof(float) * kMlpParams);
        d_v.alloc(sizeof(float) * kMlpParams);
        d_loss.alloc(sizeof(float) * std::max<int64_t>(nsteps, 1));
        CK(cudaMemcpyAsync(d_th.p, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_x.p, x, sizeof(float) * n * kMlpIn, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_t.p, t, sizeof(float) * n, cudaMemcpyHostToDevice, st));
        if (nsteps > 0)
            CK(cudaMemcpyAsync(d_ord.p, order, sizeof(int32_t) * nsteps * batch, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(d_m.p, 0, sizeof(float) * kMlpParams, st));
        CK(cudaMemsetAsync(d_v.p, 0, sizeof(float) * kMlpParams, st));
        for (int64_t k = 0; k < nsteps; k++) {
            CK(launch_mlp_grad(st, d_th.as<float>(), d_x.as<float>(), d_t.as<float>(), d_ord.as<int32_t>() + k * batch,
                               batch, d_g.as<float>(), d_loss.as<float>() + k));
            CK(launch_mlp_adam(st, d_th.as<float>(), d_g.as<float>(), d_m.as<float>(), d_v.as<float>(), (int)(k + 1),
                               lr));
        }
        CK(cudaMemcpyAsync(params, d_th.p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, st));
        if (losses && nsteps > 0)
            CK(cudaMemcpyAsync(losses, d_loss.p, sizeof(float) * nsteps, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    });
}

int hs_launch_count(int64_t* count) {
    if (!count) return HS_ERR_ARG;
    *count = launch_count();
    return HS_OK;
}

int hs_eval_pivot_reciprocals(int64_t n, const double* x, double* rsqrt_out, double* rcp_out, void* stream) {
    if (n < 0 || (n > 0 && (!x || !rsqrt_out || !rcp_out))) return HS_ERR_ARG;
    return run_guarded([&] {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        CK(launch_eval_recip(st, n, x, rsqrt_out, rcp_out));
        CK(cudaStreamSynchronize(st));
    });
}

// FMA throughput of the current device, FP64 (fp32 = 0) or FP32 pipe
static int measure_fma_peak(void* stream, double* tflops, int fp32) {
    if (!tflops) return HS_ERR_ARG;
    return run_guarded([&] {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        DBuf sink;
        sink.alloc(64);
        const int blocks = sms * 8, iters = fp32 ? 1 << 16 : 1 << 14;
        auto launch = [&](int it) {
            return fp32 ? launch_fp32_peak(st, blocks, it, sink.as<double>())
                        : launch_fp64_peak(st, blocks, it, sink.as<double>());
        };
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(launch(256));  // warm-up
        CK(cudaEventRecord(a, st));
        CK(launch(iters));
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        *tflops = 2.0 * 8.0 * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
    });
}

int hs_measure_fp64_peak(void* stream, double* tflops) { return measure_fma_peak(stream, tflops, 0); }

int hs_measure_fp32_peak(void* stream, double* tflops) { return measure_fma_peak(stream, tflops, 1); }

const char* hs_status_str(int status) {
    switch (status) {
        case HS_OK: return "ok";
        case HS_ERR_ARG: return "invalid argument";
        case HS_ERR_NOT_SPD: return "diagonal block not positive definite";
        case HS_ERR_NOCONV: return "Krylov solver did not converge";
        case HS_ERR_CUDA: return "CUDA error";
        case HS_ERR_OOM: return "out of device memory";
        case HS_ERR_UNSUPPORTED: return "block size beyond kernel limits";
        case HS_ERR_TIMEOUT: return "bounded device wait timed out";
        default: return "unknown status";
    }
}

}  // extern "C"
