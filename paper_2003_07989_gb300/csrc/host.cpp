// host.cpp -- H0 by Kruskal's union-find (Sec. "Zero-Dimensional Persistence
// Computation: Kruskal's Algorithm"), the submatrix reduction of the columns
// that are not apparent (Sec. "Core System Optimizations": the two-layer pair
// store; Sec. "Reduction Matrix vs. Oblivious Matrix Reduction"), and helpers
// for barcode assembly.
#include "host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

namespace rpp {

void decode_host(const Binomial &B, uint64_t c, int p, int64_t n, int *v) {
    int hi = (int)n - 1;
    for (int i = 0; i <= p; ++i) {
        const int k = p + 1 - i;
        int lo = k - 1, h = hi;
        while (lo < h) {
            int mid = (lo + h + 1) >> 1;
            if (B.at(k, mid) <= c) lo = mid;
            else h = mid - 1;
        }
        v[i] = lo;
        c -= B.at(k, lo);
        hi = lo - 1;
    }
}

void youngest_edge(const HostInstance &I, const int *v, int k, int32_t *u, int32_t *w) {
    float best = -1.0f;
    uint64_t best_idx = 0;
    *u = *w = -1;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            const int x = std::max(v[a], v[b]), y = std::min(v[a], v[b]);
            const float d = I.dist(x, y);
            const uint64_t idx = (uint64_t)x * (uint64_t)(x - 1) / 2 + (uint64_t)y;
            if (d > best || (d == best && idx < best_idx)) {
                best = d;
                best_idx = idx;
                *u = x;
                *w = y;
            }
        }
}

// ---------------------------------------------------------------------------
// Kruskal

void Kruskal::init(int64_t n) {
    parent.resize(n);
    size_.assign(n, 1);
    for (int64_t i = 0; i < n; ++i) parent[i] = (int32_t)i;
    components = n;
    deaths.clear();
    mst_pos.clear();
}

int32_t Kruskal::find(int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

void Kruskal::run(const uint32_t *hi, const uint64_t *lo, int64_t count, int64_t pos0,
                  const Binomial &B, int64_t n) {
    int v[2];
    for (int64_t k = 0; k < count && components > 1; ++k) {
        decode_host(B, lo[k], 1, n, v);
        int32_t a = find(v[0]), b = find(v[1]);
        if (a == b) continue;
        if (size_[a] < size_[b]) std::swap(a, b);
        parent[b] = a;
        size_[a] += size_[b];
        --components;
        HostPair P;
        P.sigma = 0;
        P.tau = lo[k];
        P.birth = 0.0f;
        uint32_t bits = ~hi[k];
        std::memcpy(&P.death, &bits, sizeof(float));
        deaths.push_back(P);
        mst_pos.push_back((uint32_t)(pos0 - k));
    }
}

// ---------------------------------------------------------------------------
// pair store

int PairStore::lookup(uint64_t tau, uint64_t *sigma, int64_t *slot) {
    ++reads;
    auto it = reduced.find(tau);
    if (it != reduced.end()) {
        *slot = it->second;
        return 2;
    }
    const uint64_t *e = app_tau + napp;
    const uint64_t *f = std::lower_bound(app_tau, e, tau);
    if (f != e && *f == tau) {
        *sigma = app_sigma[f - app_tau];
        return 1;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// submatrix reduction

namespace {

// A column entry packed so that unsigned 128-bit order is "older first":
// smaller diameter first, then larger index (the simplex-wise refinement).
typedef unsigned __int128 entry;

inline entry make_entry(float diam, uint64_t idx) {
    uint32_t bits;
    std::memcpy(&bits, &diam, sizeof(float));
    return ((entry)bits << 64) | (entry)(~idx);
}
inline uint64_t entry_index(entry e) { return ~(uint64_t)e; }
inline float entry_diam(entry e) {
    uint32_t bits = (uint32_t)(e >> 64);
    float d;
    std::memcpy(&d, &bits, sizeof(float));
    return d;
}

// Working column: a min-heap with repetitions; an entry present an even number
// of times is zero over Z/2 and cancels when it reaches the top.
struct WorkColumn {
    std::vector<entry> h;
    void push(entry e) {
        h.push_back(e);
        std::push_heap(h.begin(), h.end(), std::greater<entry>());
    }
    entry pop() {
        std::pop_heap(h.begin(), h.end(), std::greater<entry>());
        entry e = h.back();
        h.pop_back();
        return e;
    }
    // Oldest nonzero entry (kept in the column); false if the sum is zero.
    bool low(entry *out) {
        while (!h.empty()) {
            entry e = pop();
            if (!h.empty() && h.front() == e) {
                pop();
                continue;
            }
            push(e);
            *out = e;
            return true;
        }
        return false;
    }
    // Remaining nonzero entries, each once, oldest first.
    void drain(std::vector<entry> &out) {
        entry e;
        while (low(&e)) {
            pop();
            out.push_back(e);
        }
    }
};

// Push the coboundary of the p-simplex v (diameter d) restricted to diam <= t.
void push_coboundary(const HostInstance &I, int p, const int *v, float d, WorkColumn &W) {
    const Binomial &B = *I.B;
    // For w from n-1 down: j = number of vertices of v above w. The cofacet
    // index is sum_{i<j} C(v_i, p+2-i) + C(w, p+2-j) + sum_{i>=j} C(v_i, p+1-i).
    uint64_t high = 0, low = 0;
    for (int i = 0; i <= p; ++i) low += B.at(p + 1 - i, v[i]);
    int j = 0;
    for (int64_t w = I.n - 1; w >= 0; --w) {
        if (j <= p && w == v[j]) {
            high += B.at(p + 2 - j, v[j]);
            low -= B.at(p + 1 - j, v[j]);
            ++j;
            continue;
        }
        float cd = d;
        for (int i = 0; i <= p; ++i) cd = std::max(cd, I.dist(v[i], (int)w));
        if (cd > I.t) continue;
        W.push(make_entry(cd, high + B.at(p + 2 - j, w) + low));
    }
}

}  // namespace

void reduce_leftovers(const HostInstance &I, int p, const Leftover *left, int64_t nleft,
                      PairStore &store, std::vector<HostPair> &out, ReduceStats &stats) {
    std::vector<std::vector<entry>> stored(nleft);
    WorkColumn W;
    int v[RPP_MAX_DIM + 2];
    for (int64_t j = 0; j < nleft; ++j) {
        const Leftover &L = left[j];
        HostPair P;
        P.sigma = L.sigma;
        P.birth = L.diam;
        if (L.pivot == NO_PIVOT) {  // empty coboundary: an essential class
            P.tau = NO_PIVOT;
            P.death = INFINITY;
            out.push_back(P);
            continue;
        }
        uint64_t osig;
        int64_t oslot;
        if (store.lookup(L.pivot, &osig, &oslot) == 0) {  // nobody owns the pivot
            ++stats.free_pivot;
            store.reduced[L.pivot] = j;
            P.tau = L.pivot;
            P.death = L.pdiam;
            out.push_back(P);
            continue;
        }
        W.h.clear();
        decode_host(*I.B, L.sigma, p, I.n, v);
        push_coboundary(I, p, v, L.diam, W);
        entry e;
        bool nonzero;
        while ((nonzero = W.low(&e))) {
            const uint64_t tau = entry_index(e);
            const int kind = store.lookup(tau, &osig, &oslot);
            if (kind == 0) break;
            ++stats.additions;
            if (kind == 1) {  // apparent owner: its column is its coboundary
                decode_host(*I.B, osig, p, I.n, v);
                push_coboundary(I, p, v, entry_diam(e), W);
            } else if (!stored[oslot].empty()) {
                for (entry x : stored[oslot]) W.push(x);
            } else {
                const Leftover &O = left[oslot];
                decode_host(*I.B, O.sigma, p, I.n, v);
                push_coboundary(I, p, v, O.diam, W);
            }
        }
        if (nonzero) {
            const uint64_t tau = entry_index(e);
            store.reduced[tau] = j;
            P.tau = tau;
            P.death = entry_diam(e);
            out.push_back(P);
            W.drain(stored[j]);  // the reduced column, for later additions
        } else {
            P.tau = NO_PIVOT;
            P.death = INFINITY;
            out.push_back(P);
        }
    }
    stats.reads += store.reads;
}

}  // namespace rpp
