// Test harness for the host reduction's column heap (csrc/col_heap.h)
// without a GPU: random walks of lazily listed columns, the heap against an
// ordered multiset. A working column is the Z/2 sum of cursors that list
// increasing keys; its pivot is the smallest key left once equal keys cancel
// in pairs. Each step takes the pivot, then adds either one cursor starting
// at it (an apparent owner's coboundary) or an odd number of cursors whose
// entries below it are skipped (another column's reduced column, whose
// entries below its pivot sum to zero); either way the pivot cancels. The
// pivot sequences and the counts of cancelled entries must agree, with the
// heap past its switch to the radix form. Test code only.
//
//   col_heap_harness trials        exit 0 and "all ok" on success
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>

#include "col_heap.h"

using rpp::ColHeap;
using rpp::u128;

static const u128 NONE = ~(u128)0;

struct RefHeap {  // ordered multiset
    typedef std::pair<u128, int32_t> E;
    std::multiset<E> s;
    bool empty() const { return s.empty(); }
    void push(E e) { s.insert(e); }
    E top() { return *s.begin(); }
    void pop() { s.erase(s.begin()); }
    bool top_twice() {
        auto it = s.begin();
        const u128 k = it->first;
        ++it;
        return it != s.end() && it->first == k;
    }
};

struct Cur {
    std::vector<u128> keys;
    size_t pos = 0;
    u128 head() const { return pos < keys.size() ? keys[pos] : NONE; }
};

// The walk's pivot step (as in csrc/host.cpp): equal heads cancel in pairs,
// both cursors advance; the pivot itself stays in the heap.
template <class H>
u128 pivot(H &h, std::vector<Cur> &cur, long long &entries) {
    while (!h.empty()) {
        const auto a = h.top();
        if (h.top_twice()) {
            h.pop();
            const auto b = h.top();
            h.pop();
            if (b.first != a.first) return NONE - 1;  // reported as a mismatch
            entries += 2;
            for (int ci : {a.second, b.second}) {
                cur[ci].pos++;
                if (cur[ci].head() != NONE) h.push({cur[ci].head(), ci});
            }
            continue;
        }
        return a.first;
    }
    return NONE;
}

static u128 key(uint32_t d, uint64_t idx) { return ((u128)d << 64) | (u128)(~idx); }

int main(int argc, char **argv) {
    const int trials = argc > 1 ? std::atoi(argv[1]) : 100;
    for (int trial = 0; trial < trials; ++trial) {
        std::mt19937_64 rng(trial);
        std::vector<Cur> c1, c2;
        ColHeap h1;
        RefHeap h2;
        long long e1 = 0, e2 = 0;
        auto make_cursor = [&](u128 lo, bool first_is_lo, u128 floor) {
            Cur c;
            u128 k = lo;
            if (first_is_lo) c.keys.push_back(k);
            const int len = 1 + (int)(rng() % 40);
            for (int i = 0; i < len; ++i) {
                const u128 gap = rng() % 3 == 0 ? (u128)(rng() % ((uint64_t)1 << (rng() % 60)))
                                                : (u128)(rng() % 8);
                k = k + 1 + gap;
                c.keys.push_back(k);
            }
            while (c.head() != NONE && c.head() < floor) c.pos++;
            return c;
        };
        int ncur = 0;
        auto add = [&](const Cur &c) {
            c1.push_back(c);
            c2.push_back(c);
            if (c.head() != NONE) {
                h1.push({c.head(), ncur});
                h2.push({c.head(), ncur});
            }
            ++ncur;
        };
        const u128 base = key(1000, 5000);
        const int start = 3 + (int)(rng() % 5);
        for (int i = 0; i < start; ++i) add(make_cursor(base + rng() % 50, true, 0));
        int steps = 0;
        bool radix_seen = false;
        for (;;) {
            const u128 p1 = pivot(h1, c1, e1), p2 = pivot(h2, c2, e2);
            if (p1 != p2) {
                std::printf("trial %d step %d: pivots differ\n", trial, steps);
                return 1;
            }
            radix_seen |= h1.rad != nullptr;
            if (p1 == NONE || steps >= 3000) break;
            ++steps;
            const int n = (rng() % 2) ? 1 : 1 + 2 * (int)(rng() % 20);
            add(make_cursor(p1, true, p1));
            for (int i = 1; i < n; ++i) add(make_cursor(p1 - (rng() % 100), rng() % 2, p1));
        }
        if (e1 != e2) {
            std::printf("trial %d: cancelled entries differ\n", trial);
            return 1;
        }
        if (!radix_seen) {
            std::printf("trial %d: the heap never switched to its radix form\n", trial);
            return 1;
        }
    }
    std::printf("all ok\n");
    return 0;
}
