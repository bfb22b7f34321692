// col_heap.h -- the ordered set of cursor heads of one working column in
// the host reduction of dimensions p >= 2 (the submatrix reduction of Alg. 1
// over lazily listed coboundaries). Separate from host.cpp so that a CPU test
// can exercise it alone.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <functional>
#include <memory>
#include <utility>
#include <vector>

namespace rpp {

typedef unsigned __int128 u128;

typedef std::greater<std::pair<u128, int32_t>> HeapCmp;

// The heads of a column's cursors, oldest first: a binary heap while small;
// past RADIX_AT entries (the long walks) a radix heap over the 128-bit keys,
// whose pushes are O(1). A radix heap needs every key pushed to be at least
// the last one taken out; pivot() and add_cursor's floor keep that.
struct ColHeap {
    typedef std::pair<u128, int32_t> E;
    static constexpr size_t RADIX_AT = 1024;
    struct Radix {
        std::vector<E> b[129];  // b[i]: keys whose highest bit differing from `last` is i - 1
        u128 last = 0;
        size_t size = 0;
    };
    std::vector<E> bin;
    std::unique_ptr<Radix> rad;

    static int bucket(u128 k, u128 last) {
        const u128 x = k ^ last;
        if (!x) return 0;
        const uint64_t hi = (uint64_t)(x >> 64), lo = (uint64_t)x;
        return hi ? 128 - __builtin_clzll(hi) : 64 - __builtin_clzll(lo);
    }
    bool empty() const { return rad ? rad->size == 0 : bin.empty(); }
    void push(E e) {
        if (rad) {
            rad->b[bucket(e.first, rad->last)].push_back(e);
            ++rad->size;
            return;
        }
        bin.push_back(e);
        std::push_heap(bin.begin(), bin.end(), HeapCmp());
        if (bin.size() > RADIX_AT) {  // every key is at least the smallest
            rad.reset(new Radix());
            rad->last = bin.front().first;
            for (const E &x : bin) rad->b[bucket(x.first, rad->last)].push_back(x);
            rad->size = bin.size();
            std::vector<E>().swap(bin);
        }
    }
    E top() {  // requires !empty()
        if (!rad) return bin.front();
        if (rad->b[0].empty()) {  // the next smallest key becomes `last`
            int i = 1;
            while (rad->b[i].empty()) ++i;
            u128 m = rad->b[i][0].first;
            for (const E &x : rad->b[i]) m = std::min(m, x.first);
            rad->last = m;
            std::vector<E> moved;
            moved.swap(rad->b[i]);
            for (const E &x : moved) rad->b[bucket(x.first, m)].push_back(x);
        }
        return rad->b[0].back();
    }
    void pop() {  // removes what top() returned
        if (rad) {
            rad->b[0].pop_back();
            --rad->size;
            return;
        }
        std::pop_heap(bin.begin(), bin.end(), HeapCmp());
        bin.pop_back();
    }
    // Does another entry carry top()'s key? Nothing is removed, so `last`
    // stays at that key. (A binary heap's second smallest entry is a child of
    // its root; in a radix heap every entry equal to `last` is in b[0].)
    bool top_twice() {  // requires !empty()
        if (rad) {
            top();
            return rad->b[0].size() >= 2;
        }
        if (bin.size() < 2) return false;
        const u128 k = bin.front().first;
        return bin[1].first == k || (bin.size() > 2 && bin[2].first == k);
    }
    void release() {
        std::vector<E>().swap(bin);
        rad.reset();
    }
};

}  // namespace rpp
