// host.cpp -- the submatrix reduction of the columns that are not apparent
// (Sec. "Core System Optimizations"; Alg. 1 with the reduction-matrix
// technique of Sec. "Reduction Matrix vs. Oblivious Matrix Reduction").
//
// Reduction of one leftover column j follows Alg. 1: while the pivot (oldest
// nonzero entry) of the working column has an owner, add the owner's reduced
// column. Almost every owner is an apparent column, whose reduced column is
// its plain coboundary; only rarely is it another leftover column.
//   Dimension 1: every leftover column walks in its own thread, through
//     apparent owners and through earlier leftover columns once these are
//     finished; a pivot that no finished column owns is kept only when every
//     unfinished earlier column has moved past it (see Ledger).
//   Dimensions p >= 2: Phase A (in parallel over columns) walks through
//     apparent owners only, stopping at the first pivot that no apparent
//     column owns; Phase B (in column order) adds earlier leftover columns
//     where that pivot belongs to one and continues the walk.
// Both add exactly the columns Alg. 1 adds, in the same order. A reduced
// column is kept as the set V of simplices whose coboundaries it sums.
//
// The working column is a heap of lazy cursors, one per added coboundary.
// Each cursor lists its cofacets oldest first (smallest diameter, then largest
// index) without materialising them: first the cofacets of equal diameter
// (vertices w, largest first, with every distance to the simplex <= its
// diameter), then the others by a (p+1)-way merge of the vertices' neighbour
// lists sorted by distance, where a vertex is emitted at its last occurrence,
// whose distance is the cofacet's diameter.
//   Dimensions p >= 2: equal entries from two cursors cancel over Z/2 when they
//     meet at the top of the heap.
//   Dimension 1 (edges): the parity of a triangle (how many of its edges lie
//     in V) is read from V's adjacency bits when a cursor reaches it, so even
//     entries are skipped on the spot and never enter the heap.
#include "host.h"
#include "col_heap.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <type_traits>

static_assert(__BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__, "lune_word packs bytes little-endian");

namespace rpp {

// ---------------------------------------------------------------------------
// A persistent pool of host threads shared by every reduction of the process.
// parallel_for may be called from several threads at once; the caller works
// on its own job too, so a job always makes progress.

namespace {

class Pool {
  public:
    struct Job {
        std::function<void(int64_t)> fn;
        int64_t count = 0;
        std::atomic<int64_t> next{0}, done{0};
        std::mutex m;
        std::condition_variable cv;
    };

    explicit Pool(int workers) {
        for (int i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }

    void parallel_for(int64_t count, const std::function<void(int64_t)> &fn) {
        auto job = std::make_shared<Job>();
        job->fn = fn;
        job->count = count;
        {
            std::lock_guard<std::mutex> g(mu_);
            jobs_.push_back(job);
        }
        cv_.notify_all();
        work(*job);
        std::unique_lock<std::mutex> g(job->m);
        job->cv.wait(g, [&] { return job->done.load() == job->count; });
    }

  private:
    static void work(Job &j) {
        for (;;) {
            const int64_t i = j.next.fetch_add(1);
            if (i >= j.count) return;
            j.fn(i);
            if (j.done.fetch_add(1) + 1 == j.count) {
                std::lock_guard<std::mutex> g(j.m);
                j.cv.notify_all();
            }
        }
    }
    void loop() {
        for (;;) {
            std::shared_ptr<Job> job;
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_.wait(g, [&] { return stop_ || !jobs_.empty(); });
                if (stop_) return;
                job = jobs_.front();
                if (job->next.load() >= job->count) {  // exhausted: retire it
                    jobs_.pop_front();
                    continue;
                }
            }
            work(*job);
        }
    }
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<std::shared_ptr<Job>> jobs_;
    std::vector<std::thread> th_;
    bool stop_ = false;
};

Pool &pool(int threads) {
    static Pool p(std::max(0, threads - 1));
    return p;
}

}  // namespace

void parallel_for(int threads, int64_t count, const std::function<void(int64_t)> &fn) {
    if (threads <= 1 || count < 2) {
        for (int64_t i = 0; i < count; ++i) fn(i);
        return;
    }
    pool(threads).parallel_for(count, fn);
}

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

uint64_t index_host(const Binomial &B, const int *v, int p) {
    uint64_t c = 0;
    for (int i = 0; i <= p; ++i) c += B.at(p + 1 - i, v[i]);
    return c;
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
// submatrix reduction

namespace {

// Column entries packed so that unsigned 128-bit order is "older first":
// smaller diameter, then larger index (the simplex-wise refinement); u128 is
// col_heap.h's.
const u128 NONE = ~(u128)0;

inline u128 age_key(float diam, uint64_t idx) {
    uint32_t bits;
    std::memcpy(&bits, &diam, sizeof(float));
    return ((u128)bits << 64) | (u128)(~idx);
}
inline uint64_t key_index(u128 k) { return ~(uint64_t)k; }
inline float key_diam(u128 k) {
    uint32_t bits = (uint32_t)(k >> 64);
    float d;
    std::memcpy(&d, &bits, sizeof(float));
    return d;
}
inline uint32_t float_bits(float f) {
    uint32_t b;
    std::memcpy(&b, &f, sizeof(float));
    return b;
}
inline float bits_float(uint32_t b) {
    float f;
    std::memcpy(&f, &b, sizeof(float));
    return f;
}

// Index of the cofacet v + {w} of the p-simplex v[0] > ... > v[p].
inline uint64_t cofacet_idx(const Binomial &B, const int *v, int p, int w) {
    uint64_t c = 0;
    int k = p + 2;
    bool placed = false;
    for (int i = 0; i <= p; ++i) {
        if (!placed && w > v[i]) {
            c += B.at(k--, w);
            placed = true;
        }
        c += B.at(k--, v[i]);
    }
    if (!placed) c += B.at(1, w);
    return c;
}

struct Cursor {
    int v[RPP_MAX_DIM + 1];
    float d = 0.0f;
    int32_t lune = -1;
    bool merging = false;       // merge positions set up
    int32_t pos[RPP_MAX_DIM + 1];
    std::vector<int32_t> ties;  // equal-key emissions, largest vertex at the back
    float tie_key = 0.0f;
    u128 head = NONE;
};

// Index over the sorted apparent taus: every STRIDE-th key, searched first.
constexpr int64_t STRIDE = 64;

// The edges {a, b} (a > b) of diameter in [from, threshold] in coboundary
// order (diameter descending, index ascending), packed as the GPU path hands
// them over: ab = (a << 16) | b and hi = ~bits(diameter), at position
// m - 1 - f for filtration position f. One 64-bit key per edge,
// (bits(diameter) - bits(from), ~a, ~b) with a and b in w bits each, orders
// the edges into filtration order (diameter ascending; on ties the index
// descends with (a, b)). The keys are written straight into up to 2048
// buckets by their top bits (two passes over the distance rows: count, then
// place); a bucket is sorted only when a sweep first reaches it, so a short
// sweep pays for little more than the partition.
struct EdgeList {
    float from = 0.0f;
    int w = 1, sh = 0;
    uint64_t vmax = 1, kmax = 0;  // kmax: no key exceeds it
    uint32_t base = 0;
    int64_t m = 0;
    mutable std::unique_ptr<uint64_t[]> key;  // by bucket; a bucket sorted once done
    std::vector<int64_t> bstart;              // bucket i: positions [bstart[i], bstart[i + 1])
    mutable std::unique_ptr<uint32_t[]> ab, hi;
    std::unique_ptr<std::atomic<uint8_t>[]> done;
    mutable std::mutex mu;

    int nbuckets() const { return (int)bstart.size() - 1; }
    int bucket_of(uint64_t k) const { return (int)(k >> sh); }

    // Sort bucket i and fill its positions of ab and hi (once).
    void ensure(int i) const {
        if (done[i].load(std::memory_order_acquire)) return;
        std::lock_guard<std::mutex> g(mu);
        if (done[i].load(std::memory_order_relaxed)) return;
        std::sort(key.get() + bstart[i], key.get() + bstart[i + 1]);
        for (int64_t f = bstart[i]; f < bstart[i + 1]; ++f) {
            const uint64_t k = key[f];
            const uint32_t a = (uint32_t)(vmax - ((k >> w) & vmax));
            const uint32_t b = (uint32_t)(vmax - (k & vmax));
            ab[m - 1 - f] = (a << 16) | b;
            hi[m - 1 - f] = ~((uint32_t)(k >> (2 * w)) + base);
        }
        done[i].store(1, std::memory_order_release);
    }

    // Filtration position of the first edge of diameter bits >= bd, and its
    // bucket (its bucket sorted).
    int64_t first_at(uint32_t bd, int *bucket) const {
        *bucket = 0;
        if (m == 0) return 0;
        const uint64_t kb = bd <= base ? 0 : (uint64_t)(bd - base) << (2 * w);
        if (kb > kmax) {
            *bucket = nbuckets() - 1;
            return m;
        }
        const int i = bucket_of(kb);
        ensure(i);
        *bucket = i;
        return std::lower_bound(key.get() + bstart[i], key.get() + bstart[i + 1], kb) - key.get();
    }
};

void sort_edges(const HostInstance &I, float from, EdgeList &out) {
    const int64_t n = I.n;
    int w = 1;
    while ((int64_t(1) << w) < n) ++w;
    const uint64_t vmax = (uint64_t(1) << w) - 1;
    const uint32_t base = float_bits(from);
    const float t = I.t;
    // every key is at most kmax: the bucket shift follows from the range alone
    const uint64_t kmax = t >= from ? ((uint64_t)(float_bits(t) - base) << (2 * w)) |
                                          ((uint64_t(1) << (2 * w)) - 1)
                                    : 0;
    const int top = kmax ? 64 - __builtin_clzll(kmax) : 0;
    const int sh = std::max(0, top - 11);
    out.from = from;
    out.w = w;
    out.sh = sh;
    out.vmax = vmax;
    out.kmax = kmax;
    out.base = base;
    const int nb = (int)(kmax >> sh) + 1;
    auto key_of = [&](int64_t a, int64_t b, float d) {
        return ((uint64_t)(float_bits(d) - base) << (2 * w)) | ((vmax - (uint64_t)a) << w) |
               (vmax - (uint64_t)b);
    };
    std::vector<int64_t> &bs = out.bstart;
    bs.assign(nb + 1, 0);
    for (int64_t a = 1; a < n; ++a) {
        const float *Da = I.D + a * I.ld;
        for (int64_t b = 0; b < a; ++b)
            if (Da[b] >= from && Da[b] <= t) ++bs[out.bucket_of(key_of(a, b, Da[b])) + 1];
    }
    for (int i = 0; i < nb; ++i) bs[i + 1] += bs[i];
    const int64_t m = bs[nb];
    out.m = m;
    out.key.reset(new uint64_t[m > 0 ? m : 1]);
    std::vector<int64_t> at(bs.begin(), bs.end() - 1);
    for (int64_t a = 1; a < n; ++a) {
        const float *Da = I.D + a * I.ld;
        for (int64_t b = 0; b < a; ++b)
            if (Da[b] >= from && Da[b] <= t) {
                const uint64_t k = key_of(a, b, Da[b]);
                out.key[at[out.bucket_of(k)]++] = k;
            }
    }
    out.ab.reset(new uint32_t[m > 0 ? m : 1]);
    out.hi.reset(new uint32_t[m > 0 ? m : 1]);
    out.done.reset(new std::atomic<uint8_t>[nb]);
    for (int i = 0; i < nb; ++i) out.done[i].store(0, std::memory_order_relaxed);
}

// Dimensions p >= 2 up to this many points keep the threshold graph's rows
// as bitsets for the cursors' scans of equal-diameter cofacets (n^2 / 8 bytes).
constexpr int64_t LUNE_BITS_NMAX = 16384;

struct Reducer {
    const HostInstance &I;
    int p;
    int64_t n;
    std::vector<uint64_t> top;  // app_tau[0], app_tau[STRIDE], ...
    // Dimensions p >= 2: bit w of row a is set iff D[a][w] <= t and w != a.
    // A cofacet of a simplex inside the threshold adds a vertex of every one
    // of its vertices' rows, so a cursor's lune scan visits only the set bits
    // of the AND of those rows (a handful below a sparse threshold, instead
    // of all n vertices), testing each exactly.
    std::vector<uint64_t> tbits;
    int64_t tw = 0;  // words per row

    Reducer(const HostInstance &I_, int p_, int threads = 1) : I(I_), p(p_), n(I_.n) {
        for (uint64_t i = 0; i < I.napp; i += STRIDE) top.push_back(I.app_tau[i]);
        if (p >= 2 && n <= LUNE_BITS_NMAX) {
            tw = (n + 63) / 64;
            tbits.assign((size_t)(n * tw), 0);
            parallel_for(threads, n, [&](int64_t a) {
                const float *Da = I.D + a * I.ld;
                uint64_t *row = tbits.data() + a * tw;
                for (int64_t w = 0; w < n; ++w)
                    if (w != a && Da[w] <= I.t) row[w >> 6] |= 1ull << (w & 63);
            });
        }
    }

    bool is_apparent_tau(uint64_t tau) const {
        auto it = std::upper_bound(top.begin(), top.end(), tau);
        if (it == top.begin()) return false;
        const int64_t blk = (it - top.begin()) - 1;
        const uint64_t *b = I.app_tau + blk * STRIDE;
        const uint64_t *e = I.app_tau + std::min<uint64_t>(I.napp, (uint64_t)(blk + 1) * STRIDE);
        const uint64_t *f = std::lower_bound(b, e, tau);
        return f != e && *f == tau;
    }

    bool in_simplex(const int *v, int w) const {
        for (int i = 0; i <= p; ++i)
            if (v[i] == w) return true;
        return false;
    }

    // Dimension 1, the instance without the GPU's sorted edges: the edges of
    // diameter >= from sorted here for all walks of the reduction; when a
    // walk starts below the first sweep's level, all of them (twice at most).
    mutable std::mutex edges_mu;
    mutable std::shared_ptr<const EdgeList> own_edges;
    std::shared_ptr<const EdgeList> level_edges(float from) const {
        std::lock_guard<std::mutex> g(edges_mu);
        if (!own_edges || own_edges->from > from) {
            auto e = std::make_shared<EdgeList>();
            sort_edges(I, own_edges ? 0.0f : from, *e);
            own_edges = e;
        }
        return own_edges;
    }

    int nbr_vertex(int v, int64_t pos) const { return (int)(uint32_t)I.nbr[(int64_t)v * n + pos]; }
    float nbr_dist(int v, int64_t pos) const {
        return bits_float((uint32_t)(I.nbr[(int64_t)v * n + pos] >> 32));
    }

    // A cursor over the coboundary of the p-simplex v (diameter d). If
    // `first` >= 0 the caller knows the oldest cofacet adds vertex `first`.
    void init_cursor(Cursor &c, const int *v, float d, int first) const {
        for (int i = 0; i <= p; ++i) c.v[i] = v[i];
        c.d = d;
        c.merging = false;
        c.ties.clear();
        if (first >= 0) {
            c.lune = first - 1;
            c.head = age_key(d, cofacet_idx(*I.B, c.v, p, first));
            return;
        }
        c.lune = (int32_t)n - 1;
        advance(c);
    }

    void start_merge(Cursor &c) const {
        c.merging = true;
        for (int i = 0; i <= p; ++i) {  // first neighbour farther than d
            const uint64_t *row = I.nbr + (int64_t)c.v[i] * n;
            const uint64_t lim = ((uint64_t)float_bits(c.d) << 32) | 0xffffffffull;
            c.pos[i] = (int32_t)(std::upper_bound(row, row + n, lim) - row);
        }
    }

    // Next vertex at or below c.lune in the AND of the rows of c's vertices
    // (-1: none).
    int next_lune_candidate(const Cursor &c) const {
        int64_t k = c.lune >> 6;
        uint64_t mask = (c.lune & 63) == 63 ? ~0ull : ((2ull << (c.lune & 63)) - 1);
        for (; k >= 0; --k, mask = ~0ull) {
            uint64_t m = mask;
            for (int i = 0; i <= p; ++i) m &= tbits[(int64_t)c.v[i] * tw + k];
            if (m) return (int)(k << 6) + 63 - __builtin_clzll(m);
        }
        return -1;
    }

    // Move the cursor to its next cofacet inside the threshold (or NONE).
    void advance(Cursor &c) const {
        while (!tbits.empty() && c.lune >= 0) {  // the same scan over candidates only
            const int w = next_lune_candidate(c);
            c.lune = w - 1;
            if (w < 0) break;
            float m = 0.0f;
            for (int i = 0; i <= p; ++i) m = std::max(m, I.dist(c.v[i], w));
            if (m <= c.d) {
                c.head = age_key(c.d, cofacet_idx(*I.B, c.v, p, w));
                return;
            }
        }
        while (c.lune >= 0) {  // cofacets of diameter d, largest vertex first
            const int w = c.lune--;
            if (in_simplex(c.v, w)) continue;
            float m = 0.0f;
            for (int i = 0; i <= p; ++i) m = std::max(m, I.dist(c.v[i], w));
            if (m <= c.d) {
                c.head = age_key(c.d, cofacet_idx(*I.B, c.v, p, w));
                return;
            }
        }
        if (!c.merging) start_merge(c);
        if (!c.ties.empty()) {
            const int w = c.ties.back();
            c.ties.pop_back();
            c.head = age_key(c.tie_key, cofacet_idx(*I.B, c.v, p, w));
            return;
        }
        for (;;) {
            int best = -1;
            float bd = INFINITY;
            for (int i = 0; i <= p; ++i)
                if (c.pos[i] < n) {
                    const float x = nbr_dist(c.v[i], c.pos[i]);
                    if (x < bd) {
                        bd = x;
                        best = i;
                    }
                }
            if (best < 0 || bd > I.t) {
                c.head = NONE;
                return;
            }
            // every occurrence at distance bd; a vertex is emitted where its
            // (distance, list) pair is the largest of its p+1 occurrences
            for (;;) {
                int bi = -1;
                for (int i = 0; i <= p; ++i)
                    if (c.pos[i] < n && nbr_dist(c.v[i], c.pos[i]) == bd) {
                        bi = i;
                        break;
                    }
                if (bi < 0) break;
                const int w = nbr_vertex(c.v[bi], c.pos[bi]);
                ++c.pos[bi];
                bool emit = true;
                for (int k = 0; k <= p && emit; ++k) {
                    if (k == bi) continue;
                    const float e = I.dist(c.v[k], w);
                    if (e > bd || (e == bd && k > bi)) emit = false;
                }
                if (emit) c.ties.push_back(w);
            }
            if (!c.ties.empty()) {
                std::sort(c.ties.begin(), c.ties.end());
                c.tie_key = bd;
                const int w = c.ties.back();
                c.ties.pop_back();
                c.head = age_key(bd, cofacet_idx(*I.B, c.v, p, w));
                return;
            }
        }
    }

    // The apparent column owning pivot tau, if any: tau is among the apparent
    // taus, and its owner is the youngest facet of tau (vertices into s, the
    // vertex tau adds to it into *added). Given each edge's apparent vertex
    // (I.app_w), s owns tau iff that vertex is *added. Without either (I.app_tau
    // and I.app_w null) the pair is tested again from its definition: tau is
    // apparent iff its youngest facet s has tau's diameter and tau is the
    // oldest cofacet of s, i.e. no vertex w above *added lies within tau's
    // diameter of every vertex of s. (A cleared column never passes: an
    // apparent pair is a persistence pair, and a cleared simplex is already
    // paired in the dimension below.)
    bool apparent_owner(u128 key, int *s, int *added) const {
        const uint64_t tidx = key_index(key);
        if (I.app_tau && !is_apparent_tau(tidx)) return false;
        const float dt = key_diam(key);
        int u[RPP_MAX_DIM + 2];
        decode_host(*I.B, tidx, p + 1, n, u);
        int best = -1;
        float bestd = -1.0f;
        for (int r = 0; r <= p + 1; ++r) {  // facets in increasing index order
            float fd = 0.0f;
            for (int a = 0; a <= p + 1; ++a)
                for (int b = a + 1; b <= p + 1; ++b)
                    if (a != r && b != r) fd = std::max(fd, I.dist(u[a], u[b]));
            if (fd > bestd) {  // strict: the first (smallest index) wins ties
                bestd = fd;
                best = r;
            }
        }
        if (bestd != dt) return false;  // cannot happen for a stored apparent tau
        for (int a = 0, k = 0; a <= p + 1; ++a)
            if (a != best) s[k++] = u[a];
        *added = u[best];
        if (I.app_w && p == 1)  // s is apparent with tau iff tau adds its recorded vertex
            return I.app_w[(uint64_t)s[0] * (uint64_t)(s[0] - 1) / 2 + (uint64_t)s[1]] == *added;
        if (!I.app_tau)
            for (int w = (int)n - 1; w > *added; --w) {
                if (in_simplex(s, w)) continue;
                float m = 0.0f;
                for (int i = 0; i <= p; ++i) m = std::max(m, I.dist(s[i], w));
                if (m <= dt) return false;  // an older cofacet of equal diameter
            }
        return true;
    }
};

// Where a leftover column's own cursor starts, from its oldest cofacet (found
// on the GPU): a cofacet of equal diameter adds a known vertex (>= 0); a larger
// diameter means there is no cofacet of equal diameter (EMPTY_LUNE).
constexpr int EMPTY_LUNE = -2;

int first_vertex(const Reducer &R, const Leftover &L, const int *v) {
    if (L.pivot == NO_PIVOT) return -1;
    if (L.pdiam != L.diam) return EMPTY_LUNE;
    int u[RPP_MAX_DIM + 2];
    decode_host(*R.I.B, L.pivot, R.p + 1, R.n, u);
    for (int i = 0; i <= R.p + 1; ++i)
        if (!R.in_simplex(v, u[i])) return u[i];
    return -1;
}

// Heap keys of dimension 1, ordered like age_key. When every triangle index
// fits in 32 bits the key packs (diameter bits, complemented index) into 64.
struct Key64 {
    typedef uint64_t T;
    static constexpr T NIL = ~(T)0;  // diameter bits of a NaN: never a real key
    static T make(float d, uint64_t idx) {
        return ((T)float_bits(d) << 32) | (T)(uint32_t)~(uint32_t)idx;
    }
    static u128 wide(T k) {
        return k == NIL ? NONE : age_key(bits_float((uint32_t)(k >> 32)), (uint32_t)~(uint32_t)k);
    }
};
struct Key128 {
    typedef u128 T;
    static constexpr T NIL = ~(T)0;
    static T make(float d, uint64_t idx) { return age_key(d, idx); }
    static u128 wide(T k) { return k; }
};

inline int bits_of(uint64_t x) {  // bits needed to write x
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

// Pivots of the leftover columns of one dimension reduced so far, shared by
// the columns that are reduced in parallel. Column j adds column i < j once
// i is finished, and keeps a pivot that no finished column owns only when
// every unfinished column before it has moved past that pivot: pivots only
// move forward (an addition cancels the pivot and brings younger entries
// only), so none of those columns can end there. The additions are then
// those of Alg. 1 in column order, whatever the interleaving, and the lowest
// unfinished column never waits. Columns must be started in increasing order
// and each finished by the thread that started it.
template <class K, class Col = std::vector<uint64_t>>
struct Ledger {
    std::mutex m;
    std::unordered_map<uint64_t, int64_t> owner;  // pivot index -> finished column
    std::vector<Col> &V;                          // reduced columns, final once finished
    std::vector<char> done;
    int64_t low = 0;                              // columns below are finished
    // Per column, its current pivot as a 64-bit image that preserves the age
    // order (an image that is smaller or equal for every older key): exact
    // for 64-bit keys; for 128-bit ones the diameter bits over the top 32
    // bits of the complemented index, taken over idx_bits significant bits
    // (exact when they number 32 or fewer).
    std::unique_ptr<std::atomic<uint64_t>[]> front;
    // done[] again, readable without the lock (set after the column's owner
    // entry, under the lock)
    std::unique_ptr<std::atomic<char>[]> fin;
    int idx_bits = 64;

    Ledger(std::vector<Col> &V_, int64_t ncols, int idx_bits_ = 64)
        : V(V_), done(ncols, 0), front(new std::atomic<uint64_t>[ncols]),
          fin(new std::atomic<char>[ncols]), idx_bits(idx_bits_) {
        owner.reserve((size_t)ncols * 2);
        for (int64_t j = 0; j < ncols; ++j) {
            front[j].store(0, std::memory_order_relaxed);
            fin[j].store(0, std::memory_order_relaxed);
        }
    }
    uint64_t image(u128 k) const {
        if (k == NONE) return ~0ull;
        if (std::is_same<typename K::T, uint64_t>::value) return (uint64_t)K::make(key_diam(k), key_index(k));
        const uint64_t idx = key_index(k);
        const int b = idx_bits < 64 ? idx_bits : 64;
        const uint64_t rev = (b == 64 ? ~0ull : ((1ull << b) - 1)) - idx;  // larger index: smaller
        const uint64_t top = b > 32 ? rev >> (b - 32) : rev;
        return ((uint64_t)float_bits(key_diam(k)) << 32) | top;
    }
    void advance(int64_t j, u128 k) { front[j].store(image(k), std::memory_order_relaxed); }

    // The finished column that owns pivot k of column j, or -1 when k is
    // free for j; waits while an unfinished earlier column may still end at k
    // (its pivot's image is at most k's: pivots only move forward, and the
    // image keeps their order). The wait watches that one column's pivot and
    // finished flag without the lock, so waiting columns do not hold up the
    // column they wait for (its own queries take the lock).
    int64_t query(int64_t j, u128 k) {
        const uint64_t ub = image(k);
        for (;;) {
            int64_t blocker = -1;
            {
                std::lock_guard<std::mutex> g(m);
                auto it = owner.find(key_index(k));
                if (it != owner.end()) return it->second;
                while (low < j && done[low]) ++low;
                for (int64_t i = low; i < j; ++i)
                    if (!done[i] && front[i].load(std::memory_order_relaxed) <= ub) {
                        blocker = i;
                        break;
                    }
                if (blocker < 0) return -1;
            }
            // a short spin first (a sleep's timer slack is longer than most
            // waits), then yields, then short sleeps
            for (int round = 0;; ++round) {
                if (fin[blocker].load(std::memory_order_acquire) ||
                    front[blocker].load(std::memory_order_relaxed) > ub)
                    break;
                if (round < 2048) std::this_thread::yield();
                else std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
    // Column j is finished with pivot k (NONE: a zero column); V[j] is final.
    void finish(int64_t j, u128 k) {
        std::lock_guard<std::mutex> g(m);
        if (k != NONE) owner[key_index(k)] = j;
        done[j] = 1;
        fin[j].store(1, std::memory_order_release);
    }
};

// ---- dimensions p >= 2 -------------------------------------------------------

struct ColumnState {
    std::vector<Cursor> cur;
    ColHeap heap;  // (head, cursor)
    std::vector<std::pair<uint64_t, float>> V;    // simplices whose coboundaries were added
    u128 cand = NONE;
    bool started = false;
    int64_t additions = 0, reads = 0, entries = 0;
};

// Add the coboundary of simplex v (index idx, diameter d) to the working
// column; `first` as in Reducer::init_cursor, or EMPTY_LUNE. Entries older
// than `floor` are skipped: the caller adds a reduced column whose pivot is
// floor, the working column's own pivot, so those entries sum to zero.
void add_cursor(const Reducer &R, ColumnState &S, const int *v, uint64_t idx, float d,
                int first, u128 floor = 0) {
    S.cur.emplace_back();
    Cursor &c = S.cur.back();
    if (first == EMPTY_LUNE) {
        for (int i = 0; i <= R.p; ++i) c.v[i] = v[i];
        c.d = d;
        c.lune = -1;
        c.merging = false;
        R.advance(c);
    } else {
        R.init_cursor(c, v, d, first);
    }
    while (c.head != NONE && c.head < floor) R.advance(c);
    if (c.head != NONE) S.heap.push({c.head, (int32_t)(S.cur.size() - 1)});
    S.V.emplace_back(idx, d);
}

void add_cursor(const Reducer &R, ColumnState &S, uint64_t idx, float d, u128 floor) {
    int v[RPP_MAX_DIM + 1];
    decode_host(*R.I.B, idx, R.p, R.n, v);
    add_cursor(R, S, v, idx, d, -1, floor);
}

// Oldest nonzero entry of the working column (NONE if it is zero).
u128 pivot(const Reducer &R, ColumnState &S) {
    while (!S.heap.empty()) {
        const std::pair<u128, int32_t> a = S.heap.top();
        if (S.heap.top_twice()) {  // cancels over Z/2
            S.heap.pop();
            const std::pair<u128, int32_t> b = S.heap.top();  // the same key
            S.heap.pop();
            S.entries += 2;
            for (int32_t ci : {a.second, b.second}) {
                Cursor &c = S.cur[ci];
                R.advance(c);
                if (c.head != NONE) S.heap.push({c.head, ci});
            }
            continue;
        }
        return a.first;  // the pivot stays in the column
    }
    return NONE;
}

typedef std::vector<std::pair<uint64_t, float>> SimplexSet;  // (index, diameter)

// Walk column j: add the owners of its pivot until the pivot is free or the
// column is zero. Apparent owners come from the pair store; pivots of earlier
// leftover columns from the ledger, which also holds back a pivot that an
// unfinished earlier column may still reach (as in dimension 1).
void walk(const Reducer &R, ColumnState &S, Ledger<Key128, SimplexSet> &led, int64_t j) {
    for (;;) {
        const u128 k = pivot(R, S);
        if (k == NONE) {
            S.cand = NONE;
            return;
        }
        led.advance(j, k);
        ++S.reads;
        int s[RPP_MAX_DIM + 1], added;
        if (R.apparent_owner(k, s, &added)) {
            ++S.additions;  // its oldest cofacet is the pivot, which adds `added`
            add_cursor(R, S, s, index_host(*R.I.B, s, R.p), key_diam(k), added);
            continue;
        }
        const int64_t i = led.query(j, k);
        if (i >= 0) {
            ++S.additions;
            for (const auto &x : led.V[i]) add_cursor(R, S, x.first, x.second, k);
            continue;
        }
        S.cand = k;
        return;
    }
}

void start_column(const Reducer &R, ColumnState &S, const Leftover &L) {
    S.started = true;
    int v[RPP_MAX_DIM + 1];
    decode_host(*R.I.B, L.sigma, R.p, R.n, v);
    add_cursor(R, S, v, L.sigma, L.diam, first_vertex(R, L, v));
}

// Z/2 sum of the simplices in V: sort and drop pairs.
void reduce_set(SimplexSet &V) {
    std::sort(V.begin(), V.end(),
              [](const std::pair<uint64_t, float> &a, const std::pair<uint64_t, float> &b) {
                  return a.first < b.first;
              });
    size_t o = 0;
    for (size_t i = 0; i < V.size();) {
        size_t j = i;
        while (j < V.size() && V[j].first == V[i].first) ++j;
        if ((j - i) & 1) V[o++] = V[i];
        i = j;
    }
    V.resize(o);
}

constexpr double PHASE_B_SERIAL_MS = 4.0;

// Two phases. A: every column walks on its own (in parallel, no shared
// state) while its pivots have apparent owners, and stops at the first pivot
// without one. B: the columns then finish concurrently, one per host thread
// at a time, in index order: a column whose pivot an earlier leftover column
// owns adds that column's reduced column and walks on under the ledger, which
// makes the additions those of Alg. 1 in column order whatever the
// interleaving (as in dimension 1). Most columns leave phase B after one
// ledger query; phase B runs in order on the calling thread until it proves
// long, then concurrently.
void reduce_general(const HostInstance &I, int p, const Leftover *left, int64_t nleft,
                    int threads, std::vector<HostPair> &out, ReduceStats &stats) {
    Reducer R(I, p, threads);
    std::vector<ColumnState> col(nleft);
    std::vector<SimplexSet> V(nleft);
    // cofacet indices (the pivots) stay below C(n, p+2)
    Ledger<Key128, SimplexSet> led(V, nleft, bits_of(I.B->at(p + 2, I.n)));

    auto phase_a_column = [&](int64_t j) {
        const Leftover &L = left[j];
        ColumnState &S = col[j];
        if (L.pivot == NO_PIVOT) {
            S.cand = NONE;
            return;
        }
        const u128 k0 = age_key(L.pdiam, L.pivot);
        int s[RPP_MAX_DIM + 1], added;
        ++S.reads;
        if (!R.apparent_owner(k0, s, &added)) {
            S.cand = k0;  // the unreduced pivot is free of apparent owners
            return;
        }
        start_column(R, S, L);
        for (;;) {  // apparent owners only
            const u128 k = pivot(R, S);
            if (k == NONE) {
                S.cand = NONE;
                return;
            }
            ++S.reads;
            if (!R.apparent_owner(k, s, &added)) {
                S.cand = k;
                return;
            }
            ++S.additions;
            add_cursor(R, S, s, index_host(*R.I.B, s, R.p), key_diam(k), added);
        }
    };
    auto phase_b_column = [&](int64_t j) {
        const Leftover &L = left[j];
        ColumnState &S = col[j];
        if (S.cand != NONE) {
            const int64_t i = led.query(j, S.cand);
            if (i >= 0) {  // owned by an earlier leftover column: add it and walk on
                if (!S.started) start_column(R, S, L);
                ++S.additions;
                for (const auto &x : led.V[i]) add_cursor(R, S, x.first, x.second, S.cand);
                walk(R, S, led, j);
            }
        }
        if (S.started) {
            reduce_set(S.V);
            V[j].swap(S.V);
        } else {
            V[j].emplace_back(L.sigma, L.diam);
        }
        std::vector<Cursor>().swap(S.cur);
        S.heap.release();
        led.finish(j, S.cand);
    };
    if (threads <= 1 || nleft < 16) {
        for (int64_t j = 0; j < nleft; ++j) phase_a_column(j);
    } else {
        pool(threads).parallel_for(nleft, phase_a_column);
    }
    for (int64_t j = 0; j < nleft; ++j) led.advance(j, col[j].cand);  // NONE: past everything
    // In order on this thread while that stays cheap (most columns leave
    // after one query, and then the ledger's coordination would cost more
    // than it saves); once phase B has taken PHASE_B_SERIAL_MS, the remaining
    // columns go to the host threads (they start in increasing order: the
    // pool hands out indices in order).
    const auto b0 = std::chrono::steady_clock::now();
    int64_t j = 0;
    for (; j < nleft; ++j) {
        if (threads > 1 && (j & 63) == 0 &&
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - b0)
                    .count() > PHASE_B_SERIAL_MS)
            break;
        phase_b_column(j);
    }
    if (j < nleft) {
        const int64_t first = j;
        pool(threads).parallel_for(nleft - first, [&](int64_t i) { phase_b_column(first + i); });
    }

    for (int64_t j = 0; j < nleft; ++j) {
        const Leftover &L = left[j];
        const ColumnState &S = col[j];
        HostPair P;
        P.sigma = L.sigma;
        P.birth = L.diam;
        if (S.cand == NONE) {
            P.tau = NO_PIVOT;
            P.death = INFINITY;
        } else {
            P.tau = key_index(S.cand);
            P.death = key_diam(S.cand);
            if (!S.started) ++stats.free_pivot;
        }
        out.push_back(P);
        stats.additions += S.additions;
        stats.reads += S.reads;
        stats.entries += S.entries;
    }
}

// ---- dimension 1 -------------------------------------------------------------
//
// The working column of leftover j is the coboundary of a set V of edges; a
// triangle is a nonzero entry iff an odd number of its edges lie in V. V is
// kept as adjacency bits (row a, bit b set iff the edge {a, b} is in V).
// During an apparent walk V only grows (an apparent edge is added once, when
// its own pivot is reached; an edge already in V would leave it, and the walk
// then restarts), so a triangle's parity can be read from the bits whenever a
// cursor lists it: the cursor skips it if even.
// The heap then holds only entries that were nonzero when listed; one whose
// parity changed since is dropped when it surfaces. Every nonzero triangle
// stays reachable: the last of its edges to enter V has a cursor that listed
// it (or will) after its parity last changed. Adding another leftover's column
// can remove edges from V; the walk then restarts from the new V,
// each cursor placed just past the cancelled pivot (the sum is zero up to
// there).
//
// Lune part of an edge cursor (x, y) with diameter d: the vertices w with
// D[x][w] <= d and D[y][w] <= d, largest first, taken 64 at a time as a bit
// mask from which the even triangles are masked out (D's rows are read in
// order; the parity of a word of triangles is two adjacency words).
// Merge part: the neighbour rows of x and y beyond distance d are merged. A
// vertex w met in x's row at distance e is a cofacet of diameter e exactly
// when D[y][w] < e (its other occurrence came first); on a tie D[y][w] == e it
// is taken from y's row, which is merged after x's at each distance.
//
// A walk whose V grows large switches from cursors to a sweep over the
// triangles themselves, level by level in diameter (see "sweep mode" below).

struct Cur1 {
    int32_t x = 0, y = 0;
    int32_t hw = -1;             // head vertex (-1: no more cofacets)
    float hd = 0.0f;             // head diameter
    float d = 0.0f;
    int32_t first = -1;          // known oldest cofacet vertex, emitted before anything else
    int32_t lune = -1;           // lune vertices <= lune are still to come (-1: done)
    int32_t lw = -1;             // word of lune vertices cached in lm (-1: none)
    uint64_t lm = 0;
    int32_t pa = -1, pb = -1;    // merge positions (pa < 0: merge not started)
    // The next cofacets in age order, produced in a batch while the cursor's
    // rows are in cache (their order does not depend on V; parity is read
    // when each one surfaces).
    static constexpr int NB = 4;
    uint8_t bn = 0, bi = 0;      // batch size, next position
    bool bend = false;           // no cofacets after the batch
    int32_t bw[NB];
    float bh[NB];
    float tie_key = 0.0f;
    std::vector<int32_t> ties;   // equal-diameter emissions, largest at the back
};

// 4-ary min-heap of (key, cursor) with a replace-top step (one sift where a
// pop followed by a push would take two). Four children share a cache line
// and the tree is half as deep as a binary one.
template <class T>
struct MinHeap {
    typedef std::pair<T, int32_t> E;
    std::vector<E> h;
    static bool less(const E &a, const E &b) {
        return a.first < b.first || (a.first == b.first && a.second < b.second);
    }
    bool empty() const { return h.empty(); }
    const E &top() const { return h[0]; }
    void clear() { h.clear(); }
    void push(E e) {
        size_t i = h.size();
        h.push_back(e);
        while (i > 0) {
            const size_t up = (i - 1) >> 2;
            if (!less(e, h[up])) break;
            h[i] = h[up];
            i = up;
        }
        h[i] = e;
    }
    void sift_down(E e) {  // place e at the root
        const size_t m = h.size();
        size_t i = 0;
        for (;;) {
            const size_t c0 = 4 * i + 1;
            if (c0 >= m) break;
            size_t c = c0;
            const size_t ce = std::min(c0 + 4, m);
            for (size_t k = c0 + 1; k < ce; ++k)
                if (less(h[k], h[c])) c = k;
            if (!less(h[c], e)) break;
            h[i] = h[c];
            i = c;
        }
        h[i] = e;
    }
    void replace_top(E e) { sift_down(e); }
    void pop() {
        const E last = h.back();
        h.pop_back();
        if (!h.empty()) sift_down(last);
    }
};

// Monotone priority queue of (64-bit key, cursor): every key pushed is >= the
// last key taken from the top, which holds for the walk (a new cursor starts
// at the current pivot, an advanced cursor moves past its previous entry).
// Bucket i > 0 holds keys whose highest bit differing from `last` is bit
// i - 1; bucket 0 holds keys equal to `last`. Pushes append; the top is
// found by redistributing the lowest non-empty bucket, whose elements each
// move to a strictly lower bucket.
struct RadixHeap {
    typedef std::pair<uint64_t, int32_t> E;
    std::vector<E> b[65];
    uint64_t last = 0;
    size_t size = 0;
    static int bucket(uint64_t k, uint64_t last) {
        return k == last ? 0 : 64 - __builtin_clzll(k ^ last);
    }
    bool empty() const { return size == 0; }
    void clear() {
        for (auto &v : b) v.clear();
        last = 0;
        size = 0;
    }
    void push(E e) {
        b[bucket(e.first, last)].push_back(e);
        ++size;
    }
    const E &top() {  // requires !empty()
        if (b[0].empty()) {
            int i = 1;
            while (b[i].empty()) ++i;
            uint64_t m = b[i][0].first;
            for (const E &e : b[i]) m = std::min(m, e.first);
            last = m;
            for (const E &e : b[i]) b[bucket(e.first, last)].push_back(e);
            b[i].clear();
        }
        return b[0].back();
    }
    void pop() {  // removes the element top() returned
        b[0].pop_back();
        --size;
    }
    void replace_top(E e) {
        pop();
        push(e);
    }
};

template <class K>
struct Walk1 {
    typedef typename K::T Key;
    const HostInstance &I;
    const Reducer &R;
    int64_t n, W, S;              // vertices, words per bit row, words per vertex
    // Per vertex a, S = 2W words: the sweep's bits P[a] (words 0..W-1), then
    // V's adjacency bits of a (words W..2W-1); next to each other, so that a
    // level reads two contiguous stretches. All clear when idle.
    uint64_t *rows;
    uint64_t *adj;                // rows + W: V as adjacency bits
    std::vector<Cur1> cur;
    typename std::conditional<std::is_same<Key, uint64_t>::value, RadixHeap, MinHeap<Key>>::type
        heap;
    std::vector<uint64_t> V;      // edges of V (indices)
    int64_t additions = 0, reads = 0, entries = 0, levels = 0;
    int64_t sweep_pivots = 0;
    mutable int64_t sweep_idle = 0;
    bool swept = false;  // the walk entered sweep mode at least once
    int threads = 1;

    // rows_: the calling thread's scratch of n x 2 ceil(n / 64) words, all
    // clear; it is left clear again when the walk ends.
    Walk1(const HostInstance &I_, const Reducer &R_, uint64_t *rows_, int threads_ = 1)
        : I(I_), R(R_), n(I_.n), W((I_.n + 63) / 64), S(2 * ((I_.n + 63) / 64)), rows(rows_),
          adj(rows_ + (I_.n + 63) / 64), threads(threads_) {}
    ~Walk1() {
        clear_bits();
        clear_plane();
    }

    static uint64_t edge_index(int x, int y) {
        return (uint64_t)x * (uint64_t)(x - 1) / 2 + (uint64_t)y;
    }
    // Vertices x > y of the edge with index e.
    static void edge_vertices(uint64_t e, int &x, int &y) {
        uint64_t a = (uint64_t)((1.0 + std::sqrt(1.0 + 8.0 * (double)e)) / 2.0);
        while (a * (a - 1) / 2 > e) --a;
        while ((a + 1) * a / 2 <= e) ++a;
        x = (int)a;
        y = (int)(e - a * (a - 1) / 2);
    }
    bool vbit(int a, int b) const { return (adj[(int64_t)a * S + (b >> 6)] >> (b & 63)) & 1ull; }
    void set_edge(int x, int y) {
        adj[(int64_t)x * S + (y >> 6)] |= 1ull << (y & 63);
        adj[(int64_t)y * S + (x >> 6)] |= 1ull << (x & 63);
    }
    void clear_bits() {
        if ((int64_t)V.size() * 8 > n * W) {
            for (int64_t a = 0; a < n; ++a)
                std::memset(adj + a * S, 0, (size_t)W * sizeof(uint64_t));
            return;
        }
        for (uint64_t e : V) {
            int x, y;
            edge_vertices(e, x, y);
            adj[(int64_t)x * S + (y >> 6)] = 0;
            adj[(int64_t)y * S + (x >> 6)] = 0;
        }
    }

    void start_merge(Cur1 &c) const {
        const uint64_t *rx = I.nbr + (int64_t)c.x * n, *ry = I.nbr + (int64_t)c.y * n;
        const uint64_t lim = ((uint64_t)float_bits(c.d) << 32) | 0xffffffffull;
        c.pa = (int32_t)(std::upper_bound(rx, rx + n, lim) - rx);
        c.pb = (int32_t)(std::upper_bound(ry, ry + n, lim) - ry);
    }

    // Lune vertices of the cursor in word k: bit i set iff w = 64 k + i is
    // within c.d of both x and y (x and y themselves excluded).
    uint64_t lune_word(const Cur1 &c, int64_t k) const {
        const float *Dx = I.D + (int64_t)c.x * I.ld, *Dy = I.D + (int64_t)c.y * I.ld;
        const int64_t b = k << 6, e = std::min<int64_t>(b + 64, n);
        const float d = c.d;
        uint64_t m = 0;
        if (e - b == 64) {
            // one flag byte per vertex (a loop the compiler vectorises), then
            // eight 0/1 bytes at a time into eight bits: the product with
            // sum_i 2^(56 - 7 i) gathers byte i into bit 56 + i, and every other
            // partial product falls below bit 56 without carrying into it or
            // beyond bit 63
            uint8_t f[64];
            for (int i = 0; i < 64; ++i) f[i] = (uint8_t)((Dx[b + i] <= d) & (Dy[b + i] <= d));
            for (int j = 0; j < 8; ++j) {
                uint64_t x;
                std::memcpy(&x, f + 8 * j, 8);  // little-endian: byte i at bits 8i..8i+7
                m |= ((x * 0x0102040810204080ull) >> 56) << (8 * j);
            }
        } else {
            for (int64_t i = b; i < e; ++i)
                m |= (uint64_t)((Dx[i] <= d) & (Dy[i] <= d)) << (i - b);
        }
        if ((c.x >> 6) == k) m &= ~(1ull << (c.x & 63));
        if ((c.y >> 6) == k) m &= ~(1ull << (c.y & 63));
        return m;
    }

    // Next cofacet of the cursor in age order: every one of the merge part,
    // the odd ones of the lune.
    bool raw_next(Cur1 &c) {
        ++entries;
        return fetch(c);
    }

    bool fetch(Cur1 &c) const {
        if (c.bi == c.bn) {
            c.bi = c.bn = 0;
            while (!c.bend && c.bn < Cur1::NB) {
                if (!step(c)) {
                    c.bend = true;
                    break;
                }
                c.bw[c.bn] = c.hw;
                c.bh[c.bn] = c.hd;
                ++c.bn;
            }
            if (c.bn == 0) {
                c.hw = -1;
                return false;
            }
        }
        c.hw = c.bw[c.bi];
        c.hd = c.bh[c.bi];
        ++c.bi;
        return true;
    }

    // The cofacet after the current one, into (hw, hd); false if none.
    bool step(Cur1 &c) const {
        if (c.first >= 0) {  // the oldest cofacet, known in advance
            c.hw = c.first;
            c.hd = c.d;
            c.lune = c.first - 1;
            c.first = -1;
            return true;
        }
        while (c.lune >= 0) {  // diameter d, largest vertex first
            const int64_t k = c.lune >> 6;
            if (c.lw != k) {
                c.lm = lune_word(c, k);
                c.lw = (int32_t)k;
            }
            uint64_t m = c.lm;
            const int sh = c.lune & 63;
            if (sh < 63) m &= (2ull << sh) - 1;
            m &= ~(adj[(int64_t)c.x * S + k] ^ adj[(int64_t)c.y * S + k]);  // odd ones only
            if (m) {
                const int w = (int)(k << 6) + 63 - __builtin_clzll(m);
                c.lune = w - 1;
                c.hw = w;
                c.hd = c.d;
                return true;
            }
            c.lune = (int32_t)(k << 6) - 1;
        }
        if (!c.ties.empty()) {
            c.hw = c.ties.back();
            c.ties.pop_back();
            c.hd = c.tie_key;
            return true;
        }
        if (c.pa < 0) start_merge(c);
        const uint64_t *rx = I.nbr + (int64_t)c.x * n, *ry = I.nbr + (int64_t)c.y * n;
        const float *Dx = I.D + (int64_t)c.x * I.ld, *Dy = I.D + (int64_t)c.y * I.ld;
        for (;;) {
            const uint32_t da = c.pa < n ? (uint32_t)(rx[c.pa] >> 32) : 0xffffffffu;
            const uint32_t db = c.pb < n ? (uint32_t)(ry[c.pb] >> 32) : 0xffffffffu;
            if (c.pa >= n && c.pb >= n) break;
            const uint32_t bd = std::min(da, db);
            const float e = bits_float(bd);
            if (e > I.t) break;
            if (da != db) {  // the common case: a lone occurrence at distance e
                const bool sa = da < db;
                const uint64_t *row = sa ? rx : ry;
                int32_t &pos = sa ? c.pa : c.pb;
                if (pos + 1 >= n || (uint32_t)(row[pos + 1] >> 32) != bd) {
                    // the other row has nothing left at e, so D[other][w] != e
                    const uint32_t w = (uint32_t)row[pos++];
                    if ((sa ? Dy : Dx)[w] < e) {
                        c.hw = (int32_t)w;
                        c.hd = e;
                        return true;
                    }
                    continue;
                }
            }
            merge_level(c, bd);
            if (!c.ties.empty()) {
                c.hw = c.ties.back();
                c.ties.pop_back();
                c.hd = c.tie_key;
                return true;
            }
        }
        c.hw = -1;
        return false;
    }

    // Consume every occurrence at distance bits bd in both rows; the cofacets
    // of diameter bd become the cursor's ties (sorted, largest at the back).
    void merge_level(Cur1 &c, uint32_t bd) const {
        const uint64_t *rx = I.nbr + (int64_t)c.x * n, *ry = I.nbr + (int64_t)c.y * n;
        const float *Dx = I.D + (int64_t)c.x * I.ld, *Dy = I.D + (int64_t)c.y * I.ld;
        const float e = bits_float(bd);
        while (c.pa < n && (uint32_t)(rx[c.pa] >> 32) == bd) {
            const uint32_t w = (uint32_t)rx[c.pa++];
            if (Dy[w] < e) c.ties.push_back((int32_t)w);
        }
        while (c.pb < n && (uint32_t)(ry[c.pb] >> 32) == bd) {
            const uint32_t w = (uint32_t)ry[c.pb++];
            if (Dx[w] <= e) c.ties.push_back((int32_t)w);
        }
        std::sort(c.ties.begin(), c.ties.end());
        c.tie_key = e;
    }

    // Colex comparison of the triangle {x, y, w} with the triangle kv[0] >
    // kv[1] > kv[2]: true if {x, y, w} has the smaller index. For fixed x, y
    // the sorted tuple never decreases as w grows (also at w = x or w = y), so
    // the predicate holds on a prefix of w.
    static bool tri_before(int x, int y, int w, const int *kv) {
        int a = x, b = y, c = w;  // x > y
        if (c > a) std::swap(a, c), std::swap(b, c);
        else if (c > b) std::swap(b, c);
        if (a != kv[0]) return a < kv[0];
        if (b != kv[1]) return b < kv[1];
        return c < kv[2];
    }

    // Position a fresh cursor so that its next cofacet is the first one younger
    // than the triangle k = (dk, kv): a column whose entries up to k are known
    // to be zero need not list them.
    void seek(Cur1 &c, float dk, const int *kv) const {
        c.first = -1;
        if (dk < c.d) return;  // every cofacet is younger than k
        if (dk == c.d) {  // lune vertices w (largest first) with index below k's
            int lo = -1, hi = (int)n;  // largest w with tri_before(w): in [lo, hi)
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (tri_before(c.x, c.y, mid, kv)) lo = mid;
                else hi = mid;
            }
            c.lune = lo;
            return;
        }
        c.lune = -1;  // the whole lune is older than k
        const uint64_t *rx = I.nbr + (int64_t)c.x * n, *ry = I.nbr + (int64_t)c.y * n;
        const uint32_t bd = float_bits(dk);
        const uint64_t lim = (uint64_t)bd << 32;
        c.pa = (int32_t)(std::lower_bound(rx, rx + n, lim) - rx);
        c.pb = (int32_t)(std::lower_bound(ry, ry + n, lim) - ry);
        merge_level(c, bd);  // cofacets of diameter dk: keep those younger than k
        while (!c.ties.empty() && !tri_before(c.x, c.y, c.ties.back(), kv)) c.ties.pop_back();
    }

    // Parity of the cursor's head (the cursor's own edge is in V).
    bool odd(const Cur1 &c) const { return vbit(c.x, c.hw) == vbit(c.y, c.hw); }

    // Next cofacet with odd parity (hw = -1 if none).
    void advance(Cur1 &c) {
        while (raw_next(c))
            if (odd(c)) return;
    }

    static void sort3(const Cur1 &c, int *v) {
        int a = c.x, b = c.y, w = c.hw;  // sort {x, y, w} decreasingly (x > y)
        if (w > a) std::swap(a, w), std::swap(b, w);
        else if (w > b) std::swap(b, w);
        v[0] = a;
        v[1] = b;
        v[2] = w;
    }
    Key head_key(const Cur1 &c) const {
        int v[3];
        sort3(c, v);
        return K::make(c.hd, I.B->at(3, v[0]) + I.B->at(2, v[1]) + (uint64_t)v[2]);
    }

    void push(int32_t ci) { heap.push({head_key(cur[ci]), ci}); }

    // Cursor of edge (x, y) (x > y); `first` as in Reducer::init_cursor, or
    // EMPTY_LUNE. The edge's bits must already be set.
    void add_cursor(int x, int y, float d, int first) {
        cur.emplace_back();
        Cur1 &c = cur.back();
        c.x = x;
        c.y = y;
        c.d = d;
        c.first = first >= 0 ? first : -1;
        c.lune = first >= 0 ? first - 1 : (first == EMPTY_LUNE ? -1 : (int32_t)n - 1);
        advance(c);
        if (c.hw >= 0) push((int32_t)cur.size() - 1);
    }

    void add_edge(int x, int y, float d, int first) {
        set_edge(x, y);
        V.push_back(edge_index(x, y));
        add_cursor(x, y, d, first);
    }

    // Restart the walk from the edge set newV (sorted, no repeats), whose
    // coboundary is known to vanish up to and including the entry k.
    void rebuild(std::vector<uint64_t> newV, u128 k) {
        clear_plane();
        sweep = false;
        clear_bits();
        cur.clear();
        heap.clear();
        V.swap(newV);
        for (uint64_t e : V) {
            int x, y;
            edge_vertices(e, x, y);
            set_edge(x, y);
        }
        if (can_sweep() && V.size() >= SWEEP_MIN) {
            enter_sweep(k);
            return;
        }
        int kv[3];
        decode_host(*I.B, key_index(k), 2, n, kv);
        const float dk = key_diam(k);
        for (uint64_t e : V) {
            cur.emplace_back();
            Cur1 &c = cur.back();
            edge_vertices(e, c.x, c.y);
            c.d = I.dist(c.x, c.y);
            c.lune = (int32_t)n - 1;
            seek(c, dk, kv);
            advance(c);
            if (c.hw >= 0) push((int32_t)cur.size() - 1);
        }
    }

    // Add the reduced column (edge set b, sorted) of the leftover owning the
    // pivot k of V: the pivot cancels and the walk restarts past it.
    void add_leftover(const std::vector<uint64_t> &b, u128 k) {
        ++additions;
        if (sweep) {
            for (uint64_t e : b) toggle_edge(e);
            return;
        }
        std::vector<uint64_t> a = edges(), sum;
        std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(),
                                      std::back_inserter(sum));
        rebuild(std::move(sum), k);
    }

    u128 pivot() {
        if (sweep) return pivot_sweep();
        while (!heap.empty()) {
            const int32_t ci = heap.top().second;
            Cur1 &c = cur[ci];
            if (odd(c)) return K::wide(heap.top().first);  // still nonzero
            advance(c);
            if (c.hw >= 0) heap.replace_top({head_key(c), ci});
            else heap.pop();
        }
        return NONE;
    }

    // Add owners of the pivot until it is free; led: the finished leftover
    // columns, j: this column's position among them.
    u128 walk(Ledger<K> &led, int64_t j) {
        for (;;) {
            const u128 k = pivot();
            if (k == NONE) return NONE;
            ++reads;
            led.advance(j, k);
            int s[3], added;
            if (sweep ? sweep_owner(s, &added) : R.apparent_owner(k, s, &added)) {
                ++additions;  // its oldest cofacet is the pivot, which adds `added`
                if (sweep) {
                    toggle_edge(edge_index(s[0], s[1]));
                } else if (vbit(s[0], s[1])) {
                    // already in V (possible after a leftover's column was
                    // added): the addition removes it, so restart past k
                    std::vector<uint64_t> nv = edges(), one{edge_index(s[0], s[1])}, rest;
                    std::set_symmetric_difference(nv.begin(), nv.end(), one.begin(), one.end(),
                                                  std::back_inserter(rest));
                    rebuild(std::move(rest), k);
                } else {
                    add_edge(s[0], s[1], key_diam(k), added);
                    if (can_sweep() && V.size() >= SWEEP_MIN) enter_sweep(k);
                }
                continue;
            }
            const int64_t i = led.query(j, k);  // a pivot has one owner at most
            if (i >= 0) {
                add_leftover(led.V[i], k);
                continue;
            }
            return k;
        }
    }

    // The edges of V, sorted (an edge listed twice has left V).
    std::vector<uint64_t> edges() const {
        std::vector<uint64_t> out = V;
        std::sort(out.begin(), out.end());
        size_t o = 0;
        for (size_t i = 0; i < out.size();) {
            size_t j = i;
            while (j < out.size() && out[j] == out[i]) ++j;
            if ((j - i) & 1) out[o++] = out[i];
            i = j;
        }
        out.resize(o);
        return out;
    }

    // ---- sweep mode --------------------------------------------------------
    // Once V holds SWEEP_MIN edges the walk stops listing coboundaries and
    // sweeps the triangles themselves, in age order, one diameter level at a
    // time. The triangles of diameter e are the lune triangles {a, b, w} of
    // the edges {a, b} of length e (w within e of a and of b); a triangle with
    // several edges of length e belongs to the one with the largest index.
    // With P[a] the set of vertices within the current level's diameter of a
    // (kept up to date by setting two bits per edge as the sweep enters its
    // level), an edge's lune is the word-wise P[a] & P[b], and the parity of
    // its triangles is adj[a] ^ adj[b] ^ [ab in V]: a level costs a few word
    // operations per 64 vertices however large V is. Parities are read from
    // the bits when the sweep gets to a triangle, and every addition changes
    // only entries at or after the pivot, so additions of any kind (apparent
    // edges, a leftover's column, an edge that leaves V) are bit flips.
    static constexpr size_t SWEEP_MIN = 256;
    static constexpr int64_t PREFETCH_AHEAD = 2;  // levels
    static constexpr int64_t SWEEP_NMAX = 8192;  // P and adj: n^2 / 8 bytes each per thread
    bool sweep = false;
    uint64_t *P = nullptr;        // n x W bits: w within the level's diameter of a (no self bits)
    // The levels: the edges inside the threshold in coboundary order (those
    // of diameter >= the sweep's first level at least), f1 the next position
    // in filtration order.
    const uint32_t *eab = nullptr, *ehi = nullptr;
    int64_t ne = 0;
    std::shared_ptr<const EdgeList> elist;  // the arrays, when sorted on the host
    int ebucket = 0;              // host-sorted: the last bucket sorted for this sweep
    int64_t eready = 0;           // positions below are sorted (from the sweep's start on)
    int64_t f1 = 0;
    float lvl_d = 0.0f;           // diameter of the current level
    struct LevelEdge {
        int a, b;                 // a > b
        uint64_t idx;
        int wpos;                 // its triangles {a, b, w} with w < wpos are still to come
        int head;                 // several-edge levels: cached oldest odd triangle (w, -1: none)
        uint32_t ver;             // version of the cached head
    };
    std::vector<LevelEdge> lev;
    int piv_a = -1, piv_b = -1, piv_w = -1;  // the last pivot's triangle
    // Degree of each vertex in V: a level edge with no edge of V at either
    // end has only even triangles (all three of its edges are outside V).
    std::vector<int32_t> deg;
    // Levels of several edges: the edges' cached heads in a max-heap by
    // triangle index (stale entries are skipped by version), the level edges
    // at each vertex, and the vertices whose edges' heads must be recomputed
    // (an addition flips only triangles that contain the added edge).
    std::vector<std::pair<uint64_t, std::pair<int32_t, uint32_t>>> lheap;
    std::vector<int32_t> inc_start, inc_edge, inc_v, inc_order;
    static constexpr size_t SMALL_LEVEL = 8;  // up to this many edges: no index, every head recomputed
    std::vector<int32_t> dirty;
    std::vector<char> is_dirty;

    bool can_sweep() const { return n <= SWEEP_NMAX; }

    // Edge at position f of the filtration order (diameter ascending).
    // Host-sorted edges: sort every bucket from the last one sorted up to the
    // one holding position f (the sweep only moves forward, and positions
    // below eready are sorted from the sweep's start on).
    void need(int64_t f) {
        while (f >= eready) {
            ++ebucket;
            elist->ensure(ebucket);
            eready = elist->bstart[ebucket + 1];
        }
    }
    void edge_at(int64_t f, int &a, int &b) const {
        const uint32_t ab = eab[ne - 1 - f];
        a = (int)(ab >> 16);
        b = (int)(ab & 0xffffu);
    }
    float diam_at(int64_t f) const { return bits_float(~ehi[ne - 1 - f]); }

    static uint64_t tri_index(const Binomial &B, int a, int b, int w) {
        int v0 = a, v1 = b, v2 = w;  // a > b
        if (v2 > v0) std::swap(v0, v2), std::swap(v1, v2);
        else if (v2 > v1) std::swap(v1, v2);
        return B.at(3, v0) + B.at(2, v1) + (uint64_t)v2;
    }

    void level_edge(int a, int b) {  // a > b
        LevelEdge E;
        E.a = a;
        E.b = b;
        E.idx = edge_index(a, b);
        E.wpos = (int)n;
        E.head = -1;
        E.ver = 0;
        P[(int64_t)a * S + (b >> 6)] |= 1ull << (b & 63);
        P[(int64_t)b * S + (a >> 6)] |= 1ull << (a & 63);
        lev.push_back(E);
    }

    // Enter the next level of equal diameter: set its bits in P and list its
    // edges with every triangle still to come; false when no edge is left.
    bool next_level() {
        lev.clear();
        if (f1 >= ne) return false;
        const int64_t f0 = f1;
        need(f0);
        lvl_d = diam_at(f0);
        while (f1 + 1 < ne && (need(f1 + 1), diam_at(f1 + 1) == lvl_d)) ++f1;
        ++f1;
        for (int64_t f = f0; f < f1; ++f) {
            int a, b;
            edge_at(f, a, b);
            level_edge(a, b);
        }
        // the sweep is bound by the latency of the bit rows: ask for the rows
        // of an edge a few levels ahead
        if (f1 + PREFETCH_AHEAD < ne) {
            int a, b;
            need(f1 + PREFETCH_AHEAD);
            edge_at(f1 + PREFETCH_AHEAD, a, b);
            for (int64_t k = 0; k < S; k += 8) {
                __builtin_prefetch(rows + (int64_t)a * S + k);
                __builtin_prefetch(rows + (int64_t)b * S + k);
            }
        }
        ++levels;
        if (lev.size() > SMALL_LEVEL) build_level_index();
        return true;
    }

    // Several-edge level: the incidence lists, every edge's head, the heap.
    void build_level_index() {
        const int m = (int)lev.size();
        inc_v.clear();
        for (int i = 0; i < m; ++i) {
            inc_v.push_back(lev[i].a);
            inc_v.push_back(lev[i].b);
        }
        std::vector<int32_t> &order = inc_order;
        order.resize(2 * m);
        for (int i = 0; i < 2 * m; ++i) order[i] = i;
        std::sort(order.begin(), order.end(),
                  [&](int32_t x, int32_t y) { return inc_v[x] < inc_v[y]; });
        inc_start.assign(n + 1, 0);
        inc_edge.resize(2 * m);
        for (int i = 0; i < 2 * m; ++i) {
            inc_edge[i] = order[i] >> 1;
            ++inc_start[inc_v[order[i]] + 1];
        }
        for (int64_t v = 0; v < n; ++v) inc_start[v + 1] += inc_start[v];
        if ((int64_t)is_dirty.size() < n) is_dirty.assign(n, 0);
        dirty.clear();
        lheap.clear();
        for (int i = 0; i < m; ++i) refresh_head(i);
    }

    void refresh_head(int i) {
        LevelEdge &E = lev[i];
        E.head = level_head(E);
        ++E.ver;
        if (E.head >= 0) {
            lheap.push_back({tri_index(*I.B, E.a, E.b, E.head), {i, E.ver}});
            std::push_heap(lheap.begin(), lheap.end());
        }
    }

    // Does the triangle {a, b, w} of level edge E belong to another edge of
    // the level (one of its other edges has the same length and a larger
    // index)?
    bool taken_by_other(const LevelEdge &E, int w) const {
        const float e = lvl_d;
        if (I.dist(E.a, w) == e) {
            const uint64_t o = E.a > w ? edge_index(E.a, w) : edge_index(w, E.a);
            if (o > E.idx) return true;
        }
        if (I.dist(E.b, w) == e) {
            const uint64_t o = E.b > w ? edge_index(E.b, w) : edge_index(w, E.b);
            if (o > E.idx) return true;
        }
        return false;
    }

    // Oldest triangle of edge E still to come that is odd now (w, or -1).
    int level_head(const LevelEdge &E) const {
        if (deg[E.a] == 0 && deg[E.b] == 0) {
            ++sweep_idle;
            return -1;
        }
        const uint64_t *Pa = P + (int64_t)E.a * S, *Pb = P + (int64_t)E.b * S;
        const uint64_t *Aa = adj + (int64_t)E.a * S, *Ab = adj + (int64_t)E.b * S;
        const uint64_t flip = vbit(E.a, E.b) ? ~0ull : 0ull;
        const bool shared = lev.size() > 1;
        int top = E.wpos - 1;
        if (top < 0) return -1;
        {  // most levels hold no odd triangle: test every word at once first
            const int64_t kt = top >> 6;
            const int sh = top & 63;
            uint64_t any = (Pa[kt] & Pb[kt] & (Aa[kt] ^ Ab[kt] ^ flip)) &
                           (sh < 63 ? (2ull << sh) - 1 : ~0ull);
            for (int64_t k = 0; k < kt; ++k) any |= Pa[k] & Pb[k] & (Aa[k] ^ Ab[k] ^ flip);
            if (!any) return -1;
        }
        while (top >= 0) {
            const int64_t k = top >> 6;
            uint64_t m = Pa[k] & Pb[k] & (Aa[k] ^ Ab[k] ^ flip);
            const int sh = top & 63;
            if (sh < 63) m &= (2ull << sh) - 1;
            while (m) {
                const int w = (int)(k << 6) + 63 - __builtin_clzll(m);
                if (!shared || !taken_by_other(E, w)) return w;
                m &= ~(1ull << (w & 63));
            }
            top = (int)(k << 6) - 1;
        }
        return -1;
    }

    // Start sweeping just past the entry k (the column is zero up to and
    // including k); the bits of V are set.
    void enter_sweep(u128 k) {
        cur.clear();
        heap.clear();
        sweep = true;
        swept = true;
        P = rows;
        deg.assign(n, 0);
        for (uint64_t e : V) {  // V has no repeats here (heap mode or a rebuilt set)
            int x, y;
            edge_vertices(e, x, y);
            ++deg[x];
            ++deg[y];
        }
        const float dk = key_diam(k);
        const uint64_t kidx = key_index(k);
        // P: every edge shorter than dk (the neighbour rows are sorted by distance)
        const uint32_t bd = float_bits(dk);
        for (int64_t a = 0; a < n; ++a) {
            const uint64_t *row = I.nbr + a * n;
            uint64_t *Pa = P + a * S;
            for (int64_t i = 0; i < n && (uint32_t)(row[i] >> 32) < bd; ++i) {
                const int w = (int)(uint32_t)row[i];
                if (w != a) Pa[w >> 6] |= 1ull << (w & 63);
            }
        }
        // position the level source at the first edge of length dk
        if (I.edge_ab) {
            eab = I.edge_ab;
            ehi = I.edge_hi;
            ne = eready = I.nedges;
            int64_t lo = 0, hi = ne;  // filtration order, diameter ascending
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (float_bits(diam_at(mid)) < bd) lo = mid + 1;
                else hi = mid;
            }
            f1 = lo;
        } else {
            elist = R.level_edges(dk);
            eab = elist->ab.get();
            ehi = elist->hi.get();
            ne = elist->m;
            f1 = elist->first_at(bd, &ebucket);
            eready = f1 < ne ? elist->bstart[ebucket + 1] : ne;
        }
        if (!next_level() || lvl_d != dk) {  // cannot happen: k is a triangle inside the threshold
            lev.clear();
            return;
        }
        int kv[3];
        decode_host(*I.B, kidx, 2, n, kv);
        for (LevelEdge &E : lev) {  // triangles of index below k's are still to come
            int l = -1, h = (int)n;
            while (h - l > 1) {
                const int mid = (l + h) >> 1;
                if (tri_before(E.a, E.b, mid, kv)) l = mid;
                else h = mid;
            }
            E.wpos = l + 1;
        }
        if (lev.size() > SMALL_LEVEL) build_level_index();  // heads from the positions just set
    }

    // Oldest nonzero entry in sweep mode; the sweep moves past it.
    u128 pivot_sweep() {
        const u128 k = pivot_sweep_levels();
        if (k != NONE) ++sweep_pivots;
        return k;
    }
    u128 pivot_sweep_levels() {
        for (;;) {
            if (lev.size() == 1) {
                LevelEdge &E = lev[0];
                const int w = level_head(E);
                if (w >= 0) {
                    E.wpos = w;
                    piv_a = E.a, piv_b = E.b, piv_w = w;
                    return age_key(lvl_d, tri_index(*I.B, E.a, E.b, w));
                }
            } else if (lev.size() <= SMALL_LEVEL) {
                int best = -1, bw = -1;
                uint64_t bidx = 0;
                for (int i = 0; i < (int)lev.size(); ++i) {
                    const int w = level_head(lev[i]);
                    if (w < 0) continue;
                    const uint64_t ti = tri_index(*I.B, lev[i].a, lev[i].b, w);
                    if (best < 0 || ti > bidx) {
                        best = i;
                        bw = w;
                        bidx = ti;
                    }
                }
                if (best >= 0) {
                    piv_a = lev[best].a, piv_b = lev[best].b, piv_w = bw;
                    for (int i = 0; i < (int)lev.size(); ++i) {  // index >= bidx has been passed
                        LevelEdge &E = lev[i];
                        if (i == best) E.wpos = bw;
                        else
                            while (E.wpos > 0 && tri_index(*I.B, E.a, E.b, E.wpos - 1) > bidx)
                                --E.wpos;
                    }
                    return age_key(lvl_d, bidx);
                }
            } else {
                for (int32_t v : dirty) {
                    is_dirty[v] = 0;
                    for (int32_t j = inc_start[v]; j < inc_start[v + 1]; ++j) refresh_head(inc_edge[j]);
                }
                dirty.clear();
                while (!lheap.empty()) {
                    const auto top = lheap.front();
                    std::pop_heap(lheap.begin(), lheap.end());
                    lheap.pop_back();
                    LevelEdge &E = lev[top.second.first];
                    if (top.second.second != E.ver || E.head < 0) continue;  // stale
                    E.wpos = E.head;  // taken: its younger triangles are still to come
                    piv_a = E.a, piv_b = E.b, piv_w = E.head;
                    refresh_head(top.second.first);
                    return age_key(lvl_d, top.first);
                }
            }
            if (!next_level()) return NONE;
        }
    }

    // The apparent column owning the last pivot, if any (as
    // Reducer::apparent_owner, from the definition): its youngest facet s
    // (largest diameter, then smallest index) owns it iff the pivot is the
    // oldest cofacet of s, i.e. the vertex it adds to s is the largest vertex
    // within the level's diameter of both ends of s, which P gives (s has the
    // pivot's diameter, the current level's).
    bool sweep_owner(int *s, int *added) const {
        int v[3] = {piv_a, piv_b, piv_w};
        if (v[2] > v[0]) std::swap(v[0], v[2]), std::swap(v[1], v[2]);
        else if (v[2] > v[1]) std::swap(v[1], v[2]);
        const float fd[3] = {I.dist(v[1], v[2]), I.dist(v[0], v[2]), I.dist(v[0], v[1])};
        int r = 0;  // facets in increasing index: without v[0], v[1], v[2]
        for (int i = 1; i < 3; ++i)
            if (fd[i] > fd[r]) r = i;
        if (fd[r] != lvl_d) return false;
        const int x = r == 0 ? v[1] : v[0], y = r == 2 ? v[1] : v[2];
        const uint64_t *Px = P + (int64_t)x * S, *Py = P + (int64_t)y * S;
        for (int64_t k = W - 1; k >= 0; --k) {
            const uint64_t m = Px[k] & Py[k];
            if (m) {
                if ((int)(k << 6) + 63 - __builtin_clzll(m) != v[r]) return false;
                s[0] = x;
                s[1] = y;
                *added = v[r];
                return true;
            }
        }
        return false;
    }

    // A sweep-mode addition of the edge e: a bit flip.
    void toggle_edge(uint64_t e) {
        int x, y;
        edge_vertices(e, x, y);
        const int32_t d = vbit(x, y) ? -1 : 1;  // leaves V, or enters it
        deg[x] += d;
        deg[y] += d;
        adj[(int64_t)x * S + (y >> 6)] ^= 1ull << (y & 63);
        adj[(int64_t)y * S + (x >> 6)] ^= 1ull << (x & 63);
        V.push_back(e);
        if (lev.size() > SMALL_LEVEL)
            for (int v : {x, y})
                if (!is_dirty[v]) {
                    is_dirty[v] = 1;
                    dirty.push_back(v);
                }
    }

    void clear_plane() {
        if (P)
            for (int64_t a = 0; a < n; ++a) std::memset(P + a * S, 0, (size_t)W * sizeof(uint64_t));
        P = nullptr;
    }
};


// The bit rows of a walk (n rows of 2 ceil(n / 64) words), owned by the
// calling thread and clear.
uint64_t *adjacency_scratch(int64_t n) {
    thread_local std::vector<uint64_t> bits;
    const size_t words = (size_t)(n * 2 * ((n + 63) / 64));
    if (bits.size() < words) bits.assign(words, 0);
    return bits.data();
}

template <class K>
void reduce_p1(const HostInstance &I, const Leftover *left, int64_t nleft, int threads,
               std::vector<HostPair> &out, ReduceStats &stats) {
    Reducer R(I, 1);
    std::vector<u128> piv(nleft, NONE);
    std::vector<std::vector<uint64_t>> V(nleft);  // reduced columns as edge sets
    std::vector<char> walked(nleft, 0);
    std::vector<int64_t> adds(nleft, 0), reads(nleft, 0), entries(nleft, 0), levels(nleft, 0);
    std::vector<int64_t> spiv(nleft, 0), sidle(nleft, 0);
    std::vector<double> sms(nleft, 0.0);
    Ledger<K> led(V, nleft, bits_of(I.B->at(3, I.n)));
    for (int64_t j = 0; j < nleft; ++j)
        if (left[j].pivot != NO_PIVOT) led.advance(j, age_key(left[j].pdiam, left[j].pivot));

    auto column = [&](int64_t j) {
        const Leftover &L = left[j];
        V[j].push_back(L.sigma);
        if (L.pivot == NO_PIVOT) {
            led.finish(j, NONE);
            return;
        }
        const u128 k0 = age_key(L.pdiam, L.pivot);
        int s[3], added;
        ++reads[j];
        if (!R.apparent_owner(k0, s, &added) && led.query(j, k0) < 0) {
            piv[j] = k0;  // the unreduced pivot is free
            led.finish(j, k0);
            return;
        }
        Walk1<K> W(I, R, adjacency_scratch(I.n), threads);
        int v[2];
        decode_host(*I.B, L.sigma, 1, I.n, v);
        const auto w0 = std::chrono::steady_clock::now();
        W.add_edge(v[0], v[1], L.diam, first_vertex(R, L, v));
        const u128 k = W.walk(led, j);
        if (W.swept)
            sms[j] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0)
                         .count();
        spiv[j] = W.sweep_pivots;
        sidle[j] = W.sweep_idle;
        V[j] = W.edges();
        piv[j] = k;
        walked[j] = 1;
        adds[j] = W.additions;
        reads[j] += W.reads;
        entries[j] = W.entries;
        levels[j] = W.levels;
        led.finish(j, k);
    };
    // columns start in increasing order (the pool hands out indices in order)
    if (threads <= 1 || nleft < 16) {
        for (int64_t j = 0; j < nleft; ++j) column(j);
    } else {
        pool(threads).parallel_for(nleft, column);
    }

    for (int64_t j = 0; j < nleft; ++j) {
        const Leftover &L = left[j];
        HostPair P;
        P.sigma = L.sigma;
        P.birth = L.diam;
        if (piv[j] == NONE) {
            P.tau = NO_PIVOT;
            P.death = INFINITY;
        } else {
            P.tau = key_index(piv[j]);
            P.death = key_diam(piv[j]);
            if (!walked[j]) ++stats.free_pivot;
        }
        out.push_back(P);
        stats.additions += adds[j];
        stats.reads += reads[j];
        stats.entries += entries[j];
        stats.levels += levels[j];
        stats.sweep_pivots += spiv[j];
        stats.sweep_idle += sidle[j];
        stats.sweep_walk_ms += sms[j];
    }
}

}  // namespace

void reduce_leftovers(const HostInstance &I, int p, const Leftover *left, int64_t nleft,
                      int threads, std::vector<HostPair> &out, ReduceStats &stats) {
#ifdef RPP_WIDE_KEYS_ONLY  // tests build the 128-bit key path for small inputs too
    const bool narrow = false;
#else
    const bool narrow = I.B->at(3, I.n) <= (1ull << 32);
#endif
    if (p == 1 && narrow)  // triangle indices fit in 32 bits
        reduce_p1<Key64>(I, left, nleft, threads, out, stats);
    else if (p == 1)
        reduce_p1<Key128>(I, left, nleft, threads, out, stats);
    else reduce_general(I, p, left, nleft, threads, out, stats);
}

}  // namespace rpp
