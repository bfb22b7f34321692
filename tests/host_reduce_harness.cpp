// Test harness for the library's host reduction (csrc/host.cpp) without a GPU.
//
// It reads a symmetric float32 distance matrix, prepares on the CPU what the
// GPU stages hand to the host reduction -- the edges inside the threshold in
// coboundary order, Kruskal's merging edges (cleared), the apparent pairs by
// their definition, the leftover columns with their unreduced pivots, and the
// per-vertex neighbour rows -- runs reduce_leftovers for dimension 1 and
// writes the nonzero H1 intervals. Test code only: the product never links it.
//
//   host_reduce_harness D.f32 n t threads flags out.f32
//     t        threshold (inf: the enclosing radius, as the library does)
//     flags    bit 0: no sorted edge array (the reduction sorts the edges itself)
//              bit 1: no apparent array (apparent pivots tested again)
//   out.f32    (birth, death) float32 pairs of the nonzero H1 intervals
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "host.h"

using namespace rpp;

static uint32_t fbits(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

int main(int argc, char **argv) {
    if (argc < 7) {
        std::fprintf(stderr, "usage: %s D.f32 n t threads flags out.f32\n", argv[0]);
        return 2;
    }
    const int n = std::atoi(argv[2]);
    const float t_user = (float)std::atof(argv[3]);
    const int threads = std::atoi(argv[4]);
    const int flags = std::atoi(argv[5]);
    std::vector<float> Din((size_t)n * n);
    FILE *f = std::fopen(argv[1], "rb");
    if (!f || std::fread(Din.data(), 4, Din.size(), f) != Din.size()) return 3;
    std::fclose(f);
    const int64_t ld = (n + 31) / 32 * 32;
    std::vector<float> D((size_t)n * ld, 0.0f);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) D[(size_t)i * ld + j] = Din[(size_t)i * n + j];
    // threshold: min(t, enclosing radius)
    float R = INFINITY;
    for (int i = 0; i < n; ++i) {
        float m = 0.0f;
        for (int j = 0; j < n; ++j) m = std::max(m, D[(size_t)i * ld + j]);
        R = std::min(R, m);
    }
    const float t = std::min(t_user, R);
    // binomial table C(v, k), k = 0..3
    std::vector<uint64_t> store(4 * (size_t)(n + 1), 0);
    for (int v = 0; v <= n; ++v) {
        store[v] = 1;
        for (int k = 1; k <= 3; ++k)
            store[(size_t)k * (n + 1) + v] =
                v == 0 ? 0 : store[(size_t)(k - 1) * (n + 1) + v - 1] + store[(size_t)k * (n + 1) + v - 1];
    }
    Binomial B;
    B.n = n;
    B.kmax = 3;
    B.host = store.data();
    // edges inside t in coboundary order: diameter descending, index ascending
    struct Edge {
        float d;
        uint64_t idx;
        int x, y;
    };
    std::vector<Edge> E;
    for (int x = 1; x < n; ++x)
        for (int y = 0; y < x; ++y) {
            const float d = D[(size_t)x * ld + y];
            if (d <= t) E.push_back({d, (uint64_t)x * (x - 1) / 2 + y, x, y});
        }
    std::sort(E.begin(), E.end(), [](const Edge &a, const Edge &b) {
        return a.d != b.d ? a.d > b.d : a.idx < b.idx;
    });
    const int64_t ne = (int64_t)E.size();
    // Kruskal in filtration order: its merging edges are cleared
    std::vector<int> par(n);
    for (int i = 0; i < n; ++i) par[i] = i;
    auto find = [&](int a) {
        while (par[a] != a) a = par[a] = par[par[a]];
        return a;
    };
    std::vector<char> cleared(ne, 0);
    for (int64_t k = ne - 1; k >= 0; --k) {
        const int a = find(E[k].x), b = find(E[k].y);
        if (a != b) {
            par[a] = b;
            cleared[k] = 1;
        }
    }
    // apparent pairs by the definition; leftovers with their oldest cofacet
    std::vector<uint64_t> app;
    std::vector<Leftover> left;
    for (int64_t k = 0; k < ne; ++k) {
        if (cleared[k]) continue;
        const Edge &e = E[k];
        int bw = -1;
        float bd = INFINITY;
        for (int w = n - 1; w >= 0; --w) {  // oldest cofacet: smallest diameter, then largest w
            if (w == e.x || w == e.y) continue;
            const float m = std::max(e.d, std::max(D[(size_t)e.x * ld + w], D[(size_t)e.y * ld + w]));
            if (m <= t && m < bd) {
                bd = m;
                bw = w;
            }
        }
        uint64_t tidx = NO_PIVOT;
        bool apparent = false;
        if (bw >= 0) {
            int v[3] = {e.x, e.y, bw};
            std::sort(v, v + 3, [](int a, int b) { return a > b; });
            tidx = B.at(3, v[0]) + B.at(2, v[1]) + (uint64_t)v[2];
            if (bd == e.d) {  // youngest facet of tau: facets in increasing index
                const int fa[3][2] = {{v[1], v[2]}, {v[0], v[2]}, {v[0], v[1]}};
                for (int r = 0; r < 3; ++r)
                    if (D[(size_t)fa[r][0] * ld + fa[r][1]] == e.d) {
                        apparent = (uint64_t)fa[r][0] * (fa[r][0] - 1) / 2 + fa[r][1] == e.idx;
                        break;
                    }
            }
        }
        if (apparent) app.push_back(tidx);
        else left.push_back({e.idx, tidx, e.d, bw >= 0 ? bd : 0.0f, (uint64_t)k});
    }
    std::sort(app.begin(), app.end());
    // neighbour rows: (bits(distance) << 32) | vertex, ascending
    std::vector<uint64_t> nbr((size_t)n * n);
    for (int r = 0; r < n; ++r) {
        uint64_t *row = &nbr[(size_t)r * n];
        for (int i = 0; i < n; ++i) row[i] = ((uint64_t)fbits(D[(size_t)r * ld + i]) << 32) | (uint64_t)i;
        std::sort(row, row + n);
    }
    std::vector<uint32_t> eab(ne), ehi(ne);
    for (int64_t k = 0; k < ne; ++k) {
        eab[k] = ((uint32_t)E[k].x << 16) | (uint32_t)E[k].y;
        ehi[k] = ~fbits(E[k].d);
    }
    HostInstance I;
    I.n = n;
    I.D = D.data();
    I.ld = ld;
    I.B = &B;
    I.nbr = nbr.data();
    I.t = t;
    if (!(flags & 1)) {
        I.edge_ab = eab.data();
        I.edge_hi = ehi.data();
        I.nedges = ne;
    }
    if (!(flags & 2)) {
        I.app_tau = app.data();
        I.napp = app.size();
    }
    std::vector<HostPair> out;
    ReduceStats st;
    reduce_leftovers(I, 1, left.data(), (int64_t)left.size(), threads, out, st);
    FILE *o = std::fopen(argv[6], "wb");
    if (!o) return 4;
    for (const HostPair &P : out)
        if (P.tau == NO_PIVOT || P.death > P.birth) {
            std::fwrite(&P.birth, 4, 1, o);
            std::fwrite(&P.death, 4, 1, o);
        }
    std::fclose(o);
    std::printf("leftover %zu additions %lld levels %lld\n", left.size(), (long long)st.additions,
                (long long)st.levels);
    return 0;
}
