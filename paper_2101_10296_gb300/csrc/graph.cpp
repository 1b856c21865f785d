// Graph validation and CSR construction.
#include <algorithm>
#include <cstdio>

#include "host.hpp"

namespace qaoa {

int build_graph(int32_t n, int64_t m, const int32_t *edges, const int32_t *weights, Graph &g, std::string &err) {
    if (n < 0 || m < 0 || (m > 0 && edges == nullptr)) {
        err = "invalid graph sizes or NULL edge array";
        return QAOA_E_INVALID;
    }
    g.n = n;
    g.m = m;
    g.eu.resize(m);
    g.ev.resize(m);
    g.ew.assign(size_t(m), 1);
    if (weights) {
        for (int64_t e = 0; e < m; ++e) {
            const int32_t w = weights[e];
            if (w == 0 || w > QAOA_MAX_CONE_EDGES || w < -QAOA_MAX_CONE_EDGES) {
                char buf[128];
                snprintf(buf, sizeof buf, "edge %lld has weight %d (need 1 <= |w| <= %d)", (long long)e, w,
                         QAOA_MAX_CONE_EDGES);
                err = buf;
                return QAOA_E_INVALID;
            }
            g.ew[e] = w;
        }
    }
    std::vector<int64_t> deg(size_t(n) + 1, 0);
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n) {
            char buf[128];
            snprintf(buf, sizeof buf, "edge %lld has a vertex outside [0, %d)", (long long)e, n);
            err = buf;
            return QAOA_E_INVALID;
        }
        if (a == b) {
            char buf[96];
            snprintf(buf, sizeof buf, "edge %lld is a self-loop", (long long)e);
            err = buf;
            return QAOA_E_INVALID;
        }
        g.eu[e] = std::min(a, b);
        g.ev[e] = std::max(a, b);
        deg[a]++;
        deg[b]++;
    }
    g.off.assign(size_t(n) + 1, 0);
    for (int32_t v = 0; v < n; ++v) g.off[v + 1] = g.off[v] + deg[v];
    g.adj.resize(size_t(2 * m));
    g.eid.resize(size_t(2 * m));
    std::vector<int64_t> fill(g.off.begin(), g.off.end() - 1);
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = g.eu[e], b = g.ev[e];
        g.adj[fill[a]] = b;
        g.eid[fill[a]++] = e;
        g.adj[fill[b]] = a;
        g.eid[fill[b]++] = e;
    }
    std::vector<std::pair<int32_t, int64_t>> tmp;
    for (int32_t v = 0; v < n; ++v) {
        int64_t s = g.off[v], t = g.off[v + 1];
        tmp.clear();
        for (int64_t k = s; k < t; ++k) tmp.emplace_back(g.adj[k], g.eid[k]);
        std::sort(tmp.begin(), tmp.end());
        for (int64_t k = s; k < t; ++k) {
            g.adj[k] = tmp[k - s].first;
            g.eid[k] = tmp[k - s].second;
            if (k > s && g.adj[k] == g.adj[k - 1]) {
                char buf[128];
                snprintf(buf, sizeof buf, "repeated edge between %d and %d", v, g.adj[k]);
                err = buf;
                return QAOA_E_INVALID;
            }
        }
    }
    return QAOA_OK;
}

int64_t find_edge(const Graph &g, int32_t a, int32_t b) {
    auto first = g.adj.begin() + g.off[a];
    auto last = g.adj.begin() + g.off[a + 1];
    auto it = std::lower_bound(first, last, b);
    if (it == last || *it != b) return -1;
    return g.eid[size_t(it - g.adj.begin())];
}

}  // namespace qaoa
