// CPU oracle for the dynamic graph store and its algorithms.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, imports or
// calls this file; only the tests, the smoke check and the benchmark's CPU
// baseline arm do.  It shares no code, header, constant or helper with the
// CUDA path.
//
// It computes the plain definitions that the paper's method reaches exactly,
// and nothing of the method itself (no slabs, hashing, frontiers, iterators
// or incremental/decremental bookkeeping): every algorithm is rerun from
// scratch on the current edge set.
//
//  * Edge set (Sec. "Experimental Evaluation", insertion/deletion/query
//    discussion): an edge is stored only if it is not already present, a
//    delete removes a present edge (and is a no-op otherwise), a query reports
//    presence and, for the weighted store, the stored weight.  A batch is
//    applied in batch order, so among repeated (src, dst) pairs of one insert
//    batch the first occurrence is the one stored.
//  * Shortest-path tree (Sec. "Dynamic Single Source Shortest Path and Breadth
//    First Search"): every vertex v carries <distance(v), parent(v)>; the source
//    is <0, SRC>, unreachable vertices are <INF, INVALID>.  Distances are
//    Dijkstra's (weighted) or FIFO BFS hop counts (unweighted).  The parent is
//    the smallest vertex id u with a live edge (u, v) and distance(u) + w(u, v)
//    == distance(v): the tie-break that a 64-bit atomicMin over the packed
//    <distance, parent> pair settles on (footnote on the tree-node packing).
//  * Weakly connected components (Sec. "Incremental WCC"): vertices joined by
//    a path that ignores edge direction share a label; the label is the
//    smallest vertex id of the component.
//  * PageRank (Sec. "Dynamic PageRank", Eq. 1 and the teleport term of its
//    algorithm): power iteration in double precision, PR[v] = (1 - d) / N +
//    d * (sum over edges u -> v of PR[u] / out(u) + T / N) with T the rank of
//    the vertices without out-edges, until the L1 change is <= eps.
//  * Triangles (Sec. "Dynamic Triangle Counting"): the number of vertex
//    triples pairwise joined by an edge of either direction (self-loops
//    ignored).
//
// Vertex ids are 32-bit; the value 0xFFFFFFFF stands for INF / INVALID.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <queue>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;

struct OracleGraph {
    uint32_t V;
    std::unordered_map<uint64_t, uint32_t> edges; // (src << 32 | dst) -> weight
};

uint64_t edge_key(uint32_t s, uint32_t d) { return (uint64_t(s) << 32) | d; }

// Adjacency in compressed-row form, built from the edge set on demand.
struct Csr {
    std::vector<uint64_t> off;
    std::vector<uint32_t> dst;
    std::vector<uint32_t> w;
};

Csr build_csr(const OracleGraph &g)
{
    Csr c;
    c.off.assign(size_t(g.V) + 1, 0);
    for (const auto &e : g.edges)
        c.off[(e.first >> 32) + 1]++;
    for (uint32_t v = 0; v < g.V; ++v)
        c.off[v + 1] += c.off[v];
    c.dst.resize(g.edges.size());
    c.w.resize(g.edges.size());
    std::vector<uint64_t> fill(c.off.begin(), c.off.end() - 1);
    for (const auto &e : g.edges) {
        uint32_t s = uint32_t(e.first >> 32);
        uint64_t at = fill[s]++;
        c.dst[at] = uint32_t(e.first);
        c.w[at] = e.second;
    }
    return c;
}

// parent(v) = min u over live (u, v) with dist[u] + w == dist[v]; the source
// is its own parent, unreachable vertices have none.
void min_tight_parents(const OracleGraph &g, uint32_t source, bool unit, const std::vector<uint64_t> &dist,
                       uint32_t *parent)
{
    const uint64_t inf = ~uint64_t(0);
    for (uint32_t v = 0; v < g.V; ++v)
        parent[v] = kNone;
    for (const auto &e : g.edges) {
        uint32_t u = uint32_t(e.first >> 32), v = uint32_t(e.first);
        if (dist[u] == inf || dist[v] == inf || v == source)
            continue;
        uint64_t w = unit ? 1 : e.second;
        if (dist[u] + w == dist[v] && u < parent[v])
            parent[v] = u;
    }
    if (source < g.V)
        parent[source] = source;
}

} // namespace

extern "C" {

void *orc_create(uint32_t V)
{
    OracleGraph *g = new OracleGraph;
    g->V = V;
    return g;
}

void orc_destroy(void *h) { delete static_cast<OracleGraph *>(h); }

uint64_t orc_num_edges(void *h) { return static_cast<OracleGraph *>(h)->edges.size(); }

// Insert in batch order; flags[i] = 1 iff edge i was absent and is now stored
// with weight w[i] (w == nullptr stores weight 1).
void orc_insert(void *h, const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t n,
                uint8_t *flags)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    for (uint64_t i = 0; i < n; ++i) {
        auto r = g->edges.emplace(edge_key(src[i], dst[i]), w ? w[i] : 1u);
        if (flags)
            flags[i] = r.second ? 1 : 0;
    }
}

// Delete in batch order; flags[i] = 1 iff edge i was present and is now gone.
void orc_delete(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *flags)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    for (uint64_t i = 0; i < n; ++i) {
        size_t erased = g->edges.erase(edge_key(src[i], dst[i]));
        if (flags)
            flags[i] = erased ? 1 : 0;
    }
}

// bitmap bit (i % 32) of word (i / 32) = presence of edge i; w_out[i] = stored
// weight if present, 0 otherwise.  bitmap has ceil(n / 32) words.
void orc_query(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint32_t *bitmap,
               uint32_t *w_out)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    std::memset(bitmap, 0, ((n + 31) / 32) * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; ++i) {
        auto it = g->edges.find(edge_key(src[i], dst[i]));
        bool hit = it != g->edges.end();
        if (hit)
            bitmap[i / 32] |= 1u << (i % 32);
        if (w_out)
            w_out[i] = hit ? it->second : 0u;
    }
}

// Live edges sorted by (src, dst).
void orc_export(void *h, uint32_t *src, uint32_t *dst, uint32_t *w)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    std::vector<std::pair<uint64_t, uint32_t>> all(g->edges.begin(), g->edges.end());
    std::sort(all.begin(), all.end());
    for (size_t i = 0; i < all.size(); ++i) {
        src[i] = uint32_t(all[i].first >> 32);
        dst[i] = uint32_t(all[i].first);
        w[i] = all[i].second;
    }
}

void orc_out_degree(void *h, uint32_t *deg)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    std::memset(deg, 0, size_t(g->V) * sizeof(uint32_t));
    for (const auto &e : g->edges)
        deg[e.first >> 32]++;
}

// Breadth-first search from `source` with a FIFO queue: dist = hop count.
// Returns 0.
int orc_bfs(void *h, uint32_t source, uint32_t *dist_out, uint32_t *parent_out)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    const uint64_t inf = ~uint64_t(0);
    Csr c = build_csr(*g);
    std::vector<uint64_t> dist(g->V, inf);
    std::queue<uint32_t> q;
    dist[source] = 0;
    q.push(source);
    while (!q.empty()) {
        uint32_t u = q.front();
        q.pop();
        for (uint64_t k = c.off[u]; k < c.off[u + 1]; ++k) {
            uint32_t v = c.dst[k];
            if (dist[v] == inf) {
                dist[v] = dist[u] + 1;
                q.push(v);
            }
        }
    }
    for (uint32_t v = 0; v < g->V; ++v)
        dist_out[v] = dist[v] == inf ? kNone : uint32_t(dist[v]);
    min_tight_parents(*g, source, true, dist, parent_out);
    return 0;
}

// Dijkstra from `source` with a binary heap and 64-bit path sums.  Returns 0,
// or 1 if some shortest distance does not fit below 0xFFFFFFFF (then the
// 32-bit outputs of those vertices are clamped to 0xFFFFFFFE).
int orc_sssp(void *h, uint32_t source, uint32_t *dist_out, uint32_t *parent_out)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    const uint64_t inf = ~uint64_t(0);
    Csr c = build_csr(*g);
    std::vector<uint64_t> dist(g->V, inf);
    using Item = std::pair<uint64_t, uint32_t>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    dist[source] = 0;
    pq.push({0, source});
    while (!pq.empty()) {
        auto [d, u] = pq.top();
        pq.pop();
        if (d != dist[u])
            continue;
        for (uint64_t k = c.off[u]; k < c.off[u + 1]; ++k) {
            uint32_t v = c.dst[k];
            uint64_t nd = d + c.w[k];
            if (nd < dist[v]) {
                dist[v] = nd;
                pq.push({nd, v});
            }
        }
    }
    int overflow = 0;
    for (uint32_t v = 0; v < g->V; ++v) {
        if (dist[v] == inf) {
            dist_out[v] = kNone;
        } else if (dist[v] >= kNone) {
            dist_out[v] = kNone - 1;
            overflow = 1;
        } else {
            dist_out[v] = uint32_t(dist[v]);
        }
    }
    min_tight_parents(*g, source, false, dist, parent_out);
    return overflow;
}

// Weakly connected components: union-find over every live edge with edge
// direction ignored, then label = smallest vertex id of each component.
void orc_wcc(void *h, uint32_t *label)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    std::vector<uint32_t> up(g->V);
    for (uint32_t v = 0; v < g->V; ++v)
        up[v] = v;
    std::function<uint32_t(uint32_t)> find = [&](uint32_t x) {
        uint32_t r = x;
        while (up[r] != r)
            r = up[r];
        while (up[x] != r) {
            uint32_t nx = up[x];
            up[x] = r;
            x = nx;
        }
        return r;
    };
    for (const auto &e : g->edges) {
        uint32_t a = find(uint32_t(e.first >> 32)), b = find(uint32_t(e.first));
        if (a != b)
            up[std::max(a, b)] = std::min(a, b);
    }
    std::vector<uint32_t> smallest(g->V, kNone);
    for (uint32_t v = 0; v < g->V; ++v) {
        uint32_t r = find(v);
        smallest[r] = std::min(smallest[r], v);
    }
    for (uint32_t v = 0; v < g->V; ++v)
        label[v] = smallest[find(v)];
}

// PageRank by power iteration (see the header).  init (nullable): starting
// ranks, else 1 / V each.  Writes V ranks to out and the number of
// iterations run to *iters.
void orc_pagerank(void *h, double damping, double eps, uint32_t max_iter, const double *init, double *out,
                  uint32_t *iters)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    const uint32_t V = g->V;
    std::vector<uint32_t> outdeg(V, 0);
    for (const auto &e : g->edges)
        outdeg[e.first >> 32]++;
    std::vector<double> pr(V), next(V);
    for (uint32_t v = 0; v < V; ++v)
        pr[v] = init ? init[v] : 1.0 / V;
    uint32_t it = 0;
    while (it < max_iter) {
        double teleport = 0;
        for (uint32_t v = 0; v < V; ++v)
            if (outdeg[v] == 0)
                teleport += pr[v];
        std::vector<double> sum(V, 0.0);
        for (const auto &e : g->edges) {
            const uint32_t u = uint32_t(e.first >> 32), v = uint32_t(e.first);
            sum[v] += pr[u] / outdeg[u];
        }
        double delta = 0;
        for (uint32_t v = 0; v < V; ++v) {
            next[v] = (1.0 - damping) / V + damping * (sum[v] + teleport / V);
            delta += std::fabs(next[v] - pr[v]);
        }
        pr.swap(next);
        ++it;
        if (delta <= eps)
            break;
    }
    for (uint32_t v = 0; v < V; ++v)
        out[v] = pr[v];
    *iters = it;
}

// Triangles of the undirected simple graph underlying the edge set: each
// triple u < v < w with all three pairs adjacent is counted once.
uint64_t orc_triangles(void *h)
{
    OracleGraph *g = static_cast<OracleGraph *>(h);
    std::vector<std::vector<uint32_t>> nb(g->V);
    for (const auto &e : g->edges) {
        const uint32_t u = uint32_t(e.first >> 32), v = uint32_t(e.first);
        if (u == v)
            continue;
        nb[u].push_back(v);
        nb[v].push_back(u);
    }
    for (auto &x : nb) {
        std::sort(x.begin(), x.end());
        x.erase(std::unique(x.begin(), x.end()), x.end());
    }
    uint64_t count = 0;
    for (uint32_t u = 0; u < g->V; ++u)
        for (uint32_t v : nb[u]) {
            if (v <= u)
                continue;
            for (uint32_t w : nb[v])
                if (w > v && std::binary_search(nb[u].begin(), nb[u].end(), w))
                    ++count;
        }
    return count;
}

} // extern "C"
