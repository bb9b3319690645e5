// Multi-core CPU baseline of the batched edge operations (TEST AND
// BENCHMARK INFRASTRUCTURE ONLY; nothing in the library path uses it).
//
// The same edge-set semantics as oracle.cpp (Sec. "Experimental
// Evaluation", insertion/deletion/query: an edge is stored only if absent,
// a delete removes a present edge, a query reports presence and the stored
// weight; a batch is applied in batch order), with the edge set partitioned
// by source vertex over T shards, one host thread per shard.  Every thread
// scans the whole batch and applies, in batch order, the edges whose source
// falls in its shard; since all edges of one (src, dst) pair fall in one
// shard, the outcome equals the sequential one.  Plain C++17 with
// std::thread, no platform intrinsics.
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

struct Sharded {
    uint32_t V;
    uint32_t T;
    std::vector<std::unordered_map<uint64_t, uint32_t>> shard; // (src << 32 | dst) -> weight
};

inline uint64_t key_of(uint32_t s, uint32_t d) { return (uint64_t(s) << 32) | d; }
inline uint32_t shard_of(const Sharded &g, uint32_t s) { return s % g.T; }

template <class F> void on_all_shards(const Sharded &g, F f)
{
    std::vector<std::thread> th;
    th.reserve(g.T);
    for (uint32_t t = 0; t < g.T; ++t)
        th.emplace_back(f, t);
    for (auto &x : th)
        x.join();
}

} // namespace

extern "C" {

void *shd_create(uint32_t V, uint32_t threads)
{
    Sharded *g = new Sharded;
    g->V = V;
    g->T = threads ? threads : 1;
    g->shard.resize(g->T);
    return g;
}

void shd_destroy(void *h) { delete static_cast<Sharded *>(h); }

uint64_t shd_num_edges(void *h)
{
    const Sharded *g = static_cast<Sharded *>(h);
    uint64_t m = 0;
    for (const auto &s : g->shard)
        m += s.size();
    return m;
}

// flags[i] (nullable) = 1 iff edge i was absent and is now stored.
void shd_insert(void *h, const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t n, uint8_t *flags)
{
    Sharded *g = static_cast<Sharded *>(h);
    on_all_shards(*g, [&](uint32_t t) {
        auto &m = g->shard[t];
        for (uint64_t i = 0; i < n; ++i) {
            if (shard_of(*g, src[i]) != t)
                continue;
            const bool added = m.emplace(key_of(src[i], dst[i]), w ? w[i] : 1u).second;
            if (flags)
                flags[i] = added ? 1 : 0;
        }
    });
}

// flags[i] (nullable) = 1 iff edge i was present and is now removed.
void shd_delete(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *flags)
{
    Sharded *g = static_cast<Sharded *>(h);
    on_all_shards(*g, [&](uint32_t t) {
        auto &m = g->shard[t];
        for (uint64_t i = 0; i < n; ++i) {
            if (shard_of(*g, src[i]) != t)
                continue;
            const bool gone = m.erase(key_of(src[i], dst[i])) != 0;
            if (flags)
                flags[i] = gone ? 1 : 0;
        }
    });
}

// hit[i] = presence of edge i, w_out[i] (nullable) = stored weight or 0.
void shd_query(void *h, const uint32_t *src, const uint32_t *dst, uint64_t n, uint8_t *hit, uint32_t *w_out)
{
    Sharded *g = static_cast<Sharded *>(h);
    on_all_shards(*g, [&](uint32_t t) {
        const auto &m = g->shard[t];
        for (uint64_t i = 0; i < n; ++i) {
            if (shard_of(*g, src[i]) != t)
                continue;
            auto it = m.find(key_of(src[i], dst[i]));
            hit[i] = it != m.end() ? 1 : 0;
            if (w_out)
                w_out[i] = it != m.end() ? it->second : 0u;
        }
    });
}

} // extern "C"
