// Serving engine: continuous batching of mixed requests on one graph.  The
// paper has no serving layer; this is a project addition built on the
// library's calls.
//
// Requests (query, insert, delete, incremental SSSP) are queued in arrival
// order and admitted by mk_server_progress as in-flight slots and slab-pool
// memory allow.  Consecutive read requests form one group: all its queries
// go out as one CUDA-graph replay of the multi-request query kernel (the
// batcher) on the query stream, its SSSP requests run on the SSSP stream, so
// the two overlap on the device; both wait for the last update.  A run of
// consecutive updates of one kind is one merged batch (mk_update_multi) and
// a barrier: its stream waits for every read group launched before it, and
// the next reads wait for it, so every request sees exactly the updates that
// arrived before it -- the results are those of running the requests one at
// a time in arrival order.  Completion is detected with events; requests that
// arrive while others run are admitted at the next progress call.
#include "mk_host.h"

#include <algorithm>
#include <deque>
#include <vector>

using namespace mk;

namespace {

struct Group {
    cudaEvent_t done_q = nullptr, done_s = nullptr, done_u = nullptr;
    std::vector<uint64_t> tags;
    std::vector<int> status;
};

} // namespace

struct mk_server {
    mk_graph *g = nullptr;
    mk_batcher *batcher = nullptr;
    uint32_t max_inflight = 0;
    uint32_t inflight = 0;
    uint32_t commit_every = 0;
    uint32_t updates_since_commit = 0;
    uint64_t pool_free_est = 0;
    cudaStream_t sq = nullptr, ss = nullptr, su = nullptr;
    cudaEvent_t last_update = nullptr;
    bool have_update = false;
    std::vector<cudaEvent_t> reads_since_update;
    std::deque<mk_request> queue;
    std::deque<Group> flight;
    std::vector<cudaEvent_t> spare;
    std::vector<std::pair<uint64_t, int>> finished;
    uint64_t groups = 0, merged_queries = 0, merged_updates = 0;
};

namespace {

cudaEvent_t ev(mk_server *s)
{
    if (!s->spare.empty()) {
        cudaEvent_t e = s->spare.back();
        s->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

bool is_read(int kind) { return kind == MK_REQ_QUERY || kind == MK_REQ_SSSP || kind == MK_REQ_BFS; }

// Free pool slabs, read exactly (synchronises).
mk_status refresh_pool(mk_server *s)
{
    uint64_t free_slabs = 0;
    MK_TRY(mk_pool_free(s->g, &free_slabs, s->su));
    s->pool_free_est = free_slabs;
    return MK_OK;
}

// Launches the read group at the head of the queue (up to `room` requests).
mk_status launch_reads(mk_server *s, uint32_t room)
{
    Group grp;
    // the group: the reads at the head of the queue
    std::vector<mk_request> reqs;
    uint32_t n_query = 0;
    while (room && !s->queue.empty() && is_read(s->queue.front().kind)) {
        reqs.push_back(s->queue.front());
        n_query += reqs.back().kind == MK_REQ_QUERY;
        s->queue.pop_front();
        --room;
    }
    const bool any_q = n_query > 0, any_s = reqs.size() > n_query;
    if (s->have_update) {
        if (any_q)
            MK_CUDA(cudaStreamWaitEvent(s->sq, s->last_update, 0));
        if (any_s)
            MK_CUDA(cudaStreamWaitEvent(s->ss, s->last_update, 0));
    }
    for (const mk_request &r : reqs) {
        int st = MK_OK;
        if (r.kind == MK_REQ_QUERY && n_query == 1) {
            // a lone query needs no merging: one direct launch
            st = mk_query_batch(s->g, r.d_src, r.d_dst, r.n, r.d_out0, r.d_out1, s->sq);
        } else if (r.kind == MK_REQ_QUERY) {
            st = mk_batcher_add_query(s->batcher, r.d_src, r.d_dst, r.n, r.d_out0, r.d_out1);
            if (st == MK_ERR_INVALID_ARG && r.n) { // batcher full: flush and retry
                MK_TRY(mk_batcher_launch(s->batcher, s->sq));
                st = mk_batcher_add_query(s->batcher, r.d_src, r.d_dst, r.n, r.d_out0, r.d_out1);
            }
            s->merged_queries++;
        } else {
            st = r.kind == MK_REQ_SSSP ? mk_incr_sssp(s->g, r.source, r.d_out0, r.d_out1, s->ss)
                                       : mk_incr_bfs(s->g, r.source, r.d_out0, r.d_out1, s->ss);
        }
        grp.tags.push_back(r.tag);
        grp.status.push_back(st);
    }
    if (n_query > 1)
        MK_TRY(mk_batcher_launch(s->batcher, s->sq));
    if (any_q) {
        grp.done_q = ev(s);
        MK_CUDA(cudaEventRecord(grp.done_q, s->sq));
        s->reads_since_update.push_back(grp.done_q);
    }
    if (any_s) {
        grp.done_s = ev(s);
        MK_CUDA(cudaEventRecord(grp.done_s, s->ss));
        s->reads_since_update.push_back(grp.done_s);
    }
    s->inflight += (uint32_t)grp.tags.size();
    s->flight.push_back(std::move(grp));
    s->groups++;
    return MK_OK;
}

// Launches the run of updates of one kind at the head of the queue (a
// barrier), up to the next commit point and the free in-flight slots, as
// one mk_update_multi call (merged into one staged batch; results identical
// to one call per request in order).
mk_status launch_update(mk_server *s)
{
    const int kind = s->queue.front().kind;
    const uint32_t to_commit = s->commit_every ? s->commit_every - s->updates_since_commit : 0xFFFFFFFFu;
    const uint32_t slots = std::max<uint32_t>(1, s->max_inflight - std::min(s->inflight, s->max_inflight));
    Group grp;
    std::vector<mk_update_req> reqs;
    std::vector<size_t> member; // position in grp of each request in reqs
    uint64_t need = 0;
    while (!s->queue.empty() && s->queue.front().kind == kind && grp.tags.size() < std::min(to_commit, slots)) {
        const mk_request r = s->queue.front();
        int st = MK_OK;
        if (kind == MK_REQ_INSERT) {
            // admission by slab-pool memory: at most one new slab per edge
            if (s->pool_free_est < need + r.n)
                MK_TRY(refresh_pool(s));
            if (s->pool_free_est < need + r.n)
                st = MK_ERR_POOL_EXHAUSTED; // refused, nothing enqueued
            else
                need += r.n;
        }
        s->queue.pop_front();
        if (st == MK_OK) {
            mk_update_req q{};
            q.kind = kind;
            q.d_src = r.d_src;
            q.d_dst = r.d_dst;
            q.d_w = r.d_w;
            q.n = r.n;
            q.d_flags = (uint8_t *)r.d_out0;
            reqs.push_back(q);
            member.push_back(grp.tags.size());
        }
        grp.tags.push_back(r.tag);
        grp.status.push_back(st);
    }
    for (cudaEvent_t e : s->reads_since_update)
        MK_CUDA(cudaStreamWaitEvent(s->su, e, 0));
    s->reads_since_update.clear();
    if (!reqs.empty()) {
        int st = mk_update_multi(s->g, reqs.data(), (uint32_t)reqs.size(), s->su);
        s->pool_free_est -= std::min<uint64_t>(s->pool_free_est, need);
        s->updates_since_commit += (uint32_t)reqs.size();
        if (st == MK_OK && s->commit_every && s->updates_since_commit >= s->commit_every) {
            st = mk_commit_batch(s->g, s->su);
            s->updates_since_commit = 0;
        }
        if (st != MK_OK)
            for (size_t i : member)
                grp.status[i] = st;
        s->merged_updates += reqs.size() > 1 ? reqs.size() : 0;
    }
    grp.done_u = ev(s);
    MK_CUDA(cudaEventRecord(grp.done_u, s->su));
    MK_CUDA(cudaEventRecord(s->last_update, s->su));
    s->have_update = true;
    s->inflight += (uint32_t)grp.tags.size();
    s->flight.push_back(std::move(grp));
    s->groups++;
    return MK_OK;
}

bool group_done(const Group &grp)
{
    for (cudaEvent_t e : {grp.done_q, grp.done_s, grp.done_u})
        if (e && cudaEventQuery(e) != cudaSuccess)
            return false;
    return true;
}

} // namespace

extern "C" {

mk_status mk_server_create(mk_graph *g, uint32_t max_inflight, uint32_t commit_every, mk_server **out)
{
    if (!g || !out || !max_inflight)
        return MK_ERR_INVALID_ARG;
    mk_server *s = new mk_server;
    s->g = g;
    s->max_inflight = max_inflight;
    s->commit_every = commit_every;
    mk_status st = mk_batcher_create(g, std::max<uint32_t>(max_inflight, 1), &s->batcher);
    if (st == MK_OK && (cudaStreamCreateWithFlags(&s->sq, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&s->ss, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&s->su, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&s->last_update, cudaEventDisableTiming) != cudaSuccess))
        st = MK_ERR_CUDA;
    if (st == MK_OK)
        st = refresh_pool(s);
    if (st != MK_OK) {
        mk_server_destroy(s);
        return st;
    }
    *out = s;
    return MK_OK;
}

mk_status mk_server_destroy(mk_server *s)
{
    if (!s)
        return MK_ERR_INVALID_ARG;
    for (cudaStream_t st : {s->sq, s->ss, s->su})
        if (st)
            cudaStreamSynchronize(st);
    if (s->batcher)
        mk_batcher_destroy(s->batcher);
    for (auto &grp : s->flight)
        for (cudaEvent_t e : {grp.done_q, grp.done_s, grp.done_u})
            if (e)
                cudaEventDestroy(e);
    for (cudaEvent_t e : s->spare)
        cudaEventDestroy(e);
    if (s->last_update)
        cudaEventDestroy(s->last_update);
    for (cudaStream_t st : {s->sq, s->ss, s->su})
        if (st)
            cudaStreamDestroy(st);
    delete s;
    return MK_OK;
}

mk_status mk_server_submit(mk_server *s, const mk_request *r)
{
    if (!s || !r || r->kind < MK_REQ_QUERY || r->kind > MK_REQ_BFS)
        return MK_ERR_INVALID_ARG;
    const bool upd = r->kind == MK_REQ_INSERT || r->kind == MK_REQ_DELETE;
    if ((r->kind == MK_REQ_QUERY || upd) && r->n && (!r->d_src || !r->d_dst))
        return MK_ERR_INVALID_ARG;
    if (r->kind == MK_REQ_QUERY && r->n && !r->d_out0)
        return MK_ERR_INVALID_ARG;
    s->queue.push_back(*r);
    return MK_OK;
}

mk_status mk_server_progress(mk_server *s, uint64_t *done_tags, int *done_status, uint32_t cap, uint32_t *n_done)
{
    if (!s || !n_done || (cap && !done_tags))
        return MK_ERR_INVALID_ARG;
    // retire finished groups (in order)
    while (!s->flight.empty() && group_done(s->flight.front())) {
        Group &grp = s->flight.front();
        for (size_t i = 0; i < grp.tags.size(); ++i)
            s->finished.push_back({grp.tags[i], grp.status[i]});
        s->inflight -= (uint32_t)grp.tags.size();
        for (cudaEvent_t e : {grp.done_q, grp.done_s, grp.done_u})
            if (e)
                s->spare.push_back(e);
        s->flight.pop_front();
    }
    // admit while slots are free
    while (!s->queue.empty() && s->inflight < s->max_inflight) {
        if (is_read(s->queue.front().kind))
            MK_TRY(launch_reads(s, s->max_inflight - s->inflight));
        else
            MK_TRY(launch_update(s));
    }
    const uint32_t n = (uint32_t)std::min<size_t>(cap, s->finished.size());
    for (uint32_t i = 0; i < n; ++i) {
        done_tags[i] = s->finished[i].first;
        if (done_status)
            done_status[i] = s->finished[i].second;
    }
    s->finished.erase(s->finished.begin(), s->finished.begin() + n);
    *n_done = n;
    return MK_OK;
}

mk_status mk_server_pending(mk_server *s, uint64_t *queued, uint64_t *inflight)
{
    if (!s)
        return MK_ERR_INVALID_ARG;
    if (queued)
        *queued = s->queue.size();
    if (inflight)
        *inflight = s->inflight + s->finished.size();
    return MK_OK;
}

} // extern "C"
