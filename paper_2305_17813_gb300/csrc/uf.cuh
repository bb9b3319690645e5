// Union-find helpers shared by the weighted store's WCC and the set
// layout's WCC (paper, Sec. "Auxiliary Data Structures", Union-Find, with
// the Union-Async hooking of Sec. "Incremental WCC").
#pragma once

#include "mk_device.cuh"

namespace mk {

// Parent loads.  The coherent form reads L2 (the point of coherence); the
// cached form may also hit a stale line in the SM's L1.  A stale parent is
// still a correct one from an earlier moment: parents only ever move to
// smaller ids of the same set (a hook replaces a root's self-link, path
// halving replaces a parent by an ancestor), and a vertex that is not a root
// never becomes one again.  So a find on cached loads returns a vertex that
// is, or was, the root of the element's set -- always a member of that set.
// Path halving may then store a parent older than the current one, which
// is still an ancestor in the same set.  The union below only acts on a
// found root through a CAS that succeeds while it is still a root, and
// retries on coherent loads.  The cached form
// keeps the roots that every find ends at (above all the giant component's
// vertex 0) in L1 instead of sending every find's last load to the same L2
// line.
template <bool kCached>
__device__ __forceinline__ uint32_t uf_load(const uint32_t *p, uint32_t x)
{
    return kCached ? p[x] : __ldcg(&p[x]);
}

// N finds in lockstep, so that their dependent loads overlap; kNil entries
// are left alone.  Parents strictly decrease along every path (p[x] < x
// except at roots), so every walk ends.
template <int N, bool kCached>
__device__ __forceinline__ void uf_find_n(uint32_t *p, uint32_t (&x)[N])
{
    bool done[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
        done[i] = x[i] == kNil;
    for (;;) {
        bool all = true;
#pragma unroll
        for (int i = 0; i < N; ++i)
            all = all && done[i];
        if (all)
            return;
        uint32_t px[N], ppx[N];
#pragma unroll
        for (int i = 0; i < N; ++i)
            px[i] = done[i] ? x[i] : uf_load<kCached>(p, x[i]);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            done[i] = done[i] || px[i] == x[i];
            ppx[i] = done[i] ? px[i] : uf_load<kCached>(p, px[i]);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (!done[i]) {
                if (ppx[i] == px[i]) {
                    x[i] = px[i]; // px is the root: no third load
                    done[i] = true;
                } else {
                    p[x[i]] = ppx[i]; // path halving: ppx is an ancestor of x
                    x[i] = ppx[i];
                }
            }
        }
    }
}

// Union of the sets of the elements held by one group of G lanes, N per lane
// (act[i] says which are present): all roots are found in parallel, the
// group's smallest root m is the anchor, and every other root r is hooked
// under it with one CAS on p[r] from r to m.  The CAS succeeds only while r
// is still a root; m need not be one any more, because any vertex with a
// smaller id lies in another tree (ids never increase towards a root), so
// the hook joins the two sets and keeps parents decreasing.  Elements of one
// lane with the same root share one CAS.  An element whose CAS loses (its
// root was hooked by another warp meanwhile) retries with fresh roots of
// itself and of the anchor, hooking the larger under the smaller.  Returns
// false if the retry bound was hit.  Must be called by the full warp.
template <int G, int N>
__device__ __forceinline__ bool group_union(uint32_t *p, const uint32_t (&e)[N], const bool (&act)[N],
                                            uint32_t limit)
{
    uint32_t r[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
        r[i] = act[i] ? e[i] : kNil;
    uf_find_n<N, true>(p, r);
    uint32_t m = kNil;
#pragma unroll
    for (int i = 0; i < N; ++i)
        m = min(m, r[i]);
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1)
        m = min(m, __shfl_xor_sync(kFull, m, o));
    bool pend[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        pend[i] = act[i] && r[i] != m;
        if (!pend[i])
            continue;
        // first attempt with the roots just found (r > m for every pending r)
        bool decided = false, val = false;
#pragma unroll
        for (int j = 0; j < i; ++j)
            if (!decided && act[j] && r[j] == r[i]) {
                decided = true;
                val = pend[j];
            }
        if (decided)
            pend[i] = val;
        else if (atomicCAS(&p[r[i]], r[i], m) == r[i])
            pend[i] = false;
    }
    for (uint32_t it = 0; it < limit; ++it) {
        bool any = false;
#pragma unroll
        for (int i = 0; i < N; ++i)
            any = any || pend[i];
        if (!__any_sync(kFull, any))
            return true;
        uint32_t anc[1] = {any ? m : kNil};
        uf_find_n<1, false>(p, anc);
        const uint32_t a = anc[0];
        uint32_t x[N];
#pragma unroll
        for (int i = 0; i < N; ++i)
            x[i] = pend[i] ? r[i] : kNil;
        uf_find_n<N, false>(p, x);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (pend[i]) {
                r[i] = x[i];
                const uint32_t hi = max(r[i], a), lo = min(r[i], a);
                if (r[i] == a || atomicCAS(&p[hi], hi, lo) == hi)
                    pend[i] = false;
            }
        }
    }
    return false;
}

} // namespace mk
