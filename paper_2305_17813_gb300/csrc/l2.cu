// L2 residency controls: an access-policy window on a stream that marks one
// part of the store as persisting in L2 (the north star's "L2 residency
// controls cover the hot slab pool").  The window and the set-aside are
// properties of this process's context and stream; they end with the
// context (nothing here changes a setting of the device itself), and
// MK_L2_NONE removes them.
#include "mk_host.h"

#include <algorithm>

using namespace mk;

extern "C" mk_status mk_l2_window(mk_graph *g, int region, void *stream, mk_l2_info *out)
{
    if (!g || region < MK_L2_NONE || region > MK_L2_POOL)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, max_persist = 0, max_window = 0;
    MK_CUDA(cudaGetDevice(&dev));
    MK_CUDA(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev));
    MK_CUDA(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev));
    cudaStreamAttrValue attr{};
    mk_l2_info info{};
    info.max_bytes = (uint64_t)max_persist;
    if (region == MK_L2_NONE || max_persist <= 0 || max_window <= 0) {
        attr.accessPolicyWindow.base_ptr = nullptr;
        attr.accessPolicyWindow.num_bytes = 0;
        attr.accessPolicyWindow.hitRatio = 0.f;
        attr.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
        attr.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
        MK_CUDA(cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &attr));
        MK_CUDA(cudaCtxResetPersistingL2Cache());
        MK_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0));
    } else {
        void *base = nullptr;
        uint64_t bytes = 0;
        if (region == MK_L2_VINFO) {
            base = (void *)g->v.vinfo;
            bytes = (uint64_t)g->v.V * 8;
        } else if (region == MK_L2_HEADS) {
            base = g->v.slabs;
            bytes = (uint64_t)g->v.H * 128;
        } else {
            base = g->v.slabs + (size_t)g->v.H * 32;
            bytes = (uint64_t)g->v.P * 128;
        }
        const uint64_t win = std::min<uint64_t>(bytes, (uint64_t)max_window);
        const uint64_t aside = std::min<uint64_t>(win, (uint64_t)max_persist);
        MK_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, aside));
        attr.accessPolicyWindow.base_ptr = base;
        attr.accessPolicyWindow.num_bytes = win;
        // the share of the window's lines that may persist: all of them when
        // the window fits the set-aside, else the fraction that fits
        attr.accessPolicyWindow.hitRatio = win ? std::min(1.f, (float)aside / (float)win) : 0.f;
        attr.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        MK_CUDA(cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &attr));
        info.window_bytes = win;
        info.hit_ratio = attr.accessPolicyWindow.hitRatio;
    }
    if (out)
        *out = info;
    return MK_OK;
}
