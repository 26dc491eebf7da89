// gs_contrib_prune_noalloc: the contribution prune for callers that cannot
// allocate device memory (see include/gs.h).  Its scan scratch is a
// file-scope static device array instead of a caller-provided workspace.
#include <cstdio>
#include <mutex>

#include "gs_internal.cuh"

namespace {

// Scratch of the prune's two-kernel scan: one 32-bit partial count per scan
// block (at most kMaxSortBlocks), sized like the prune workspace, which also
// reserves the bytes of a control block after them.  The partial counts are
// 32-bit, so at most 2^31 - 1 items fit one call.
constexpr size_t kNoallocScratchBytes = 8192;
constexpr int64_t kNoallocMaxItems = 0x7FFFFFFF;
static_assert(gs::kMaxSortBlocks * 4 + sizeof(gs::Ctl) <= kNoallocScratchBytes, "static prune scratch too small");

static __device__ __align__(256) unsigned char g_prune_scratch[kNoallocScratchBytes];

// Device address of g_prune_scratch per device ordinal.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device, with that device current, by cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int gs_contrib_prune_noalloc(const float *contrib_max, int64_t n, float threshold, uint8_t *keep,
                                        int32_t *keep_index, int64_t *n_keep, void *stream) {
    if (n < 0 || n > kNoallocMaxItems) {
        char msg[160];
        snprintf(msg, sizeof msg, "gs_contrib_prune_noalloc: n = %lld is outside 0..%lld, the range its static "
                 "scratch (32-bit partial counts) holds", (long long)n, (long long)kNoallocMaxItems);
        return gs::report(GS_ERR_INVALID, msg);
    }
    size_t need = 0;
    int rc = gs_prune_workspace_size(n, &need);
    if (rc != GS_OK) return rc;
    if (need > kNoallocScratchBytes)
        return gs::report(GS_ERR_WORKSPACE, "gs_contrib_prune_noalloc: scan scratch exceeds the static array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gs::report(GS_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return gs::report(GS_ERR_INVALID, "gs_contrib_prune_noalloc: device ordinal above 63");
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_prune_scratch);
            if (e != cudaSuccess || !p)
                return gs::report(GS_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                : "cudaGetSymbolAddress returned NULL");
            g_addr[dev] = p;
        }
        ptr = g_addr[dev];
    }
    // Nothing in the scratch has to start at zero: the scan writes every
    // partial count and control field it later reads.
    return gs_contrib_prune(contrib_max, n, threshold, keep, keep_index, n_keep, ptr, kNoallocScratchBytes, stream);
}
