// gs_contrib_prune_noalloc: the contribution prune for callers that cannot
// allocate device memory (see include/gs.h).  Its scan scratch is a
// file-scope static device array instead of a caller-provided workspace.
#include <cstdio>

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
    // In host code g_prune_scratch names a host-side stand-in, not device
    // memory, so its device address is looked up on every call, with the
    // calling thread's current device.  No address is cached: after a
    // cudaDeviceReset (or a new primary context) the array lives elsewhere.
    // The first lookup on a device loads this file's module there, which is
    // when the driver backs the array with device memory; later lookups only
    // read the loaded module's symbol table.
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_prune_scratch);
    if (e != cudaSuccess) return gs::report(GS_ERR_CUDA, cudaGetErrorString(e));
    if (!ptr) return gs::report(GS_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    // Nothing in the scratch has to start at zero: the scan writes every
    // partial count and control field it later reads.
    return gs_contrib_prune(contrib_max, n, threshold, keep, keep_index, n_keep, ptr, kNoallocScratchBytes, stream);
}
