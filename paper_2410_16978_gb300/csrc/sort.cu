// S2 - tile binning with depth-keyed radix sorts (Sec. 3.3: the Gaussians are
// sorted relative to the camera; the paper's renderer uses GPU radix sorts).
//
// Order of the tile lists: (tile, depth, Gaussian index).  It is produced by
//   1. compacting the visible Gaussians in index order,
//   2. a stable LSD radix sort of them by the float bits of their depth,
//   3. an exclusive scan of their tile counts in that depth order,
//   4. emitting one (tile id, Gaussian) pair per covered tile at the scanned
//      offsets (so the pairs are in depth order), and
//   5. a stable LSD radix sort of the pairs by tile id,
// which equals a stable sort of the keys (tile << 32 | depth bits) emitted in
// index order, with 32-bit keys and far fewer passes over the pair list.
//
// Every kernel runs on a fixed grid of sort_blocks() CTAs that each own a
// contiguous range of the items, so item counts produced on the device never
// need to travel to the host.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ void block_range(uint32_t n, uint32_t &beg, uint32_t &end) {
    const uint64_t tiles = (static_cast<uint64_t>(n) + kSortTile - 1) / kSortTile;
    const uint64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const uint64_t b = static_cast<uint64_t>(blockIdx.x) * per * kSortTile;
    const uint64_t e = b + per * kSortTile;
    beg = static_cast<uint32_t>(b < n ? b : n);
    end = static_cast<uint32_t>(e < n ? e : n);
}

// Exclusive scan over the 256 threads of a block; *total = sum of all v.
__device__ __forceinline__ uint32_t block_scan_256(uint32_t v, uint32_t *s_w, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < 8 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? s_w[warp - 1] : 0;
    *total = s_w[7];
    __syncthreads();
    return base + x - v;
}

// ---------------------------------------------------------------------------
// Generic three-kernel scan: reduce per block, scan the block sums, rescan.

struct NSrc {               // item count: min(*dev, cap) if dev, else cap
    const uint32_t *dev;
    uint32_t cap;
    __device__ __forceinline__ uint32_t get() const {
        if (!dev) return cap;
        const uint32_t d = *dev;
        return d < cap ? d : cap;
    }
};

template <class F>
__global__ void __launch_bounds__(256) k_scan_reduce(F f, NSrc ns, uint32_t *__restrict__ partials) {
    __shared__ uint32_t s_w[8];
    uint32_t beg, end;
    block_range(ns.get(), beg, end);
    uint32_t acc = 0;
    for (uint32_t i = beg + threadIdx.x; i < end; i += 256) acc += f(i);
    uint32_t tot;
    block_scan_256(acc, s_w, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

enum ScanFinal { FIN_NONE = 0, FIN_NVIS = 1, FIN_NKEEP = 2 };

__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *__restrict__ partials, int G, int mode,
                                                        Ctl *ctl, uint64_t cap, int64_t *n_keep) {
    __shared__ uint32_t s_w[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t v = t < G ? partials[t] : 0;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = (warp > 0 ? s_w[warp - 1] : 0) + x - v;
    if (t < G) partials[t] = excl;
    if (t == 0) {
        const uint32_t total = s_w[31];
        if (mode == FIN_NVIS) {
            ctl->n_vis = total;
            ctl->st.n_visible = total;
        } else if (mode == FIN_NKEEP) {
            *n_keep = total;
        }
        ctl->scan_total = total;
    }
}

template <class F, class Out>
__global__ void __launch_bounds__(256) k_scan_down(F f, NSrc ns, const uint32_t *__restrict__ partials, Out out) {
    __shared__ uint32_t s_w[8];
    uint32_t beg, end;
    block_range(ns.get(), beg, end);
    uint32_t run = partials[blockIdx.x];
    for (uint32_t t0 = beg; t0 < end; t0 += kSortTile) {
        uint32_t v[kSortItems];
        uint32_t sum = 0;
        const uint32_t i0 = t0 + threadIdx.x * kSortItems;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            v[k] = (i0 + k < end) ? f(i0 + k) : 0;
            sum += v[k];
        }
        uint32_t tot;
        uint32_t off = run + block_scan_256(sum, s_w, &tot);
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            if (i0 + k < end) out(i0 + k, off, v[k]);
            off += v[k];
        }
        run += tot;
    }
}

// --- functors ---
struct VisFlag {
    const uint32_t *tiles;
    __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return tiles[i] > 0 ? 1u : 0u; }
};
struct CompactOut {
    const uint32_t *depth_key;
    uint32_t *keys, *vals;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t off, uint32_t v) const {
        if (v) { keys[off] = depth_key[i]; vals[off] = i; }
    }
};
struct VisFlag2 {           // visible to either of two views
    const uint32_t *tiles_a, *tiles_b;
    __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
        return (tiles_a[i] > 0 || tiles_b[i] > 0) ? 1u : 0u;
    }
};
struct CompactOut2 {        // key: view a's depth when view a sees it, else view b's
    const uint32_t *tiles_a, *depth_a, *depth_b;
    uint32_t *keys, *vals;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t off, uint32_t v) const {
        if (v) {
            keys[off] = tiles_a[i] > 0 ? depth_a[i] : depth_b[i];
            vals[off] = i;
        }
    }
};
struct KeepFlag {
    const float *cmax;
    float thr;
    __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return cmax[i] >= thr ? 1u : 0u; }
};
struct ActiveFlag {         // keep unless trainable and activity / samples <= thr
    const float *act;
    const uint8_t *layer;
    uint32_t mask;
    float inv_samples, thr;
    __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
        const bool trainable = (mask >> layer[i]) & 1u;
        return (trainable && act[i] * inv_samples <= thr) ? 0u : 1u;
    }
};
struct KeepOut {
    uint8_t *keep;
    int32_t *idx;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t off, uint32_t v) const {
        keep[i] = static_cast<uint8_t>(v);
        if (v && idx) idx[off] = static_cast<int32_t>(i);
    }
};

// ---------------------------------------------------------------------------
// Radix sort pass: 8-bit digits, histogram per (digit, block) in digit-major
// order.  The first pass of a sort also records min and max key (as max of
// ~key and max of key); a later pass whose digit is the same in every key
// (all keys agree on the bits at and above its shift) is an identity
// permutation and only copies.

__device__ __forceinline__ bool pass_is_constant(const uint32_t *mm, int shift) {
    const uint32_t kmin = ~mm[0], kmax = mm[1];
    return ((kmin ^ kmax) >> shift) == 0;
}

__global__ void __launch_bounds__(256) k_radix_up(const uint32_t *__restrict__ keys, NSrc ns, int shift,
                                                  uint32_t *__restrict__ hist, uint32_t *__restrict__ mm, int first) {
    __shared__ uint32_t s_h[8][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!first && pass_is_constant(mm, shift)) return;
    for (int k = threadIdx.x; k < 8 * 256; k += 256) (&s_h[0][0])[k] = 0;
    __syncthreads();
    uint32_t beg, end;
    block_range(ns.get(), beg, end);
    uint32_t kinv = 0, kmax = 0;
    for (uint32_t t0 = beg; t0 < end; t0 += kSortTile) {
        uint32_t key[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {        // issue all loads of the tile first
            const uint32_t i = t0 + r * 256 + threadIdx.x;
            key[r] = i < end ? keys[i] : 0;
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint32_t i = t0 + r * 256 + threadIdx.x;
            const bool valid = i < end;
            uint32_t d = 256u + lane;
            if (valid) {
                d = (key[r] >> shift) & 255u;
                kinv = max(kinv, ~key[r]);
                kmax = max(kmax, key[r]);
            }
            const unsigned peers = __match_any_sync(FULL, d);
            if (valid && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&s_h[warp][d], __popc(peers));
        }
    }
    if (first) {
        kinv = __reduce_max_sync(FULL, kinv);
        kmax = __reduce_max_sync(FULL, kmax);
        if (lane == 0) {    // 0 is neutral for both maxima: warps without items change nothing
            atomicMax(&mm[0], kinv);
            atomicMax(&mm[1], kmax);
        }
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += s_h[w][d];
    hist[static_cast<size_t>(d) * gridDim.x + blockIdx.x] = sum;
}

// Per digit (one CTA each): exclusive scan of its G block counts in place and
// the digit's total.
__global__ void __launch_bounds__(256) k_radix_rowscan(uint32_t *__restrict__ hist, int G,
                                                       uint32_t *__restrict__ rowtot, const uint32_t *__restrict__ mm,
                                                       int shift, int first) {
    __shared__ uint32_t s_w[8];
    if (!first && pass_is_constant(mm, shift)) return;
    uint32_t *row = hist + static_cast<size_t>(blockIdx.x) * G;
    constexpr int per = kMaxSortBlocks / 256;
    uint32_t v[per];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int b = threadIdx.x * per + k;
        v[k] = b < G ? row[b] : 0;
        sum += v[k];
    }
    uint32_t tot;
    uint32_t run = block_scan_256(sum, s_w, &tot);
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int b = threadIdx.x * per + k;
        if (b < G) row[b] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) rowtot[blockIdx.x] = tot;
}

// Stable scatter.  A block walks its range in tiles of 2048 items; warp w
// ranks the contiguous run [256 w, 256 w + 256) of the tile in 8 rounds of 32
// with warp-private digit counters, so items are ranked in (warp, round,
// lane) = index order.  The tile is then sorted by digit in shared memory and
// written out in that order, so consecutive threads store consecutive
// addresses of the same digit's run.
__global__ void __launch_bounds__(256) k_radix_down(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                    uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, NSrc ns,
                                                    int shift, const uint32_t *__restrict__ hist,
                                                    const uint32_t *__restrict__ rowtot,
                                                    const uint32_t *__restrict__ mm, int first) {
    __shared__ uint32_t s_off[256];       // global offset of each digit for this block's next tile
    __shared__ uint32_t s_wc[8][256];     // per-warp digit counts, then per-warp digit bases
    __shared__ uint32_t s_lstart[256];    // start of each digit's run in the locally sorted tile
    __shared__ uint32_t s_key[kSortTile], s_val[kSortTile];
    __shared__ uint32_t s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t beg, end;
    block_range(ns.get(), beg, end);
    if (!first && pass_is_constant(mm, shift)) {
        for (uint32_t i = beg + threadIdx.x; i < end; i += 256) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    {
        uint32_t tot;
        const uint32_t digit_base = block_scan_256(rowtot[threadIdx.x], s_w, &tot);
        s_off[threadIdx.x] = digit_base + hist[static_cast<size_t>(threadIdx.x) * gridDim.x + blockIdx.x];
    }
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t t0 = beg; t0 < end; t0 += kSortTile) {
#pragma unroll
        for (int w = 0; w < 8; ++w) s_wc[w][threadIdx.x] = 0;
        __syncthreads();
        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        const uint32_t run0 = t0 + warp * 256;
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint32_t i = run0 + r * 32 + lane;
            key[r] = i < end ? kin[i] : 0u;
            val[r] = i < end ? vin[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint32_t i = run0 + r * 32 + lane;
            const bool valid = i < end;
            const uint32_t d = valid ? (key[r] >> shift) & 255u : 256u + lane;
            const unsigned peers = __match_any_sync(FULL, d);
            const uint32_t before = valid ? s_wc[warp][d] : 0;
            rank[r] = before + __popc(peers & lt);
            __syncwarp();
            if (valid && (peers & lt) == 0) s_wc[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit d = thread: exclusive prefix over the warps and the tile total
        const int d = threadIdx.x;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_wc[w][d];
            s_wc[w][d] = acc;
            acc += c;
        }
        uint32_t ntile;
        s_lstart[d] = block_scan_256(acc, s_w, &ntile);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (run0 + r * 32 + lane < end) {
                const uint32_t dd = (key[r] >> shift) & 255u;
                const uint32_t lpos = s_lstart[dd] + s_wc[warp][dd] + rank[r];
                s_key[lpos] = key[r];
                s_val[lpos] = val[r];
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < ntile; i += 256) {
            const uint32_t k = s_key[i];
            const uint32_t dd = (k >> shift) & 255u;
            const uint32_t pos = s_off[dd] + (i - s_lstart[dd]);
            kout[pos] = k;
            vout[pos] = s_val[i];
        }
        __syncthreads();
        s_off[d] += acc;
    }
}

// ---------------------------------------------------------------------------

}  // namespace

int sort_blocks() {
    static int cached = 0;
    if (cached) return cached;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int g = 4 * (sms > 0 ? sms : 80);
    if (g > kMaxSortBlocks) g = kMaxSortBlocks;
    cached = g;
    return g;
}

cudaError_t launch_compact_visible(const uint32_t *tiles, const uint32_t *depth_key, int n, uint32_t *keys_out,
                                   uint32_t *vals_out, uint32_t *partials, Ctl *ctl, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{nullptr, static_cast<uint32_t>(n)};
    VisFlag f{tiles};
    k_scan_reduce<<<G, 256, 0, st>>>(f, ns, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, G, FIN_NVIS, ctl, 0, nullptr);
    k_scan_down<<<G, 256, 0, st>>>(f, ns, partials, CompactOut{depth_key, keys_out, vals_out});
    return cudaGetLastError();
}

cudaError_t launch_compact_visible2(const uint32_t *tiles_a, const uint32_t *depth_a, const uint32_t *tiles_b,
                                    const uint32_t *depth_b, int n, uint32_t *keys_out, uint32_t *vals_out,
                                    uint32_t *partials, Ctl *ctl, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{nullptr, static_cast<uint32_t>(n)};
    VisFlag2 f{tiles_a, tiles_b};
    k_scan_reduce<<<G, 256, 0, st>>>(f, ns, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, G, FIN_NVIS, ctl, 0, nullptr);
    k_scan_down<<<G, 256, 0, st>>>(f, ns, partials, CompactOut2{tiles_a, depth_a, depth_b, keys_out, vals_out});
    return cudaGetLastError();
}

cudaError_t launch_radix_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                              const uint32_t *n_dev, uint32_t n_cap, int shift, uint32_t *hist, uint32_t *minmax,
                              bool first, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{n_dev, n_cap};
    uint32_t *rowtot = hist + static_cast<size_t>(256) * kMaxSortBlocks;
    k_radix_up<<<G, 256, 0, st>>>(kin, ns, shift, hist, minmax, first ? 1 : 0);
    k_radix_rowscan<<<256, 256, 0, st>>>(hist, G, rowtot, minmax, shift, first ? 1 : 0);
    k_radix_down<<<G, 256, 0, st>>>(kin, vin, kout, vout, ns, shift, hist, rowtot, minmax, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_activity_prune(const float *activity, const uint8_t *layer, uint32_t train_mask, int n,
                                  float samples, float thr, uint8_t *keep, int32_t *keep_index, int64_t *n_keep,
                                  uint32_t *partials, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{nullptr, static_cast<uint32_t>(n)};
    ActiveFlag f{activity, layer, train_mask, 1.f / samples, thr};
    Ctl *ctl = reinterpret_cast<Ctl *>(partials + kMaxSortBlocks);
    k_scan_reduce<<<G, 256, 0, st>>>(f, ns, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, G, FIN_NKEEP, ctl, 0, n_keep);
    k_scan_down<<<G, 256, 0, st>>>(f, ns, partials, KeepOut{keep, keep_index});
    return cudaGetLastError();
}

cudaError_t launch_prune(const float *contrib_max, int n, float thr, uint8_t *keep, int32_t *keep_index,
                         int64_t *n_keep, uint32_t *partials, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{nullptr, static_cast<uint32_t>(n)};
    KeepFlag f{contrib_max, thr};
    Ctl *ctl = reinterpret_cast<Ctl *>(partials + kMaxSortBlocks);
    k_scan_reduce<<<G, 256, 0, st>>>(f, ns, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, G, FIN_NKEEP, ctl, 0, n_keep);
    k_scan_down<<<G, 256, 0, st>>>(f, ns, partials, KeepOut{keep, keep_index});
    return cudaGetLastError();
}

}  // namespace gs
