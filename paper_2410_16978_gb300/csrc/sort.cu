// S2 - the depth sort of the visible Gaussians (Sec. 3.3: the Gaussians are
// sorted relative to the camera; the paper's renderer uses GPU radix sorts),
// and the scans of the prune entry points.
//
// The depth order is a stable LSD radix sort of the visible Gaussians, taken
// in index order, by the float bits of their depth (so ties keep index
// order).  It runs as
//   1. one pass over all Gaussians that counts the visible ones, the four
//      8-bit digit histograms of their keys and the smallest and largest key;
//   2. one kernel per digit.  A CTA takes a tile of 4096 items, ranks them
//      by digit in shared memory, and places every digit's run of the tile
//      at the count of that digit in all smaller keys (the histogram) plus
//      its count in the tiles before this one.  The first digit kernel reads
//      the Gaussians directly, keeps the visible ones and also writes their
//      indices in index order (the visible list of the backward).  Its tiles
//      are the histogram pass's, which counts the first digit per tile and
//      per group of G consecutive tiles (G^2 at or above the tile count): a
//      tile's prefix is the groups before its group plus the tiles before it
//      in its group: two threads per digit, one loading at most sqrt(tiles)
//      group counts and the other fewer than 2 sqrt(tiles) tile counts, all
//      independent loads.
//      The later digit kernels, over the visible Gaussians only, take their
//      tiles by ticket and find the prefix by a decoupled look-back over the
//      tiles before them (the single-pass prefix scan of Merrill and Garland,
//      used per digit as in Adinets and Merrill's Onesweep radix sort).
// A digit at and above the highest bit where the smallest and largest key
// differ is the same in every key: its kernel returns at once, and the last
// digit kernel that runs writes the final order.  A tile waits only on tiles
// with smaller tickets, whose CTAs are already running, and every wait is
// bounded (GS_ERR_TIMEOUT in the status word when it gives up).
//
// The scans of the prune entry points keep a fixed grid of sort_blocks() CTAs
// that each own a contiguous range of the items, so item counts produced on
// the device never need to travel to the host.
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
// Generic two-kernel scan: reduce per block, then rescan, each block first
// adding up the counts of the blocks before it (at most kMaxSortBlocks).

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

template <class F, class Out>
__global__ void __launch_bounds__(256) k_scan_down(F f, NSrc ns, const uint32_t *__restrict__ partials, Out out,
                                                   int64_t *__restrict__ n_total) {
    __shared__ uint32_t s_w[8];
    uint32_t beg, end;
    block_range(ns.get(), beg, end);
    uint32_t before = 0;                       // the counts of the blocks before this one
    for (uint32_t b = threadIdx.x; b < blockIdx.x; b += 256) before += partials[b];
    uint32_t run;
    block_scan_256(before, s_w, &run);
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
    if (n_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *n_total = run;   // the last block: the total
}

// --- functors ---
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
// Depth sort.

struct VisSrc {             // one view: visible where its tile count is non-zero
    const uint32_t *tiles, *depth;
    __device__ __forceinline__ bool visible(uint32_t i) const { return tiles[i] > 0; }
    __device__ __forceinline__ uint32_t key(uint32_t i) const { return depth[i]; }
};
struct VisSrc2 {            // two eyes: visible to either; keyed by view a's depth where view a sees it
    const uint32_t *tiles_a, *depth_a, *tiles_b, *depth_b;
    __device__ __forceinline__ bool visible(uint32_t i) const { return tiles_a[i] > 0 || tiles_b[i] > 0; }
    __device__ __forceinline__ uint32_t key(uint32_t i) const { return tiles_a[i] > 0 ? depth_a[i] : depth_b[i]; }
};

constexpr int kLookCounters = 256;                 // one per digit
constexpr uint64_t kLookAgg = 1ull << 32;          // the tile's own count is published
constexpr uint64_t kLookIncl = 2ull << 32;         // the count of every tile up to and including it
constexpr uint32_t kSpinLimit = 1u << 20;
#ifdef GS_DEBUG
// Test hooks of the look-back wait (gs_debug_sort_wait): its iteration limit,
// and a digit kernel whose first tile never publishes its counts.
uint32_t g_dbg_spin_limit = kSpinLimit;
int g_dbg_withhold_pass = -1;
#endif

__device__ __forceinline__ void st_volatile(uint64_t *p, uint64_t v) { *reinterpret_cast<volatile uint64_t *>(p) = v; }
__device__ __forceinline__ uint64_t ld_volatile(const uint64_t *p) {
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

// Digit kernels that run: one per 8-bit digit below the highest bit where the
// smallest and largest visible key differ, and always the first (it also
// compacts the visible Gaussians).
__device__ __forceinline__ int sort_passes(const Ctl *ctl) {
    const uint32_t v = ctl->n_vis > 1 ? (~ctl->depth_mm[0]) ^ ctl->depth_mm[1] : 0u;
    const int m = v ? (39 - __clz(v)) / 8 : 0;     // ceil((32 - clz) / 8)
    return m > 1 ? m : 1;
}

constexpr int kPassThreads = 512;
constexpr int kPassWarps = kPassThreads / 32;
constexpr int kPassTile = kPassThreads * kSortItems;
static_assert(kPassTile % kSortTile == 0, "a digit-kernel tile is whole histogram rounds");

// Tile counts of the first digit kernel: cnt[tile][digit] and their sums
// over groups of 2^lg consecutive tiles, grp[group][digit].
struct TileCounts {
    uint32_t *cnt, *grp;
    int lg;
};

// One CTA per tile of the first digit kernel: the visible count, the key
// range, the four digit histograms, and the tile's count of every first digit.
// Exclusive prefix of counter c over the tiles before tile t (whose own count
// `own` is already published as an aggregate unless t == 0); publishes the
// inclusive prefix of tile t.  The predecessors are read kLookWindow at a time,
// nearest first, so a walk over tiles that only hold aggregates costs one
// memory latency per window instead of one per tile.
constexpr int kLookWindow = 8;
__device__ uint32_t look_back(uint64_t *status, uint32_t t, int c, uint32_t own, Ctl *ctl, uint32_t spin_limit,
                              bool publish) {
    uint32_t excl = 0;
    int64_t j = static_cast<int64_t>(t) - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        uint64_t w[kLookWindow];
#pragma unroll
        for (int k = 0; k < kLookWindow; ++k)
            w[k] = j - k >= 0 ? ld_volatile(status + static_cast<size_t>(j - k) * kLookCounters + c) : kLookIncl;
        int used = 0;
        bool incl = false, waiting = false;
#pragma unroll
        for (int k = 0; k < kLookWindow; ++k) {
            if (incl || waiting) continue;
            const uint64_t flag = w[k] & ~0xFFFFFFFFull;
            if (flag == 0) {
                waiting = true;
                continue;
            }
            excl += static_cast<uint32_t>(w[k]);
            ++used;
            incl = flag == kLookIncl;
        }
        if (incl) break;
        j -= used;
        if (waiting) {
            if (++spins > spin_limit) {
                ctl->st.error = GS_ERR_TIMEOUT;
                break;
            }
            __nanosleep(64);
        }
    }
    if (publish) st_volatile(status + static_cast<size_t>(t) * kLookCounters + c, kLookIncl | (excl + own));
    return excl;
}

template <class Src>
__global__ void __launch_bounds__(256) k_sort_hist(Src src, uint32_t n, uint32_t *__restrict__ ghist, Ctl *ctl,
                                                   TileCounts tc) {
    __shared__ uint32_t s_h[4][256];
    __shared__ uint32_t s_w[8];
    const int lane = threadIdx.x & 31;
    const uint32_t t = blockIdx.x;
    for (int k = threadIdx.x; k < 4 * 256; k += 256) (&s_h[0][0])[k] = 0;
    __syncthreads();
    const uint32_t beg = t * kPassTile, end = min(n, beg + kPassTile);
    uint32_t kinv = 0, kmax = 0, cnt = 0;
    for (uint32_t t0 = beg; t0 < end; t0 += kSortTile) {
        bool vis[kSortItems];
        uint32_t key[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const uint32_t i = t0 + r * 256 + threadIdx.x;
            vis[r] = i < end && src.visible(i);
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) key[r] = vis[r] ? src.key(t0 + r * 256 + threadIdx.x) : 0u;
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (vis[r]) {
                kinv = max(kinv, ~key[r]);
                kmax = max(kmax, key[r]);
                ++cnt;
            }
            const unsigned vm = __ballot_sync(FULL, vis[r]);
            if (vm == 0) continue;
            const int leader = __ffs(vm) - 1;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                // one atomic when the warp's visible keys share the digit (the high digits
                // of depths in a narrow range), else one per key
                const uint32_t d = (key[r] >> (8 * p)) & 255u;
                const uint32_t dl = __shfl_sync(FULL, d, leader);
                if (__all_sync(FULL, !vis[r] || d == dl)) {
                    if (lane == leader) atomicAdd(&s_h[p][dl], __popc(vm));
                } else if (vis[r]) {
                    atomicAdd(&s_h[p][d], 1u);
                }
            }
        }
    }
    kinv = __reduce_max_sync(FULL, kinv);
    kmax = __reduce_max_sync(FULL, kmax);
    if (lane == 0) {        // 0 is neutral for both maxima
        atomicMax(&ctl->depth_mm[0], kinv);
        atomicMax(&ctl->depth_mm[1], kmax);
    }
    uint32_t tot;
    block_scan_256(cnt, s_w, &tot);
    if (threadIdx.x == 0 && tot) {
        atomicAdd(&ctl->n_vis, tot);
        atomicAdd(&ctl->st.n_visible, tot);
    }
    for (int k = threadIdx.x; k < 4 * 256; k += 256) {
        const uint32_t c = (&s_h[0][0])[k];
        if (c) atomicAdd(&ghist[k], c);
    }
    const uint32_t c0 = s_h[0][threadIdx.x];
    tc.cnt[static_cast<size_t>(t) * kLookCounters + threadIdx.x] = c0;
    if (c0) atomicAdd(&tc.grp[static_cast<size_t>(t >> tc.lg) * kLookCounters + threadIdx.x], c0);
}

struct SortBufs {
    const uint32_t *kin, *vin;       // digit kernels after the first: this pass's input
    uint32_t *kout, *vout;           // the next digit kernel's input
    uint32_t *final_out;             // Gaussian indices in depth order (last digit kernel)
    uint32_t *vis_index;             // first digit kernel: visible indices in index order
    const uint32_t *ghist;           // [4][256] digit histograms of the visible keys
    TileCounts tc;                   // first digit kernel: tile and group counts
    uint64_t *status, *status_next;  // look-back words [tile][256] of this (after the first) and the next pass
    uint32_t spin_limit;             // iterations a look-back waits for a predecessor before GS_ERR_TIMEOUT
    int withhold;                    // GS_DEBUG test hook: this kernel's first tile publishes nothing (-1: off)
};

// One digit (bits 8 pass .. 8 pass + 7) of the stable LSD sort, on tiles of
// kPassTile items and CTAs of kPassThreads threads.  Warp w ranks the
// contiguous run [256 w, 256 w + 256) of its tile in 8 rounds of 32 with
// warp-private 16-bit digit counters, so items are ranked in index order; the
// tile is then sorted by digit in shared memory and written out in that order,
// so consecutive threads store consecutive addresses of one digit's run.

// Exclusive scan over the 512 threads of a block; *total = sum of all v.
__device__ __forceinline__ uint32_t block_scan_512(uint32_t v, uint32_t *s_w, uint32_t *total) {
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
        uint32_t w = lane < kPassWarps ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < kPassWarps; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kPassWarps) s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? s_w[warp - 1] : 0;
    *total = s_w[kPassWarps - 1];
    __syncthreads();
    return base + x - v;
}

template <class Src, bool FIRST>
__global__ void __launch_bounds__(kPassThreads) k_sort_pass(Src src, uint32_t n_all, int pass, SortBufs B, Ctl *ctl) {
    __shared__ uint16_t s_wc[kPassWarps][256];   // per-warp digit counts, then per-warp digit bases
    __shared__ uint32_t s_lstart[256];            // start of each digit's run in the locally sorted tile
    __shared__ uint32_t s_off[256];               // global position of each digit's run
    __shared__ uint32_t s_key[kPassTile], s_val[kPassTile];
    __shared__ uint32_t s_w[kPassWarps], s_vw[kPassWarps];
    __shared__ uint32_t s_part[256];               // per digit: its count in this group's tiles before this one
    __shared__ uint32_t s_ticket, s_visbase;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int passes = sort_passes(ctl);
    if (pass >= passes) return;
    const bool last = pass == passes - 1;
    const uint32_t n_vis = min(ctl->n_vis, n_all);
    const uint32_t n = FIRST ? n_all : n_vis;
    const uint32_t ntiles = (n + kPassTile - 1) / kPassTile;
    uint32_t t = blockIdx.x;                       // the first digit kernel: the histogram pass's tiles
    if (FIRST && t >= ntiles) return;
    if (!FIRST && threadIdx.x == 0) s_ticket = atomicAdd(&ctl->sort_ticket[pass], 1u);
    for (int e = threadIdx.x; e < kPassWarps * 256; e += kPassThreads) (&s_wc[0][0])[e] = 0;
    __syncthreads();
    if (!FIRST) {
        t = s_ticket;
        if (t >= ntiles) return;
    }
#ifdef GS_DEBUG
    const bool publish = !(pass == B.withhold && t == 0);
#else
    constexpr bool publish = true;
#endif
    if (!last && t < (n_vis + kPassTile - 1) / kPassTile)
        for (int c = threadIdx.x; c < kLookCounters; c += kPassThreads)
            B.status_next[static_cast<size_t>(t) * kLookCounters + c] = 0;
    const int shift = 8 * pass;
    const uint32_t run0 = t * kPassTile + warp * 256;
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems], vrank[kSortItems];
    bool valid[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = run0 + r * 32 + lane;
        if constexpr (FIRST) {
            valid[r] = i < n && src.visible(i);
            val[r] = i;
        } else {
            valid[r] = i < n;
            val[r] = valid[r] ? B.vin[i] : 0u;
        }
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = run0 + r * 32 + lane;
        if constexpr (FIRST) key[r] = valid[r] ? src.key(i) : 0u;
        else key[r] = valid[r] ? B.kin[i] : 0u;
    }
    uint32_t vw = 0;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t d = valid[r] ? (key[r] >> shift) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(FULL, d);
        const uint32_t before = valid[r] ? s_wc[warp][d] : 0;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid[r] && (peers & lt) == 0) s_wc[warp][d] = static_cast<uint16_t>(before + __popc(peers));
        __syncwarp();
        if constexpr (FIRST) {
            const unsigned vb = __ballot_sync(FULL, valid[r]);
            vrank[r] = vw + __popc(vb & lt);
            vw += __popc(vb);
        }
    }
    if constexpr (FIRST) {
        if (lane == 0) s_vw[warp] = vw;
    }
    __syncthreads();
    const int d = threadIdx.x & 255;
    const bool dig = threadIdx.x < 256;
    uint32_t part = 0;
    if constexpr (FIRST) {
        // the count of digit d in the tiles before this one: the first 256 threads sum the groups before
        // this tile's group, the others the tiles before it in its group
        const uint32_t g0 = t >> B.tc.lg;
        if (dig) {
            const uint32_t *gp = B.tc.grp + d;
#pragma unroll 8
            for (uint32_t g = 0; g < g0; ++g) part += gp[static_cast<size_t>(g) * kLookCounters];
        } else {
            const uint32_t *cp = B.tc.cnt + d;
#pragma unroll 8
            for (uint32_t u = g0 << B.tc.lg; u < t; ++u) part += cp[static_cast<size_t>(u) * kLookCounters];
            s_part[d] = part;
        }
    }
    // per digit d (the first 256 threads): exclusive prefix over the warps, the tile's count, and (after
    // the first digit kernel) its publication
    uint32_t acc = 0;
    if (dig) {
#pragma unroll
        for (int w = 0; w < kPassWarps; ++w) {
            const uint32_t c = s_wc[w][d];
            s_wc[w][d] = static_cast<uint16_t>(acc);
            acc += c;
        }
        if (!FIRST && publish)
            st_volatile(B.status + static_cast<size_t>(t) * kLookCounters + d, (t == 0 ? kLookIncl : kLookAgg) | acc);
    }
    uint32_t ntile;
    const uint32_t ls = block_scan_512(acc, s_w, &ntile);      // synchronises: s_part is complete
    if (dig) s_lstart[d] = ls;
    uint32_t gtot;
    const uint32_t gbase = block_scan_512(dig ? B.ghist[pass * 256 + d] : 0u, s_w, &gtot);
    uint32_t excl = 0;
    if (dig) excl = FIRST ? part + s_part[d] : look_back(B.status, t, d, acc, ctl, B.spin_limit, publish);
    if (dig) s_off[d] = gbase + excl;
    if constexpr (FIRST) {
        // the items of all digits in the tiles before this one are the visible Gaussians before it
        uint32_t before;
        block_scan_512(excl, s_w, &before);
        if (d == 0) s_visbase = before;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (valid[r]) {
            const uint32_t dd = (key[r] >> shift) & 255u;
            const uint32_t lpos = s_lstart[dd] + s_wc[warp][dd] + rank[r];
            s_key[lpos] = key[r];
            s_val[lpos] = val[r];
        }
    }
    if constexpr (FIRST) {
        uint32_t vbase = s_visbase;
        for (int w = 0; w < warp; ++w) vbase += s_vw[w];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r)
            if (valid[r]) B.vis_index[vbase + vrank[r]] = val[r];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ntile; i += kPassThreads) {
        const uint32_t k = s_key[i];
        const uint32_t dd = (k >> shift) & 255u;
        const uint32_t pos = s_off[dd] + (i - s_lstart[dd]);
        if (!GS_CHECK(pos < n_vis, ctl, kSiteSortScatter)) continue;
        if (last) {
            B.final_out[pos] = s_val[i];
        } else {
            B.kout[pos] = k;
            B.vout[pos] = s_val[i];
        }
    }
}

// 2^lg tiles per group: the least with 2^(2 lg) >= tiles.
int sort_group_log(uint32_t nt) {
    int lg = 0;
    while ((static_cast<uint64_t>(1) << (2 * lg)) < nt) ++lg;
    return lg;
}

TileCounts tile_counts(const SortWork &w, int n) {
    TileCounts tc;
    tc.cnt = w.cnt;
    tc.grp = w.grp;
    tc.lg = sort_group_log(sort_tiles(n));
    return tc;
}

template <class Src>
cudaError_t sort_histograms(const Src &src, int n, const SortWork &w, Ctl *ctl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // the histograms and the group counts were cleared with the control block
    const TileCounts tc = tile_counts(w, n);
    k_sort_hist<<<sort_tiles(n), 256, 0, st>>>(src, static_cast<uint32_t>(n), w.ghist, ctl, tc);
    return cudaGetLastError();
}

template <class Src>
cudaError_t sort_digits(const Src &src, int n, const SortWork &w, Ctl *ctl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const TileCounts tc = tile_counts(w, n);
    const uint32_t nt = sort_tiles(n);
    uint32_t *A[2] = {w.keys[0], w.vals[0]}, *Bb[2] = {w.keys[1], w.vals[1]};
    for (int p = 0; p < 4; ++p) {
        SortBufs b;
        uint32_t *const *in = (p & 1) ? A : Bb;       // pass p reads what pass p - 1 wrote
        uint32_t *const *out = (p & 1) ? Bb : A;
        b.kin = in[0];
        b.vin = in[1];
        b.kout = out[0];
        b.vout = out[1];
        b.final_out = w.order;
        b.vis_index = w.vis_index;
        b.ghist = w.ghist;
        b.tc = tc;
        b.status = p > 0 ? w.status + static_cast<size_t>(p - 1) * nt * kLookCounters : nullptr;
        b.status_next = p < 3 ? w.status + static_cast<size_t>(p) * nt * kLookCounters : nullptr;
#ifdef GS_DEBUG
        b.spin_limit = g_dbg_spin_limit;
        b.withhold = g_dbg_withhold_pass;
#else
        b.spin_limit = kSpinLimit;
        b.withhold = -1;
#endif
        if (p == 0) k_sort_pass<Src, true><<<nt, kPassThreads, 0, st>>>(src, static_cast<uint32_t>(n), p, b, ctl);
        else k_sort_pass<Src, false><<<nt, kPassThreads, 0, st>>>(src, static_cast<uint32_t>(n), p, b, ctl);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

}  // namespace

int sort_blocks() {
    static PerDevice cache;
    return cache.get([] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int g = 4 * (sms > 0 ? sms : 80);
        return g < kMaxSortBlocks ? g : kMaxSortBlocks;
    });
}

uint32_t sort_tiles(int64_t n) { return static_cast<uint32_t>((n + kPassTile - 1) / kPassTile); }

size_t sort_count_bytes(int64_t n) {
    return static_cast<size_t>(sort_tiles(n > 0 ? n : 1)) * kLookCounters * sizeof(uint32_t);
}

size_t sort_status_bytes(int64_t n) {
    return 3 * static_cast<size_t>(sort_tiles(n > 0 ? n : 1)) * kLookCounters * sizeof(uint64_t);
}

size_t sort_group_bytes(int64_t n) {
    // ceil(sqrt(tiles)) groups: never fewer than the ceil(tiles / 2^lg) in use (2^lg >= sqrt(tiles)), and
    // non-decreasing in n, so a workspace sized for n Gaussians also holds any smaller scene
    const uint32_t nt = sort_tiles(n > 0 ? n : 1);
    uint32_t g = 1;
    while (static_cast<uint64_t>(g) * g < nt) ++g;
    return static_cast<size_t>(g) * kLookCounters * sizeof(uint32_t);
}

cudaError_t launch_sort_histograms(const uint32_t *tiles, const uint32_t *depth, int n, const SortWork &w, Ctl *ctl,
                                   cudaStream_t st) {
    return sort_histograms(VisSrc{tiles, depth}, n, w, ctl, st);
}

cudaError_t launch_sort_digits(const uint32_t *tiles, const uint32_t *depth, int n, const SortWork &w, Ctl *ctl,
                               cudaStream_t st) {
    return sort_digits(VisSrc{tiles, depth}, n, w, ctl, st);
}

cudaError_t launch_sort_histograms2(const uint32_t *tiles_a, const uint32_t *depth_a, const uint32_t *tiles_b,
                                    const uint32_t *depth_b, int n, const SortWork &w, Ctl *ctl, cudaStream_t st) {
    return sort_histograms(VisSrc2{tiles_a, depth_a, tiles_b, depth_b}, n, w, ctl, st);
}

cudaError_t launch_sort_digits2(const uint32_t *tiles_a, const uint32_t *depth_a, const uint32_t *tiles_b,
                                const uint32_t *depth_b, int n, const SortWork &w, Ctl *ctl, cudaStream_t st) {
    return sort_digits(VisSrc2{tiles_a, depth_a, tiles_b, depth_b}, n, w, ctl, st);
}

cudaError_t launch_activity_prune(const float *activity, const uint8_t *layer, uint32_t train_mask, int n,
                                  float samples, float thr, uint8_t *keep, int32_t *keep_index, int64_t *n_keep,
                                  uint32_t *partials, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{nullptr, static_cast<uint32_t>(n)};
    ActiveFlag f{activity, layer, train_mask, 1.f / samples, thr};
    k_scan_reduce<<<G, 256, 0, st>>>(f, ns, partials);
    k_scan_down<<<G, 256, 0, st>>>(f, ns, partials, KeepOut{keep, keep_index}, n_keep);
    return cudaGetLastError();
}

cudaError_t launch_prune(const float *contrib_max, int n, float thr, uint8_t *keep, int32_t *keep_index,
                         int64_t *n_keep, uint32_t *partials, cudaStream_t st) {
    const int G = sort_blocks();
    NSrc ns{nullptr, static_cast<uint32_t>(n)};
    KeepFlag f{contrib_max, thr};
    k_scan_reduce<<<G, 256, 0, st>>>(f, ns, partials);
    k_scan_down<<<G, 256, 0, st>>>(f, ns, partials, KeepOut{keep, keep_index}, n_keep);
    return cudaGetLastError();
}

}  // namespace gs

extern "C" int gs_debug_sort_wait(uint32_t spin_limit, int32_t withhold_pass) {
#ifdef GS_DEBUG
    if (withhold_pass != -1 && (withhold_pass < 1 || withhold_pass > 3))
        return gs::report(GS_ERR_INVALID, "gs_debug_sort_wait: withhold_pass must be -1 or 1..3");
    gs::g_dbg_spin_limit = spin_limit ? spin_limit : gs::kSpinLimit;
    gs::g_dbg_withhold_pass = withhold_pass;
    return GS_OK;
#else
    (void)spin_limit;
    (void)withhold_pass;
    return gs::report(GS_ERR_INVALID, "gs_debug_sort_wait: only in GS_DEBUG builds");
#endif
}
