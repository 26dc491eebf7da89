// S3 / S4a - front-to-back compositing of each 16x16 tile over its sorted
// splat list (Sec. 3.3: Gaussians rendered as splats in camera-sorted order),
// and its exact backward with the per-Gaussian blend weight alpha*T that
// drives contribution pruning (Sec. 3.2.2).
//
// Work decomposition (compositing is FP32 FMA + MUFU work, not a dense
// contraction, so no tensor cores are involved):
//  * Forward: persistent warps take work items (tile, 8x4 pixel block) from
//    per-view device queues in heaviest-first tile order (the views of a
//    batch in turn) and composite one pixel per lane until the block's 32
//    pixels are done.  The walk goes segment by segment (kSeg list
//    positions), each segment blended from a local product that the
//    transmittance at its start scales; at every segment boundary the warp
//    stores each pixel's transmittance as a checkpoint, with the colour
//    blended from there to the end of the pixel's walk (filled in when the
//    walk ends).
//  * Both passes drop, 32 records at a time, the splats that provably stay
//    below alpha = 1/255 over the warp's whole pixel block (see
//    splat_reaches_block); list positions are kept, so nothing changes.
//  * Backward: the blended prefix of a pixel can be thousands of splats long,
//    and walking it serially would make the longest pixel the critical path
//    of the whole kernel.  The checkpoints cut every 8x8 block's walk into
//    segments of at most kSeg positions; persistent warps take (tile, block,
//    segment) items from a queue and each walks its segment back to front
//    from the checkpoint at the segment's end.  The forward writes the items:
//    the second 8x4 block of an 8x8 block to finish knows the block's longest
//    blended prefix, so no ordering pass runs between the two.
//
// splat_alpha() is the single definition of the per-(pixel, splat) alpha used
// by both passes; every operation is an explicitly rounded intrinsic, so the
// backward reproduces the forward's skip decisions bit for bit.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr float kLn2 = 0x1.62e430p-1f;
constexpr int kFwdThreads = 256;
// One pixel per lane, an 8x4 block per warp.  (Two pixels per lane, an 8x8 block, gives each lane two blend
// chains but culls on a larger block and needs 70 registers; on the 1.2M-Gaussian frame it measured 0.28 ms
// against 0.22 ms.)
constexpr int kBwdThreads = 128;
// Backward pixels per lane: 2 (an 8x8 block per warp) or 4 (16x8).  4 halves the per-splat reduction and
// atomics per pixel but needs 96 registers (5 blocks per SM instead of 7) and culls on a coarser block;
// on the 1.2M-Gaussian frame it measured 0.403 ms against 0.362 ms for 2.
constexpr int kBwdPx = 2;
// The forward writes the backward's work items per 8x8 block (two pixels per lane).
static_assert(kBwdPx == 2, "backward work items are 8x8 blocks");

// 1/x to about 1 ulp (the hardware reciprocal approximation; x = 1 - alpha is in [0.01, 1]).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha = min(0.99, o * 2^(A2 (dx + beta dy)^2 + G2 dy^2)), d = pixel - mean.
// Returns alpha; p, dy, ex (= 2^e) and the unclamped product ao are outputs.
__device__ __forceinline__ float splat_alpha(float px, float py, const float4 a, const float4 b, float &p, float &dy,
                                             float &ex, float &ao) {
    const float dx = __fsub_rn(px, a.x);
    dy = __fsub_rn(py, a.y);
    p = __fmaf_rn(a.w, dy, dx);
    const float e = __fmaf_rn(__fmul_rn(a.z, p), p, __fmul_rn(__fmul_rn(b.x, dy), dy));
    ex = ex2_approx(e);
    ao = __fmul_rn(b.y, ex);
    return fminf(kAlphaMax, ao);
}

__device__ __forceinline__ uint32_t ceil_seg(uint32_t n) { return (n + kSeg - 1) / kSeg; }

// Can the splat reach alpha >= 1/255 at some pixel centre of the block
// [x0, x1] x [y0, y1]?  The exponent A2 p^2 + G2 dy^2 (p = dx + beta dy) is a
// sum of two non-positive terms, so max(A2 p^2) + max(G2 dy^2) over the block
// bounds it from above; p is linear, so its range over the block comes from
// the corners.  The test keeps a splat unless even that bound, raised by a
// margin far above single-precision rounding of the per-pixel exponent, gives
// alpha < 1/255: a dropped splat is one the per-pixel test would skip at every
// pixel of the block, so dropping it changes no result.
__device__ __forceinline__ bool splat_reaches_block(const float4 a, const float4 b, float x0, float x1, float y0,
                                                    float y1) {
    const float dylo = y0 - a.y, dyhi = y1 - a.y;
    const float mdy = dylo > 0.f ? dylo : (dyhi < 0.f ? -dyhi : 0.f);
    const float blo = a.w * dylo, bhi = a.w * dyhi;
    const float plo = (x0 - a.x) + fminf(blo, bhi), phi = (x1 - a.x) + fmaxf(blo, bhi);
    const float mp = plo > 0.f ? plo : (phi < 0.f ? -phi : 0.f);
    const float emax = a.z * mp * mp + b.x * mdy * mdy;
    return b.y * ex2_approx(emax + 1e-3f) >= kAlphaMin;
}

// Exclusive scan over a 1024-thread block; returns the prefix, *total the sum.
__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t *s_w, uint32_t *total) {
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
        uint32_t w = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? s_w[warp - 1] : 0;
    *total = s_w[31];
    __syncthreads();
    return base + x - v;
}

// Bucket of a work amount for a heaviest-first counting sort: a logarithmic
// scale with 16 sub-steps per octave; zero work goes last.
constexpr int kBuckets = 513;
__device__ __forceinline__ int work_bucket(uint32_t w) {
    if (w == 0) return kBuckets - 1;
    const int lz = 31 - __clz(w);
    const uint32_t sub = lz >= 4 ? (w >> (lz - 4)) & 15u : (w << (4 - lz)) & 15u;
    return (kBuckets - 2) - (lz * 16 + static_cast<int>(sub));
}

// One CTA (1024 threads) sorts the tiles heaviest first (by list length) into
// order[] (ties in no particular order: tiles are independent, so the order
// changes no result).
__device__ void order_tiles(int Tn, uint32_t *order, uint32_t *s_cnt, uint32_t *s_w, const uint2 *ranges) {
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < Tn; t += blockDim.x) atomicAdd(&s_cnt[work_bucket(ranges[t].y - ranges[t].x)], 1u);
    __syncthreads();
    {
        const uint32_t c = threadIdx.x < kBuckets ? s_cnt[threadIdx.x] : 0;
        uint32_t tot;
        const uint32_t ex = block_scan_1024(c, s_w, &tot);
        if (threadIdx.x < kBuckets) s_cnt[threadIdx.x] = ex;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Tn; t += blockDim.x)
        order[atomicAdd(&s_cnt[work_bucket(ranges[t].y - ranges[t].x)], 1u)] = t;
    __syncthreads();
}

// Forward set-up (one CTA): heaviest-first tile order by list length, the
// checkpoint base of every tile (exclusive prefix of its segment count), and
// zeroed meeting words of the 8x8 blocks and queue.
// The set-up is a single CTA walking every tile several times; up to
// kSetupSmemTiles tiles, the tile ranges are first staged in dynamic shared
// memory so the later passes cost no memory round trips.
constexpr int kSetupSmemTiles = 8192;

__global__ void __launch_bounds__(1024) k_fwd_setup(const uint2 *__restrict__ g_ranges, int Tn,
                                                    uint32_t *__restrict__ order, uint32_t *__restrict__ seg_base,
                                                    uint32_t *__restrict__ queue, uint32_t *__restrict__ qdone) {
    __shared__ uint32_t s_cnt[kBuckets];
    __shared__ uint32_t s_w[32];
    extern __shared__ uint2 s_ranges[];
    if (threadIdx.x == 0) *queue = 0;
    const uint2 *ranges = g_ranges;
    if (Tn <= kSetupSmemTiles) {
        for (int t = threadIdx.x; t < Tn; t += blockDim.x) s_ranges[t] = g_ranges[t];
        __syncthreads();
        ranges = s_ranges;
    }
    for (int q = threadIdx.x; q < 8 * Tn; q += blockDim.x) qdone[q] = 0;   // 4 x 64-bit meeting words per tile
    order_tiles(Tn, order, s_cnt, s_w, ranges);
    uint32_t carry = 0;
    for (int t0 = 0; t0 < Tn; t0 += 1024) {
        const int t = t0 + threadIdx.x;
        const uint32_t v = t < Tn ? ceil_seg(ranges[t].y - ranges[t].x) : 0;
        uint32_t tot;
        const uint32_t ex = block_scan_1024(v, s_w, &tot);
        if (t < Tn) seg_base[t] = carry + ex;
        carry += tot;
    }
}

struct Chunk {
    float4 a, b;
    float c;
    uint32_t g;
    uint32_t ly;      // backward: the splat's layer, consumed one chunk later
};

// n, ctl, site: the Gaussian count and the bounds check of GS_DEBUG builds
// (nothing in release builds).
__device__ __forceinline__ void fetch_chunk(const uint32_t *__restrict__ list, const Rec *__restrict__ rec,
                                            uint32_t pos, uint32_t end, Chunk &ch, uint32_t n, const Ctl *ctl,
                                            uint32_t site) {
    if (pos < end) {
        const uint32_t g = list[pos];
        if (!GS_CHECK(g < n, ctl, site)) {
            ch = Chunk{};          // an inert splat (opacity 0): no block keeps it
            return;
        }
        ch.g = g;
        const Rec *r = rec + ch.g;
        ch.a = r->a;
        ch.b = r->b;
        ch.c = r->c.x;
    }
}

// The backward also needs each splat's layer (frozen layers get no gradient).
__device__ __forceinline__ void fetch_chunk_layer(const uint32_t *__restrict__ list, const Rec *__restrict__ rec,
                                                  const uint8_t *__restrict__ layer, uint32_t pos, uint32_t end,
                                                  Chunk &ch, uint32_t n, const Ctl *ctl) {
    fetch_chunk(list, rec, pos, end, ch, n, ctl, kSiteBwdId);
    if (pos < end && GS_CHECK(ch.g < n, ctl, kSiteBwdId)) ch.ly = layer[ch.g];
}

// The record of an id loaded one chunk earlier: list and record loads of a
// chunk are issued a chunk apart, so the record load does not wait on the
// list load in the same iteration.
__device__ __forceinline__ void fetch_rec(const Rec *__restrict__ rec, uint32_t g, bool valid, Chunk &ch) {
    if (valid) {
        ch.g = g;
        const Rec *r = rec + g;
        ch.a = r->a;
        ch.b = r->b;
        ch.c = r->c.x;
    }
}

__device__ __forceinline__ void fetch_rec_layer(const Rec *__restrict__ rec, const uint8_t *__restrict__ layer,
                                                uint32_t g, bool valid, Chunk &ch, uint32_t n, const Ctl *ctl) {
    if (valid && !GS_CHECK(g < n, ctl, kSiteBwdId)) {
        ch = Chunk{};              // an inert splat (opacity 0): no block keeps it
        return;
    }
    fetch_rec(rec, g, valid, ch);
    if (valid) ch.ly = layer[g];
}

struct FwdBatch {
    FwdJob job[kMaxBatch];
    int n;
};

// Forward compositing, segment by segment.  A pixel's walk is cut at the
// checkpoint segments (kSeg list positions).  In every segment the pixel
// blends from a local product P = 1: the colour D it blends there is relative
// to Ts, its transmittance at the segment's start, and the segment ends with
// colour Ts * D and transmittance Ts * P.  The stop test of a splat is
// Ts * P * (1 - alpha) < kTMin, the paper's T < 1e-4 on this factorisation.
// The checkpoints store Ts and the colour blended from the segment on, which
// is all the backward needs to start a segment's walk from its end.
constexpr int kFwdWarps = kFwdThreads / 32;

struct FwdLane {        // one pixel's walk
    float Ts;           // transmittance at the start of the current segment
    float P;            // product of (1 - alpha) over the splats blended in the segment
    float D0, D1, D2;   // colour blended in the segment, relative to Ts
    uint32_t last;      // 1 + list position (from the tile's first entry) of the last blended splat
    uint32_t nb;        // blended splats
    bool done;          // stopped (or outside the image)
};

struct FwdPipe {        // list ids and records fetched ahead of the walk
    Chunk nxt;          // records of the 32 entries at pos
    uint32_t gid;       // ids of the 32 entries at pos + 32
    uint32_t pos;       // list position (from the tile's first entry) of nxt
};

struct FwdSmem {
    float4 a[kFwdWarps][32], b[kFwdWarps][32];
    float c[kFwdWarps][32];
    uint32_t pos[kFwdWarps][32];
};

// Walks list positions [pp.pos, e) of the block at (bx0, by0) (an 8x4 block of
// pixel centres), 32 entries at a time: the entries that can reach the block
// are staged in shared memory, and each lane blends them into its pixel's
// segment state.  Returns early once every lane has stopped.
__device__ __forceinline__ void walk_segment(FwdPipe &pp, uint32_t e, const FwdJob &J, uint2 rg, float bx0, float by0,
                                             float px, float py, FwdLane &L, int lane, int warp, FwdSmem &sm) {
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t len = rg.y - rg.x;
    bool mine = L.done;
    for (; pp.pos < e; pp.pos += 32) {
        if (__all_sync(FULL, mine)) break;
        const uint32_t base = pp.pos;
        const bool keep =
            base + lane < len && splat_reaches_block(pp.nxt.a, pp.nxt.b, bx0, bx0 + 7.f, by0, by0 + 3.f);
        const unsigned km = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) {
            const int slot = __popc(km & lt);
            sm.a[warp][slot] = pp.nxt.a;
            sm.b[warp][slot] = pp.nxt.b;
            sm.c[warp][slot] = pp.nxt.c;
            sm.pos[warp][slot] = base + lane;
        }
        __syncwarp();
        const bool v1 = base + 32 + lane < len;
        if (v1 && !GS_CHECK(pp.gid < J.n, J.ctl, kSiteFwdId))
            pp.nxt = Chunk{};      // an inert splat (opacity 0): no block keeps it
        else
            fetch_rec(J.rec, pp.gid, v1, pp.nxt);
        pp.gid = base + 64 + lane < len ? J.list[rg.x + base + 64 + lane] : 0u;
        const int cnt = __popc(km);
        int lastk = -1;
        for (int k = 0; k < cnt && !mine; ++k) {
            const float4 a = sm.a[warp][k], b = sm.b[warp][k];
            float p, dy, ex, ao;
            const float al = splat_alpha(px, py, a, b, p, dy, ex, ao);
            if (al >= kAlphaMin) {
                const float Pn = __fmul_rn(L.P, __fsub_rn(1.f, al));
                if (__fmul_rn(L.Ts, Pn) < kTMin) {
                    L.done = true;
                    mine = true;
                } else {
                    const float w = __fmul_rn(al, L.P);
                    L.D0 = __fmaf_rn(b.z, w, L.D0);
                    L.D1 = __fmaf_rn(b.w, w, L.D1);
                    L.D2 = __fmaf_rn(sm.c[warp][k], w, L.D2);
                    L.P = Pn;
                    lastk = k;
                    ++L.nb;
                }
            }
        }
        if (lastk >= 0) L.last = sm.pos[warp][lastk] + 1;    // position of the chunk's last blend, read once
    }
}

// The live view after v in turn (live != 0, v < 31).
__device__ __forceinline__ int next_live(uint32_t live, int v) {
    const uint32_t after = live & ~((2u << v) - 1u);
    return __ffs(after ? after : live) - 1;
}

__global__ void __launch_bounds__(kFwdThreads) k_composite_fwd(const __grid_constant__ FwdBatch batch) {
    __shared__ FwdSmem sm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Views of a batch are taken in turn, each from its own heaviest-first queue, so the heaviest blocks of
    // every view start first; a view whose queue has run out leaves the rotation.
    uint32_t live = (1u << batch.n) - 1u;
    int v = static_cast<int>((blockIdx.x * kFwdWarps + warp) % static_cast<uint32_t>(batch.n));
    for (;;) {
        uint32_t local = 0;
        if (lane == 0) {
            for (;;) {
                local = atomicAdd(batch.job[v].queue, 1u);
                if (local < static_cast<uint32_t>(batch.job[v].Tn) * 8u) break;
                live &= ~(1u << v);
                if (!live) break;
                v = next_live(live, v);
            }
        }
        live = __shfl_sync(FULL, live, 0);
        if (!live) break;
        local = __shfl_sync(FULL, local, 0);
        v = __shfl_sync(FULL, v, 0);
        const FwdJob &J = batch.job[v];
        const int W = J.W, H = J.H, Tx = J.Tx;
        const int tile = J.order[local / 8];
        const int sub = local % 8;                      // block column sub & 1, block row sub >> 1
        const int ox = (sub & 1) * 8, oy = (sub >> 1) * 4;
        const uint2 rg = J.ranges[tile];
        const float bx0 = (tile % Tx) * kTile + ox + 0.5f, by0 = (tile / Tx) * kTile + oy + 0.5f;
        const int lx = ox + (lane & 7), ly = oy + (lane >> 3);
        const int x = (tile % Tx) * kTile + lx, y = (tile / Tx) * kTile + ly;
        const bool inside = x < W && y < H;
        FwdLane L{1.f, 1.f, 0.f, 0.f, 0.f, 0u, 0u, !inside};
        float C0 = 0.f, C1 = 0.f, C2 = 0.f;             // colour of the last finished segment
        const uint32_t len = rg.y - rg.x, nseg = ceil_seg(len);
        float4 *ck0 = J.ckpt + static_cast<size_t>(J.seg_base[tile]) * kTilePix + lx;
        FwdPipe pp;
        pp.pos = 0;
        fetch_chunk(J.list, J.rec, rg.x + lane, rg.y, pp.nxt, J.n, J.ctl, kSiteFwdId);
        pp.gid = rg.x + 32 + lane < rg.y ? J.list[rg.x + 32 + lane] : 0u;   // ids one chunk ahead
        uint32_t sd = 0;
        for (uint32_t s = 0; s < nseg; ++s) {
            if (s > 0) {
                if (__all_sync(FULL, L.done)) break;
                sd = s;
                if (!GS_CHECK(J.seg_base[tile] + sd < J.n_segs, J.ctl, kSiteCkpt)) break;
                // checkpoint s: (T at the segment's start, colour of segment s - 1); rewritten below
                ck0[static_cast<size_t>(sd) * kTilePix + ly * kTile] = make_float4(L.Ts, C0, C1, C2);
            }
            walk_segment(pp, min((s + 1) * kSeg, len), J, rg, bx0, by0, x + 0.5f, y + 0.5f, L, lane, warp, sm);
            // the segment ends: its colour, the transmittance at the next segment's start
            C0 = __fmul_rn(L.Ts, L.D0);
            C1 = __fmul_rn(L.Ts, L.D1);
            C2 = __fmul_rn(L.Ts, L.D2);
            L.Ts = __fmul_rn(L.Ts, L.P);
            L.P = 1.f;
            L.D0 = L.D1 = L.D2 = 0.f;
        }
        // Checkpoint s holds (T at segment start, colour of segment s-1) as written
        // above; rewrite it, deepest segment first, to (T at segment start, F_s),
        // F_s = colour blended at list positions >= s kSeg.  F_0 is the pixel's colour.
        for (uint32_t s = sd; s > 0; --s) {
            float4 *slot = ck0 + static_cast<size_t>(s) * kTilePix + ly * kTile;
            const float4 raw = *slot;
            *slot = make_float4(raw.x, C0, C1, C2);
            C0 = __fadd_rn(raw.y, C0);
            C1 = __fadd_rn(raw.z, C1);
            C2 = __fadd_rn(raw.w, C2);
        }
        if (inside) {
            const size_t plane = static_cast<size_t>(W) * H;
            const size_t pix = static_cast<size_t>(y) * W + x;
            J.image[pix] = __fmaf_rn(L.Ts, J.bg.x, C0);
            J.image[plane + pix] = __fmaf_rn(L.Ts, J.bg.y, C1);
            J.image[2 * plane + pix] = __fmaf_rn(L.Ts, J.bg.z, C2);
            if (J.alpha) J.alpha[pix] = 1.f - L.Ts;
            J.t_final[pix] = L.Ts;
            J.n_contrib[pix] = L.last;
        }
        const uint32_t wm = __reduce_max_sync(FULL, L.last);
        const int qd = (sub & 1) + 2 * (oy >> 3);      // the 8x8 block of the tile this 8x4 block is half of
        const uint32_t wb = __reduce_add_sync(FULL, L.nb);
        if (lane == 0 && wb) atomicAdd(J.n_blended, static_cast<unsigned long long>(wb));
        // The two 8x4 blocks of an 8x8 block meet in one 64-bit word (finished blocks << 32 | longest blended
        // prefix).  The second to finish knows the 8x8 block's longest blended prefix: it stores it for the
        // backward and appends the block's backward work items, one per kSeg positions of the prefix.  They come
        // out in the order the forward finishes them, the heaviest tiles last; the backward takes them from the end.
        uint32_t nsg = 0, ibase = 0;
        if (lane == 0) {
            unsigned long long *meet = reinterpret_cast<unsigned long long *>(J.qdone) + 4 * tile + qd;
            unsigned long long seen = 0ull, prev = ~0ull;
            bool ok = false;
            for (int round = 0; round < 3 && !ok; ++round) {   // two rounds at most: one other writer, once
                const unsigned long long want =
                    ((seen >> 32) + 1ull) << 32 | max(static_cast<uint32_t>(seen), wm);
                prev = atomicCAS(meet, seen, want);
                ok = prev == seen;
                seen = prev;
            }
            if (ok && (prev >> 32) == 1ull) {
                const uint32_t qm = max(static_cast<uint32_t>(prev), wm);
                J.qwork[4 * tile + qd] = qm;
                nsg = ceil_seg(qm);
                if (nsg) ibase = atomicAdd(J.n_items, nsg);
            }
        }
        nsg = __shfl_sync(FULL, nsg, 0);
        ibase = __shfl_sync(FULL, ibase, 0);
        for (uint32_t sg = lane; sg < nsg; sg += 32)
            J.items[ibase + sg] = make_uint2(static_cast<uint32_t>(tile), (static_cast<uint32_t>(qd) << 24) | sg);
        v = next_live(live, v);
    }
}

// Backward set-up: the work items (tile, 8x8 block q, segment s) were written
// by the forward as it finished each 8x8 block; this kernel restarts the work
// queue and zeroes the record-gradient rows of the visible Gaussians (visible
// list of the last render, n_vis entries), the only rows the compositor adds
// to and the chain rule reads.
__global__ void __launch_bounds__(1024) k_bwd_setup(uint32_t *__restrict__ queue,
                                                    const uint32_t *__restrict__ vis_index,
                                                    const uint32_t *__restrict__ n_vis, int n,
                                                    float4 *__restrict__ rec_grad) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *queue = 0;
    const uint32_t nv = min(*n_vis, static_cast<uint32_t>(n));
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nv; p += gridDim.x * blockDim.x) {
        const size_t i = vis_index[p];
        rec_grad[3 * i] = z;
        rec_grad[3 * i + 1] = z;
        rec_grad[3 * i + 2] = z;
    }
}

// Reduce-scatter of 10 values across a warp in 12 shuffles.  Halving by lane
// bit: bit 4 splits the values 5 / 5, bit 3 splits each half 3 / 2, bit 2
// splits those 2 / 1 and 1 / 1, bit 1 splits the remaining pair, and bit 0
// completes the sums.  Lane l ends with the warp sum of value
// reduce10_owner(l); value i is held by the lanes of one aligned group.
__device__ __forceinline__ int reduce10_owner(int lane) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    return 5 * b4 + (b3 ? 3 + b2 : (b2 ? 2 : b1));
}

// The lowest lane holding each value (lanes 0, 2, 4, 8, 12, 16, 18, 20, 24, 28).
__device__ __forceinline__ bool reduce10_writer(int lane) {
    return !(lane & 1) && (((lane & 12) == 0) || !(lane & 2));
}

__device__ __forceinline__ float reduce_scatter10(const float v[10], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float keep = b4 ? v[i + 5] : v[i];
        const float send = b4 ? v[i] : v[i + 5];
        a[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    float c[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float hi = i < 2 ? a[i + 3] : 0.f;
        const float send = b3 ? a[i] : hi;
        const float keep = b3 ? hi : a[i];
        c[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    const float s0 = b3 ? (b2 ? c[0] : c[1]) : (b2 ? c[0] : c[2]);
    const float s1 = (!b3 && b2) ? c[1] : 0.f;
    const float r0 = __shfl_xor_sync(FULL, s0, 4);
    const float r1 = __shfl_xor_sync(FULL, s1, 4);
    const float d0 = (b3 ? (b2 ? c[1] : c[0]) : (b2 ? c[2] : c[0])) + r0;
    const float d1 = c[1] + r1;
    const bool two = !b3 && !b2;
    const float s2 = two ? (b1 ? d0 : d1) : d0;
    const float e = (two ? (b1 ? d1 : d0) : d0) + __shfl_xor_sync(FULL, s2, 2);
    return e + __shfl_xor_sync(FULL, e, 1);
}

// Backward, back to front within a segment.  With
//   S_i = sum_{j>i} c_j a_j T_j + T_N bg   (T_j: transmittance before splat j)
//   dL/da_i = T_i (dC.c_i) - (dC.S_i - dA T_N) / (1 - a_i).
// The scalar R_i = dC.S_i - dA T_N is carried from the back: a work item
// covers list positions [s kSeg, (s+1) kSeg) of one 8x8 block (two pixels per
// lane) and starts from the forward's checkpoint of segment s+1, which holds
// the transmittance there and the colour blended from there on (or from T_N
// and zero when the pixel stopped inside segment s).  Going back, T_i =
// T_{i+1} / (1 - a_i) and R_{i-1} = R_i + (dC.c_i) a_i T_i: every term of R
// is at most of the size of T there, so deep splats keep their relative
// accuracy (a running total minus a prefix would not).
//
// Each splat's 10 sums are reduce-scattered over the warp and added to the
// record gradient, float 12 g + i for value i, by ten lanes at once:
//   (du, dv, dA2, dbeta, dG2, dopacity, dr, dg, db, sum of alpha*T);
//   contrib_max[g] = max(.., alpha*T).
// The five geometric values are summed as moments of dL/de' (e' the natural
// exponent) and scaled by the splat's constants once, after the warp sum.
// 1 / (1 - a_i) is the hardware reciprocal approximation (about 1 ulp): a
// correctly rounded reciprocal costs several instructions per pixel and
// splat and changes the gradients only at the last bits.
// Six CTAs per SM (at most 80 registers) measured faster than five at 89.
template <int PX>
__global__ void __launch_bounds__(kBwdThreads, 6) k_composite_bwd(
    const uint2 *__restrict__ items, const uint32_t *__restrict__ n_items, uint32_t *__restrict__ queue,
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ list, const Rec *__restrict__ rec, int W, int H,
    int Tx, float3 bg, const float *__restrict__ t_final, const uint32_t *__restrict__ n_contrib,
    const uint32_t *__restrict__ seg_base, const float4 *__restrict__ ckpt, const uint32_t *__restrict__ qwork,
    const float *__restrict__ dL_dimage, const float *__restrict__ dL_dalpha, const uint8_t *__restrict__ layer,
    uint32_t grad_layer_mask, float4 *__restrict__ rec_grad, float *__restrict__ contrib_max, uint32_t n_rec,
    const Ctl *__restrict__ ctl) {
    __shared__ float4 s_a[kBwdThreads / 32][32], s_b[kBwdThreads / 32][32];
    __shared__ float s_c[kBwdThreads / 32][32];
    __shared__ uint32_t s_g[kBwdThreads / 32][32];
    __shared__ uint32_t s_pos[kBwdThreads / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int own = reduce10_owner(lane);
    const bool writer = reduce10_writer(lane);
    // per-lane factors of the value it holds after the reduce-scatter:
    //   du = -2 ln2 A2 S0, dv = -2 ln2 (A2 beta S0 + G2 S1), dA2 = ln2 S2, dbeta = 2 ln2 A2 S3, dG2 = ln2 S4
    const float cA = own == 0 ? -2.f * kLn2 : (own == 3 ? 2.f * kLn2 : 0.f);
    const float cB = own == 1 ? -2.f * kLn2 : 0.f;
    const float cC = (own == 2 || own == 4) ? kLn2 : (own >= 5 ? 1.f : 0.f);
    const uint32_t total = *n_items;
    const size_t plane = static_cast<size_t>(W) * H;
    for (;;) {
        uint32_t id = 0;
        if (lane == 0) id = atomicAdd(queue, 1u);
        id = __shfl_sync(FULL, id, 0);
        if (id >= total) break;
        const uint2 it = items[total - 1 - id];       // the forward appended the heaviest tiles' items last
        const int tile = static_cast<int>(it.x);
        const int q = static_cast<int>(it.y >> 24);
        const uint32_t seg = it.y & 0xFFFFFFu;
        const uint2 rg = ranges[tile];
        const uint32_t s0 = rg.x + seg * kSeg;
        // block of the item: PX = 2: 8x8 quadrant q of the tile; PX = 4: 16x8 half q
        constexpr int BW = PX == 2 ? 8 : 16;
        const int ox = PX == 2 ? (q & 1) * 8 : 0, oy = PX == 2 ? (q >> 1) * 8 : q * 8;
        const uint32_t qmax = PX == 2 ? qwork[4 * tile + q] : max(qwork[4 * tile + 2 * q], qwork[4 * tile + 2 * q + 1]);
        const uint32_t s1 = rg.x + min(min((seg + 1) * kSeg, qmax), rg.y - rg.x);
        const float4 *nck = ckpt + (static_cast<size_t>(seg_base[tile]) + seg + 1) * kTilePix;
        const float bx0 = (tile % Tx) * kTile + ox + 0.5f, by0 = (tile / Tx) * kTile + oy + 0.5f;
        float px[PX], py[PX], dC0[PX], dC1[PX], dC2[PX], R[PX], T[PX];
        uint32_t nc[PX];
#pragma unroll
        for (int j = 0; j < PX; ++j) {
            const int lx = ox + (lane % BW), ly = oy + (lane / BW) + (32 / BW) * j;
            const int x = (tile % Tx) * kTile + lx, y = (tile / Tx) * kTile + ly;
            px[j] = x + 0.5f;
            py[j] = y + 0.5f;
            nc[j] = 0;
            dC0[j] = dC1[j] = dC2[j] = R[j] = 0.f;
            T[j] = 1.f;
            if (x < W && y < H) {
                const size_t pix = static_cast<size_t>(y) * W + x;
                const uint32_t n = n_contrib[pix];
                if (n > seg * kSeg) {
                    nc[j] = n;
                    const float TN = t_final[pix];
                    float dA = 0.f;
                    if (dL_dimage) {
                        dC0[j] = dL_dimage[pix];
                        dC1[j] = dL_dimage[plane + pix];
                        dC2[j] = dL_dimage[2 * plane + pix];
                    }
                    if (dL_dalpha) dA = dL_dalpha[pix];
                    R[j] = TN * (dC0[j] * bg.x + dC1[j] * bg.y + dC2[j] * bg.z) - dA * TN;
                    T[j] = TN;
                    if (n > (seg + 1) * kSeg) {
                        const float4 ck = nck[ly * kTile + lx];
                        T[j] = ck.x;
                        R[j] += dC0[j] * ck.y + dC1[j] * ck.z + dC2[j] * ck.w;
                    }
                }
            }
        }
        const uint32_t nchunk = (s1 - s0 + 31) / 32;
        Chunk nxt;
        if (nchunk) fetch_chunk_layer(list, rec, layer, s0 + (nchunk - 1) * 32 + lane, s1, nxt, n_rec, ctl);
        // ids one chunk ahead of the records (the walk goes back to front; every chunk below the last is full)
        uint32_t gid = nchunk >= 2 ? list[s0 + (nchunk - 2) * 32 + lane] : 0u;
        for (uint32_t c = nchunk; c-- > 0;) {
            const uint32_t base = s0 + c * 32;
            const bool keep =
                base + lane < s1 && splat_reaches_block(nxt.a, nxt.b, bx0, bx0 + (BW - 1.f), by0, by0 + 7.f);
            const unsigned km = __ballot_sync(FULL, keep);
            __syncwarp();
            if (keep) {
                const int slot = __popc(km & lt);
                s_a[warp][slot] = nxt.a;
                s_b[warp][slot] = nxt.b;
                s_c[warp][slot] = nxt.c;
                s_g[warp][slot] = nxt.g | (((grad_layer_mask >> nxt.ly) & 1u) << 31);   // bit 31: trainable
                s_pos[warp][slot] = base + lane - rg.x;
            }
            __syncwarp();
            fetch_rec_layer(rec, layer, gid, c > 0, nxt, n_rec, ctl);
            if (c > 1) gid = list[base - 64 + lane];
            const int cnt = __popc(km);
            for (int k = cnt - 1; k >= 0; --k) {
                const uint32_t pos = s_pos[warp][k];
                const float4 a = s_a[warp][k], b = s_b[warp][k];
                const float cb = s_c[warp][k];
                float p[PX], dy[PX], ex[PX], ao[PX], al[PX];
                bool act[PX];
                bool any = false;
#pragma unroll
                for (int j = 0; j < PX; ++j) {
                    al[j] = splat_alpha(px[j], py[j], a, b, p[j], dy[j], ex[j], ao[j]);
                    act[j] = pos < nc[j] && al[j] >= kAlphaMin;
                    any |= act[j];
                }
                if (!__any_sync(FULL, any)) continue;
                // v: du, dv, dA2, dbeta, dG2, dopacity, dr, dg, db, sum of alpha*T
                float v[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float wmx = 0.f;
#pragma unroll
                for (int j = 0; j < PX; ++j) {
                    if (!act[j]) continue;
                    const float dcc = dC0[j] * b.z + dC1[j] * b.w + dC2[j] * cb;
                    const float inv = rcp_approx(__fsub_rn(1.f, al[j]));
                    const float Ti = T[j] * inv;
                    const float wgt = al[j] * Ti;
                    const float dLda = Ti * dcc - R[j] * inv;
                    R[j] = fmaf(wgt, dcc, R[j]);
                    T[j] = Ti;
                    v[6] += wgt * dC0[j];
                    v[7] += wgt * dC1[j];
                    v[8] += wgt * dC2[j];
                    if (ao[j] < kAlphaMax) {
                        // moments of dL/de' = dL/da alpha (e' = e ln 2 = ln(alpha / o)); the splat's
                        // constant factors are applied once to the warp sums (see below)
                        const float dLde = dLda * al[j];
                        const float tp = dLde * p[j], td = dLde * dy[j];
                        v[5] += dLda * ex[j];
                        v[0] += tp;
                        v[1] += td;
                        v[2] += tp * p[j];
                        v[3] += tp * dy[j];
                        v[4] += td * dy[j];
                    }
                    v[9] += wgt;
                    wmx = fmaxf(wmx, wgt);
                }
                const float sv0 = reduce_scatter10(v, lane);
                // sum of tp, for the lanes holding the sum of td (dv needs both)
                const float stp = __shfl_sync(FULL, sv0, lane & ~2);
                const float sv = sv0 * (cA * a.z + cC) + cB * (a.z * a.w * stp + b.x * sv0);
                const uint32_t smx = __reduce_max_sync(FULL, __float_as_uint(wmx));
                const uint32_t gt = s_g[warp][k];
                const uint32_t g = gt & 0x7FFFFFFFu;
                const bool train = gt >> 31;
                // value i is float 12 g + i of the record gradient: one atomic per value, one instruction
                if (writer && (train || own == 9))
                    atomicAdd(reinterpret_cast<float *>(rec_grad) + 12 * static_cast<size_t>(g) + own, sv);
                if (lane == 1 && contrib_max) atomicMax(reinterpret_cast<unsigned int *>(&contrib_max[g]), smx);
            }
        }
    }
}

// Blocks that fill every SM once for a persistent kernel (at most max_per
// blocks per SM).
template <class K>
int persistent_blocks(K kernel, int threads, int max_per = 1 << 30) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    return max(1, sms) * max(1, min(per, max_per));
}

// Forward CTAs per SM.  The frame's longest items (8x4 blocks of tiles whose
// walks run to thousands of list positions) start first and end last, and
// while their SM is crowded each gets only its warp's share of the issue
// slots.  Sixteen warps per SM still keep the SM issuing, and give those items
// twice the share that the 32 resident warps allowed: on the 1.2M-Gaussian
// frame the kernel took 0.19 ms instead of 0.22 (one block per SM: 0.27).
// A launch of many pixels has many more items per warp than its longest item
// is long, so the tail weighs less and a third CTA per SM pays: a 2064 x 2208
// view of 3M Gaussians took 0.606 ms instead of 0.666 (the 1.2M-Gaussian
// 1024 x 1024 frame 0.20 ms instead of 0.176, a 3M-Gaussian one 0.294 either
// way).  Batched serving launches keep two: they run beside the launches of a
// companion stream, and a third CTA per SM lowered the saturated served
// throughput from 7,530 to 7,270 Mpixels/s.
constexpr int kFwdBlocksPerSm = 2;
constexpr int kFwdBlocksPerSmWide = 3;
constexpr uint64_t kFwdWidePixels = 2u << 20;   // pixels of a launch from which it takes kFwdBlocksPerSmWide

}  // namespace

cudaError_t launch_fwd_setup(const CompositeBufs &cb, const uint2 *ranges, int Tn, cudaStream_t st) {
    if (Tn == 0) return cudaSuccess;
    static PerDevice attr;
    attr.get([] {
        cudaFuncSetAttribute(k_fwd_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, kSetupSmemTiles * 8);
        return 1;
    });
    const size_t smem = Tn <= kSetupSmemTiles ? static_cast<size_t>(Tn) * 8 : 0;
    k_fwd_setup<<<1, 1024, smem, st>>>(ranges, Tn, cb.order, cb.seg_base, cb.queue, cb.qdone);
    return cudaGetLastError();
}

cudaError_t launch_composite_forward(const FwdJob *jobs, int n, cudaStream_t st, bool wide_ok) {
    FwdBatch batch;
    batch.n = 0;
    uint32_t total = 0;
    uint64_t pixels = 0;
    for (int i = 0; i < n && batch.n < kMaxBatch; ++i) {
        if (jobs[i].Tn == 0) continue;
        batch.job[batch.n++] = jobs[i];
        total += static_cast<uint32_t>(jobs[i].Tn) * 8u;
        pixels += static_cast<uint64_t>(jobs[i].W) * jobs[i].H;
    }
    if (total == 0) return cudaSuccess;
    static PerDevice cache, cache_wide;
    const int blocks = wide_ok && pixels >= kFwdWidePixels
                           ? cache_wide.get([] {
                                 return persistent_blocks(k_composite_fwd, kFwdThreads, kFwdBlocksPerSmWide);
                             })
                           : cache.get([] { return persistent_blocks(k_composite_fwd, kFwdThreads, kFwdBlocksPerSm); });
    const int b = min(blocks, static_cast<int>((total + kFwdWarps - 1) / kFwdWarps));
    k_composite_fwd<<<b, kFwdThreads, 0, st>>>(batch);
    return cudaGetLastError();
}

cudaError_t launch_bwd_setup(const CompositeBufs &cb, int Tx, int Ty, float4 *rec_grad, const uint32_t *vis_index,
                             const uint32_t *n_vis, int n, cudaStream_t st) {
    if (Tx * Ty == 0) return cudaSuccess;
    static PerDevice cache;
    const int sms = cache.get([] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return max(1, v);
    });
    k_bwd_setup<<<sms, 1024, 0, st>>>(cb.queue, vis_index, n_vis, n, rec_grad);
    return cudaGetLastError();
}

cudaError_t launch_composite_backward(const CompositeBufs &cb, const uint2 *ranges, const uint32_t *list,
                                      const Rec *rec, int W, int H, int Tx, int Ty, float3 bg, const float *t_final,
                                      const uint32_t *n_contrib, const float *dL_dimage,
                                      const float *dL_dalpha, const uint8_t *layer, uint32_t grad_layer_mask,
                                      float4 *rec_grad, float *contrib_max, uint32_t n, const Ctl *ctl,
                                      cudaStream_t st) {
    if (Tx * Ty == 0) return cudaSuccess;
    static PerDevice cache;
    const int blocks = cache.get([] { return persistent_blocks(k_composite_bwd<kBwdPx>, kBwdThreads); });
    k_composite_bwd<kBwdPx><<<blocks, kBwdThreads, 0, st>>>(cb.items, cb.n_items, cb.queue, ranges, list, rec, W, H, Tx, bg,
                                                    t_final, n_contrib, cb.seg_base, cb.ckpt, cb.qwork,
                                                    dL_dimage, dL_dalpha, layer, grad_layer_mask, rec_grad,
                                                    contrib_max, n, ctl);
    return cudaGetLastError();
}

}  // namespace gs
