// S2 (second half) - tile binning by two stable bucket passes (Sec. 3.3: the
// splats of each tile are composited in camera-sorted order).
//
// Input: the visible Gaussians in depth order (order[p], p < n_vis, from the
// depth radix sort) and their tile rectangles.  Output: for every tile the
// Gaussians whose rectangle covers it, in depth order (ties by index, as the
// depth sort is stable), concatenated in tile order, and each tile's range.
// That is the stable sort of the (tile, Gaussian) pairs by tile, built
// without sorting the pairs:
//
//  1. Rows.  The (Gaussian, tile row) pairs, in depth order, are split into
//     one list per tile row.  K = gridDim.x * 8 warps each take a contiguous
//     chunk of the depth order; a first pass counts each chunk's entries per
//     row in shared memory, an exclusive scan over the chunks of every row
//     (row-major count matrices [Ty][K] of entries and of pairs) gives each chunk its place, and a
//     second pass writes the entries (Gaussian, x0 | x1 << 16) there.  Within
//     a chunk the entries go out in depth order: a warp expands 32 Gaussians
//     into their row pairs 32 at a time and ranks equal rows by lane
//     (__match_any_sync or ballots), and lanes hold consecutive pairs in depth order.
//  2. Tiles.  Every row list is cut into pieces of a fixed number of entries
//     (thousands of pieces per frame, so heavy rows spread over all SMs); a
//     warp per piece counts its pairs per tile, a per-row scan over the
//     pieces gives each (piece, tile) its first list position and each tile
//     its range, and a second pass writes the Gaussian ids, again ranked in
//     depth order within a warp.
//
// Per pair this writes the row entry once (8 B, per row of the rectangle, not
// per tile) and the final Gaussian id once (4 B); the count matrix is a few MB.
// Requires Tx, Ty <= kBinMaxDim (images up to 4096 x 4096).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Inclusive warp scan.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan over a block of NT threads (NT / 32 <= 32 warps).
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_w, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    const uint32_t x = warp_incl_scan(v, lane);
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_w[lane] : 0;
        w = warp_incl_scan(w, lane);
        if (lane < NW) s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? s_w[warp - 1] : 0;
    *total = s_w[NW - 1];
    __syncthreads();
    return base + x - v;
}

__device__ __forceinline__ uint32_t shfl_payload(uint32_t v, int j) { return __shfl_sync(FULL, v, j); }
__device__ __forceinline__ uint2 shfl_payload(uint2 v, int j) {
    return make_uint2(__shfl_sync(FULL, v.x, j), __shfl_sync(FULL, v.y, j));
}

// Lanes hold 32 consecutive list entries in order (the valid ones first),
// entry j covering slots [start_j, start_j + w_j) of the expanded sequence.
// Returns the entry that owns slot k0 + lane: entries starting before k0 plus
// those starting in [k0, k0 + lane], minus one.  Valid entries have w > 0.
__device__ __forceinline__ int window_owner(uint32_t start, uint32_t w, uint32_t k0, int lane) {
    const unsigned before = __ballot_sync(FULL, w > 0 && start < k0);
    const bool in = w > 0 && start >= k0 && start - k0 < 32u;
    const unsigned mask = __reduce_or_sync(FULL, in ? 1u << (start - k0) : 0u);
    return __popc(before) - 1 + __popc(mask & (0xFFFFFFFFu >> (31 - lane)));
}

// Lanes with equal keys of nb bits (among the active ones), from nb + 1 ballots.
__device__ __forceinline__ unsigned match_keyn(uint32_t key, bool act, int lane, int nb) {
    unsigned m = __ballot_sync(FULL, act);
#pragma unroll 8
    for (int b = 0; b < nb; ++b) {
        const unsigned bb = __ballot_sync(FULL, (key >> b) & 1u);
        m &= ((key >> b) & 1u) ? bb : ~bb;
    }
    return act ? m : (1u << lane);
}

// The 32 lanes hold consecutive list entries in order; entry j covers the
// buckets [b0_j, b0_j + n_j) (n_j = 0: no entry) and carries the payload v_j.
// The (bucket, payload) items are expanded in that order, 32 per window, and
// each is stored at its bucket's running position s_pos[bucket] (per-warp
// counters in shared memory), so every bucket receives its items in order:
// the lanes of a window that share a bucket are ranked by lane, and the first
// of them moves the counter.  Windows go in pairs whose rankings run on
// different pipes, __match_any_sync for the first and ballots on the nb key
// bits for the second; either alone saturates its pipe on large frames.
// store(pos, payload) writes one item.
template <class V, class Store>
__device__ __forceinline__ void expand_scatter(uint32_t b0, uint32_t n, V v, uint32_t *s_pos, int lane, int nb,
                                               Store store) {
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t incl = warp_incl_scan(n, lane);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t start = incl - n;
    for (uint32_t k0 = 0; k0 < total; k0 += 64) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint32_t kw = k0 + 32u * u;
            const uint32_t k = kw + lane;
            const bool act = k < total;
            const int j = window_owner(start, n, kw, lane);
            const uint32_t sj = __shfl_sync(FULL, start, j), bj = __shfl_sync(FULL, b0, j);
            const V vj = shfl_payload(v, j);
            const uint32_t bk = act ? bj + (k - sj) : 0u;
            // the two windows rank on different pipes: __match_any_sync and ballots
            const unsigned peers = u == 0 ? __match_any_sync(FULL, act ? bk : 0x10000u + lane)
                                          : match_keyn(bk, act, lane, nb);
            const uint32_t before = act ? s_pos[bk] : 0u;
            __syncwarp();
            if (act && (peers & lt) == 0) s_pos[bk] = before + __popc(peers);
            if (act) store(before + __popc(peers & lt), vj);
            __syncwarp();
        }
    }
}

// In-place inclusive prefix sum of a[0..n) (shared memory) by one warp.
__device__ __forceinline__ void warp_prefix_inplace(uint32_t *a, int n, int lane) {
    const int per = (n + 31) / 32;
    const int b = min(n, lane * per), e = min(n, b + per);
    uint32_t sum = 0;
    for (int i = b; i < e; ++i) sum += a[i];
    uint32_t run = warp_incl_scan(sum, lane) - sum;
    for (int i = b; i < e; ++i) {
        run += a[i];
        a[i] = run;
    }
    __syncwarp();
}

// The per-row scan of the row pass splits every row's kBinChunks chunk
// counts into kRowParts parts, one CTA each.
constexpr int kRowParts = 2;
constexpr int kPartChunks = kBinChunks / kRowParts;
static_assert(kPartChunks % 1024 == 0 && kPartChunks / 1024 <= kBinChunksPerThread, "row-scan part shape");

struct RowInfo {           // per tile row, in the workspace
    uint32_t start;        // first row-list entry of the row
    uint32_t entries;      // row-list entries of the row
    uint32_t pair_start;   // first pair (final list position) of the row
    uint32_t pairs;        // pairs of the row
    uint32_t piece_start;  // first piece of the row (pieces: kPiece-entry parts of row lists)
    uint32_t part_base[kRowParts - 1];   // entries of the row in the chunk parts before parts 1 ..
    uint32_t pad_[4 - kRowParts];        // (32 bytes in all)
};

// Pass 1 (SCATTER = false: count, true: write) over the chunks of the depth order.
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_bin_rows(const uint32_t *__restrict__ order, const Rec *__restrict__ rec,
                                                  uint32_t n_cap, int Ty, uint32_t *__restrict__ M,
                                                  RowInfo *__restrict__ rows, uint2 *__restrict__ rowlist,
                                                  const Ctl *__restrict__ ctl) {
    __shared__ uint32_t s_cnt[8][kBinMaxDim + 1];
    __shared__ uint32_t s_px[SCATTER ? 1 : 8][kBinMaxDim + 1];
    // an error before the binning (a depth sort that timed out) leaves the order unfinished: do not read it
    if (ctl->st.error != GS_OK) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t K = gridDim.x * 8u, c = blockIdx.x * 8u + warp;
    const uint32_t n = min(ctl->n_vis, n_cap);
    const uint32_t b = static_cast<uint32_t>(static_cast<uint64_t>(n) * c / K);
    const uint32_t e = static_cast<uint32_t>(static_cast<uint64_t>(n) * (c + 1) / K);
    // the block's 8 chunks are 8 consecutive columns of the row-major count
    // matrix: thread t moves (row t / 8, column t % 8), so every row segment
    // is one 32-byte transaction
    for (int t = threadIdx.x; t < 8 * (Ty + 1); t += blockDim.x) {
        const int r = t >> 3, w = t & 7;
        const uint32_t ch = blockIdx.x * 8u + w, part = ch / (K / kRowParts);
        s_cnt[w][r] = (SCATTER && r < Ty)
                          ? rows[r].start + (part ? rows[r].part_base[part - 1] : 0u) + M[static_cast<size_t>(r) * K + ch]
                          : 0u;
        if (!SCATTER) s_px[w][r] = 0;
    }
    __syncthreads();
    // ids two groups ahead and records one group ahead of the group being binned, so the gathers overlap
    // the binning of the groups before them
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t g_nx = b + lane < e ? order[b + lane] : 0u;
    float4 c_nx = b + lane < e ? rec[g_nx].c : z4;
    uint32_t gid = b + 32 + lane < e ? order[b + 32 + lane] : 0u;
    for (uint32_t p0 = b; p0 < e; p0 += 32) {
        const bool valid = p0 + lane < e;
        const uint32_t g = g_nx;
        const float4 cc = c_nx;
        g_nx = gid;
        c_nx = p0 + 32 + lane < e ? rec[g_nx].c : z4;
        gid = p0 + 64 + lane < e ? order[p0 + 64 + lane] : 0u;
        uint32_t y0 = 0, x01 = 0, nrows = 0;
        if (valid) {
            const uint32_t r0 = __float_as_uint(cc.z), r1 = __float_as_uint(cc.w);
            y0 = r0 >> 16;
            nrows = (r1 >> 16) - y0;
            x01 = (r0 & 0xFFFFu) | (r1 << 16);     // x0 | x1 << 16
        }
        if (!SCATTER) {
            // rows [y0, y0 + nrows) each get one entry and w pairs: difference array
            if (nrows) {
                const uint32_t w = (x01 >> 16) - (x01 & 0xFFFFu);
                atomicAdd(&s_cnt[warp][y0], 1u);
                atomicSub(&s_cnt[warp][y0 + nrows], 1u);
                atomicAdd(&s_px[warp][y0], w);
                atomicSub(&s_px[warp][y0 + nrows], w);
            }
            continue;
        }
        expand_scatter(y0, nrows, make_uint2(g, x01), s_cnt[warp], lane, 32 - __clz(max(Ty - 1, 1)), [&](uint32_t pos, uint2 en) {
            if (GS_CHECK(pos < ctl->st.dup_capacity, ctl, kSiteRowList)) rowlist[pos] = en;
        });
    }
    if (!SCATTER) {
        __syncwarp();
        warp_prefix_inplace(s_cnt[warp], Ty, lane);
        warp_prefix_inplace(s_px[warp], Ty, lane);
        __syncthreads();
        // entries and pairs per (row, chunk), written as 32-byte row segments; the
        // pairs matrix follows the entries matrix and is summed per row by the scan
        for (int t = threadIdx.x; t < 8 * Ty; t += blockDim.x) {
            const int r = t >> 3, w = t & 7;
            const size_t at = static_cast<size_t>(r) * K + blockIdx.x * 8u + w;
            M[at] = s_cnt[w][r];
            M[static_cast<size_t>(Ty) * K + at] = s_px[w][r];
        }
    }
}

// Per (row, part) (one CTA each, kRowParts parts of K / kRowParts chunks per
// row): exclusive scan of the part's chunk counts in place, and the part's
// entry and pair totals.  The part moves through shared memory with
// coalesced loads and stores (each thread scans a contiguous run of counts);
// the pair total needs only a sum, read coalesced.  The last CTA to finish
// (a counter in the control block) then does the per-row work for the whole
// frame: part bases, row totals, the row, pair and piece starts, the pair
// total and the capacity check.
__global__ void __launch_bounds__(1024) k_bin_rowscan(uint32_t *__restrict__ M, int K, int Ty,
                                                      RowInfo *__restrict__ rows, uint2 *__restrict__ part_tot,
                                                      Ctl *__restrict__ ctl, uint64_t cap, uint32_t piece) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_row[kPartChunks];
    __shared__ bool s_last;
    if (ctl->st.error != GS_OK) return;      // uniform: an error set before this kernel (a sort that timed out)
    const int r = blockIdx.x / kRowParts, part = blockIdx.x % kRowParts;
    const int KP = K / kRowParts;
    uint32_t *row = M + static_cast<size_t>(r) * K + static_cast<size_t>(part) * KP;
    const uint32_t *prow = M + static_cast<size_t>(Ty + r) * K + static_cast<size_t>(part) * KP;   // pairs
    uint32_t psum = 0;
    for (int i = threadIdx.x; i < KP; i += 1024) {
        s_row[i] = row[i];
        psum += prow[i];
    }
    uint32_t ptot;
    block_excl_scan<1024>(psum, s_w, &ptot);             // synchronises the block, so s_row is complete
    const int per = KP / 1024;
    uint32_t v[kBinChunksPerThread];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kBinChunksPerThread; ++q) {
        v[q] = q < per ? s_row[threadIdx.x * per + q] : 0u;
        sum += v[q];
    }
    uint32_t tot;
    uint32_t run = block_excl_scan<1024>(sum, s_w, &tot);
#pragma unroll
    for (int q = 0; q < kBinChunksPerThread; ++q) {
        if (q < per) s_row[threadIdx.x * per + q] = run;
        run += v[q];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < KP; i += 1024) row[i] = s_row[i];
    if (threadIdx.x == 0) {
        part_tot[blockIdx.x] = make_uint2(tot, ptot);
        __threadfence();
        s_last = atomicAdd(&ctl->bin_scan_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last CTA: per row (thread r < Ty <= 256) the part bases and totals, then the starts
    const volatile uint2 *pt = part_tot;
    uint32_t ent = 0, prs = 0;
    if (threadIdx.x < Ty) {
        for (int p = 0; p < kRowParts; ++p) {
            const uint32_t e = pt[threadIdx.x * kRowParts + p].x;
            if (p > 0) rows[threadIdx.x].part_base[p - 1] = ent;
            ent += e;
            prs += pt[threadIdx.x * kRowParts + p].y;
        }
        rows[threadIdx.x].entries = ent;
        rows[threadIdx.x].pairs = prs;
    }
    uint32_t te, tp, tq;
    const bool in = threadIdx.x < Ty;
    const uint32_t s0 = block_excl_scan<1024>(in ? ent : 0u, s_w, &te);
    const uint32_t s1 = block_excl_scan<1024>(in ? prs : 0u, s_w, &tp);
    const uint32_t s2 = block_excl_scan<1024>(in ? (ent + piece - 1) / piece : 0u, s_w, &tq);
    if (in) {
        rows[threadIdx.x].start = s0;
        rows[threadIdx.x].pair_start = s1;
        rows[threadIdx.x].piece_start = s2;
    }
    if (threadIdx.x == 0) {
        ctl->st.n_dup = tp;
        ctl->st.dup_capacity = cap;
        ctl->n_pieces = tq;
        if (tp > cap) ctl->st.error = GS_ERR_WORKSPACE;
    }
}

// Pass 2 (SCATTER = false: count, true: write), one warp per piece of a row
// list.  Count: per-(piece, tile) counts into P[piece][Tx].  Write: P holds
// the first list position of every (piece, tile) (k_bin_tiles_scan).
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_bin_tiles(const uint2 *__restrict__ rowlist, const RowInfo *__restrict__ rows,
                                                   int Tx, int Ty, uint32_t piece, uint32_t *__restrict__ P,
                                                   uint32_t *__restrict__ list, const Ctl *__restrict__ ctl) {
    __shared__ uint32_t s_cnt[8][kBinMaxDim + 1];
    __shared__ uint32_t s_ps[kBinMaxDim + 1];
    if (ctl->st.error != GS_OK) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t npieces = ctl->n_pieces;
    for (int r = threadIdx.x; r < Ty; r += blockDim.x) s_ps[r] = rows[r].piece_start;
    if (threadIdx.x == 0) s_ps[Ty] = npieces;
    __syncthreads();
    const uint32_t nwarps = gridDim.x * 8u;
    for (uint32_t p = blockIdx.x * 8u + warp; p < npieces; p += nwarps) {
        int lo = 0, hi = Ty - 1;                 // largest row r with s_ps[r] <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_ps[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const RowInfo ri = rows[lo];
        const uint32_t e0 = ri.start + (p - s_ps[lo]) * piece;
        const uint32_t e1 = min(e0 + piece, ri.start + ri.entries);
        uint32_t *Pp = P + static_cast<size_t>(p) * Tx;
        for (int t = lane; t <= Tx; t += 32) s_cnt[warp][t] = (SCATTER && t < Tx) ? Pp[t] : 0u;
        __syncwarp();
        uint2 en_nx = e0 + lane < e1 ? rowlist[e0 + lane] : make_uint2(0u, 0u);   // entries one group ahead
        for (uint32_t q0 = e0; q0 < e1; q0 += 32) {
            const uint2 en = en_nx;
            en_nx = q0 + 32 + lane < e1 ? rowlist[q0 + 32 + lane] : make_uint2(0u, 0u);
            uint32_t g = 0, x0 = 0, w = 0;
            if (q0 + lane < e1) {
                g = en.x;
                x0 = en.y & 0xFFFFu;
                w = (en.y >> 16) - x0;
            }
            if (!SCATTER) {
                // tiles [x0, x0 + w) each get one pair: difference array
                if (w) {
                    atomicAdd(&s_cnt[warp][x0], 1u);
                    atomicSub(&s_cnt[warp][x0 + w], 1u);
                }
                continue;
            }
            expand_scatter(x0, w, g, s_cnt[warp], lane, 32 - __clz(max(Tx - 1, 1)), [&](uint32_t pos, uint32_t id) {
                if (GS_CHECK(pos < ctl->st.n_dup, ctl, kSitePairList)) list[pos] = id;
            });
        }
        if (!SCATTER) {
            __syncwarp();
            warp_prefix_inplace(s_cnt[warp], Tx, lane);
            for (int t = lane; t < Tx; t += 32) Pp[t] = s_cnt[warp][t];
        }
        __syncwarp();
    }
}

// Per row (one CTA of 1024 threads): the threads form S slices of TW tiles
// (TW the power of two at or above Tx, at least 16, so S = 1024 / TW <= 64);
// thread (slice s, tile t) sums the counts of tile t over its share of the
// row's pieces; the slice sums give each tile's total and range; then every
// (piece, tile) count is replaced by its first list position.
__global__ void __launch_bounds__(1024) k_bin_tiles_scan(const RowInfo *__restrict__ rows, int Tx, uint32_t piece,
                                                         uint32_t *__restrict__ P, uint2 *__restrict__ ranges,
                                                         const Ctl *__restrict__ ctl) {
    __shared__ uint32_t s_sum[1024];         // [slice][tile]
    __shared__ uint32_t s_off[kBinMaxDim];
    __shared__ uint32_t s_w[32];
    if (ctl->st.error != GS_OK) return;
    int TW = 16;
    while (TW < Tx) TW <<= 1;
    const int S = 1024 / TW;
    const int r = blockIdx.x;
    const int t = threadIdx.x & (TW - 1), sl = threadIdx.x / TW;
    const RowInfo ri = rows[r];
    const uint32_t npc = (ri.entries + piece - 1) / piece;
    const uint32_t per = (npc + S - 1) / S;
    const uint32_t p0 = ri.piece_start + min(npc, sl * per), p1 = ri.piece_start + min(npc, (sl + 1) * per);
    uint32_t sum = 0;
    if (t < Tx)
        for (uint32_t p = p0; p < p1; ++p) sum += P[static_cast<size_t>(p) * Tx + t];
    s_sum[sl * TW + t] = sum;
    __syncthreads();
    uint32_t tot = 0, before = 0;
    if (t < Tx)
        for (int q = 0; q < S; ++q) {
            const uint32_t v = s_sum[q * TW + t];
            if (q < sl) before += v;
            tot += v;
        }
    uint32_t all;
    const uint32_t toff = block_excl_scan<1024>(sl == 0 && t < Tx ? tot : 0u, s_w, &all);
    if (sl == 0 && t < Tx) s_off[t] = toff;   // tile offsets within the row, read by every slice below
    __syncthreads();
    if (t < Tx) {
        const uint32_t base = ri.pair_start + s_off[t];
        if (sl == 0 && GS_CHECK(base + tot <= ctl->st.n_dup, ctl, kSiteRange))
            ranges[static_cast<size_t>(r) * Tx + t] = make_uint2(base, base + tot);
        uint32_t run = base + before;
        // eight counts loaded before any of them is replaced, so the loads overlap instead of each waiting
        // behind the previous store
        constexpr int kB = 8;
        for (uint32_t p = p0; p < p1; p += kB) {
            uint32_t v[kB];
#pragma unroll
            for (int k = 0; k < kB; ++k) v[k] = p + k < p1 ? P[static_cast<size_t>(p + k) * Tx + t] : 0u;
#pragma unroll
            for (int k = 0; k < kB; ++k) {
                if (p + k < p1) P[static_cast<size_t>(p + k) * Tx + t] = run;
                run += v[k];
            }
        }
    }
}

}  // namespace

cudaError_t launch_bin_rows(const uint32_t *order, const Rec *rec, uint32_t n_cap, int Ty, uint32_t *M,
                            void *rows_buf, uint2 *rowlist, Ctl *ctl, uint64_t cap, uint32_t piece, cudaStream_t st) {
    if (Ty > kBinMaxDim) return cudaErrorInvalidValue;
    RowInfo *rows = static_cast<RowInfo *>(rows_buf);   // zero on entry (cleared with the control block)
    uint2 *part_tot = reinterpret_cast<uint2 *>(static_cast<char *>(rows_buf) + bin_rows_bytes(Ty) -
                                                 static_cast<size_t>(Ty) * kRowParts * sizeof(uint2));
    k_bin_rows<false><<<kBinBlocks, 256, 0, st>>>(order, rec, n_cap, Ty, M, rows, rowlist, ctl);
    k_bin_rowscan<<<Ty * kRowParts, 1024, 0, st>>>(M, kBinBlocks * 8, Ty, rows, part_tot, ctl, cap, piece);
    k_bin_rows<true><<<kBinBlocks, 256, 0, st>>>(order, rec, n_cap, Ty, M, rows, rowlist, ctl);
    return cudaGetLastError();
}

cudaError_t launch_bin_tiles(const uint2 *rowlist, const void *rows_buf, int Tx, int Ty, uint32_t piece, uint32_t *P,
                             uint32_t *list, uint2 *ranges, const Ctl *ctl, cudaStream_t st) {
    if (Tx > kBinMaxDim || Ty > kBinMaxDim) return cudaErrorInvalidValue;
    const RowInfo *rows = static_cast<const RowInfo *>(rows_buf);
    const int G = 4 * sort_blocks();
    k_bin_tiles<false><<<G, 256, 0, st>>>(rowlist, rows, Tx, Ty, piece, P, list, ctl);
    k_bin_tiles_scan<<<Ty, 1024, 0, st>>>(rows, Tx, piece, P, ranges, ctl);
    k_bin_tiles<true><<<G, 256, 0, st>>>(rowlist, rows, Tx, Ty, piece, P, list, ctl);
    return cudaGetLastError();
}

uint32_t bin_piece_entries(int64_t dup_cap, int Tx) {
    // Pieces of 256 entries at every size: measured against 128, 512 and 1024 on the 1.2M-Gaussian 1024 x 1024
    // frame and on 3M-Gaussian views of 1024 x 1024 and 2064 x 2208 (40M and 123M pairs), 256 was fastest or
    // within 1% of it.  (Growing the pieces with the capacity, to keep the count matrix near 64 MB, made the pieces
    // of the 2064 x 2208 view 2048 entries long and its tile pass 1.3 times slower.)  The count matrix then takes
    // at most 4 B per pair of capacity.
    (void)dup_cap;
    (void)Tx;
    return 256u;
}

size_t bin_piece_bytes(int64_t dup_cap, int Tx, int Ty) {
    // A row list of E entries has ceil(E / piece) pieces and the row lists hold at most dup_cap entries, so
    // dup_cap / piece + Ty rows of counts always suffice; the size grows with the capacity.
    const uint32_t piece = bin_piece_entries(dup_cap, Tx);
    return (static_cast<size_t>(dup_cap) / piece + Ty + 1) * Tx * 4;
}

// The RowInfo of every row, then the (entries, pairs) totals of every (row, part) of the row scan.
size_t bin_rows_bytes(int Ty) {
    return static_cast<size_t>(Ty) * sizeof(RowInfo) + static_cast<size_t>(Ty) * kRowParts * sizeof(uint2);
}
static_assert(sizeof(RowInfo) == 32, "RowInfo layout");

}  // namespace gs
