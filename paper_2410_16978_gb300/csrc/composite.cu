// S3 / S4a - front-to-back compositing of each 16x16 tile over its sorted
// splat list (Sec. 3.3: Gaussians rendered as splats in camera-sorted order),
// and its exact backward with the per-Gaussian blend weight alpha*T that
// drives contribution pruning (Sec. 3.2.2).
//
// Work layout: one CTA per tile.  Every warp walks the tile's list on its own
// (no CTA-wide barriers, so a warp whose pixels are done leaves at once): the
// forward warp owns an 8x4 pixel block (one pixel per lane), the backward warp
// an 8x8 block (two pixels per lane, which halves the cost of reducing each
// splat's gradient over the warp).  Tiles are launched heaviest first
// (k_tile_order) so that the long lists do not end up in the last wave.  Compositing is FP32 FMA + MUFU work, not a
// dense contraction, so no tensor cores are involved.
//
// splat_alpha() is the single definition of the per-(pixel, splat) alpha used
// by both passes; every operation is an explicitly rounded intrinsic, so the
// backward reproduces the forward's skip decisions and transmittance bit for
// bit.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr float kLn2 = 0x1.62e430p-1f;
constexpr int kThreads = 128;

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

// Pixel of lane `lane` of warp `warp`, j-th of its two pixels.
__device__ __forceinline__ void pixel_of(int tile, int Tx, int warp, int lane, int j, int &x, int &y) {
    x = (tile % Tx) * kTile + (warp & 1) * 8 + (lane & 7);
    y = (tile / Tx) * kTile + (warp >> 1) * 8 + (lane >> 3) + 4 * j;
}

// Heaviest-first launch order of the tiles: a one-CTA counting sort of the
// tiles by a logarithmic bucket of their work (list length, or the longest
// blended prefix for the backward).  Ties keep no particular order; tiles are
// independent, so the order changes no result.
__global__ void __launch_bounds__(1024) k_tile_order(const uint2 *__restrict__ ranges,
                                                     const uint32_t *__restrict__ work, int Tn,
                                                     uint32_t *__restrict__ order) {
    constexpr int kBuckets = 513;
    __shared__ uint32_t s_cnt[kBuckets];
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    auto bucket = [&](int t) -> int {
        const uint32_t w = work ? work[t] : ranges[t].y - ranges[t].x;
        if (w == 0) return kBuckets - 1;                      // empty tiles last
        const int lz = 31 - __clz(w);
        const uint32_t sub = lz >= 4 ? (w >> (lz - 4)) & 15u : (w << (4 - lz)) & 15u;
        return (kBuckets - 2) - (lz * 16 + static_cast<int>(sub));   // heavier -> smaller bucket
    };
    for (int t = threadIdx.x; t < Tn; t += blockDim.x) atomicAdd(&s_cnt[bucket(t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < kBuckets; ++b) {
            const uint32_t c = s_cnt[b];
            s_cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Tn; t += blockDim.x) order[atomicAdd(&s_cnt[bucket(t)], 1u)] = t;
}

// Each warp walks the tile's list on its own (no CTA barriers): it stages 32
// records at a time in a warp-private shared buffer while the next 32 are
// already in flight in registers, and stops once all 64 of its pixels are done.
struct Chunk {
    float4 a, b;
    float c;
    uint32_t g;
};

__device__ __forceinline__ void fetch_chunk(const uint32_t *__restrict__ list, const Rec *__restrict__ rec,
                                            uint32_t pos, uint32_t end, Chunk &ch) {
    if (pos < end) {
        ch.g = list[pos];
        const Rec *r = rec + ch.g;
        ch.a = r->a;
        ch.b = r->b;
        ch.c = r->c.x;
    }
}

constexpr int kFwdThreads = 256;

// Forward: 256 threads per tile, one pixel per lane; warp w owns the 8x4 block
// ((w & 1) * 8, (w >> 1) * 4) and walks the list until its 32 pixels are done.
__global__ void __launch_bounds__(kFwdThreads) k_composite_fwd(const uint32_t *__restrict__ order,
                                                               const uint2 *__restrict__ ranges,
                                                               const uint32_t *__restrict__ list,
                                                               const Rec *__restrict__ rec, int W, int H, int Tx,
                                                               float3 bg, float *__restrict__ image,
                                                               float *__restrict__ alpha_out, float *__restrict__ t_final,
                                                               uint32_t *__restrict__ n_contrib, float *__restrict__ c_sum,
                                                               uint32_t *__restrict__ tile_work) {
    __shared__ float4 s_a[kFwdThreads / 32][32], s_b[kFwdThreads / 32][32];
    __shared__ float s_c[kFwdThreads / 32][32];
    __shared__ uint32_t s_wmax[kFwdThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = order[blockIdx.x];
    const uint2 rg = ranges[tile];
    const int x = (tile % Tx) * kTile + (warp & 1) * 8 + (lane & 7);
    const int y = (tile / Tx) * kTile + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = x < W && y < H;
    const float px = x + 0.5f, py = y + 0.5f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    Chunk nxt;
    fetch_chunk(list, rec, rg.x + lane, rg.y, nxt);
    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        if (__all_sync(FULL, done)) break;
        __syncwarp();
        s_a[warp][lane] = nxt.a;
        s_b[warp][lane] = nxt.b;
        s_c[warp][lane] = nxt.c;
        __syncwarp();
        fetch_chunk(list, rec, base + 32 + lane, rg.y, nxt);
        const int cnt = min(32u, rg.y - base);
        for (int k = 0; k < cnt && !done; ++k) {
            const float4 a = s_a[warp][k], b = s_b[warp][k];
            float p, dy, ex, ao;
            const float al = splat_alpha(px, py, a, b, p, dy, ex, ao);
            if (al < kAlphaMin) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
            if (Tn < kTMin) { done = true; break; }
            const float w = __fmul_rn(al, T);
            C0 = __fmaf_rn(b.z, w, C0);
            C1 = __fmaf_rn(b.w, w, C1);
            C2 = __fmaf_rn(s_c[warp][k], w, C2);
            T = Tn;
            last = base + k - rg.x + 1;
        }
    }
    if (inside) {
        const size_t plane = static_cast<size_t>(W) * H;
        const size_t pix = static_cast<size_t>(y) * W + x;
        image[pix] = __fmaf_rn(T, bg.x, C0);
        image[plane + pix] = __fmaf_rn(T, bg.y, C1);
        image[2 * plane + pix] = __fmaf_rn(T, bg.z, C2);
        if (alpha_out) alpha_out[pix] = 1.f - T;
        t_final[pix] = T;
        n_contrib[pix] = last;
        c_sum[pix] = C0;
        c_sum[plane + pix] = C1;
        c_sum[2 * plane + pix] = C2;
    }
    const uint32_t wm = __reduce_max_sync(FULL, last);
    if (lane == 0) s_wmax[warp] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t m = 0;
#pragma unroll
        for (int w = 0; w < kFwdThreads / 32; ++w) m = max(m, s_wmax[w]);
        tile_work[tile] = m;
    }
}

// Reduce-scatter of 16 values across a warp: at step o (16, 8, 4, 2) each
// lane keeps the half of its values selected by bit o of its lane id and adds
// its partner's copy of that half; a last exchange at 1 completes the sums.
// Afterwards lanes 2i and 2i+1 hold the warp sum of value i.
__device__ __forceinline__ float reduce_scatter16(float v[16], int lane) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const int o = 2 * h;                    // xor distance 16, 8, 4, 2
        const bool hi = lane & o;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            const float send = hi ? v[q] : v[q + h];
            const float recv = __shfl_xor_sync(FULL, send, o);
            v[q] = (hi ? v[q + h] : v[q]) + recv;
        }
    }
    return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}

// Backward, front to back.  With S_i = sum_{j>i} c_j a_j T_j + T_N bg:
//   dL/da_i = dC.(c_i T_i - S_i/(1-a_i)) + dA T_N/(1-a_i)
//           = T_i (dC.c_i) - (dC.(Csum - P_i) + T_N (dC.bg) - dA T_N)/(1-a_i)
// where P_i is the running colour sum including splat i; dC.P_i is carried as
// the scalar Q.  Each warp walks the list only up to the longest blended
// prefix of its own 64 pixels, reduces each splat's 10 sums over its pixels
// and adds them to the record gradient with vector atomics:
//   rec_grad[3g]   += (du, dv, dA2, dbeta)
//   rec_grad[3g+1] += (dG2, dopacity, dr, dg)
//   rec_grad[3g+2] += (db, sum of alpha*T, 0, 0);  contrib_max[g] = max(.., alpha*T)
__global__ void __launch_bounds__(kThreads) k_composite_bwd(
    const uint32_t *__restrict__ order, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ list,
    const Rec *__restrict__ rec, int W, int H, int Tx, float3 bg, const float *__restrict__ t_final,
    const uint32_t *__restrict__ n_contrib, const float *__restrict__ c_sum, const float *__restrict__ dL_dimage,
    const float *__restrict__ dL_dalpha, const uint8_t *__restrict__ layer, uint32_t grad_layer_mask,
    float4 *__restrict__ rec_grad, float *__restrict__ contrib_max) {
    __shared__ float4 s_a[kThreads / 32][32], s_b[kThreads / 32][32];
    __shared__ float s_c[kThreads / 32][32];
    __shared__ uint32_t s_g[kThreads / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = order[blockIdx.x];
    const uint2 rg = ranges[tile];
    const size_t plane = static_cast<size_t>(W) * H;
    float px[2], py[2], TN[2], dC0[2], dC1[2], dC2[2], QC[2], K0[2], T[2], Q[2];
    uint32_t nc[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        int x, y;
        pixel_of(tile, Tx, warp, lane, j, x, y);
        px[j] = x + 0.5f;
        py[j] = y + 0.5f;
        nc[j] = 0;
        TN[j] = 1.f;
        dC0[j] = dC1[j] = dC2[j] = QC[j] = 0.f;
        float dA = 0.f;
        if (x < W && y < H) {
            const size_t pix = static_cast<size_t>(y) * W + x;
            nc[j] = n_contrib[pix];
            TN[j] = t_final[pix];
            if (dL_dimage) {
                dC0[j] = dL_dimage[pix];
                dC1[j] = dL_dimage[plane + pix];
                dC2[j] = dL_dimage[2 * plane + pix];
            }
            if (dL_dalpha) dA = dL_dalpha[pix];
            QC[j] = dC0[j] * c_sum[pix] + dC1[j] * c_sum[plane + pix] + dC2[j] * c_sum[2 * plane + pix];
        }
        K0[j] = TN[j] * (dC0[j] * bg.x + dC1[j] * bg.y + dC2[j] * bg.z) - dA * TN[j];
        T[j] = 1.f;
        Q[j] = 0.f;
    }
    const uint32_t wbound = __reduce_max_sync(FULL, max(nc[0], nc[1]));
    const uint32_t stop = rg.x + min(wbound, rg.y - rg.x);
    Chunk nxt;
    fetch_chunk(list, rec, rg.x + lane, stop, nxt);
    for (uint32_t base = rg.x; base < stop; base += 32) {
        __syncwarp();
        s_a[warp][lane] = nxt.a;
        s_b[warp][lane] = nxt.b;
        s_c[warp][lane] = nxt.c;
        s_g[warp][lane] = nxt.g;
        __syncwarp();
        fetch_chunk(list, rec, base + 32 + lane, stop, nxt);
        const int cnt = min(32u, stop - base);
        for (int k = 0; k < cnt; ++k) {
            const uint32_t pos = base + k - rg.x;
            const float4 a = s_a[warp][k], b = s_b[warp][k];
            const float cb = s_c[warp][k];
            float p[2], dy[2], ex[2], ao[2], al[2];
            al[0] = splat_alpha(px[0], py[0], a, b, p[0], dy[0], ex[0], ao[0]);
            al[1] = splat_alpha(px[1], py[1], a, b, p[1], dy[1], ex[1], ao[1]);
            bool act[2];
            act[0] = pos < nc[0] && al[0] >= kAlphaMin;
            act[1] = pos < nc[1] && al[1] >= kAlphaMin;
            if (!__any_sync(FULL, act[0] || act[1])) continue;
            // v: du, dv, dA2, dbeta, dG2, dopacity, dr, dg, db, sum of alpha*T (10..15 unused)
            float v[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float wmx = 0.f;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (!act[j]) continue;
                const float dcc = dC0[j] * b.z + dC1[j] * b.w + dC2[j] * cb;
                const float wgt = __fmul_rn(al[j], T[j]);
                Q[j] = fmaf(wgt, dcc, Q[j]);
                const float inv = __frcp_rn(1.f - al[j]);
                const float dLda = T[j] * dcc - ((QC[j] - Q[j]) + K0[j]) * inv;
                v[6] += wgt * dC0[j];
                v[7] += wgt * dC1[j];
                v[8] += wgt * dC2[j];
                if (ao[j] < kAlphaMax) {
                    const float dLde = dLda * al[j] * kLn2;
                    const float A2p = a.z * p[j];
                    v[5] += dLda * ex[j];
                    v[2] += dLde * p[j] * p[j];
                    v[3] += dLde * 2.f * A2p * dy[j];
                    v[4] += dLde * dy[j] * dy[j];
                    v[0] -= dLde * 2.f * A2p;
                    v[1] -= dLde * (2.f * A2p * a.w + 2.f * b.x * dy[j]);
                }
                v[9] += wgt;
                wmx = fmaxf(wmx, wgt);
                T[j] = __fmul_rn(T[j], __fsub_rn(1.f, al[j]));
            }
            const float sv = reduce_scatter16(v, lane);
            // value i sits in lane 2i: lanes 0, 8, 16 gather (i, i+1, i+2, i+3)
            const float s1 = __shfl_down_sync(FULL, sv, 2);
            const float s2 = __shfl_down_sync(FULL, sv, 4);
            const float s3 = __shfl_down_sync(FULL, sv, 6);
            const uint32_t smx = __reduce_max_sync(FULL, __float_as_uint(wmx));
            const uint32_t g = s_g[warp][k];
            const bool train = (grad_layer_mask >> layer[g]) & 1u;
            if (lane == 0 && train) atomicAdd(&rec_grad[3 * g], make_float4(sv, s1, s2, s3));
            if (lane == 8 && train) atomicAdd(&rec_grad[3 * g + 1], make_float4(sv, s1, s2, s3));
            if (lane == 16) atomicAdd(reinterpret_cast<float2 *>(&rec_grad[3 * g + 2]), make_float2(train ? sv : 0.f, s1));
            if (lane == 1 && contrib_max) atomicMax(reinterpret_cast<unsigned int *>(&contrib_max[g]), smx);
        }
    }
}

}  // namespace

cudaError_t launch_tile_order(const uint2 *ranges, const uint32_t *work, int Tn, uint32_t *order, cudaStream_t st) {
    if (Tn == 0) return cudaSuccess;
    k_tile_order<<<1, 1024, 0, st>>>(ranges, work, Tn, order);
    return cudaGetLastError();
}

cudaError_t launch_composite_forward(const uint32_t *order, const uint2 *ranges, const uint32_t *list, const Rec *rec,
                                     int W, int H, int Tx, int Ty, float3 bg, float *image, float *alpha,
                                     float *t_final, uint32_t *n_contrib, float *c_sum, uint32_t *tile_work,
                                     cudaStream_t st) {
    const int tiles = Tx * Ty;
    if (tiles == 0) return cudaSuccess;
    k_composite_fwd<<<tiles, kFwdThreads, 0, st>>>(order, ranges, list, rec, W, H, Tx, bg, image, alpha, t_final,
                                                   n_contrib, c_sum, tile_work);
    return cudaGetLastError();
}

cudaError_t launch_composite_backward(const uint32_t *order, const uint2 *ranges, const uint32_t *list, const Rec *rec,
                                      int W, int H, int Tx, int Ty, float3 bg, const float *t_final,
                                      const uint32_t *n_contrib, const float *c_sum, const float *dL_dimage,
                                      const float *dL_dalpha, const uint8_t *layer, uint32_t grad_layer_mask,
                                      float4 *rec_grad, float *contrib_max, cudaStream_t st) {
    const int tiles = Tx * Ty;
    if (tiles == 0) return cudaSuccess;
    k_composite_bwd<<<tiles, kThreads, 0, st>>>(order, ranges, list, rec, W, H, Tx, bg, t_final, n_contrib, c_sum,
                                                dL_dimage, dL_dalpha, layer, grad_layer_mask, rec_grad, contrib_max);
    return cudaGetLastError();
}

}  // namespace gs
