// S3 / S4a - front-to-back compositing of each 16x16 tile over its sorted
// splat list (Sec. 3.3: Gaussians rendered as splats in camera-sorted order),
// and its exact backward with the per-Gaussian blend weight alpha*T that
// drives contribution pruning (Sec. 3.2.2).
//
// One CTA per tile, one thread per pixel; each warp owns an 8x4 pixel block.
// Splat records are gathered 256 at a time into shared memory; the CTA stops
// when every pixel has reached T < 1e-4 (vote with __syncthreads_count).
// Compositing is FP32 FMA + MUFU work, not a dense contraction, so no tensor
// cores are involved.
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

__device__ __forceinline__ void pixel_of(int tile, int Tx, int &x, int &y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = (tile % Tx) * kTile + (warp & 1) * 8 + (lane & 7);
    y = (tile / Tx) * kTile + (warp >> 1) * 4 + (lane >> 3);
}

__global__ void __launch_bounds__(256) k_composite_fwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ list,
                                                       const Rec *__restrict__ rec, int W, int H, int Tx, float3 bg,
                                                       float *__restrict__ image, float *__restrict__ alpha_out,
                                                       float *__restrict__ t_final, uint32_t *__restrict__ n_contrib,
                                                       float *__restrict__ c_sum) {
    __shared__ float4 s_a[256], s_b[256];
    __shared__ float s_c[256];
    const int tile = blockIdx.x;
    int x, y;
    pixel_of(tile, Tx, x, y);
    const bool inside = x < W && y < H;
    const float px = x + 0.5f, py = y + 0.5f;
    const uint2 rg = ranges[tile];
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t base = rg.x; base < rg.y; base += 256) {
        if (__syncthreads_count(done) == 256) break;
        const uint32_t j = base + threadIdx.x;
        if (j < rg.y) {
            const Rec *r = rec + list[j];
            s_a[threadIdx.x] = r->a;
            s_b[threadIdx.x] = r->b;
            s_c[threadIdx.x] = r->c.x;
        }
        __syncthreads();
        const int cnt = min(256u, rg.y - base);
        for (int k = 0; k < cnt && !done; ++k) {
            const float4 a = s_a[k], b = s_b[k];
            float p, dy, ex, ao;
            const float al = splat_alpha(px, py, a, b, p, dy, ex, ao);
            if (al < kAlphaMin) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
            if (Tn < kTMin) { done = true; break; }
            const float w = __fmul_rn(al, T);
            C0 = __fmaf_rn(b.z, w, C0);
            C1 = __fmaf_rn(b.w, w, C1);
            C2 = __fmaf_rn(s_c[k], w, C2);
            T = Tn;
            last = base + k - rg.x + 1;
        }
    }
    if (inside) {
        const size_t pix = static_cast<size_t>(y) * W + x;
        const size_t plane = static_cast<size_t>(W) * H;
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
}

// Backward, front to back.  With S_i = sum_{j>i} c_j a_j T_j + T_N bg:
//   dL/da_i = dC.(c_i T_i - S_i/(1-a_i)) + dA T_N/(1-a_i)
//           = T_i (dC.c_i) - (dC.(Csum - P_i) + T_N (dC.bg) - dA T_N)/(1-a_i)
// where P_i is the running colour sum including splat i.  dC.P_i is carried
// as the scalar Q.
__global__ void __launch_bounds__(256) k_composite_bwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ list, const Rec *__restrict__ rec, int W, int H,
    int Tx, float3 bg, const float *__restrict__ t_final, const uint32_t *__restrict__ n_contrib,
    const float *__restrict__ c_sum, const float *__restrict__ dL_dimage, const float *__restrict__ dL_dalpha,
    const uint8_t *__restrict__ layer, uint32_t grad_layer_mask, float4 *__restrict__ rec_grad,
    float *__restrict__ contrib_sum, float *__restrict__ contrib_max) {
    __shared__ float4 s_a[256], s_b[256];
    __shared__ float s_c[256];
    __shared__ uint32_t s_idx[256];
    __shared__ float s_acc[256][12];
    __shared__ uint32_t s_wmax[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    int x, y;
    pixel_of(tile, Tx, x, y);
    const bool inside = x < W && y < H;
    const float px = x + 0.5f, py = y + 0.5f;
    const uint2 rg = ranges[tile];
    const size_t plane = static_cast<size_t>(W) * H;
    const size_t pix = inside ? static_cast<size_t>(y) * W + x : 0;
    uint32_t nc = 0;
    float TN = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dA = 0.f, QC = 0.f;
    if (inside) {
        nc = n_contrib[pix];
        TN = t_final[pix];
        if (dL_dimage) { dC0 = dL_dimage[pix]; dC1 = dL_dimage[plane + pix]; dC2 = dL_dimage[2 * plane + pix]; }
        if (dL_dalpha) dA = dL_dalpha[pix];
        QC = dC0 * c_sum[pix] + dC1 * c_sum[plane + pix] + dC2 * c_sum[2 * plane + pix];
    }
    const float K0 = TN * (dC0 * bg.x + dC1 * bg.y + dC2 * bg.z) - dA * TN;
    // longest blended prefix in the tile
    const uint32_t wm = __reduce_max_sync(FULL, nc);
    if (lane == 0) s_wmax[warp] = wm;
    for (int k = 0; k < 12; ++k) s_acc[threadIdx.x][k] = 0.f;
    __syncthreads();
    uint32_t maxnc = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) maxnc = max(maxnc, s_wmax[w]);
    const uint32_t stop = rg.x + min(maxnc, rg.y - rg.x);

    float T = 1.f, Q = 0.f;
    for (uint32_t base = rg.x; base < stop; base += 256) {
        const uint32_t j = base + threadIdx.x;
        if (j < stop) {
            const uint32_t g = list[j];
            const Rec *r = rec + g;
            s_a[threadIdx.x] = r->a;
            s_b[threadIdx.x] = r->b;
            s_c[threadIdx.x] = r->c.x;
            s_idx[threadIdx.x] = g;
        }
        __syncthreads();
        const int cnt = min(256u, stop - base);
        for (int k = 0; k < cnt; ++k) {
            const uint32_t pos = base + k - rg.x;
            bool act = pos < nc;
            const float4 a = s_a[k], b = s_b[k];
            const float cb = s_c[k];
            float p = 0.f, dy = 0.f, ex = 0.f, ao = 0.f, al = 0.f;
            if (act) {
                al = splat_alpha(px, py, a, b, p, dy, ex, ao);
                act = al >= kAlphaMin;
            }
            if (!__any_sync(FULL, act)) continue;
            float v[10];
            float wgt = 0.f;
#pragma unroll
            for (int q = 0; q < 10; ++q) v[q] = 0.f;
            if (act) {
                const float dcc = dC0 * b.z + dC1 * b.w + dC2 * cb;
                wgt = __fmul_rn(al, T);
                Q = fmaf(wgt, dcc, Q);
                const float inv = 1.f / (1.f - al);
                const float dLda = T * dcc - ((QC - Q) + K0) * inv;
                v[6] = wgt * dC0;
                v[7] = wgt * dC1;
                v[8] = wgt * dC2;
                if (ao < kAlphaMax) {
                    const float dLde = dLda * al * kLn2;
                    const float A2p = a.z * p;
                    v[5] = dLda * ex;
                    v[2] = dLde * p * p;
                    v[3] = dLde * 2.f * A2p * dy;
                    v[4] = dLde * dy * dy;
                    v[0] = -dLde * 2.f * A2p;
                    v[1] = -dLde * (2.f * A2p * a.w + 2.f * b.x * dy);
                }
                v[9] = wgt;
                T = __fmul_rn(T, __fsub_rn(1.f, al));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 10; ++q) v[q] += __shfl_xor_sync(FULL, v[q], o);
            const uint32_t wmx = __reduce_max_sync(FULL, __float_as_uint(wgt));
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < 10; ++q) atomicAdd(&s_acc[k][q], v[q]);
                atomicMax(reinterpret_cast<unsigned int *>(&s_acc[k][10]), wmx);
            }
        }
        __syncthreads();
        if (j < stop) {
            float *acc = s_acc[threadIdx.x];
            const uint32_t g = s_idx[threadIdx.x];
            if (acc[9] > 0.f) {
                if ((grad_layer_mask >> layer[g]) & 1u) {
                    atomicAdd(&rec_grad[3 * g], make_float4(acc[0], acc[1], acc[2], acc[3]));
                    atomicAdd(&rec_grad[3 * g + 1], make_float4(acc[4], acc[5], acc[6], acc[7]));
                    atomicAdd(&rec_grad[3 * g + 2], make_float4(acc[8], 0.f, 0.f, 0.f));
                }
                if (contrib_sum) atomicAdd(&contrib_sum[g], acc[9]);
                if (contrib_max) atomicMax(reinterpret_cast<unsigned int *>(&contrib_max[g]),
                                           __float_as_uint(acc[10]));
            }
#pragma unroll
            for (int q = 0; q < 12; ++q) acc[q] = 0.f;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_composite_forward(const uint2 *ranges, const uint32_t *list, const Rec *rec, int W, int H, int Tx,
                                     int Ty, float3 bg, float *image, float *alpha, float *t_final, uint32_t *n_contrib,
                                     float *c_sum, cudaStream_t st) {
    const int tiles = Tx * Ty;
    if (tiles == 0) return cudaSuccess;
    k_composite_fwd<<<tiles, 256, 0, st>>>(ranges, list, rec, W, H, Tx, bg, image, alpha, t_final, n_contrib, c_sum);
    return cudaGetLastError();
}

cudaError_t launch_composite_backward(const uint2 *ranges, const uint32_t *list, const Rec *rec, int W, int H, int Tx,
                                      int Ty, float3 bg, const float *t_final, const uint32_t *n_contrib,
                                      const float *c_sum, const float *dL_dimage, const float *dL_dalpha,
                                      const uint8_t *layer, uint32_t grad_layer_mask, float4 *rec_grad,
                                      float *contrib_sum, float *contrib_max, cudaStream_t st) {
    const int tiles = Tx * Ty;
    if (tiles == 0) return cudaSuccess;
    k_composite_bwd<<<tiles, 256, 0, st>>>(ranges, list, rec, W, H, Tx, bg, t_final, n_contrib, c_sum, dL_dimage,
                                           dL_dalpha, layer, grad_layer_mask, rec_grad, contrib_sum, contrib_max);
    return cudaGetLastError();
}

}  // namespace gs
