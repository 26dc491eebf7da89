// The training step around the rasterizer (Sec. 3.2: every layer is
// optimised with the layers below it frozen, a random background per frame
// and the alpha channel in the loss): the image loss with its gradient, Adam
// on the Gaussian parameters, and the row compaction that applies a prune.
//
// Loss (the 3DGS image loss the paper's training builds on):
//   Y    = C_t + (1 - A_t) bg                 target under this frame's background
//   loss = (1 - lam) mean|X - Y| + lam (1 - mean SSIM(X, Y)) + w_a mean|A - A_t|
// SSIM per channel with an 11x11 Gaussian window (sigma 1.5, normalised),
// zero outside the image, C1 = 0.01^2, C2 = 0.03^2.  Its gradient is three
// window sums of per-pixel maps (the window is symmetric):
//   dSSIM/dx_p = (G*a)_p + 2 x_p (G*b)_p + y_p (G*c)_p,
//   a = df/dmu_x - 2 mu_x df/dsx - mu_y df/dsxy,  b = df/dsx,  c = df/dsxy.
// Both kernels stage a (32 + 10) x (8 + 10) halo tile in shared memory and run
// the window as a horizontal then a vertical 11-tap pass (HBM-bound: a few
// floats per pixel and channel in and out).
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kLW = 32, kLH = 16, kHalo = 5, kWin = 11;
constexpr int kRW = kLW + 2 * kHalo, kRH = kLH + 2 * kHalo;   // 42 x 26 staged region
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Win {
    float g[kWin];
};

__device__ __forceinline__ float target_at(const float *trgb, const float *talpha, float bgc, size_t pc, size_t p) {
    return trgb[pc] + (1.f - talpha[p]) * bgc;
}

__device__ __forceinline__ float sgn(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// SSIM's window moments are taken of x - kSsimShift and y - kSsimShift (image
// values lie in [0, 1]); zero padding outside the image enters as -kSsimShift.
constexpr float kSsimShift = 0.5f;

// Pass 1: per pixel and channel, SSIM and the maps a, b, c; block sums of
// SSIM, |X - Y| and (channel 0) |A - A_t|.
__global__ void __launch_bounds__(kLW *kLH) k_loss_maps(const float *__restrict__ X, const float *__restrict__ A,
                                                        const float *__restrict__ Ct, const float *__restrict__ At,
                                                        float3 bg, int W, int H, const Win win,
                                                        float *__restrict__ maps, float *__restrict__ partials) {
    __shared__ float s_x[kRH][kRW], s_y[kRH][kRW];
    __shared__ float s_h[5][kRH][kLW];
    __shared__ float s_red[3][kLW * kLH / 32];
    const int ch = blockIdx.z;
    const float bgc = ch == 0 ? bg.x : (ch == 1 ? bg.y : bg.z);
    const size_t plane = static_cast<size_t>(W) * H;
    const int x0 = blockIdx.x * kLW - kHalo, y0 = blockIdx.y * kLH - kHalo;
    const int tid = threadIdx.x;
    for (int i = tid; i < kRW * kRH; i += kLW * kLH) {
        const int ry = i / kRW, rx = i % kRW;
        const int gx = x0 + rx, gy = y0 + ry;
        float xv = 0.f, yv = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t p = static_cast<size_t>(gy) * W + gx;
            xv = X[ch * plane + p];
            yv = target_at(Ct, At, bgc, ch * plane + p, p);
        }
        s_x[ry][rx] = xv;
        s_y[ry][rx] = yv;
    }
    __syncthreads();
    for (int i = tid; i < kRH * kLW; i += kLW * kLH) {
        const int ry = i / kLW, cx = i % kLW;
        float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
            const float a = s_x[ry][cx + j] - kSsimShift, b = s_y[ry][cx + j] - kSsimShift, w = win.g[j];
            mx = fmaf(w, a, mx);
            my = fmaf(w, b, my);
            xx = fmaf(w, a * a, xx);
            yy = fmaf(w, b * b, yy);
            xy = fmaf(w, a * b, xy);
        }
        s_h[0][ry][cx] = mx;
        s_h[1][ry][cx] = my;
        s_h[2][ry][cx] = xx;
        s_h[3][ry][cx] = yy;
        s_h[4][ry][cx] = xy;
    }
    __syncthreads();
    const int lx = tid % kLW, ly = tid / kLW;
    const int gx = blockIdx.x * kLW + lx, gy = blockIdx.y * kLH + ly;
    float f = 0.f, l1 = 0.f, la = 0.f;
    if (gx < W && gy < H) {
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kWin; ++i)
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmaf(win.g[i], s_h[q][ly + i][lx], m[q]);
        // moments of the shifted values x - kSsimShift, y - kSsimShift: the (co)variances are shift
        // invariant, and the shift takes most of E[x^2] - mu^2's cancellation out for values in [0, 1]
        const float mcx = m[0], mcy = m[1];
        const float sx = m[2] - mcx * mcx, sy = m[3] - mcy * mcy, sxy = m[4] - mcx * mcy;
        const float mux = mcx + kSsimShift, muy = mcy + kSsimShift;
        const float n1 = 2.f * mux * muy + kC1, n2 = 2.f * sxy + kC2;
        const float d1 = mux * mux + muy * muy + kC1, d2 = sx + sy + kC2;
        f = (n1 * n2) / (d1 * d2);
        const float df_dmx = f * (2.f * muy / n1 - 2.f * mux / d1);
        const float df_dsx = -f / d2;
        const float df_dsxy = 2.f * f / n2;
        const size_t p = static_cast<size_t>(gy) * W + gx;
        float *mp = maps + static_cast<size_t>(ch) * 3 * plane;
        mp[p] = df_dmx - 2.f * mcx * df_dsx - mcy * df_dsxy;
        mp[plane + p] = df_dsx;
        mp[2 * plane + p] = df_dsxy;
        l1 = fabsf(s_x[ly + kHalo][lx + kHalo] - s_y[ly + kHalo][lx + kHalo]);
        if (ch == 0 && A) la = fabsf(A[p] - At[p]);
    }
    // block sums (fixed order: deterministic)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_down_sync(0xFFFFFFFFu, f, o);
        l1 += __shfl_down_sync(0xFFFFFFFFu, l1, o);
        la += __shfl_down_sync(0xFFFFFFFFu, la, o);
    }
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = f;
        s_red[1][tid >> 5] = l1;
        s_red[2][tid >> 5] = la;
    }
    __syncthreads();
    if (tid < 3) {
        float s = 0.f;
        for (int w = 0; w < kLW * kLH / 32; ++w) s += s_red[tid][w];
        const size_t b = (static_cast<size_t>(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[3 * b + tid] = s;
    }
}

// loss = (1 - lam) L1 + lam (1 - SSIM) + w_a LA from the block sums, by one CTA
// of kLW * kLH threads in a fixed order (deterministic): each thread adds its
// strided share of the block sums in single precision, then a tree in shared
// memory (scratch: 3 * kLW * kLH floats).  The GB300's double-precision pipe is
// narrow; converting and adding every block sum in double took 20 us.
__device__ void loss_from_block_sums(const float *__restrict__ partials, int nb, size_t plane, float lam, float w_a,
                                     float *__restrict__ loss, float *scratch) {
    constexpr int NT = kLW * kLH;
    const int tid = threadIdx.x;
    float a[3] = {0.f, 0.f, 0.f};
    for (int b = tid; b < nb; b += NT)
#pragma unroll
        for (int q = 0; q < 3; ++q) a[q] += partials[3 * b + q];
#pragma unroll
    for (int q = 0; q < 3; ++q) scratch[q * NT + tid] = a[q];
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (tid < o)
#pragma unroll
            for (int q = 0; q < 3; ++q) scratch[q * NT + tid] += scratch[q * NT + tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        const double n = 3.0 * static_cast<double>(plane);
        *loss = static_cast<float>((1.0 - lam) * scratch[NT] / n + lam * (1.0 - scratch[0] / n) +
                                   w_a * scratch[2 * NT] / static_cast<double>(plane));
    }
    __syncthreads();
}

// Pass 2: window sums of a, b, c and the gradient of the loss; the first CTA
// also adds up pass 1's block sums into the loss.
__global__ void __launch_bounds__(kLW *kLH) k_loss_grad(const float *__restrict__ X, const float *__restrict__ A,
                                                        const float *__restrict__ Ct, const float *__restrict__ At,
                                                        float3 bg, int W, int H, const Win win, float lam, float w_a,
                                                        const float *__restrict__ maps, float *__restrict__ dX,
                                                        float *__restrict__ dA, const float *__restrict__ partials,
                                                        float w_a_loss, float *__restrict__ loss) {
    __shared__ float s_m[3][kRH][kRW];
    __shared__ float s_h[3][kRH][kLW];
    static_assert(3 * kRH * kRW >= 3 * kLW * kLH, "loss scratch in s_m");
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
        loss_from_block_sums(partials, static_cast<int>(gridDim.x * gridDim.y * gridDim.z), static_cast<size_t>(W) * H,
                             lam, w_a_loss, loss, &s_m[0][0][0]);
    const int ch = blockIdx.z;
    const float bgc = ch == 0 ? bg.x : (ch == 1 ? bg.y : bg.z);
    const size_t plane = static_cast<size_t>(W) * H;
    const float *mp = maps + static_cast<size_t>(ch) * 3 * plane;
    const int x0 = blockIdx.x * kLW - kHalo, y0 = blockIdx.y * kLH - kHalo;
    const int tid = threadIdx.x;
    for (int i = tid; i < kRW * kRH; i += kLW * kLH) {
        const int ry = i / kRW, rx = i % kRW;
        const int gx = x0 + rx, gy = y0 + ry;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const size_t p = in ? static_cast<size_t>(gy) * W + gx : 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) s_m[q][ry][rx] = in ? mp[q * plane + p] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kRH * kLW; i += kLW * kLH) {
        const int ry = i / kLW, cx = i % kLW;
        float h[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < kWin; ++j)
#pragma unroll
            for (int q = 0; q < 3; ++q) h[q] = fmaf(win.g[j], s_m[q][ry][cx + j], h[q]);
#pragma unroll
        for (int q = 0; q < 3; ++q) s_h[q][ry][cx] = h[q];
    }
    __syncthreads();
    const int lx = tid % kLW, ly = tid / kLW;
    const int gx = blockIdx.x * kLW + lx, gy = blockIdx.y * kLH + ly;
    if (gx >= W || gy >= H) return;
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kWin; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) s[q] = fmaf(win.g[i], s_h[q][ly + i][lx], s[q]);
    const size_t p = static_cast<size_t>(gy) * W + gx;
    const float x = X[ch * plane + p];
    const float y = target_at(Ct, At, bgc, ch * plane + p, p);
    const float inv_n = 1.f / (3.f * static_cast<float>(plane));
    const float dS = s[0] + 2.f * (x - kSsimShift) * s[1] + (y - kSsimShift) * s[2];
    dX[ch * plane + p] = ((1.f - lam) * sgn(x - y) - lam * dS) * inv_n;
    if (ch == 0 && dA) dA[p] = A ? w_a * sgn(A[p] - At[p]) / static_cast<float>(plane) : 0.f;
}

// Adam over the five parameter arrays seen as one index space; a Gaussian
// whose layer is not in train_mask keeps parameters and moments.
struct AdamArrays {
    float *p[5];
    const float *g[5];
    float *m[5], *v[5];
    uint64_t end[5];       // cumulative element counts
    uint32_t width[5];     // elements per Gaussian
    float step[5];         // lr / (1 - beta1^t)
};

__global__ void __launch_bounds__(256) k_adam(const AdamArrays arr, const uint8_t *__restrict__ layer,
                                              uint32_t train_mask, float beta1, float beta2, float inv_sqrt_bc2,
                                              float eps) {
    const uint64_t total = arr.end[4];
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        int k = 0;
        while (e >= arr.end[k]) ++k;
        const uint64_t i = e - (k ? arr.end[k - 1] : 0);
        const uint64_t row = i / arr.width[k];
        if (!((train_mask >> layer[row]) & 1u)) continue;
        const float g = arr.g[k][i];
        const float m = fmaf(beta1, arr.m[k][i], (1.f - beta1) * g);
        const float v = fmaf(beta2, arr.v[k][i], (1.f - beta2) * g * g);
        arr.m[k][i] = m;
        arr.v[k][i] = v;
        arr.p[k][i] -= arr.step[k] * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
    }
}

// The same update four elements at a time: a thread takes one 16-byte unit of
// one array (the last unit of an array may be partial) with vector loads and
// stores; the layer test runs only when some layer is frozen (a frozen
// element's values are written back unchanged).  Used when every array is
// 16-byte aligned; every element gets the same arithmetic as in k_adam.
struct Adam4 {
    float *p[5];
    const float *g[5];
    float *m[5], *v[5];
    uint32_t len[5];       // elements of each array
    uint32_t uend[5];      // cumulative 16-byte units
    uint32_t width[5];     // elements per Gaussian
    float step[5];
};

__global__ void __launch_bounds__(256) k_adam4(const Adam4 a, const uint8_t *__restrict__ layer, uint32_t train_mask,
                                               float beta1, float beta2, float inv_sqrt_bc2, float eps) {
    const bool all = train_mask == 0xFFFFFFFFu;
    const uint32_t total = a.uend[4];
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
        int k = 0;
        while (u >= a.uend[k]) ++k;
        const uint32_t e0 = 4u * (u - (k ? a.uend[k - 1] : 0u));
        const uint32_t cnt = min(4u, a.len[k] - e0);
        bool tr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            tr[q] = q < static_cast<int>(cnt) &&
                    (all || ((train_mask >> layer[(e0 + q) / a.width[k]]) & 1u));
        if (cnt == 4) {
            const float4 g4 = *reinterpret_cast<const float4 *>(a.g[k] + e0);
            float4 m4 = *reinterpret_cast<const float4 *>(a.m[k] + e0);
            float4 v4 = *reinterpret_cast<const float4 *>(a.v[k] + e0);
            float4 p4 = *reinterpret_cast<const float4 *>(a.p[k] + e0);
            float *gg = reinterpret_cast<float *>(const_cast<float4 *>(&g4));
            float *mm = reinterpret_cast<float *>(&m4), *vv = reinterpret_cast<float *>(&v4),
                  *pp = reinterpret_cast<float *>(&p4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!tr[q]) continue;
                const float g = gg[q];
                const float m = fmaf(beta1, mm[q], (1.f - beta1) * g);
                const float v = fmaf(beta2, vv[q], (1.f - beta2) * g * g);
                mm[q] = m;
                vv[q] = v;
                pp[q] -= a.step[k] * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
            }
            *reinterpret_cast<float4 *>(a.m[k] + e0) = m4;
            *reinterpret_cast<float4 *>(a.v[k] + e0) = v4;
            *reinterpret_cast<float4 *>(a.p[k] + e0) = p4;
        } else {
            for (uint32_t q = 0; q < cnt; ++q) {
                if (!tr[q]) continue;
                const uint32_t i = e0 + q;
                const float g = a.g[k][i];
                const float m = fmaf(beta1, a.m[k][i], (1.f - beta1) * g);
                const float v = fmaf(beta2, a.v[k][i], (1.f - beta2) * g * g);
                a.m[k][i] = m;
                a.v[k][i] = v;
                a.p[k][i] -= a.step[k] * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
            }
        }
    }
}

// Activity of the inactive pruning (Sec. 3.2.2): per trainable Gaussian,
// activity += 2 |d mean| + 0.1 |d SH| + 0.1 |d log-scale|, the norms of the
// update the last Adam step applied, recomputed from the new moments with
// the same expression as k_adam.
struct ActArgs {
    const float *m[3], *v[3];   // means, SH, log-scales
    uint32_t width[3];          // 3, 3K, 3
    float step[3];              // lr / (1 - beta1^t)
    float inv_sqrt_bc2, eps;
};

__global__ void __launch_bounds__(256) k_activity(const ActArgs a, const uint8_t *__restrict__ layer,
                                                  uint32_t train_mask, int n, float *__restrict__ activity) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || !((train_mask >> layer[g]) & 1u)) return;
    float nrm[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *m = a.m[k] + static_cast<size_t>(g) * a.width[k];
        const float *v = a.v[k] + static_cast<size_t>(g) * a.width[k];
        float acc = 0.f;
        for (uint32_t e = 0; e < a.width[k]; ++e) {
            const float d = a.step[k] * m[e] / (sqrtf(v[e]) * a.inv_sqrt_bc2 + a.eps);
            acc = fmaf(d, d, acc);
        }
        nrm[k] = sqrtf(acc);
    }
    activity[g] += 2.f * nrm[0] + 0.1f * nrm[1] + 0.1f * nrm[2];
}

// dst row i = src row idx[i], rows of `words` words of type T.
template <typename T>
__global__ void __launch_bounds__(256) k_gather_rows(const T *__restrict__ src, T *__restrict__ dst, uint32_t words,
                                                     const int32_t *__restrict__ idx, uint64_t n) {
    const uint64_t total = n * words;
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t r = e / words, w = e - r * words;
        dst[e] = src[static_cast<uint64_t>(idx[r]) * words + w];
    }
}

}  // namespace

size_t loss_workspace_bytes(int W, int H) {
    const size_t plane = static_cast<size_t>(W) * H;
    const size_t nb = static_cast<size_t>((W + kLW - 1) / kLW) * ((H + kLH - 1) / kLH) * 3;
    return 9 * plane * 4 + ((3 * nb * 4 + 255) / 256) * 256;
}

cudaError_t launch_image_loss(const float *X, const float *A, const float *Ct, const float *At, float3 bg, int W,
                              int H, float lam, float w_a, void *ws, float *loss, float *dX, float *dA,
                              cudaStream_t st) {
    Win win;
    double g[kWin], sum = 0.0;
    for (int j = 0; j < kWin; ++j) {
        const double r = j - kHalo;
        g[j] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
        sum += g[j];
    }
    for (int j = 0; j < kWin; ++j) win.g[j] = static_cast<float>(g[j] / sum);
    const size_t plane = static_cast<size_t>(W) * H;
    float *maps = static_cast<float *>(ws);
    float *partials = maps + 9 * plane;
    const dim3 grid((W + kLW - 1) / kLW, (H + kLH - 1) / kLH, 3);
    k_loss_maps<<<grid, kLW * kLH, 0, st>>>(X, A, Ct, At, bg, W, H, win, maps, partials);
    k_loss_grad<<<grid, kLW * kLH, 0, st>>>(X, A, Ct, At, bg, W, H, win, lam, w_a, maps, dX, dA, partials,
                                            A ? w_a : 0.f, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *const p[5], const float *const g[5], float *const m[5], float *const v[5],
                        const uint32_t width[5], int64_t n, const uint8_t *layer, uint32_t train_mask,
                        const float lr[5], float beta1, float beta2, float eps, int step, cudaStream_t st) {
    AdamArrays a;
    uint64_t acc = 0;
    const double bc1 = 1.0 - std::pow(static_cast<double>(beta1), step);
    const double bc2 = 1.0 - std::pow(static_cast<double>(beta2), step);
    for (int k = 0; k < 5; ++k) {
        a.p[k] = p[k];
        a.g[k] = g[k];
        a.m[k] = m[k];
        a.v[k] = v[k];
        a.width[k] = width[k];
        acc += static_cast<uint64_t>(n) * width[k];
        a.end[k] = acc;
        a.step[k] = static_cast<float>(lr[k] / bc1);
    }
    if (acc == 0) return cudaSuccess;
    const float inv_sqrt_bc2 = static_cast<float>(1.0 / std::sqrt(bc2));
    bool vec = acc < (1ull << 32);
    for (int k = 0; k < 5; ++k)
        vec = vec && width[k] > 0 && (reinterpret_cast<uintptr_t>(p[k]) | reinterpret_cast<uintptr_t>(g[k]) |
                                      reinterpret_cast<uintptr_t>(m[k]) | reinterpret_cast<uintptr_t>(v[k])) % 16 == 0;
    if (vec) {
        Adam4 b;
        uint32_t units = 0;
        for (int k = 0; k < 5; ++k) {
            b.p[k] = p[k];
            b.g[k] = g[k];
            b.m[k] = m[k];
            b.v[k] = v[k];
            b.width[k] = width[k];
            b.step[k] = a.step[k];
            b.len[k] = static_cast<uint32_t>(static_cast<uint64_t>(n) * width[k]);
            units += (b.len[k] + 3) / 4;
            b.uend[k] = units;
        }
        const int blocks = static_cast<int>(std::min<uint64_t>((units + 255) / 256, 8ull * 1024));
        k_adam4<<<blocks, 256, 0, st>>>(b, layer, train_mask, beta1, beta2, inv_sqrt_bc2, eps);
        return cudaGetLastError();
    }
    const int blocks = static_cast<int>(std::min<uint64_t>((acc + 255) / 256, 8ull * 1024));
    k_adam<<<blocks, 256, 0, st>>>(a, layer, train_mask, beta1, beta2, inv_sqrt_bc2, eps);
    return cudaGetLastError();
}

cudaError_t launch_activity(const float *const m[3], const float *const v[3], int sh_coeffs, int64_t n,
                            const uint8_t *layer, uint32_t train_mask, const float lr[3], float beta1, float beta2,
                            float eps, int step, float *activity, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    ActArgs a;
    const double bc1 = 1.0 - std::pow(static_cast<double>(beta1), step);
    const double bc2 = 1.0 - std::pow(static_cast<double>(beta2), step);
    const uint32_t width[3] = {3, static_cast<uint32_t>(3 * sh_coeffs), 3};
    for (int k = 0; k < 3; ++k) {
        a.m[k] = m[k];
        a.v[k] = v[k];
        a.width[k] = width[k];
        a.step[k] = static_cast<float>(lr[k] / bc1);
    }
    a.inv_sqrt_bc2 = static_cast<float>(1.0 / std::sqrt(bc2));
    a.eps = eps;
    k_activity<<<static_cast<int>((n + 255) / 256), 256, 0, st>>>(a, layer, train_mask, static_cast<int>(n), activity);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void *src, void *dst, int64_t row_bytes, const int32_t *idx, int64_t n,
                               cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int wb = (row_bytes % 4 == 0 && (reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 4 == 0)
                       ? 4 : (row_bytes % 2 == 0 ? 2 : 1);
    const uint32_t words = static_cast<uint32_t>(row_bytes / wb);
    const uint64_t total = static_cast<uint64_t>(n) * words;
    const int blocks = static_cast<int>(std::min<uint64_t>((total + 255) / 256, 8ull * 1024));
    if (wb == 4)
        k_gather_rows<uint32_t><<<blocks, 256, 0, st>>>(static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst),
                                                        words, idx, static_cast<uint64_t>(n));
    else if (wb == 2)
        k_gather_rows<uint16_t><<<blocks, 256, 0, st>>>(static_cast<const uint16_t *>(src), static_cast<uint16_t *>(dst),
                                                        words, idx, static_cast<uint64_t>(n));
    else
        k_gather_rows<uint8_t><<<blocks, 256, 0, st>>>(static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst),
                                                       words, idx, static_cast<uint64_t>(n));
    return cudaGetLastError();
}

}  // namespace gs
