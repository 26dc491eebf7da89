// S4b - per-Gaussian chain rule from the record gradient (d/du, dv, dA2,
// dbeta, dG2, dopacity, drgb) to the stored parameters (means, log-scales,
// quaternions, opacity logit, SH), the backward of the EWA projection used by
// the layered training (Sec. 3.2).  Gaussians that were culled or whose layer
// is frozen (not in grad_layer_mask; Sec. 3.2: lower layers stay fixed) get 0.
//
// One launch, two kinds of block.  Live blocks take the visible Gaussians
// from the sort's index-ordered visible list, one thread each, so every warp
// does the chain rule on 32 live Gaussians instead of the third of its lanes
// that a pass over all indices would keep; they are bound by memory latency.
// Zero blocks give each warp 256 consecutive Gaussians and store zeros to the
// rows that are not live, 32 rows at a time with coalesced stores; they are
// bound by store bandwidth.  The zero blocks are spread evenly among the live
// blocks that have work, so the two kinds share the GPU for the whole launch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ float ldv(const void *p, int64_t idx, int dtype) {
    if (dtype == GS_DTYPE_F16) return __half2float(static_cast<const __half *>(p)[idx]);
    if (dtype == GS_DTYPE_BF16) return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[idx]);
    return static_cast<const float *>(p)[idx];
}

// Cartesian real SH (Condon-Shortley phase) and the gradient of each
// polynomial with respect to (x, y, z).
template <int deg>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float *b, float3 *db) {
    b[0] = 0x1.20dd76p-2f;
    db[0] = make_float3(0.f, 0.f, 0.f);
    if constexpr (deg < 1) return;
    const float C1 = 0x1.f45438p-2f;
    b[1] = -C1 * y; db[1] = make_float3(0.f, -C1, 0.f);
    b[2] = C1 * z;  db[2] = make_float3(0.f, 0.f, C1);
    b[3] = -C1 * x; db[3] = make_float3(-C1, 0.f, 0.f);
    if constexpr (deg < 2) return;
    const float C2A = 0x1.17b142p+0f, C2C = 0x1.42f602p-2f, C2E = 0x1.17b142p-1f;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    b[4] = C2A * xy;                     db[4] = make_float3(C2A * y, C2A * x, 0.f);
    b[5] = -C2A * yz;                    db[5] = make_float3(0.f, -C2A * z, -C2A * y);
    b[6] = C2C * ((2.f * zz - xx) - yy); db[6] = make_float3(-2.f * C2C * x, -2.f * C2C * y, 4.f * C2C * z);
    b[7] = -C2A * xz;                    db[7] = make_float3(-C2A * z, 0.f, -C2A * x);
    b[8] = C2E * (xx - yy);              db[8] = make_float3(2.f * C2E * x, -2.f * C2E * y, 0.f);
    if constexpr (deg < 3) return;
    const float C3A = 0x1.2e1a32p-1f, C3B = 0x1.71ff8ep+1f, C3C = 0x1.d403d0p-2f, C3D = 0x1.7e21f0p-2f,
                C3F = 0x1.71ff8ep+0f;
    b[9] = (-C3A * y) * (3.f * xx - yy);
    db[9] = make_float3(-6.f * C3A * xy, -C3A * (3.f * xx - 3.f * yy), 0.f);
    b[10] = (C3B * xy) * z;
    db[10] = make_float3(C3B * yz, C3B * xz, C3B * xy);
    b[11] = (-C3C * y) * ((4.f * zz - xx) - yy);
    db[11] = make_float3(2.f * C3C * xy, -C3C * (4.f * zz - xx - 3.f * yy), -8.f * C3C * yz);
    b[12] = (C3D * z) * ((2.f * zz - 3.f * xx) - 3.f * yy);
    db[12] = make_float3(-6.f * C3D * xz, -6.f * C3D * yz, C3D * (6.f * zz - 3.f * xx - 3.f * yy));
    b[13] = (-C3C * x) * ((4.f * zz - xx) - yy);
    db[13] = make_float3(-C3C * (4.f * zz - 3.f * xx - yy), 2.f * C3C * xy, -8.f * C3C * xz);
    b[14] = (C3F * z) * (xx - yy);
    db[14] = make_float3(2.f * C3F * xz, -2.f * C3F * yz, C3F * (xx - yy));
    b[15] = (-C3A * x) * (xx - 3.f * yy);
    db[15] = make_float3(-C3A * (3.f * xx - 3.f * yy), 6.f * C3A * xy, 0.f);
}

constexpr int kBwdThreads = 128;

// Everything the chain rule of Gaussian i reads, issued together before any
// branch: the inline-PTX loads are volatile, so the compiler keeps them at
// this point instead of moving them behind the visibility and layer tests.
template <int K>
struct RowIn {
    float4 ga, gb, gc;       // record gradient
    float m[3], ol;
    float ls[3], q[4];       // log-scales and quaternion, widened
    float sh[3 * K];         // [k][channel]
};

__device__ __forceinline__ float4 ld_now4(const void *p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_now(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <int K>
__device__ __forceinline__ void load_row(const SceneView &s, int i, const float4 *rec_grad, RowIn<K> &r) {
    r.ga = ld_now4(rec_grad + 3 * i);
    r.gb = ld_now4(rec_grad + 3 * i + 1);
    r.gc = ld_now4(rec_grad + 3 * i + 2);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.m[k] = ld_now(s.means + 3 * static_cast<int64_t>(i) + k);
    r.ol = ld_now(s.opacity_logit + i);
    if (s.dtype_sr == GS_DTYPE_F32) {
        const float *ls = static_cast<const float *>(s.log_scales) + 3 * static_cast<int64_t>(i);
        const float *q = static_cast<const float *>(s.quats) + 4 * static_cast<int64_t>(i);
#pragma unroll
        for (int k = 0; k < 3; ++k) r.ls[k] = ld_now(ls + k);
#pragma unroll
        for (int k = 0; k < 4; ++k) r.q[k] = ld_now(q + k);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) r.ls[k] = ldv(s.log_scales, 3 * static_cast<int64_t>(i) + k, s.dtype_sr);
#pragma unroll
        for (int k = 0; k < 4; ++k) r.q[k] = ldv(s.quats, 4 * static_cast<int64_t>(i) + k, s.dtype_sr);
    }
    const int64_t base = static_cast<int64_t>(i) * 3 * K;
    if constexpr ((3 * K) % 4 == 0) {
        if (s.dtype_sh == GS_DTYPE_F32 && (reinterpret_cast<uintptr_t>(s.sh) & 15u) == 0) {
            const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(s.sh) + base);
#pragma unroll
            for (int q = 0; q < 3 * K / 4; ++q) {
                const float4 x = ld_now4(p + q);
                r.sh[4 * q] = x.x; r.sh[4 * q + 1] = x.y; r.sh[4 * q + 2] = x.z; r.sh[4 * q + 3] = x.w;
            }
            return;
        }
    }
    if (s.dtype_sh == GS_DTYPE_F32) {
#pragma unroll
        for (int e = 0; e < 3 * K; ++e) r.sh[e] = ld_now(static_cast<const float *>(s.sh) + base + e);
    } else {
#pragma unroll
        for (int e = 0; e < 3 * K; ++e) r.sh[e] = ldv(s.sh, base + e, s.dtype_sh);
    }
}

// A gradient row of W floats; 16-byte stores where the row allows them.
template <int W>
__device__ __forceinline__ void store_row(float *dst, const float *v) {
    if constexpr (W % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
#pragma unroll
            for (int q = 0; q < W / 4; ++q)
                reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < W; ++e) dst[e] = v[e];
}

constexpr unsigned FULL = 0xFFFFFFFFu;

// The gradient rows of the Gaussians that are not live (tiles[i] == 0 or
// layer not in the mask): the arrays, and per launch the zero-block count,
// whether 16-byte stores apply, the SH row in stored words and its reciprocal.
struct ZeroRows {
    float *means, *log_scales, *quats, *opacity, *sh;
    const uint32_t *tiles;
    int n;
    int sh_row;          // 3K floats per SH gradient row
    uint32_t items;
    bool vec_q, vec_sh;
    int sh_w;
    uint32_t sh_m;
};

constexpr int kZeroRows = 256;             // Gaussians per zero-block warp

// Stores `zero` to the words of the rows r < nrows of a [32][w] block whose
// bit is set in `rows`, one warp, 32 consecutive words per step.  The row of
// word q is (q m) >> 20 with m = 2^20 / w + 1, exact for q < 32 w and w < 181.
template <class V>
__device__ __forceinline__ void zero_rows(V *base, int w, uint32_t m, unsigned rows, int nrows, int lane, V zero) {
    const int total = nrows * w;
    for (int q = lane; q < total; q += 32)
        if ((rows >> ((static_cast<uint32_t>(q) * m) >> 20)) & 1u) base[q] = zero;
}

__device__ __forceinline__ void zero_item(const ZeroRows &zr, uint32_t z, const uint8_t *__restrict__ layer,
                                          uint32_t mask, int lane) {
    constexpr int kSteps = kZeroRows / 32;
    constexpr uint32_t m1 = (1u << 20) + 1, m3 = (1u << 20) / 3 + 1, m4 = (1u << 20) / 4 + 1;
    const int64_t r0 = static_cast<int64_t>(z) * kZeroRows;
    uint32_t tc[kSteps], ly[kSteps];
#pragma unroll
    for (int k = 0; k < kSteps; ++k) {     // every liveness load of the item first
        const int64_t i = r0 + 32 * k + lane;
        tc[k] = i < zr.n ? zr.tiles[i] : 1u;
        ly[k] = i < zr.n ? layer[i] : 0u;
    }
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kSteps; ++k) {
        const int64_t i0 = r0 + 32 * k;
        if (i0 >= zr.n) break;
        const int nrows = zr.n - i0 < 32 ? static_cast<int>(zr.n - i0) : 32;
        const bool live = tc[k] > 0 && ((mask >> ly[k]) & 1u);
        unsigned rows = ~__ballot_sync(FULL, live);
        if (nrows < 32) rows &= (1u << nrows) - 1u;
        if (rows == 0) continue;
        zero_rows(zr.means + 3 * i0, 3, m3, rows, nrows, lane, 0.f);
        zero_rows(zr.log_scales + 3 * i0, 3, m3, rows, nrows, lane, 0.f);
        if (zr.vec_q) zero_rows(reinterpret_cast<float4 *>(zr.quats + 4 * i0), 1, m1, rows, nrows, lane, z4);
        else zero_rows(zr.quats + 4 * i0, 4, m4, rows, nrows, lane, 0.f);
        zero_rows(zr.opacity + i0, 1, m1, rows, nrows, lane, 0.f);
        if (zr.vec_sh)
            zero_rows(reinterpret_cast<float4 *>(zr.sh + static_cast<int64_t>(zr.sh_row) * i0), zr.sh_w, zr.sh_m,
                      rows, nrows, lane, z4);
        else
            zero_rows(zr.sh + static_cast<int64_t>(zr.sh_row) * i0, zr.sh_w, zr.sh_m, rows, nrows, lane, 0.f);
    }
}

// The chain rule of one live Gaussian.
template <int DEG>
__device__ __forceinline__ void grad_one(const CamView &c, int i, const RowIn<(DEG + 1) * (DEG + 1)> &r,
                                         const gs_grads &g) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float4 ga = r.ga, gb = r.gb, gc = r.gc;
    const float dU = ga.x, dV = ga.y, dA2 = ga.z, dBeta = ga.w, dG2 = gb.x, dOp = gb.y;
    const float dRgb[3] = {gb.z, gb.w, gc.x};
    const float mx = r.m[0], my_ = r.m[1], mz = r.m[2];
    const float *R = c.R;

    // opacity
    const float o = 1.f / (1.f + expf(-r.ol));
    g.opacity_logit[i] = dOp * o * (1.f - o);

    // colour and the view-direction part of d(mean)
    const float cp0 = -(R[0] * c.t[0] + R[3] * c.t[1] + R[6] * c.t[2]);
    const float cp1 = -(R[1] * c.t[0] + R[4] * c.t[1] + R[7] * c.t[2]);
    const float cp2 = -(R[2] * c.t[0] + R[5] * c.t[1] + R[8] * c.t[2]);
    const float vx = mx - cp0, vy = my_ - cp1, vz = mz - cp2;
    const float ivn = rsqrtf(vx * vx + vy * vy + vz * vz);
    const float dx = vx * ivn, dy = vy * ivn, dz = vz * ivn;
    float b[K];
    float3 db[K];
    sh_basis_grad<DEG>(dx, dy, dz, b, db);
    const float *shv = r.sh;
    float gch[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc += b[k] * shv[3 * k + ch];
        gch[ch] = acc + 0.5f > 0.f ? dRgb[ch] : 0.f;
    }
    float ddx = 0.f, ddy = 0.f, ddz = 0.f;
    float gsh[3 * K];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            gsh[3 * k + ch] = gch[ch] * b[k];
            const float t = shv[3 * k + ch] * gch[ch];
            ddx += t * db[k].x; ddy += t * db[k].y; ddz += t * db[k].z;
        }
    }
    store_row<3 * K>(g.sh + static_cast<int64_t>(i) * 3 * K, gsh);
    const float dd = ddx * dx + ddy * dy + ddz * dz;
    float gmx = (ddx - dx * dd) * ivn, gmy = (ddy - dy * dd) * ivn, gmz = (ddz - dz * dd) * ivn;

    // recompute the projection
    const float px = R[0] * mx + R[1] * my_ + R[2] * mz + c.t[0];
    const float py = R[3] * mx + R[4] * my_ + R[5] * mz + c.t[1];
    const float pz = R[6] * mx + R[7] * my_ + R[8] * mz + c.t[2];
    float sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = expf(r.ls[k]);
    float q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = r.q[k];
    const float iqn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] * iqn, x = q[1] * iqn, y = q[2] * iqn, z = q[3] * iqn;
    const float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                         2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                         2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * a + j] = Rq[3 * a + j] * sc[j];
    float Sg[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
            Sg[3 * a + bb] = M[3 * a] * M[3 * bb] + M[3 * a + 1] * M[3 * bb + 1] + M[3 * a + 2] * M[3 * bb + 2];
    const float limx = 1.3f * (0.5f * c.W / c.fx), limy = 1.3f * (0.5f * c.H / c.fy);
    const float iz = 1.f / pz;
    const float rx = px * iz, ry = py * iz;
    const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
    const float cxz = fminf(limx, fmaxf(-limx, rx)), cyz = fminf(limy, fmaxf(-limy, ry));
    const float J00 = c.fx * iz, J02 = -c.fx * cxz * iz, J11 = c.fy * iz, J12 = -c.fy * cyz * iz;
    float T[6];
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
        T[bb] = J00 * R[bb] + J02 * R[6 + bb];
        T[3 + bb] = J11 * R[3 + bb] + J12 * R[6 + bb];
    }
    float U[6];   // T Sigma
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
            U[3 * a + bb] = T[3 * a] * Sg[bb] + T[3 * a + 1] * Sg[3 + bb] + T[3 * a + 2] * Sg[6 + bb];
    const float s00 = U[0] * T[0] + U[1] * T[1] + U[2] * T[2] + 0.3f;
    const float s01 = U[0] * T[3] + U[1] * T[4] + U[2] * T[5];
    const float s11 = U[3] * T[3] + U[4] * T[4] + U[5] * T[5] + 0.3f;
    const float det = s00 * s11 - s01 * s01;
    const float NHL = -0x1.715476p-1f;
    const float idet2 = 1.f / (det * det);
    const float is11 = 1.f / s11;
    const float ds00 = dA2 * (-NHL * s11 * s11 * idet2);
    const float ds11 = dA2 * (-NHL * s01 * s01 * idet2) + dBeta * (s01 * is11 * is11) + dG2 * (-NHL * is11 * is11);
    const float ds01 = dA2 * (2.f * NHL * s11 * s01 * idet2) - dBeta * is11;
    const float G00 = ds00, G01 = 0.5f * ds01, G11 = ds11;

    // dSigma = T^T G T (symmetric), dT = 2 G T Sigma = 2 G U
    float dSg[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
            dSg[3 * a + bb] = T[a] * (G00 * T[bb] + G01 * T[3 + bb]) + T[3 + a] * (G01 * T[bb] + G11 * T[3 + bb]);
    float dT[6];
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
        dT[bb] = 2.f * (G00 * U[bb] + G01 * U[3 + bb]);
        dT[3 + bb] = 2.f * (G01 * U[bb] + G11 * U[3 + bb]);
    }
    // dJ = dT W^T (only the entries that are not identically zero)
    const float dJ00 = dT[0] * R[0] + dT[1] * R[1] + dT[2] * R[2];
    const float dJ02 = dT[0] * R[6] + dT[1] * R[7] + dT[2] * R[8];
    const float dJ11 = dT[3] * R[3] + dT[4] * R[4] + dT[5] * R[5];
    const float dJ12 = dT[3] * R[6] + dT[4] * R[7] + dT[5] * R[8];
    const float iz2 = iz * iz;
    float dpx = 0.f, dpy = 0.f, dpz = 0.f;
    dpz += -dJ00 * c.fx * iz2 + dJ02 * c.fx * cxz * iz2 - dJ11 * c.fy * iz2 + dJ12 * c.fy * cyz * iz2;
    const float dcx = -dJ02 * c.fx * iz, dcy = -dJ12 * c.fy * iz;
    if (!clx) { dpx += dcx * iz; dpz -= dcx * px * iz2; }
    if (!cly) { dpy += dcy * iz; dpz -= dcy * py * iz2; }
    dpx += dU * c.fx * iz;
    dpy += dV * c.fy * iz;
    dpz -= (dU * c.fx * px + dV * c.fy * py) * iz2;
    gmx += R[0] * dpx + R[3] * dpy + R[6] * dpz;
    gmy += R[1] * dpx + R[4] * dpy + R[7] * dpz;
    gmz += R[2] * dpx + R[5] * dpy + R[8] * dpz;
    g.means[3 * i] = gmx; g.means[3 * i + 1] = gmy; g.means[3 * i + 2] = gmz;

    // Sigma = M M^T: dM = 2 dSigma M;  M = Rq diag(s)
    float dR[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float ds = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float dM = 2.f * (dSg[3 * a] * M[j] + dSg[3 * a + 1] * M[3 + j] + dSg[3 * a + 2] * M[6 + j]);
            ds += dM * Rq[3 * a + j];
            dR[3 * a + j] = dM * sc[j];
        }
        g.log_scales[3 * i + j] = ds * sc[j];
    }
    // rotation matrix of the unit quaternion -> (w, x, y, z)
    const float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    const float dxq = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                             w * dR[7] - 2.f * x * dR[8]);
    const float dyq = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                             z * dR[7] - 2.f * y * dR[8]);
    const float dzq = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                             x * dR[6] + y * dR[7]);
    const float qd = dw * w + dxq * x + dyq * y + dzq * z;
    g.quats[4 * i] = (dw - w * qd) * iqn;
    g.quats[4 * i + 1] = (dxq - x * qd) * iqn;
    g.quats[4 * i + 2] = (dyq - y * qd) * iqn;
    g.quats[4 * i + 3] = (dzq - z * qd) * iqn;
}

template <int DEG>
__global__ void __launch_bounds__(kBwdThreads) k_preprocess_bwd(SceneView s, CamView c,
                                                                const uint32_t *__restrict__ tiles,
                                                                const uint32_t *__restrict__ vis_index,
                                                                const Ctl *__restrict__ ctl,
                                                                const float4 *__restrict__ rec_grad,
                                                                uint32_t grad_layer_mask, gs_grads g,
                                                                float *__restrict__ contrib_sum, const ZeroRows zr) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const uint32_t nl = (min(ctl->n_vis, static_cast<uint32_t>(s.n)) + kBwdThreads - 1) / kBwdThreads;
    const uint32_t stride = zr.items ? (nl + zr.items) / zr.items : 0xFFFFFFFFu;
    uint32_t b = blockIdx.x;
    if (b % stride == stride - 1 && b / stride < zr.items) {
        const uint32_t z = (b / stride) * (kBwdThreads / 32) + (threadIdx.x >> 5);
        if (static_cast<int64_t>(z) * kZeroRows < s.n) zero_item(zr, z, s.layer, grad_layer_mask, threadIdx.x & 31);
        return;
    }
    b -= min(zr.items, (b + 1) / stride);
    const uint32_t p = b * kBwdThreads + threadIdx.x;
    if (p >= min(ctl->n_vis, static_cast<uint32_t>(s.n))) return;
    const int i = static_cast<int>(vis_index[p]);
    const uint32_t tc = tiles[i];
    const uint32_t ly = s.layer[i];
    RowIn<K> r;
    load_row<K>(s, i, rec_grad, r);
    if (tc == 0) return;                        // a two-eye list also holds Gaussians only the other eye sees
    if (contrib_sum) contrib_sum[i] += r.gc.y;
    if (!((grad_layer_mask >> ly) & 1u)) return;   // frozen: a zero row
    grad_one<DEG>(c, i, r, g);
}

}  // namespace

cudaError_t launch_preprocess_backward(const SceneView &s, const CamView &c, const uint32_t *tiles,
                                       const uint32_t *vis_index, const Ctl *ctl, const float4 *rec_grad,
                                       uint32_t grad_layer_mask, const gs_grads &g, float *contrib_sum,
                                       cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    ZeroRows zr{g.means, g.log_scales, g.quats, g.opacity_logit, g.sh, tiles, s.n,
                3 * (s.sh_degree + 1) * (s.sh_degree + 1), 0, false, false, 0, 0};
    const int64_t zitems = (static_cast<int64_t>(s.n) + kZeroRows - 1) / kZeroRows;
    zr.items = static_cast<uint32_t>((zitems + kBwdThreads / 32 - 1) / (kBwdThreads / 32));   // zero blocks
    zr.vec_q = (reinterpret_cast<uintptr_t>(zr.quats) & 15u) == 0;
    zr.vec_sh = zr.sh_row % 4 == 0 && (reinterpret_cast<uintptr_t>(zr.sh) & 15u) == 0;
    zr.sh_w = zr.vec_sh ? zr.sh_row / 4 : zr.sh_row;
    zr.sh_m = (1u << 20) / static_cast<uint32_t>(zr.sh_w) + 1;
    const int blocks = (s.n + kBwdThreads - 1) / kBwdThreads + static_cast<int>(zr.items);
#define GS_PBWD(D) k_preprocess_bwd<D><<<blocks, kBwdThreads, 0, st>>>(s, c, tiles, vis_index, ctl, rec_grad, \
                                                                       grad_layer_mask, g, contrib_sum, zr)
    switch (s.sh_degree) {
        case 0: GS_PBWD(0); break;
        case 1: GS_PBWD(1); break;
        case 2: GS_PBWD(2); break;
        default: GS_PBWD(3); break;
    }
#undef GS_PBWD
    return cudaGetLastError();
}

}  // namespace gs
