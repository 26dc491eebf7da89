// S1 - per-Gaussian preprocess: layer-mask / clip-plane / near culls, EWA
// projection (Sec. 2.2.1), exponent coefficients, SH colour, opacity, tile
// rectangle and depth key (Sec. 3.3: only active layers are drawn; Gaussians
// sorted relative to the camera).
//
// This translation unit is compiled with -fmad=false: every a*b+c below is a
// rounded multiply followed by a rounded add, evaluated in the written order,
// so the integer decisions (culls, radius, rectangle, depth bits) are a fixed
// function of the float32 inputs (bit-exact tile ids and sort order).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

// exp(x) by Cody-Waite range reduction (x = k ln2 + r, ln2 split in a 16-bit
// head and a tail; Cody & Waite 1980) and the degree-7 Taylor series of exp(r)
// in Horner form.  Only +, -, * and an exact power-of-two scaling are used, so
// the result is reproducible on any IEEE single-precision machine.
__device__ __forceinline__ float exp_cw(float x) {
    x = fminf(fmaxf(x, -80.0f), 80.0f);
    float k = rintf(x * 0x1.715476p+0f);
    float r = (x - k * 0x1.62e4p-1f) - k * 0x1.7f7d1cp-20f;
    float p = 0x1.a01a02p-13f;
    p = p * r + 0x1.6c16c2p-10f;
    p = p * r + 0x1.111112p-7f;
    p = p * r + 0x1.555556p-5f;
    p = p * r + 0x1.555556p-3f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    return p * __int_as_float((static_cast<int>(k) + 127) << 23);
}

__device__ __forceinline__ float ld_half(const void *p, int64_t idx, int dtype) {
    if (dtype == GS_DTYPE_F16) return __half2float(static_cast<const __half *>(p)[idx]);
    if (dtype == GS_DTYPE_BF16) return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[idx]);
    return static_cast<const float *>(p)[idx];
}

// Real SH basis (Condon-Shortley phase, index l*l+l+m) from the textbook
// Cartesian forms; constants are the float nearest the exact normalisations.
template <int deg>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *b) {
    b[0] = 0x1.20dd76p-2f;                                  // 1/(2 sqrt(pi))
    if constexpr (deg < 1) return;
    const float C1 = 0x1.f45438p-2f;                        // sqrt(3/(4 pi))
    b[1] = -C1 * y;
    b[2] = C1 * z;
    b[3] = -C1 * x;
    if constexpr (deg < 2) return;
    const float C2A = 0x1.17b142p+0f, C2C = 0x1.42f602p-2f, C2E = 0x1.17b142p-1f;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    b[4] = C2A * xy;
    b[5] = -C2A * yz;
    b[6] = C2C * ((2.0f * zz - xx) - yy);
    b[7] = -C2A * xz;
    b[8] = C2E * (xx - yy);
    if constexpr (deg < 3) return;
    const float C3A = 0x1.2e1a32p-1f, C3B = 0x1.71ff8ep+1f, C3C = 0x1.d403d0p-2f, C3D = 0x1.7e21f0p-2f,
                C3F = 0x1.71ff8ep+0f;
    b[9] = (-C3A * y) * (3.0f * xx - yy);
    b[10] = (C3B * xy) * z;
    b[11] = (-C3C * y) * ((4.0f * zz - xx) - yy);
    b[12] = (C3D * z) * ((2.0f * zz - 3.0f * xx) - 3.0f * yy);
    b[13] = (-C3C * x) * ((4.0f * zz - xx) - yy);
    b[14] = (C3F * z) * (xx - yy);
    b[15] = (-C3A * x) * (xx - 3.0f * yy);
}

template <int DEG>
__global__ void __launch_bounds__(128) k_preprocess(SceneView s, CamView c, uint32_t layer_mask, Planes pl,
                                                    Rec *__restrict__ rec, uint32_t *__restrict__ tiles,
                                                    uint32_t *__restrict__ depth_key, const Ctl *__restrict__ ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    uint32_t ntiles = 0;
    uint32_t dkey = 0xFFFFFFFFu;
    const int lay = s.layer[i];
    const float mx = s.means[3 * i], my = s.means[3 * i + 1], mz = s.means[3 * i + 2];
    // the other per-Gaussian inputs but SH, loaded with these before the culling tests so that one memory
    // latency covers them all
    const float ls0 = ld_half(s.log_scales, 3 * (int64_t)i, s.dtype_sr);
    const float ls1 = ld_half(s.log_scales, 3 * (int64_t)i + 1, s.dtype_sr);
    const float ls2 = ld_half(s.log_scales, 3 * (int64_t)i + 2, s.dtype_sr);
    float qw, qx, qy, qz;
    if (s.dtype_sr == GS_DTYPE_F32) {
        const float4 q = reinterpret_cast<const float4 *>(s.quats)[i];
        qw = q.x; qx = q.y; qy = q.z; qz = q.w;
    } else {
        qw = ld_half(s.quats, 4 * (int64_t)i, s.dtype_sr);
        qx = ld_half(s.quats, 4 * (int64_t)i + 1, s.dtype_sr);
        qy = ld_half(s.quats, 4 * (int64_t)i + 2, s.dtype_sr);
        qz = ld_half(s.quats, 4 * (int64_t)i + 3, s.dtype_sr);
    }
    const float ol = s.opacity_logit[i];
    bool keep = (layer_mask >> lay) & 1u;
    for (int k = 0; k < pl.n && keep; ++k) {
        if (!((pl.bits[k] >> lay) & 1u)) continue;
        const float4 p = pl.p[k];
        const float dist = ((p.x * mx + p.y * my) + p.z * mz) + p.w;
        if (dist < 0.0f) keep = false;
    }
    const float *R = c.R;
    const float pz = ((R[6] * mx + R[7] * my) + R[8] * mz) + c.t[2];
    if (keep && !(pz > c.znear)) keep = false;
    if (keep) {
        // the SH row (read only if the splat turns out visible) is brought into L2 while the projection runs
        if (s.dtype_sh == GS_DTYPE_F32) {
            constexpr int K = (DEG + 1) * (DEG + 1);
            const char *row = reinterpret_cast<const char *>(static_cast<const float *>(s.sh) +
                                                             static_cast<int64_t>(i) * 3 * K);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row));                  // first and last byte of the
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + 3 * K * 4 - 1));  // row: its one or two lines
        }
        const float px = ((R[0] * mx + R[1] * my) + R[2] * mz) + c.t[0];
        const float py = ((R[3] * mx + R[4] * my) + R[5] * mz) + c.t[1];
        const float s0 = exp_cw(ls0);
        const float s1 = exp_cw(ls1);
        const float s2 = exp_cw(ls2);
        const float qq = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
        const float qn = sqrtf(qq);
        const float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
        const float r00 = 1.0f - 2.0f * (y * y + z * z), r01 = 2.0f * (x * y - w * z), r02 = 2.0f * (x * z + w * y);
        const float r10 = 2.0f * (x * y + w * z), r11 = 1.0f - 2.0f * (x * x + z * z), r12 = 2.0f * (y * z - w * x);
        const float r20 = 2.0f * (x * z - w * y), r21 = 2.0f * (y * z + w * x), r22 = 1.0f - 2.0f * (x * x + y * y);
        const float m00 = r00 * s0, m01 = r01 * s1, m02 = r02 * s2;
        const float m10 = r10 * s0, m11 = r11 * s1, m12 = r12 * s2;
        const float m20 = r20 * s0, m21 = r21 * s1, m22 = r22 * s2;
        const float S00 = (m00 * m00 + m01 * m01) + m02 * m02;
        const float S01 = (m00 * m10 + m01 * m11) + m02 * m12;
        const float S02 = (m00 * m20 + m01 * m21) + m02 * m22;
        const float S11 = (m10 * m10 + m11 * m11) + m12 * m12;
        const float S12 = (m10 * m20 + m11 * m21) + m12 * m22;
        const float S22 = (m20 * m20 + m21 * m21) + m22 * m22;

        const float limx = kFrustumClamp * ((0.5f * static_cast<float>(c.W)) / c.fx);
        const float limy = kFrustumClamp * ((0.5f * static_cast<float>(c.H)) / c.fy);
        const float izx = px / pz, izy = py / pz;
        const float cxz = fminf(limx, fmaxf(-limx, izx));
        const float cyz = fminf(limy, fmaxf(-limy, izy));
        const float j00 = c.fx / pz, j02 = -(c.fx * cxz) / pz;
        const float j11 = c.fy / pz, j12 = -(c.fy * cyz) / pz;
        const float t00 = j00 * R[0] + j02 * R[6], t01 = j00 * R[1] + j02 * R[7], t02 = j00 * R[2] + j02 * R[8];
        const float t10 = j11 * R[3] + j12 * R[6], t11 = j11 * R[4] + j12 * R[7], t12 = j11 * R[5] + j12 * R[8];
        const float u00 = (t00 * S00 + t01 * S01) + t02 * S02;
        const float u01 = (t00 * S01 + t01 * S11) + t02 * S12;
        const float u02 = (t00 * S02 + t01 * S12) + t02 * S22;
        const float u10 = (t10 * S00 + t11 * S01) + t12 * S02;
        const float u11 = (t10 * S01 + t11 * S11) + t12 * S12;
        const float u12 = (t10 * S02 + t11 * S12) + t12 * S22;
        const float c00 = ((u00 * t00 + u01 * t01) + u02 * t02) + kDilation;
        const float c01 = (u00 * t10 + u01 * t11) + u02 * t12;
        const float c11 = ((u10 * t10 + u11 * t11) + u12 * t12) + kDilation;
        const float det = c00 * c11 - c01 * c01;
        if (det > 0.0f) {
            const float mid = 0.5f * (c00 + c11);
            const float disc = fmaxf(kEigenFloor, mid * mid - det);
            const float lam = mid + sqrtf(disc);
            const float r = ceilf(kRadiusSigmas * sqrtf(lam));
            const float uu = c.fx * izx + c.cx, vv = c.fy * izy + c.cy;
            const float fTx = static_cast<float>(c.Tx), fTy = static_cast<float>(c.Ty);
            const float fx0 = fminf(fTx, fmaxf(0.0f, truncf((uu - r) * 0.0625f)));
            const float fy0 = fminf(fTy, fmaxf(0.0f, truncf((vv - r) * 0.0625f)));
            const float fx1 = fminf(fTx, fmaxf(0.0f, truncf(((uu + r) + 15.0f) * 0.0625f)));
            const float fy1 = fminf(fTy, fmaxf(0.0f, truncf(((vv + r) + 15.0f) * 0.0625f)));
            const int x0 = static_cast<int>(fx0), y0 = static_cast<int>(fy0);
            const int x1 = static_cast<int>(fx1), y1 = static_cast<int>(fy1);
            ntiles = GS_CHECK(x0 <= x1 && y0 <= y1 && x1 <= c.Tx && y1 <= c.Ty, ctl, kSiteRect)
                         ? static_cast<uint32_t>((x1 - x0) * (y1 - y0))
                         : 0u;
            if (ntiles > 0) {
                // view-dependent colour
                const float campos0 = -((R[0] * c.t[0] + R[3] * c.t[1]) + R[6] * c.t[2]);
                const float campos1 = -((R[1] * c.t[0] + R[4] * c.t[1]) + R[7] * c.t[2]);
                const float campos2 = -((R[2] * c.t[0] + R[5] * c.t[1]) + R[8] * c.t[2]);
                const float dx = mx - campos0, dy = my - campos1, dz = mz - campos2;
                const float dn = sqrtf((dx * dx + dy * dy) + dz * dz);
                constexpr int K = (DEG + 1) * (DEG + 1);
                float b[K];
                sh_basis<DEG>(dx / dn, dy / dn, dz / dn, b);
                const int64_t base = static_cast<int64_t>(i) * K * 3;
                float shv[3 * K];
                if (s.dtype_sh == GS_DTYPE_SH_CODEBOOK) {
                    // DC per Gaussian; coefficients k >= 1 from the FP16 table row (16-byte loads from L2)
                    const float *dcp = static_cast<const float *>(s.sh) + static_cast<int64_t>(i) * 3;
                    shv[0] = dcp[0]; shv[1] = dcp[1]; shv[2] = dcp[2];
                    constexpr int ROW = cb_row_halves(K);
                    const uint4 *row = reinterpret_cast<const uint4 *>(static_cast<const __half *>(s.sh_table) +
                                                                       static_cast<int64_t>(s.sh_index[i]) * ROW);
#pragma unroll
                    for (int q = 0; q < ROW / 8; ++q) {
                        const uint4 v = row[q];
                        const __half2 *h = reinterpret_cast<const __half2 *>(&v);
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const float2 f = __half22float2(h[r]);
                            const int d0 = 8 * q + 2 * r;
                            if (d0 < 3 * (K - 1)) shv[3 + d0] = f.x;
                            if (d0 + 1 < 3 * (K - 1)) shv[3 + d0 + 1] = f.y;
                        }
                    }
                } else if (s.dtype_sh == GS_DTYPE_F32 && (3 * K) % 4 == 0) {
                    // 16-byte loads of this Gaussian's coefficients (its row starts 16-byte aligned)
                    const float4 *src = reinterpret_cast<const float4 *>(static_cast<const float *>(s.sh) + base);
#pragma unroll
                    for (int k = 0; k < 3 * K / 4; ++k) {
                        const float4 v = src[k];
                        shv[4 * k] = v.x; shv[4 * k + 1] = v.y; shv[4 * k + 2] = v.z; shv[4 * k + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 3 * K; ++k) shv[k] = ld_half(s.sh, base + k, s.dtype_sh);
                }
                float rgb[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = b[0] * shv[ch];
#pragma unroll
                    for (int k = 1; k < K; ++k) acc = acc + b[k] * shv[3 * k + ch];
                    rgb[ch] = fmaxf(acc + 0.5f, 0.0f);
                }
                const float NHL = -0x1.715476p-1f;   // -log2(e)/2
                Rec o;
                o.a = make_float4(uu, vv, (c11 / det) * NHL, -(c01 / c11));
                const float opac = 1.0f / (1.0f + exp_cw(-ol));
                o.b = make_float4(NHL / c11, opac, rgb[0], rgb[1]);
                o.c = make_float4(rgb[2], pz, __uint_as_float(static_cast<uint32_t>(x0) | (static_cast<uint32_t>(y0) << 16)),
                                  __uint_as_float(static_cast<uint32_t>(x1) | (static_cast<uint32_t>(y1) << 16)));
                rec[i] = o;
                dkey = __float_as_uint(pz);
            }
        }
    }
    tiles[i] = ntiles;
    depth_key[i] = dkey;
}

}  // namespace

cudaError_t launch_preprocess(const SceneView &s, const CamView &c, uint32_t layer_mask, const Planes &pl, Rec *rec,
                              uint32_t *tiles, uint32_t *depth_key, const Ctl *ctl, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    const int threads = 128, blocks = (s.n + threads - 1) / threads;
    switch (s.sh_degree) {
        case 0: k_preprocess<0><<<blocks, threads, 0, st>>>(s, c, layer_mask, pl, rec, tiles, depth_key, ctl); break;
        case 1: k_preprocess<1><<<blocks, threads, 0, st>>>(s, c, layer_mask, pl, rec, tiles, depth_key, ctl); break;
        case 2: k_preprocess<2><<<blocks, threads, 0, st>>>(s, c, layer_mask, pl, rec, tiles, depth_key, ctl); break;
        default: k_preprocess<3><<<blocks, threads, 0, st>>>(s, c, layer_mask, pl, rec, tiles, depth_key, ctl); break;
    }
    return cudaGetLastError();
}

}  // namespace gs
