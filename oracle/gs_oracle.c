/*
 * FP64 CPU oracle of the layered Gaussian-splatting tile rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code with the CUDA path and never calls it.
 *
 * What it computes (paper: "Multi-Layer Gaussian Splatting for Immersive
 * Anatomy Visualization"):
 *   - Sec. 3.2: one Gaussian cloud whose points carry a layer id next to their
 *     colour and scale attributes; layers are shown alone or together (Sec. 1,
 *     Sec. 3.3) and can be cut (Sec. 5, "Layering Approach").
 *   - Sec. 2.2.1 / Sec. 3.3: rendering by EWA splatting of the 3D Gaussians
 *     with a depth sort relative to the camera, as in the cited 3DGS renderer.
 *     The paper prints none of these equations; the math below is the EWA /
 *     3DGS formulation it adopts by reference:
 *        Sigma  = R(q) S S^T R(q)^T,            S = diag(exp(log_scale))
 *        Sigma' = J W Sigma W^T J^T + 0.3 I     (W = camera rotation)
 *        alpha  = min(0.99, o * exp(-1/2 d^T Sigma'^-1 d)),  o = sigmoid(logit)
 *        skip alpha < 1/255, stop before a splat once T*(1-alpha) < 1e-4
 *        C = sum_i c_i alpha_i T_i + T_final * bg
 *   - Sec. 3.2 (layered training): the gradient of the render with respect to
 *     every Gaussian parameter, plus the per-Gaussian blend weight alpha*T used
 *     to find Gaussians that do not contribute (Sec. 3.2.2).
 *
 * The exponent is evaluated as  g*log2(e) = A2*(dx + beta*dy)^2 + G2*dy^2  with
 *     A2 = -log2(e)/2 * Sigma'_11/det,  beta = -Sigma'_01/Sigma'_11,
 *     G2 = -log2(e)/2 / Sigma'_11,      d = pixel centre - projected mean,
 * which is the same quadratic form -1/2 d^T Sigma'^-1 d (completing the
 * square); it is written as a sum of two non-positive terms.
 *
 * Two preprocess variants exist:
 *   or_preprocess64: every quantity in double precision (the plain definition).
 *   or_preprocess32: the same steps in IEEE single precision with a fixed
 *     evaluation order (no contraction) so that the integer decisions (culls,
 *     radius, tile rectangle, depth key) are taken in the precision of the
 *     GPU path, as required for bit-exact tile ids and sort order.
 * Compositing and the backward pass always run in double precision.
 *
 * Build with -ffp-contract=off (see oracle/__init__.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TILE 16
#define ALPHA_MAX 0.99
#define ALPHA_MIN (1.0 / 255.0)
#define T_MIN 1e-4
#define DILATION 0.3
#define FRUSTUM_CLAMP 1.3

static const double LOG2E = 1.4426950408889634073599;
static const double LN2 = 0.6931471805599453094172;
static const double PI = 3.14159265358979323846264;

/* ------------------------------------------------------------------------- */
/* camera layout: cam[0..8] = R (row-major, world->cam), cam[9..11] = t,
 * cam[12..15] = fx, fy, cx, cy, cam[16] = znear.                              */

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics from their definition.
 *   Y_l^0  = K_l0 P_l(z)
 *   Y_l^m  = sqrt(2) K_lm (-1)^m P_l^(m)(z) Re((x+iy)^m)   m > 0
 *   Y_l^-m = sqrt(2) K_lm (-1)^m P_l^(m)(z) Im((x+iy)^m)   m > 0
 * with K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l the Legendre polynomial,
 * P_l^(m) its m-th derivative; (-1)^m is the Condon-Shortley phase and
 * (1-z^2)^(m/2) cos(m phi) = Re((x+iy)^m) on the unit sphere.  Coefficient
 * index k = l*l + l + m.                                                      */

static double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* coefficients (ascending powers of z) of Legendre P_l, l <= 3, Bonnet recurrence */
static void legendre_coeffs(int l, double c[4]) {
    double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0};
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    if (l == 1) { memcpy(c, p1, sizeof p1); return; }
    double pm[4], pc[4];
    memcpy(pm, p0, sizeof pm); memcpy(pc, p1, sizeof pc);
    for (int n = 1; n < l; ++n) {           /* (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1} */
        double nx[4] = {0, 0, 0, 0};
        for (int i = 0; i < 3; ++i) nx[i + 1] += (2 * n + 1) * pc[i];
        for (int i = 0; i < 4; ++i) nx[i] = (nx[i] - n * pm[i]) / (n + 1);
        memcpy(pm, pc, sizeof pm); memcpy(pc, nx, sizeof pc);
    }
    memcpy(c, pc, sizeof pc);
}

/* value of the k-th derivative of the polynomial c at z */
static double poly_deriv(const double c[4], int k, double z) {
    double s = 0;
    for (int i = k; i < 4; ++i) s += c[i] * (factorial(i) / factorial(i - k)) * pow(z, i - k);
    return s;
}

/* Re/Im of (x+iy)^m */
static void cpow_xy(double x, double y, int m, double *re, double *im) {
    double a = 1, b = 0;
    for (int i = 0; i < m; ++i) { double na = a * x - b * y, nb = a * y + b * x; a = na; b = nb; }
    *re = a; *im = b;
}

/* Y[k] and dY[k][3] = dY/d(x,y,z) of the polynomial extension, for deg <= 3 */
void or_sh_basis(int deg, const double d[3], double *Y, double *dY) {
    double x = d[0], y = d[1], z = d[2];
    for (int l = 0; l <= deg; ++l) {
        double c[4];
        legendre_coeffs(l, c);
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int k = l * l + l + m;
            double K = sqrt((2 * l + 1) / (4 * PI) * factorial(l - am) / factorial(l + am));
            if (m == 0) {
                Y[k] = K * poly_deriv(c, 0, z);
                if (dY) { dY[3 * k] = 0; dY[3 * k + 1] = 0; dY[3 * k + 2] = K * poly_deriv(c, 1, z); }
                continue;
            }
            double sgn = (am % 2) ? -1.0 : 1.0;
            double pre = sqrt(2.0) * K * sgn;
            double q = poly_deriv(c, am, z), dq = poly_deriv(c, am + 1, z);
            double re, im, re1, im1;
            cpow_xy(x, y, am, &re, &im);
            cpow_xy(x, y, am - 1, &re1, &im1);
            if (m > 0) {
                Y[k] = pre * q * re;
                if (dY) {
                    dY[3 * k] = pre * q * am * re1;
                    dY[3 * k + 1] = pre * q * (-am * im1);
                    dY[3 * k + 2] = pre * dq * re;
                }
            } else {
                Y[k] = pre * q * im;
                if (dY) {
                    dY[3 * k] = pre * q * am * im1;
                    dY[3 * k + 1] = pre * q * am * re1;
                    dY[3 * k + 2] = pre * dq * im;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Quaternions (w, x, y, z), Hamilton product; rotation v -> q v q*.          */

static void qmul(const double a[4], const double b[4], double o[4]) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static void qconj(const double a[4], double o[4]) { o[0] = a[0]; o[1] = -a[1]; o[2] = -a[2]; o[3] = -a[3]; }

/* rotation matrix of a unit quaternion: column j = q e_j q* */
void or_quat_to_rot(const double q[4], double R[9]) {
    double qc[4];
    qconj(q, qc);
    for (int j = 0; j < 3; ++j) {
        double e[4] = {0, 0, 0, 0}, t[4], r[4];
        e[j + 1] = 1.0;
        qmul(q, e, t);
        qmul(t, qc, r);
        for (int i = 0; i < 3; ++i) R[3 * i + j] = r[i + 1];
    }
}

/* dR[i][j]/dq_k for the bilinear map q -> q e_j q* (q not renormalised):
 * d/dq_k (q e_j q*) = b_k e_j q* + q e_j conj(b_k), b_k the k-th unit quaternion */
static void quat_rot_jacobian(const double q[4], double dR[4][9]) {
    double qc[4];
    qconj(q, qc);
    for (int k = 0; k < 4; ++k) {
        double b[4] = {0, 0, 0, 0}, bc[4];
        b[k] = 1.0;
        qconj(b, bc);
        for (int j = 0; j < 3; ++j) {
            double e[4] = {0, 0, 0, 0}, t1[4], r1[4], t2[4], r2[4];
            e[j + 1] = 1.0;
            qmul(b, e, t1); qmul(t1, qc, r1);
            qmul(q, e, t2); qmul(t2, bc, r2);
            for (int i = 0; i < 3; ++i) dR[k][3 * i + j] = r1[i + 1] + r2[i + 1];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Per-Gaussian FP64 preprocess.  Outputs (per Gaussian i):
 *   vis[i] (1 = kept), u, v, depth, A2, beta, G2, opac, rgb[3], radius, rect[4]
 *   (x0, y0, x1, y1 half-open tile rectangle), cov2d[3] (Sigma'_00, _01, _11). */
void or_preprocess64(int64_t n, const double *means, const double *log_scales,
                     const double *quats, const double *opac_logit, const double *sh,
                     const uint8_t *layer, int sh_degree, const double *cam, int W, int H,
                     uint32_t layer_mask, const double *planes, const uint32_t *plane_bits,
                     int n_planes,
                     int32_t *vis, double *u, double *v, double *depth, double *A2, double *beta,
                     double *G2, double *opac, double *rgb, int32_t *radius, int32_t *rect,
                     double *cov2d) {
    const double *Rc = cam, *tc = cam + 9;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15], znear = cam[16];
    int Tx = (W + TILE - 1) / TILE, Ty = (H + TILE - 1) / TILE;
    double limx = FRUSTUM_CLAMP * (0.5 * W / fx), limy = FRUSTUM_CLAMP * (0.5 * H / fy);
    int K = (sh_degree + 1) * (sh_degree + 1);
    double campos[3];
    for (int j = 0; j < 3; ++j) campos[j] = -(Rc[j] * tc[0] + Rc[3 + j] * tc[1] + Rc[6 + j] * tc[2]);

    for (int64_t i = 0; i < n; ++i) {
        vis[i] = 0; radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        const double *mu = means + 3 * i;
        /* layer enable mask (Sec. 3.3: only active layers are rendered) */
        if (!((layer_mask >> layer[i]) & 1u)) continue;
        /* clip planes: a Gaussian of a cut layer is removed whole when its centre
         * is on the negative side (Sec. 5, cut edges depend on point density) */
        int cut = 0;
        for (int k = 0; k < n_planes; ++k) {
            if (!((plane_bits[k] >> layer[i]) & 1u)) continue;
            const double *pl = planes + 4 * k;
            if (pl[0] * mu[0] + pl[1] * mu[1] + pl[2] * mu[2] + pl[3] < 0) cut = 1;
        }
        if (cut) continue;
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = Rc[3 * r] * mu[0] + Rc[3 * r + 1] * mu[1] + Rc[3 * r + 2] * mu[2] + tc[r];
        if (!(p[2] > znear)) continue;

        /* 3D covariance */
        double q[4], qn = 0;
        for (int k = 0; k < 4; ++k) qn += quats[4 * i + k] * quats[4 * i + k];
        qn = sqrt(qn);
        for (int k = 0; k < 4; ++k) q[k] = quats[4 * i + k] / qn;
        double R[9], s[3], Sig[9];
        or_quat_to_rot(q, R);
        for (int j = 0; j < 3; ++j) s[j] = exp(log_scales[3 * i + j]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += R[3 * a + j] * s[j] * s[j] * R[3 * b + j];
                Sig[3 * a + b] = acc;
            }
        /* EWA: local affine approximation of the perspective map */
        double z = p[2];
        double cxz = fmin(limx, fmax(-limx, p[0] / z)), cyz = fmin(limy, fmax(-limy, p[1] / z));
        double xp = cxz * z, yp = cyz * z;
        double J[6] = {fx / z, 0, -fx * xp / (z * z), 0, fy / z, -fy * yp / (z * z)};
        double T[6];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += J[3 * a + j] * Rc[3 * j + b];
                T[3 * a + b] = acc;
            }
        double S2[4];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0;
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k) acc += T[3 * a + j] * Sig[3 * j + k] * T[3 * b + k];
                S2[2 * a + b] = acc;
            }
        S2[0] += DILATION; S2[3] += DILATION;
        double det = S2[0] * S2[3] - S2[1] * S2[2];
        if (!(det > 0)) continue;
        double mid = 0.5 * (S2[0] + S2[3]);
        double lam = mid + sqrt(fmax(0.1, mid * mid - det));
        double r = ceil(3.0 * sqrt(lam));
        double uu = fx * p[0] / z + cx, vv = fy * p[1] / z + cy;
        double fx0 = fmin((double)Tx, fmax(0.0, trunc((uu - r) / TILE)));
        double fy0 = fmin((double)Ty, fmax(0.0, trunc((vv - r) / TILE)));
        double fx1 = fmin((double)Tx, fmax(0.0, trunc((uu + r + TILE - 1) / TILE)));
        double fy1 = fmin((double)Ty, fmax(0.0, trunc((vv + r + TILE - 1) / TILE)));
        int x0 = (int)fx0, y0 = (int)fy0, x1 = (int)fx1, y1 = (int)fy1;
        if ((x1 - x0) * (y1 - y0) == 0) continue;

        /* view-dependent colour from SH */
        double dir[3], dn = 0, Y[16];
        for (int j = 0; j < 3; ++j) { dir[j] = mu[j] - campos[j]; dn += dir[j] * dir[j]; }
        dn = sqrt(dn);
        for (int j = 0; j < 3; ++j) dir[j] /= dn;
        or_sh_basis(sh_degree, dir, Y, NULL);
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < K; ++k) acc += Y[k] * sh[(i * K + k) * 3 + c];
            rgb[3 * i + c] = fmax(acc + 0.5, 0.0);
        }
        vis[i] = 1;
        u[i] = uu; v[i] = vv; depth[i] = z;
        A2[i] = -0.5 * LOG2E * S2[3] / det;
        beta[i] = -S2[1] / S2[3];
        G2[i] = -0.5 * LOG2E / S2[3];
        opac[i] = 1.0 / (1.0 + exp(-opac_logit[i]));
        radius[i] = (int32_t)r;
        rect[4 * i] = x0; rect[4 * i + 1] = y0; rect[4 * i + 2] = x1; rect[4 * i + 3] = y1;
        cov2d[3 * i] = S2[0]; cov2d[3 * i + 1] = S2[1]; cov2d[3 * i + 2] = S2[3];
    }
}

/* ------------------------------------------------------------------------- */
/* Single-precision decision path.  Every operation below is one IEEE binary32
 * operation rounded to nearest, evaluated in the written order (this file is
 * compiled with -ffp-contract=off, so a*b+c is two roundings).  The exponential
 * is the Cody-Waite reduction exp(x) = 2^k exp(r), r = x - k ln2 with ln2 split
 * in a 16-bit head and a tail (Cody & Waite, 1980), and exp(r) by its Taylor
 * series to degree 7 in Horner form; only +, -, * and an exact power-of-two
 * scaling are used, so the result is the same on any IEEE machine.  The float
 * constants are written as hexadecimal literals (the float nearest the exact
 * value).                                                                     */

float or_expf32(float x) {
    x = fminf(fmaxf(x, -80.0f), 80.0f);
    float k = rintf(x * 0x1.715476p+0f);                   /* x * log2(e) */
    float r = (x - k * 0x1.62e4p-1f) - k * 0x1.7f7d1cp-20f;  /* ln2 = head + tail */
    float p = 0x1.a01a02p-13f;                             /* 1/5040 */
    p = p * r + 0x1.6c16c2p-10f;                           /* 1/720 */
    p = p * r + 0x1.111112p-7f;                            /* 1/120 */
    p = p * r + 0x1.555556p-5f;                            /* 1/24 */
    p = p * r + 0x1.555556p-3f;                            /* 1/6 */
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    /* 2^k for |k| <= 116 is a normal float: build it from its exponent bits */
    union { uint32_t u; float f; } two_k;
    two_k.u = (uint32_t)((int)k + 127) << 23;
    return p * two_k.f;
}

/* The FP32 SH basis: the textbook Cartesian real SH (Condon-Shortley phase)
 * with each product evaluated in the written order.  Constants are the float
 * nearest to the exact normalisation constants.                              */
static void sh_basis32(int deg, float x, float y, float z, float *b) {
    const float C0 = 0x1.20dd76p-2f;   /* 1/(2 sqrt(pi)) */
    const float C1 = 0x1.f45438p-2f;   /* sqrt(3/(4 pi)) */
    const float C2A = 0x1.17b142p+0f;  /* sqrt(15/pi)/2 */
    const float C2C = 0x1.42f602p-2f;  /* sqrt(5/pi)/4 */
    const float C2E = 0x1.17b142p-1f;  /* sqrt(15/pi)/4 */
    const float C3A = 0x1.2e1a32p-1f;  /* sqrt(35/(2 pi))/4 */
    const float C3B = 0x1.71ff8ep+1f;  /* sqrt(105/pi)/2 */
    const float C3C = 0x1.d403d0p-2f;  /* sqrt(21/(2 pi))/4 */
    const float C3D = 0x1.7e21f0p-2f;  /* sqrt(7/pi)/4 */
    const float C3F = 0x1.71ff8ep+0f;  /* sqrt(105/pi)/4 */
    b[0] = C0;
    if (deg < 1) return;
    b[1] = -C1 * y;
    b[2] = C1 * z;
    b[3] = -C1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    b[4] = C2A * xy;
    b[5] = -C2A * yz;
    b[6] = C2C * ((2.0f * zz - xx) - yy);
    b[7] = -C2A * xz;
    b[8] = C2E * (xx - yy);
    if (deg < 3) return;
    b[9] = (-C3A * y) * (3.0f * xx - yy);
    b[10] = (C3B * xy) * z;
    b[11] = (-C3C * y) * ((4.0f * zz - xx) - yy);
    b[12] = (C3D * z) * ((2.0f * zz - 3.0f * xx) - 3.0f * yy);
    b[13] = (-C3C * x) * ((4.0f * zz - xx) - yy);
    b[14] = (C3F * z) * (xx - yy);
    b[15] = (-C3A * x) * (xx - 3.0f * yy);
}

/* Outputs mirror the GPU per-Gaussian record: vis, u, v, depth (float; its
 * bit pattern is the sort key), A2, beta, G2, opac, rgb[3], radius, rect[4].  */
void or_preprocess32(int64_t n, const float *means, const float *log_scales, const float *quats,
                     const float *opac_logit, const float *sh, const uint8_t *layer,
                     int sh_degree, const float *cam, int W, int H, uint32_t layer_mask,
                     const float *planes, const uint32_t *plane_bits, int n_planes,
                     int32_t *vis, float *u, float *v, float *depth, float *A2, float *beta,
                     float *G2, float *opac, float *rgb, int32_t *radius, int32_t *rect) {
    const float *Rc = cam, *tc = cam + 9;
    float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15], znear = cam[16];
    int Tx = (W + TILE - 1) / TILE, Ty = (H + TILE - 1) / TILE;
    float limx = 1.3f * ((0.5f * (float)W) / fx);
    float limy = 1.3f * ((0.5f * (float)H) / fy);
    float campos[3];
    for (int j = 0; j < 3; ++j) campos[j] = -((Rc[j] * tc[0] + Rc[3 + j] * tc[1]) + Rc[6 + j] * tc[2]);
    int K = (sh_degree + 1) * (sh_degree + 1);
    const float NHL = -0x1.715476p-1f;     /* -log2(e)/2 */

    for (int64_t i = 0; i < n; ++i) {
        vis[i] = 0; radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        u[i] = v[i] = depth[i] = A2[i] = beta[i] = G2[i] = opac[i] = 0.0f;
        rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0.0f;
        float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        if (!((layer_mask >> layer[i]) & 1u)) continue;
        int cut = 0;
        for (int k = 0; k < n_planes; ++k) {
            if (!((plane_bits[k] >> layer[i]) & 1u)) continue;
            const float *pl = planes + 4 * k;
            float dist = ((pl[0] * mx + pl[1] * my) + pl[2] * mz) + pl[3];
            if (dist < 0.0f) cut = 1;
        }
        if (cut) continue;
        float pz = ((Rc[6] * mx + Rc[7] * my) + Rc[8] * mz) + tc[2];
        if (!(pz > znear)) continue;
        float px = ((Rc[0] * mx + Rc[1] * my) + Rc[2] * mz) + tc[0];
        float py = ((Rc[3] * mx + Rc[4] * my) + Rc[5] * mz) + tc[1];

        float s0 = or_expf32(log_scales[3 * i]);
        float s1 = or_expf32(log_scales[3 * i + 1]);
        float s2 = or_expf32(log_scales[3 * i + 2]);
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        float qq = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
        float qnrm = sqrtf(qq);
        float w = qw / qnrm, x = qx / qnrm, y = qy / qnrm, z = qz / qnrm;
        float r00 = 1.0f - 2.0f * (y * y + z * z), r01 = 2.0f * (x * y - w * z), r02 = 2.0f * (x * z + w * y);
        float r10 = 2.0f * (x * y + w * z), r11 = 1.0f - 2.0f * (x * x + z * z), r12 = 2.0f * (y * z - w * x);
        float r20 = 2.0f * (x * z - w * y), r21 = 2.0f * (y * z + w * x), r22 = 1.0f - 2.0f * (x * x + y * y);
        float m00 = r00 * s0, m01 = r01 * s1, m02 = r02 * s2;
        float m10 = r10 * s0, m11 = r11 * s1, m12 = r12 * s2;
        float m20 = r20 * s0, m21 = r21 * s1, m22 = r22 * s2;
        float S00 = (m00 * m00 + m01 * m01) + m02 * m02;
        float S01 = (m00 * m10 + m01 * m11) + m02 * m12;
        float S02 = (m00 * m20 + m01 * m21) + m02 * m22;
        float S11 = (m10 * m10 + m11 * m11) + m12 * m12;
        float S12 = (m10 * m20 + m11 * m21) + m12 * m22;
        float S22 = (m20 * m20 + m21 * m21) + m22 * m22;

        float izx = px / pz, izy = py / pz;
        float cxz = fminf(limx, fmaxf(-limx, izx));
        float cyz = fminf(limy, fmaxf(-limy, izy));
        float j00 = fx / pz, j02 = -(fx * cxz) / pz;
        float j11 = fy / pz, j12 = -(fy * cyz) / pz;
        float t00 = j00 * Rc[0] + j02 * Rc[6], t01 = j00 * Rc[1] + j02 * Rc[7], t02 = j00 * Rc[2] + j02 * Rc[8];
        float t10 = j11 * Rc[3] + j12 * Rc[6], t11 = j11 * Rc[4] + j12 * Rc[7], t12 = j11 * Rc[5] + j12 * Rc[8];
        float u00 = (t00 * S00 + t01 * S01) + t02 * S02;
        float u01 = (t00 * S01 + t01 * S11) + t02 * S12;
        float u02 = (t00 * S02 + t01 * S12) + t02 * S22;
        float u10 = (t10 * S00 + t11 * S01) + t12 * S02;
        float u11 = (t10 * S01 + t11 * S11) + t12 * S12;
        float u12 = (t10 * S02 + t11 * S12) + t12 * S22;
        float c00 = ((u00 * t00 + u01 * t01) + u02 * t02) + 0.3f;
        float c01 = (u00 * t10 + u01 * t11) + u02 * t12;
        float c11 = ((u10 * t10 + u11 * t11) + u12 * t12) + 0.3f;
        float det = c00 * c11 - c01 * c01;
        if (!(det > 0.0f)) continue;
        float mid = 0.5f * (c00 + c11);
        float disc = fmaxf(0.1f, mid * mid - det);
        float lam = mid + sqrtf(disc);
        float r = ceilf(3.0f * sqrtf(lam));
        float uu = fx * izx + cx, vv = fy * izy + cy;
        float fx0 = fminf((float)Tx, fmaxf(0.0f, truncf((uu - r) * 0.0625f)));
        float fy0 = fminf((float)Ty, fmaxf(0.0f, truncf((vv - r) * 0.0625f)));
        float fx1 = fminf((float)Tx, fmaxf(0.0f, truncf(((uu + r) + 15.0f) * 0.0625f)));
        float fy1 = fminf((float)Ty, fmaxf(0.0f, truncf(((vv + r) + 15.0f) * 0.0625f)));
        int x0 = (int)fx0, y0 = (int)fy0, x1 = (int)fx1, y1 = (int)fy1;
        if ((x1 - x0) * (y1 - y0) == 0) continue;

        float dx = mx - campos[0], dy = my - campos[1], dz = mz - campos[2];
        float dn = sqrtf((dx * dx + dy * dy) + dz * dz);
        float b[16];
        sh_basis32(sh_degree, dx / dn, dy / dn, dz / dn, b);
        for (int c = 0; c < 3; ++c) {
            float acc = b[0] * sh[(i * K) * 3 + c];
            for (int k = 1; k < K; ++k) acc = acc + b[k] * sh[(i * K + k) * 3 + c];
            rgb[3 * i + c] = fmaxf(acc + 0.5f, 0.0f);
        }
        vis[i] = 1;
        u[i] = uu; v[i] = vv; depth[i] = pz;
        A2[i] = (c11 / det) * NHL;
        beta[i] = -(c01 / c11);
        G2[i] = NHL / c11;
        opac[i] = 1.0f / (1.0f + or_expf32(-opac_logit[i]));
        radius[i] = (int32_t)r;
        rect[4 * i] = x0; rect[4 * i + 1] = y0; rect[4 * i + 2] = x1; rect[4 * i + 3] = y1;
    }
}

/* ------------------------------------------------------------------------- */
/* Tile binning: every visible Gaussian is listed in each tile of its
 * rectangle; each tile's list is ordered by (depth, Gaussian index), i.e. a
 * stable sort of the keys (tile << 32 | depth) emitted in index order.        */

typedef struct { int64_t tile; double depth; int64_t idx; } bin_entry;

static int bin_cmp(const void *pa, const void *pb) {
    const bin_entry *a = pa, *b = pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

int64_t or_count_dups(int64_t n, const int32_t *vis, const int32_t *rect) {
    int64_t d = 0;
    for (int64_t i = 0; i < n; ++i)
        if (vis[i]) d += (int64_t)(rect[4 * i + 2] - rect[4 * i]) * (rect[4 * i + 3] - rect[4 * i + 1]);
    return d;
}

/* ranges[2*t] = start, ranges[2*t+1] = end into list (length D) */
void or_bin(int64_t n, const int32_t *vis, const int32_t *rect, const double *depth, int W, int H,
            int64_t *ranges, int32_t *list) {
    int Tx = (W + TILE - 1) / TILE, Ty = (H + TILE - 1) / TILE;
    int64_t D = or_count_dups(n, vis, rect);
    bin_entry *e = (bin_entry *)malloc(sizeof(bin_entry) * (D > 0 ? D : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!vis[i]) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                e[k].tile = (int64_t)ty * Tx + tx; e[k].depth = depth[i]; e[k].idx = i; ++k;
            }
    }
    qsort(e, (size_t)D, sizeof(bin_entry), bin_cmp);
    for (int64_t t = 0; t < (int64_t)Tx * Ty; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t j = 0; j < D; ++j) {
        list[j] = (int32_t)e[j].idx;
        if (j == 0 || e[j - 1].tile != e[j].tile) ranges[2 * e[j].tile] = j;
        if (j == D - 1 || e[j + 1].tile != e[j].tile) ranges[2 * e[j].tile + 1] = j + 1;
    }
    free(e);
}

/* ------------------------------------------------------------------------- */
/* Front-to-back compositing of one pixel over an ordered splat list.
 * flip >= 0 inverts the outcome of the flip-th "fragile" decision: a
 * threshold test (alpha vs 1/255, T' vs 1e-4) whose operands lie within a
 * relative margin of the threshold (FRAGILE_*_REL), where single-precision
 * evaluation may legitimately fall on the other side.  Returns the number of fragile
 * decisions met.                                                             */

/* Margins of a fragile decision.  The single-precision alpha of a pixel and
 * splat is a few correctly rounded operations plus an approximate 2^x on
 * bit-identical inputs, a relative error near 2e-6; the single-precision
 * transmittance is a product of up to thousands of factors, each adding a
 * rounding.                                                                   */
#define FRAGILE_ALPHA_REL 1e-5
#define FRAGILE_T_REL 1e-4

typedef struct {
    double C[3], T;
    int64_t ncontrib;        /* 1 + list position of the last blended splat */
    int64_t nevaluated;      /* list positions examined, including the stopping one */
    int nadd;
    uint64_t dhash;          /* FNV-1a hash of the discrete decisions (blended ids, clamp state, stop) */
} pix_result;

static uint64_t fnv1a(uint64_t h, uint64_t v) {
    for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xFF; h *= 0x100000001b3ULL; }
    return h;
}

static double splat_exponent(double px, double py, double u, double v, double A2, double beta, double G2,
                             double *p_out, double *dy_out) {
    double dx = px - u, dy = py - v;
    double p = dx + beta * dy;
    if (p_out) *p_out = p;
    if (dy_out) *dy_out = dy;
    return A2 * p * p + G2 * dy * dy;
}

static int composite_pixel(double px, double py, const int32_t *list, int64_t start, int64_t end,
                           const double *u, const double *v, const double *A2, const double *beta,
                           const double *G2, const double *opac, const double *rgb, int flip,
                           pix_result *res, int32_t *added, double *Tbefore, double *alphas) {
    double T = 1.0, C[3] = {0, 0, 0};
    int64_t last = 0, j;
    int nfr = 0, nadd = 0;
    uint64_t h = 0xcbf29ce484222325ULL;
    for (j = start; j < end; ++j) {
        int32_t g = list[j];
        double e = splat_exponent(px, py, u[g], v[g], A2[g], beta[g], G2[g], NULL, NULL);
        double a = fmin(ALPHA_MAX, opac[g] * exp2(e));
        int skip = a < ALPHA_MIN;
        if (fabs(a - ALPHA_MIN) <= FRAGILE_ALPHA_REL * ALPHA_MIN) { if (nfr == flip) skip = !skip; ++nfr; }
        if (skip) continue;
        double Tn = T * (1.0 - a);
        int stop = Tn < T_MIN;
        if (fabs(Tn - T_MIN) <= FRAGILE_T_REL * T_MIN) { if (nfr == flip) stop = !stop; ++nfr; }
        if (stop) break;
        if (added) { added[nadd] = g; Tbefore[nadd] = T; alphas[nadd] = a; }
        h = fnv1a(h, ((uint64_t)(uint32_t)g << 1) | (uint64_t)(a >= ALPHA_MAX));
        ++nadd;
        for (int c = 0; c < 3; ++c) C[c] += rgb[3 * g + c] * a * T;
        T = Tn;
        last = j - start + 1;
    }
    for (int c = 0; c < 3; ++c) res->C[c] = C[c];
    res->T = T;
    res->ncontrib = last;
    res->nevaluated = (j < end ? j + 1 : end) - start;
    res->nadd = nadd;
    res->dhash = fnv1a(h, (uint64_t)res->nevaluated);
    return nfr;
}

/* image[3][H][W] (planar), alpha[H][W] = 1 - T, ncontrib[H][W],
 * Tfinal[H][W]; fragile[H][W] = number of fragile decisions; alt_* = the
 * result with the first fragile decision inverted (valid where fragile > 0). */
void or_composite(int W, int H, const int64_t *ranges, const int32_t *list, const double *u,
                  const double *v, const double *A2, const double *beta, const double *G2,
                  const double *opac, const double *rgb, const double *bg, double *image,
                  double *alpha, int64_t *ncontrib, double *Tfinal, int32_t *fragile,
                  double *alt_image, double *alt_alpha, int64_t *alt_ncontrib, uint64_t *dhash) {
    int Tx = (W + TILE - 1) / TILE;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t t = (int64_t)(y / TILE) * Tx + (x / TILE);
            int64_t pidx = (int64_t)y * W + x;
            pix_result r, ra;
            int nfr = composite_pixel(x + 0.5, y + 0.5, list, ranges[2 * t], ranges[2 * t + 1], u, v, A2,
                                      beta, G2, opac, rgb, -1, &r, NULL, NULL, NULL);
            for (int c = 0; c < 3; ++c) image[(int64_t)c * W * H + pidx] = r.C[c] + r.T * bg[c];
            alpha[pidx] = 1.0 - r.T;
            ncontrib[pidx] = r.ncontrib;
            Tfinal[pidx] = r.T;
            fragile[pidx] = nfr;
            dhash[pidx] = r.dhash;
            if (nfr > 0) {
                int nfr2 = composite_pixel(x + 0.5, y + 0.5, list, ranges[2 * t], ranges[2 * t + 1], u, v,
                                           A2, beta, G2, opac, rgb, 0, &ra, NULL, NULL, NULL);
                if (nfr2 > fragile[pidx]) fragile[pidx] = nfr2;
                for (int c = 0; c < 3; ++c) alt_image[(int64_t)c * W * H + pidx] = ra.C[c] + ra.T * bg[c];
                alt_alpha[pidx] = 1.0 - ra.T;
                alt_ncontrib[pidx] = ra.ncontrib;
            } else {
                for (int c = 0; c < 3; ++c) alt_image[(int64_t)c * W * H + pidx] = image[(int64_t)c * W * H + pidx];
                alt_alpha[pidx] = alpha[pidx];
                alt_ncontrib[pidx] = ncontrib[pidx];
            }
        }
}

/* The compositing of or_composite at npix selected pixels (xs[k], ys[k]). */
void or_composite_pixels(int W, int H, const int64_t *ranges, const int32_t *list, const double *u,
                         const double *v, const double *A2, const double *beta, const double *G2,
                         const double *opac, const double *rgb, const double *bg, int64_t npix,
                         const int32_t *xs, const int32_t *ys, double *rgb_out, double *alpha,
                         int64_t *ncontrib, int32_t *fragile, double *alt_rgb, double *alt_alpha,
                         int64_t *alt_ncontrib) {
    int Tx = (W + TILE - 1) / TILE;
    (void)H;
    for (int64_t k = 0; k < npix; ++k) {
        int x = xs[k], y = ys[k];
        int64_t t = (int64_t)(y / TILE) * Tx + (x / TILE);
        pix_result r, ra;
        int nfr = composite_pixel(x + 0.5, y + 0.5, list, ranges[2 * t], ranges[2 * t + 1], u, v, A2, beta, G2,
                                  opac, rgb, -1, &r, NULL, NULL, NULL);
        for (int c = 0; c < 3; ++c) rgb_out[3 * k + c] = r.C[c] + r.T * bg[c];
        alpha[k] = 1.0 - r.T;
        ncontrib[k] = r.ncontrib;
        fragile[k] = nfr;
        ra = r;
        if (nfr > 0) {
            int nfr2 = composite_pixel(x + 0.5, y + 0.5, list, ranges[2 * t], ranges[2 * t + 1], u, v, A2, beta,
                                       G2, opac, rgb, 0, &ra, NULL, NULL, NULL);
            if (nfr2 > nfr) fragile[k] = nfr2;
        }
        for (int c = 0; c < 3; ++c) alt_rgb[3 * k + c] = ra.C[c] + ra.T * bg[c];
        alt_alpha[k] = 1.0 - ra.T;
        alt_ncontrib[k] = ra.ncontrib;
    }
}

/* Brute force: every visible Gaussian at every pixel, in (depth, index)
 * order, with no tiles.  Equal to or_composite wherever every splat's
 * alpha >= 1/255 support lies inside its tile rectangle.                     */
void or_composite_bruteforce(int W, int H, int64_t n, const int32_t *order, int64_t n_order,
                             const double *u, const double *v, const double *A2, const double *beta,
                             const double *G2, const double *opac, const double *rgb, const double *bg,
                             double *image, double *alpha) {
    (void)n;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            pix_result r;
            composite_pixel(x + 0.5, y + 0.5, order, 0, n_order, u, v, A2, beta, G2, opac, rgb, -1, &r,
                            NULL, NULL, NULL);
            int64_t pidx = (int64_t)y * W + x;
            for (int c = 0; c < 3; ++c) image[(int64_t)c * W * H + pidx] = r.C[c] + r.T * bg[c];
            alpha[pidx] = 1.0 - r.T;
        }
}

/* ------------------------------------------------------------------------- */
/* Backward of the compositing, exact derivative of the forward as written:
 *   C = sum_i c_i a_i T_i + T_N bg,  T_i = prod_{j<i} (1 - a_j),  A = 1 - T_N
 *   dC/da_i = c_i T_i - S_i / (1 - a_i),  S_i = sum_{j>i} c_j a_j T_j + T_N bg
 *   dA/da_i = T_N / (1 - a_i),           dC/dc_i = a_i T_i
 *   a = min(0.99, o 2^e): da/do = 2^e, da/de = a ln2 below the clamp, 0 above
 *   e = A2 p^2 + G2 dy^2, p = dx + beta dy, dx = px - u, dy = py - v
 * Culls, skips, the stop and the tile lists are constants.  Also accumulates
 * contrib_sum[g] += a T and contrib_max[g] = max(.., a T) over blended pixels.
 * rec_grad layout per Gaussian: [du, dv, dA2, dbeta, dG2, dopac, dr, dg, db].
 * touched_fragile[g] is set when a fragile pixel blends or skips g.
 * contrib_count[g] (may be NULL) is the number of pixels at which g was
 * blended, i.e. the number of terms of contrib_sum[g].
 * tile_mask (may be NULL) restricts the pass to the marked tiles; the result
 * is then exact for every Gaussian whose tile rectangle lies in marked tiles. */
void or_composite_backward(int W, int H, int64_t n, const int64_t *ranges, const int32_t *list,
                           const double *u, const double *v, const double *A2, const double *beta,
                           const double *G2, const double *opac, const double *rgb, const double *bg,
                           const double *dL_dimage, const double *dL_dalpha, const uint8_t *tile_mask,
                           double *rec_grad, double *contrib_sum, double *contrib_max, int32_t *touched_fragile,
                           int64_t *contrib_count) {
    int Tx = (W + TILE - 1) / TILE;
    int64_t maxlen = 0;
    int64_t ntiles = (int64_t)Tx * ((H + TILE - 1) / TILE);
    for (int64_t t = 0; t < ntiles; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    int32_t *added = (int32_t *)malloc(sizeof(int32_t) * (maxlen + 1));
    double *Tb = (double *)malloc(sizeof(double) * (maxlen + 1));
    double *al = (double *)malloc(sizeof(double) * (maxlen + 1));
    memset(rec_grad, 0, sizeof(double) * 9 * n);
    for (int64_t g = 0; g < n; ++g) {
        contrib_sum[g] = 0; contrib_max[g] = 0; touched_fragile[g] = 0;
        if (contrib_count) contrib_count[g] = 0;
    }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t t = (int64_t)(y / TILE) * Tx + (x / TILE);
            int64_t pidx = (int64_t)y * W + x;
            double px = x + 0.5, py = y + 0.5;
            pix_result r;
            if (tile_mask && !tile_mask[t]) continue;
            int nfr = composite_pixel(px, py, list, ranges[2 * t], ranges[2 * t + 1], u, v, A2, beta, G2,
                                      opac, rgb, -1, &r, added, Tb, al);
            if (nfr > 0)
                for (int64_t j = ranges[2 * t]; j < ranges[2 * t] + r.nevaluated; ++j)
                    touched_fragile[list[j]] = 1;
            double TN = r.T;
            double dC[3], dA = dL_dalpha ? dL_dalpha[pidx] : 0.0;
            for (int c = 0; c < 3; ++c) dC[c] = dL_dimage ? dL_dimage[(int64_t)c * W * H + pidx] : 0.0;
            double S[3];
            for (int c = 0; c < 3; ++c) S[c] = TN * bg[c];
            for (int k = r.nadd - 1; k >= 0; --k) {
                int32_t g = added[k];
                double a = al[k], T = Tb[k];
                double inv = 1.0 / (1.0 - a);
                double dLda = dA * TN * inv;
                for (int c = 0; c < 3; ++c) {
                    dLda += dC[c] * (rgb[3 * g + c] * T - S[c] * inv);
                    rec_grad[9 * g + 6 + c] += dC[c] * a * T;
                }
                double p, dy;
                double e = splat_exponent(px, py, u[g], v[g], A2[g], beta[g], G2[g], &p, &dy);
                double ex = exp2(e);
                if (fabs(opac[g] * ex - ALPHA_MAX) <= FRAGILE_ALPHA_REL * ALPHA_MAX) touched_fragile[g] = 1;
                if (opac[g] * ex < ALPHA_MAX) {
                    double dLde = dLda * a * LN2;
                    rec_grad[9 * g + 5] += dLda * ex;
                    rec_grad[9 * g + 2] += dLde * p * p;
                    rec_grad[9 * g + 3] += dLde * 2.0 * A2[g] * p * dy;
                    rec_grad[9 * g + 4] += dLde * dy * dy;
                    rec_grad[9 * g + 0] += dLde * (-2.0 * A2[g] * p);
                    rec_grad[9 * g + 1] += dLde * (-2.0 * A2[g] * p * beta[g] - 2.0 * G2[g] * dy);
                }
                double w = a * T;
                contrib_sum[g] += w;
                if (w > contrib_max[g]) contrib_max[g] = w;
                if (contrib_count) contrib_count[g] += 1;
                for (int c = 0; c < 3; ++c) S[c] += rgb[3 * g + c] * w;
            }
        }
    free(added); free(Tb); free(al);
}

/* ------------------------------------------------------------------------- */
/* Chain rule from the per-Gaussian record gradient to the stored parameters,
 * in double precision, exact derivative of or_preprocess64 (clamps and culls
 * contribute zero).  rec_grad layout as in or_composite_backward.
 * Outputs: d_means[3n], d_log_scales[3n], d_quats[4n], d_opac_logit[n],
 * d_sh[n*K*3]; Gaussians with vis == 0 or whose layer is not in
 * grad_layer_mask get zeros (frozen layers, Sec. 3.2).                       */
void or_chain(int64_t n, const double *means, const double *log_scales, const double *quats,
              const double *opac_logit, const double *sh, const uint8_t *layer, int sh_degree,
              const double *cam, int W, int H, const int32_t *vis, const double *rec_grad,
              uint32_t grad_layer_mask, double *d_means, double *d_log_scales, double *d_quats,
              double *d_opac, double *d_sh) {
    const double *Rc = cam, *tc = cam + 9;
    double fx = cam[12], fy = cam[13];
    double limx = FRUSTUM_CLAMP * (0.5 * W / fx), limy = FRUSTUM_CLAMP * (0.5 * H / fy);
    int K = (sh_degree + 1) * (sh_degree + 1);
    double campos[3];
    for (int j = 0; j < 3; ++j) campos[j] = -(Rc[j] * tc[0] + Rc[3 + j] * tc[1] + Rc[6 + j] * tc[2]);
    memset(d_means, 0, sizeof(double) * 3 * n);
    memset(d_log_scales, 0, sizeof(double) * 3 * n);
    memset(d_quats, 0, sizeof(double) * 4 * n);
    memset(d_opac, 0, sizeof(double) * n);
    memset(d_sh, 0, sizeof(double) * n * K * 3);

    for (int64_t i = 0; i < n; ++i) {
        if (!vis[i] || !((grad_layer_mask >> layer[i]) & 1u)) continue;
        const double *gr = rec_grad + 9 * i;
        const double *mu = means + 3 * i;
        double dmu[3] = {0, 0, 0};

        /* opacity */
        double o = 1.0 / (1.0 + exp(-opac_logit[i]));
        d_opac[i] = gr[5] * o * (1.0 - o);

        /* colour */
        double dir[3], dn = 0, Y[16], dY[48];
        for (int j = 0; j < 3; ++j) { dir[j] = mu[j] - campos[j]; dn += dir[j] * dir[j]; }
        dn = sqrt(dn);
        for (int j = 0; j < 3; ++j) dir[j] /= dn;
        or_sh_basis(sh_degree, dir, Y, dY);
        double ddir[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < K; ++k) acc += Y[k] * sh[(i * K + k) * 3 + c];
            if (!(acc + 0.5 > 0.0)) continue;           /* clamped at zero */
            for (int k = 0; k < K; ++k) {
                d_sh[(i * K + k) * 3 + c] = gr[6 + c] * Y[k];
                for (int j = 0; j < 3; ++j) ddir[j] += gr[6 + c] * sh[(i * K + k) * 3 + c] * dY[3 * k + j];
            }
        }
        double dd = ddir[0] * dir[0] + ddir[1] * dir[1] + ddir[2] * dir[2];
        for (int j = 0; j < 3; ++j) dmu[j] += (ddir[j] - dir[j] * dd) / dn;

        /* recompute the projection */
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = Rc[3 * r] * mu[0] + Rc[3 * r + 1] * mu[1] + Rc[3 * r + 2] * mu[2] + tc[r];
        double q[4], qn = 0;
        for (int k = 0; k < 4; ++k) qn += quats[4 * i + k] * quats[4 * i + k];
        qn = sqrt(qn);
        for (int k = 0; k < 4; ++k) q[k] = quats[4 * i + k] / qn;
        double R[9], s[3], M[9], Sig[9];
        or_quat_to_rot(q, R);
        for (int j = 0; j < 3; ++j) s[j] = exp(log_scales[3 * i + j]);
        for (int a = 0; a < 3; ++a)
            for (int j = 0; j < 3; ++j) M[3 * a + j] = R[3 * a + j] * s[j];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += M[3 * a + j] * M[3 * b + j];
                Sig[3 * a + b] = acc;
            }
        double z = p[2];
        double rx = p[0] / z, ry = p[1] / z;
        int clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
        double cxz = fmin(limx, fmax(-limx, rx)), cyz = fmin(limy, fmax(-limy, ry));
        double J[6] = {fx / z, 0, -fx * cxz / z, 0, fy / z, -fy * cyz / z};
        double T[6];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += J[3 * a + j] * Rc[3 * j + b];
                T[3 * a + b] = acc;
            }
        double S2[4];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0;
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k) acc += T[3 * a + j] * Sig[3 * j + k] * T[3 * b + k];
                S2[2 * a + b] = acc;
            }
        S2[0] += DILATION; S2[3] += DILATION;
        double s00 = S2[0], s01 = S2[1], s11 = S2[3];
        double det = s00 * s11 - s01 * s01;
        double NHL = -0.5 * LOG2E;

        /* record -> Sigma' (symmetric; off-diagonal gradient split evenly) */
        double dA2 = gr[2], dbeta = gr[3], dG2 = gr[4];
        double ds00 = dA2 * (-NHL * s11 * s11 / (det * det));
        double ds11 = dA2 * (-NHL * s01 * s01 / (det * det)) + dbeta * (s01 / (s11 * s11)) + dG2 * (-NHL / (s11 * s11));
        double ds01 = dA2 * (2.0 * NHL * s11 * s01 / (det * det)) + dbeta * (-1.0 / s11);
        double G[4] = {ds00, 0.5 * ds01, 0.5 * ds01, ds11};

        /* Sigma' = T Sig T^T: dSig = T^T G T, dT = 2 G T Sig */
        double dSig[9], dT[6], GT[6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int c = 0; c < 2; ++c)
                    for (int d = 0; d < 2; ++d) acc += T[3 * c + a] * G[2 * c + d] * T[3 * d + b];
                dSig[3 * a + b] = acc;
            }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int c = 0; c < 2; ++c) acc += G[2 * a + c] * T[3 * c + b];
                GT[3 * a + b] = acc;
            }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += GT[3 * a + k] * Sig[3 * k + b];
                dT[3 * a + b] = 2.0 * acc;
            }
        /* T = J W: dJ = dT W^T */
        double dJ[6];
        for (int a = 0; a < 2; ++a)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int b = 0; b < 3; ++b) acc += dT[3 * a + b] * Rc[3 * j + b];
                dJ[3 * a + j] = acc;
            }
        /* J(p): J00 = fx/z, J02 = -fx c_x/z, J11 = fy/z, J12 = -fy c_y/z,
         * c_x = clamp(x/z): dc_x/dx = 1/z, dc_x/dz = -x/z^2 when unclamped */
        double dp[3] = {0, 0, 0};
        double dcx = dJ[2] * (-fx / z), dcy = dJ[5] * (-fy / z);
        dp[2] += dJ[0] * (-fx / (z * z)) + dJ[2] * (fx * cxz / (z * z));
        dp[2] += dJ[4] * (-fy / (z * z)) + dJ[5] * (fy * cyz / (z * z));
        if (!clx) { dp[0] += dcx / z; dp[2] += dcx * (-p[0] / (z * z)); }
        if (!cly) { dp[1] += dcy / z; dp[2] += dcy * (-p[1] / (z * z)); }
        /* u = fx x/z + cx, v = fy y/z + cy */
        dp[0] += gr[0] * fx / z; dp[2] += -gr[0] * fx * p[0] / (z * z);
        dp[1] += gr[1] * fy / z; dp[2] += -gr[1] * fy * p[1] / (z * z);
        /* p = W mu + t */
        for (int j = 0; j < 3; ++j) dmu[j] += Rc[j] * dp[0] + Rc[3 + j] * dp[1] + Rc[6 + j] * dp[2];
        for (int j = 0; j < 3; ++j) d_means[3 * i + j] = dmu[j];

        /* Sig = M M^T: dM = (dSig + dSig^T) M;  M = R diag(s) */
        double dM[9];
        for (int a = 0; a < 3; ++a)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int b = 0; b < 3; ++b) acc += (dSig[3 * a + b] + dSig[3 * b + a]) * M[3 * b + j];
                dM[3 * a + j] = acc;
            }
        double dR[9];
        for (int j = 0; j < 3; ++j) {
            double ds = 0;
            for (int a = 0; a < 3; ++a) { ds += dM[3 * a + j] * R[3 * a + j]; dR[3 * a + j] = dM[3 * a + j] * s[j]; }
            d_log_scales[3 * i + j] = ds * s[j];
        }
        double Jq[4][9], dqn[4];
        quat_rot_jacobian(q, Jq);
        for (int k = 0; k < 4; ++k) {
            double acc = 0;
            for (int e = 0; e < 9; ++e) acc += dR[e] * Jq[k][e];
            dqn[k] = acc;
        }
        double qd = dqn[0] * q[0] + dqn[1] * q[1] + dqn[2] * q[2] + dqn[3] * q[3];
        for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = (dqn[k] - q[k] * qd) / qn;
    }
}

/* Contribution-based prune: keep[g] = contrib_max[g] >= threshold. */
int64_t or_prune(int64_t n, const double *contrib_max, double threshold, uint8_t *keep) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) { keep[i] = contrib_max[i] >= threshold; k += keep[i]; }
    return k;
}
