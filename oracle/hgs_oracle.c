/*
 * hgs_oracle.c -- plain, slow FP64 CPU oracle for the 3D half-Gaussian
 * splatting rasterizer (3D-HGS, CVPR 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only the tests, the package's smoke check and the bench's CPU-baseline leg
 * do.  It shares no code with the CUDA path.
 *
 * What it computes, step by step, in the paper's notation:
 *   Sec. 3.1, Eq. 2        Sigma^w = R S S^T R^T  (R from the unit quaternion)
 *   Sec. 3.1, Eq. 3        Sigma   = J W Sigma^w W^T J^T, J the affine Jacobian
 *   Sec. 3.1, Eq. 4-5      hat Sigma = top-left 2x2 block (+ the 3D-GS low-pass l*I)
 *   Sec. 3.2, Eq. 7-8 and Suppl. A.1
 *                          the half-Gaussian ray integral = 1/2 I(x,y) hat G, with
 *                          I/2 = Pr[n.(x-mu) >= 0 | pixel] computed coordinate-free:
 *                          P(d) = 1/2 erfc(-w.d / sqrt(2 v)),
 *                          k = M Sigma^w n, w = hat Sigma^-1 k, v = n^T Sigma^w n - k.w
 *   Sec. 3.3, Eq. 10       pair weight  (alpha2 + (alpha1 - alpha2) P) * hat G
 *   Sec. 3.1, Eq. 6 / Sec. 3.3 (blending with the pair weight)
 *                          front-to-back alpha compositing over the depth-sorted list
 * with the tile culling, 1/255 alpha floor, 0.99 alpha clamp and 1e-4
 * transmittance stop of the vanilla 3D-GS rasterizer that Sec. 4.1 says was
 * modified.  Binning decisions (which tiles a splat touches, its depth key)
 * are integers decided by floating point; they are taken in the same
 * canonical FP32 op sequence as the GPU (one IEEE binary32 op at a time,
 * round-to-nearest, no fused multiply-add; this file is compiled with
 * -ffp-contract=off).  Every continuous quantity is FP64.
 *
 * The adjoint (or_render_bwd / or_project_bwd) is the chain rule of the same
 * steps in reverse, by hand, in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double viewmat[12];   /* world -> camera, row-major 3x4 [R | t] */
    double fx, fy, cx, cy;
    int width, height;
    double near_plane;
    double bg[3];
} or_camera;

typedef struct {
    int tile_w, tile_h;
    int sh_degree;
    int fov_clamp;   /* 1: clamp x/z, y/z to +-1.3 tan(fov/2) inside J (3D-GS convention) */
    int plain;       /* 1: plain 3D-GS, alpha = alpha1 * hat G (P unused)           */
    int rect_mode;   /* 0: 3-sigma square of 3D-GS; 1: per-half 3-sigma extents (Sec. 3.4);
                        2: the same with the splitting edge from Algorithm 1's flattened
                        covariance (Suppl. B.1) instead of the exact cut ellipse */
    int mip;         /* 1: the low-pass is a mass-preserving 2D filter (Mip-Splatting-HGS):
                        both opacities scale by sqrt(det hat Sigma_0 / det hat Sigma)   */
    double lowpass;  /* l added to the diagonal of hat Sigma (3D-GS uses 0.3)        */
} or_opts;

enum { OR_CULLED = 0, OR_NORMAL = 1, OR_STEP = 2, OR_HALF = 3 };

#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_ALPHA_MAX 0.99
#define OR_T_MIN 1e-4

int or_abi_version(void) { return 8; }

/* Algorithm 1 (Suppl. B.1), step by step in binary64: the covariance `out` (3x3,
 * row-major) of the flattened ellipsoid that holds the cut of the Gaussian of
 * covariance Sigma (3x3, row-major) by the plane through its mean with normal n.
 * The basis (v1, v2, n^) has the plane's two directions first; in it, the in-plane
 * 2x2 block is the covariance given the normal coordinate (a', b', c'), and the third
 * axis keeps a variance of min(a', c') / 100; the result is rotated back. */
void or_alg1_flat_cov(const double *Sigma, const double *n, double *out) {
    double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double h[3] = {n[0] / nl, n[1] / nl, n[2] / nl};
    double v1[3], v2[3];
    if (h[0] == 0.0 && h[1] == 0.0) {
        v1[0] = 1.0; v1[1] = 0.0; v1[2] = 0.0;
        v2[0] = 0.0; v2[1] = 1.0; v2[2] = 0.0;
    } else {
        double l1 = sqrt(h[1] * h[1] + h[0] * h[0]);
        v1[0] = h[1] / l1; v1[1] = -h[0] / l1; v1[2] = 0.0;
        double c[3] = {h[1] * v1[2] - h[2] * v1[1], h[2] * v1[0] - h[0] * v1[2], h[0] * v1[1] - h[1] * v1[0]};
        double l2 = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        for (int i = 0; i < 3; ++i) v2[i] = c[i] / l2;
    }
    double B[3][3];                     /* columns v1, v2, n^ */
    for (int i = 0; i < 3; ++i) { B[i][0] = v1[i]; B[i][1] = v2[i]; B[i][2] = h[i]; }
    double SB[3][3], cov[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            SB[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) SB[i][j] += Sigma[3 * i + k] * B[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cov[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) cov[i][j] += B[k][i] * SB[k][j];
        }
    double ap = cov[0][0] - cov[0][2] * cov[0][2] / cov[2][2];
    double bp = cov[0][1] - cov[0][2] * cov[1][2] / cov[2][2];
    double cp = cov[1][1] - cov[1][2] * cov[1][2] / cov[2][2];
    double sl[3][3] = {{ap, bp, 0.0}, {bp, cp, 0.0}, {0.0, 0.0, fmin(ap, cp) / 100.0}};
    double T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) T[i][j] += B[i][k] * sl[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += T[i][k] * B[j][k];
            out[3 * i + j] = acc;
        }
}

/* Threads of the OpenMP loops (the CPU baseline times one core and all cores). */
void or_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Canonical FP32 binning fields.                                             */
/* Every line is one binary32 operation; the order is the specification.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int culled;
    float depth;        /* camera-space z of the mean: the sort key's low 32 bits */
    float mux, muy;     /* projected centre                                        */
    float a, b, c;      /* hat Sigma (with low-pass)                               */
    float radius;       /* ceil(3 sqrt(lambda_max))                                */
    int rect[4];        /* tile rect [x0,x1) x [y0,y1)                             */
    int tiles;
} canon_t;

static void canon_bin(const double *mean, const double *scale, const double *quat,
                      const double *normal, double op1, double op2,
                      const or_camera *cam, const or_opts *o, canon_t *out)
{
    float m0 = (float)mean[0], m1 = (float)mean[1], m2 = (float)mean[2];
    float s0 = (float)scale[0], s1 = (float)scale[1], s2 = (float)scale[2];
    float qw = (float)quat[0], qx = (float)quat[1], qy = (float)quat[2], qz = (float)quat[3];
    float V[12];
    for (int i = 0; i < 12; ++i) V[i] = (float)cam->viewmat[i];
    float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    float W = (float)cam->width, H = (float)cam->height;
    float lp = (float)o->lowpass;
    memset(out, 0, sizeof(*out));
    out->culled = 1;

    /* 1. unit quaternion */
    float n2 = qw * qw;
    n2 = n2 + qx * qx;
    n2 = n2 + qy * qy;
    n2 = n2 + qz * qz;
    float qn = sqrtf(n2);
    float iq = 1.0f / qn;
    float w = qw * iq, x = qx * iq, y = qy * iq, z = qz * iq;

    /* 2. rotation matrix */
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);

    /* 3. L = R diag(s) */
    float L[3][3];
    for (int i = 0; i < 3; ++i) {
        L[i][0] = R[i][0] * s0;
        L[i][1] = R[i][1] * s1;
        L[i][2] = R[i][2] * s2;
    }

    /* 4. camera-space mean */
    float t[3];
    for (int i = 0; i < 3; ++i) {
        float acc = V[4 * i + 0] * m0;
        acc = acc + V[4 * i + 1] * m1;
        acc = acc + V[4 * i + 2] * m2;
        t[i] = acc + V[4 * i + 3];
    }
    out->depth = t[2];

    /* 5. near-plane cull */
    if (!(t[2] > (float)cam->near_plane)) return;

    /* 6. clamped x/z, y/z */
    float iz = 1.0f / t[2];
    float ux = t[0] * iz, uy = t[1] * iz;
    float uxc = ux, uyc = uy;
    if (o->fov_clamp) {
        float limx = 1.3f * ((0.5f * W) / fx);
        float limy = 1.3f * ((0.5f * H) / fy);
        uxc = fminf(fmaxf(ux, -limx), limx);
        uyc = fminf(fmaxf(uy, -limy), limy);
    }

    /* 7. Jacobian entries */
    float j00 = fx * iz;
    float j02 = -((fx * uxc) * iz);
    float j11 = fy * iz;
    float j12 = -((fy * uyc) * iz);

    /* 8. M = J W_rot (2x3) */
    float M[2][3];
    for (int k = 0; k < 3; ++k) {
        M[0][k] = j00 * V[0 * 4 + k] + j02 * V[2 * 4 + k];
        M[1][k] = j11 * V[1 * 4 + k] + j12 * V[2 * 4 + k];
    }

    /* 9. P = M L (2x3) */
    float P[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            float acc = M[i][0] * L[0][k];
            acc = acc + M[i][1] * L[1][k];
            P[i][k] = acc + M[i][2] * L[2][k];
        }

    /* 10. hat Sigma = P P^T + l I  (A0, C0: the diagonal before the low-pass) */
    float A0 = P[0][0] * P[0][0];
    A0 = A0 + P[0][1] * P[0][1];
    A0 = A0 + P[0][2] * P[0][2];
    float a = A0 + lp;
    float b = P[0][0] * P[1][0];
    b = b + P[0][1] * P[1][1];
    b = b + P[0][2] * P[1][2];
    float C0 = P[1][0] * P[1][0];
    C0 = C0 + P[1][1] * P[1][1];
    C0 = C0 + P[1][2] * P[1][2];
    float c = C0 + lp;
    out->a = a; out->b = b; out->c = c;

    /* 11. determinant cull */
    float det = a * c - b * b;
    if (!(det > 0.0f)) return;

    /* 12. 3-sigma radius from the larger eigenvalue */
    float mid = 0.5f * (a + c);
    float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    float r = ceilf(3.0f * sqrtf(lam));

    /* 13. projected centre */
    float mux = fx * ux + cx;
    float muy = fy * uy + cy;
    out->mux = mux; out->muy = muy; out->radius = r;

    /* 14. finiteness cull */
    if (!(isfinite(mux) && isfinite(muy) && isfinite(r))) return;

    /* 15. extents towards -x, +x, -y, +y: the 3-sigma radius r (3D-GS), or per half */
    float ex0 = r, ex1 = r, ey0 = r, ey1 = r;
    if (o->rect_mode == 1 || o->rect_mode == 2) {
        /* 15a. Support of the 3-sigma half-ellipsoid {|L^-1 (x - mu)| <= 3, n.(x - mu) >= 0}
         * under the affine projection M, in direction e (1-sigma, without the low-pass):
         * sqrt(e^T P P^T e) if the whole ellipsoid's extreme point in that direction lies on
         * the kept side (sign of k.e, k = P L^T n^), else the same for the cut ellipse of
         * the splitting plane, e^T P P^T e - (k.e)^2 / |L^T n^|^2.                       */
        float K0 = 0.0f, K1 = 0.0f, Ar = A0, Cr = C0;
        float nx = (float)normal[0], ny = (float)normal[1], nz = (float)normal[2];
        float nn = nx * nx;
        nn = nn + ny * ny;
        nn = nn + nz * nz;
        if (nn >= 1e-24f) {
            float nl = sqrtf(nn);
            float h0 = nx / nl, h1 = ny / nl, h2 = nz / nl;
            float u[3];
            for (int k = 0; k < 3; ++k) {
                float acc = L[0][k] * h0;
                acc = acc + L[1][k] * h1;
                u[k] = acc + L[2][k] * h2;
            }
            float vs = u[0] * u[0];
            vs = vs + u[1] * u[1];
            vs = vs + u[2] * u[2];
            K0 = P[0][0] * u[0];
            K0 = K0 + P[0][1] * u[1];
            K0 = K0 + P[0][2] * u[2];
            K1 = P[1][0] * u[0];
            K1 = K1 + P[1][1] * u[1];
            K1 = K1 + P[1][2] * u[2];
            if (vs > 0.0f && o->rect_mode == 1) {
                Ar = fmaxf(0.0f, A0 - (K0 * K0) / vs);
                Cr = fmaxf(0.0f, C0 - (K1 * K1) / vs);
            } else if (vs > 0.0f) {
                /* 15a'. Algorithm 1 (Suppl. B.1) in binary32: basis (v1, v2, n^) of the
                 * splitting plane, the covariance in that basis from the rows L^T v1,
                 * L^T v2, L^T n^ (= u), the in-plane covariance given the normal
                 * coordinate (a', b', c'), a third variance min(a', c') / 100 along n^,
                 * and the projection M sigma M^T of the resulting flattened covariance,
                 * whose diagonal replaces the cut ellipse's (Ar, Cr).                    */
                float v1[3], v2[3];
                if (h0 == 0.0f && h1 == 0.0f) {
                    v1[0] = 1.0f; v1[1] = 0.0f; v1[2] = 0.0f;
                    v2[0] = 0.0f; v2[1] = 1.0f; v2[2] = 0.0f;
                } else {
                    float l1 = h1 * h1;
                    l1 = l1 + h0 * h0;
                    l1 = sqrtf(l1);
                    v1[0] = h1 / l1; v1[1] = -(h0 / l1); v1[2] = 0.0f;
                    float c0 = -(h2 * v1[1]);             /* n^ x v1 with v1[2] = 0 */
                    float c1 = h2 * v1[0];
                    float c2 = h0 * v1[1];
                    c2 = c2 - h1 * v1[0];
                    float l2 = c0 * c0;
                    l2 = l2 + c1 * c1;
                    l2 = l2 + c2 * c2;
                    l2 = sqrtf(l2);
                    v2[0] = c0 / l2; v2[1] = c1 / l2; v2[2] = c2 / l2;
                }
                float g1[3], g2[3];
                for (int k = 0; k < 3; ++k) {
                    float acc = L[0][k] * v1[0];
                    acc = acc + L[1][k] * v1[1];
                    g1[k] = acc + L[2][k] * v1[2];
                    acc = L[0][k] * v2[0];
                    acc = acc + L[1][k] * v2[1];
                    g2[k] = acc + L[2][k] * v2[2];
                }
                float s00 = g1[0] * g1[0], s01 = g1[0] * g2[0], s11 = g2[0] * g2[0];
                float s02 = g1[0] * u[0], s12 = g2[0] * u[0];
                for (int k = 1; k < 3; ++k) {
                    s00 = s00 + g1[k] * g1[k];
                    s01 = s01 + g1[k] * g2[k];
                    s11 = s11 + g2[k] * g2[k];
                    s02 = s02 + g1[k] * u[k];
                    s12 = s12 + g2[k] * u[k];
                }
                float ap = s00 - (s02 * s02) / vs;
                float bp = s01 - (s02 * s12) / vs;
                float cp = s11 - (s12 * s12) / vs;
                float tt = fminf(ap, cp) / 100.0f;
                float q[2][3];
                for (int i = 0; i < 2; ++i) {
                    float acc = M[i][0] * v1[0];
                    acc = acc + M[i][1] * v1[1];
                    q[i][0] = acc + M[i][2] * v1[2];
                    acc = M[i][0] * v2[0];
                    acc = acc + M[i][1] * v2[1];
                    q[i][1] = acc + M[i][2] * v2[2];
                    acc = M[i][0] * h0;
                    acc = acc + M[i][1] * h1;
                    q[i][2] = acc + M[i][2] * h2;
                }
                float As = ap * (q[0][0] * q[0][0]);
                As = As + (2.0f * bp) * (q[0][0] * q[0][1]);
                As = As + cp * (q[0][1] * q[0][1]);
                As = As + tt * (q[0][2] * q[0][2]);
                float Cs = ap * (q[1][0] * q[1][0]);
                Cs = Cs + (2.0f * bp) * (q[1][0] * q[1][1]);
                Cs = Cs + cp * (q[1][1] * q[1][1]);
                Cs = Cs + tt * (q[1][2] * q[1][2]);
                Ar = fmaxf(0.0f, As);
                Cr = fmaxf(0.0f, Cs);
            }
        }
        /* 15b. a half is splatted when its opacity reaches the 1/255 floor (as binary32) */
        float amin = (float)(1.0 / 255.0);
        int keep1 = (float)op1 >= amin, keep2 = (float)op2 >= amin;
        if (!keep1 && !keep2) return;
        float hxp = 0.0f, hxm = 0.0f, hyp = 0.0f, hym = 0.0f;
        if (keep1) {          /* side n.(x - mu) >= 0 */
            hxp = fmaxf(hxp, K0 >= 0.0f ? A0 : Ar);
            hxm = fmaxf(hxm, K0 <= 0.0f ? A0 : Ar);
            hyp = fmaxf(hyp, K1 >= 0.0f ? C0 : Cr);
            hym = fmaxf(hym, K1 <= 0.0f ? C0 : Cr);
        }
        if (keep2) {          /* side n.(x - mu) <= 0 */
            hxp = fmaxf(hxp, K0 <= 0.0f ? A0 : Ar);
            hxm = fmaxf(hxm, K0 >= 0.0f ? A0 : Ar);
            hyp = fmaxf(hyp, K1 <= 0.0f ? C0 : Cr);
            hym = fmaxf(hym, K1 >= 0.0f ? C0 : Cr);
        }
        /* 15c. 3-sigma extents with the low-pass added in quadrature */
        ex1 = 3.0f * sqrtf(hxp + lp);
        ex0 = 3.0f * sqrtf(hxm + lp);
        ey1 = 3.0f * sqrtf(hyp + lp);
        ey0 = 3.0f * sqrtf(hym + lp);
        if (!(isfinite(ex0) && isfinite(ex1) && isfinite(ey0) && isfinite(ey1))) return;
    }

    /* 16. tile rect, clamped to the grid */
    int tiles_x = (cam->width + o->tile_w - 1) / o->tile_w;
    int tiles_y = (cam->height + o->tile_h - 1) / o->tile_h;
    float tw = (float)o->tile_w, th = (float)o->tile_h;
    float fx0 = floorf((mux - ex0) / tw);
    float fx1 = floorf((mux + ex1) / tw) + 1.0f;
    float fy0 = floorf((muy - ey0) / th);
    float fy1 = floorf((muy + ey1) / th) + 1.0f;
    fx0 = fminf(fmaxf(fx0, 0.0f), (float)tiles_x);
    fx1 = fminf(fmaxf(fx1, 0.0f), (float)tiles_x);
    fy0 = fminf(fmaxf(fy0, 0.0f), (float)tiles_y);
    fy1 = fminf(fmaxf(fy1, 0.0f), (float)tiles_y);
    out->rect[0] = (int)fx0; out->rect[1] = (int)fy0;
    out->rect[2] = (int)fx1; out->rect[3] = (int)fy1;
    int nx = out->rect[2] - out->rect[0], ny = out->rect[3] - out->rect[1];
    out->tiles = (nx > 0 && ny > 0) ? nx * ny : 0;
    out->culled = 0;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3, as Cartesian polynomials of the     */
/* unit direction (x,y,z).  Convention: Y_l^m complex with the Condon-Shortley */
/* phase; real basis sqrt2 Im Y_l^|m| for m<0, Y_l^0, sqrt2 Re Y_l^m for m>0; */
/* index l*l + l + m.                                                         */
/* ------------------------------------------------------------------------ */
static void sh_basis(int deg, const double d[3], double Y[16], double dY[16][3])
{
    const double x = d[0], y = d[1], z = d[2];
    const double PI = 3.14159265358979323846;
    for (int i = 0; i < 16; ++i) { Y[i] = 0; dY[i][0] = dY[i][1] = dY[i][2] = 0; }
    double k00 = 0.5 * sqrt(1.0 / PI);
    Y[0] = k00;
    if (deg < 1) return;
    double k1 = sqrt(3.0 / (4.0 * PI));
    Y[1] = -k1 * y; dY[1][1] = -k1;
    Y[2] = k1 * z;  dY[2][2] = k1;
    Y[3] = -k1 * x; dY[3][0] = -k1;
    if (deg < 2) return;
    double k2a = 0.5 * sqrt(15.0 / PI);      /* xy, yz, xz terms */
    double k2b = 0.25 * sqrt(5.0 / PI);      /* 3z^2 - 1 = 2z^2 - x^2 - y^2 */
    double k2c = 0.25 * sqrt(15.0 / PI);     /* x^2 - y^2 */
    Y[4] = k2a * x * y;          dY[4][0] = k2a * y; dY[4][1] = k2a * x;
    Y[5] = -k2a * y * z;         dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
    Y[6] = k2b * (2 * z * z - x * x - y * y);
    dY[6][0] = -2 * k2b * x; dY[6][1] = -2 * k2b * y; dY[6][2] = 4 * k2b * z;
    Y[7] = -k2a * x * z;         dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
    Y[8] = k2c * (x * x - y * y); dY[8][0] = 2 * k2c * x; dY[8][1] = -2 * k2c * y;
    if (deg < 3) return;
    double k3a = 0.125 * sqrt(70.0 / PI);    /* m = +-3 */
    double k3b = 0.5 * sqrt(105.0 / PI);     /* m = -2 : xyz */
    double k3c = 0.125 * sqrt(42.0 / PI);    /* m = +-1 */
    double k3d = 0.25 * sqrt(7.0 / PI);      /* m = 0  */
    double k3e = 0.25 * sqrt(105.0 / PI);    /* m = +2 */
    /* m=-3: -k3a * y (3x^2 - y^2) */
    Y[9] = -k3a * y * (3 * x * x - y * y);
    dY[9][0] = -k3a * 6 * x * y; dY[9][1] = -k3a * (3 * x * x - 3 * y * y);
    /* m=-2: k3b xyz */
    Y[10] = k3b * x * y * z;
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    /* m=-1: -k3c y (4z^2 - x^2 - y^2) */
    Y[11] = -k3c * y * (4 * z * z - x * x - y * y);
    dY[11][0] = -k3c * (-2 * x * y);
    dY[11][1] = -k3c * (4 * z * z - x * x - 3 * y * y);
    dY[11][2] = -k3c * (8 * y * z);
    /* m=0: k3d z (2z^2 - 3x^2 - 3y^2) */
    Y[12] = k3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    dY[12][0] = k3d * (-6 * x * z); dY[12][1] = k3d * (-6 * y * z);
    dY[12][2] = k3d * (6 * z * z - 3 * x * x - 3 * y * y);
    /* m=1: -k3c x (4z^2 - x^2 - y^2) */
    Y[13] = -k3c * x * (4 * z * z - x * x - y * y);
    dY[13][0] = -k3c * (4 * z * z - 3 * x * x - y * y);
    dY[13][1] = -k3c * (-2 * x * y);
    dY[13][2] = -k3c * (8 * x * z);
    /* m=2: k3e z (x^2 - y^2) */
    Y[14] = k3e * z * (x * x - y * y);
    dY[14][0] = k3e * 2 * x * z; dY[14][1] = -k3e * 2 * y * z; dY[14][2] = k3e * (x * x - y * y);
    /* m=3: -k3a x (x^2 - 3y^2) */
    Y[15] = -k3a * x * (x * x - 3 * y * y);
    dY[15][0] = -k3a * (3 * x * x - 3 * y * y); dY[15][1] = -k3a * (-6 * x * y);
}

/* exported for the SH pin test */
void or_sh_eval(int deg, int n, const double *dirs, double *Y /* [n,16] */)
{
    double dY[16][3];
    for (int i = 0; i < n; ++i) sh_basis(deg, dirs + 3 * i, Y + 16 * i, dY);
}

/* ------------------------------------------------------------------------ */
/* FP64 projection of one splat for one camera.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int mode;
    double q[4], qn, qh[4];
    double R[3][3], Sw[3][3];
    double t[3];
    int clampx, clampy;
    double uxc, uyc;
    double J00, J02, J11, J12;
    double M[2][3];
    double S0[3];           /* M Sigma^w M^T (before the low-pass) */
    double det0, comp;      /* its determinant; opacity factor (1 unless mip) */
    double S2[3];           /* hat Sigma a, b, c  */
    double det, Q[3];       /* conic A, B, C      */
    double mu2[2];
    double nn, nh[3];
    double var_s, k[2], w[2], v, wp[2];
    double campos[3], dvec[3], dnorm, dir[3];
    double Y[16], dY[16][3];
    double rgb_raw[3], rgb[3];
} fwd_t;

static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static void project_fp64(const double *mean, const double *scale, const double *quat,
                         const double *normal, const double *sh, int sh_deg,
                         const or_camera *cam, const or_opts *o, fwd_t *f)
{
    const double *V = cam->viewmat;
    double Rc[3][3] = {{V[0], V[1], V[2]}, {V[4], V[5], V[6]}, {V[8], V[9], V[10]}};
    double tc[3] = {V[3], V[7], V[11]};

    /* Eq. 2: Sigma^w = R S S^T R^T */
    for (int i = 0; i < 4; ++i) f->q[i] = quat[i];
    f->qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    for (int i = 0; i < 4; ++i) f->qh[i] = quat[i] / f->qn;
    quat_to_rot(f->qh, f->R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->R[i][k] * scale[k] * scale[k] * f->R[j][k];
            f->Sw[i][j] = acc;
        }

    /* viewing transformation W */
    for (int i = 0; i < 3; ++i)
        f->t[i] = Rc[i][0] * mean[0] + Rc[i][1] * mean[1] + Rc[i][2] * mean[2] + tc[i];
    double tz = f->t[2];

    /* Eq. 3: affine Jacobian J of the perspective map at t (3D-GS clamps x/z, y/z) */
    double ux = f->t[0] / tz, uy = f->t[1] / tz;
    f->uxc = ux; f->uyc = uy; f->clampx = f->clampy = 0;
    if (o->fov_clamp) {
        double limx = 1.3 * (0.5 * cam->width / cam->fx);
        double limy = 1.3 * (0.5 * cam->height / cam->fy);
        if (ux > limx) { f->uxc = limx; f->clampx = 1; }
        if (ux < -limx) { f->uxc = -limx; f->clampx = 1; }
        if (uy > limy) { f->uyc = limy; f->clampy = 1; }
        if (uy < -limy) { f->uyc = -limy; f->clampy = 1; }
    }
    f->J00 = cam->fx / tz; f->J02 = -cam->fx * f->uxc / tz;
    f->J11 = cam->fy / tz; f->J12 = -cam->fy * f->uyc / tz;
    for (int k = 0; k < 3; ++k) {
        f->M[0][k] = f->J00 * Rc[0][k] + f->J02 * Rc[2][k];
        f->M[1][k] = f->J11 * Rc[1][k] + f->J12 * Rc[2][k];
    }

    /* Eq. 4-5: hat Sigma = (M Sigma^w M^T) top-left block, plus the low-pass */
    double MS[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            MS[i][j] = f->M[i][0] * f->Sw[0][j] + f->M[i][1] * f->Sw[1][j] + f->M[i][2] * f->Sw[2][j];
    double S00 = MS[0][0] * f->M[0][0] + MS[0][1] * f->M[0][1] + MS[0][2] * f->M[0][2];
    double S01 = MS[0][0] * f->M[1][0] + MS[0][1] * f->M[1][1] + MS[0][2] * f->M[1][2];
    double S11 = MS[1][0] * f->M[1][0] + MS[1][1] * f->M[1][1] + MS[1][2] * f->M[1][2];
    f->S2[0] = S00 + o->lowpass; f->S2[1] = S01; f->S2[2] = S11 + o->lowpass;
    f->det = f->S2[0] * f->S2[2] - f->S2[1] * f->S2[1];
    f->Q[0] = f->S2[2] / f->det; f->Q[1] = -f->S2[1] / f->det; f->Q[2] = f->S2[0] / f->det;
    /* Mip-Splatting's 2D filter: convolving alpha hat G_0 with the normalised N(0, l I)
       gives sqrt(det hat Sigma_0 / det hat Sigma) alpha hat G, the same total mass; by
       the reading of the low-pass on the half-footprint (total probability) the
       half-Gaussian weight carries the same factor on both opacities. */
    f->S0[0] = S00; f->S0[1] = S01; f->S0[2] = S11;
    f->det0 = S00 * S11 - S01 * S01;
    f->comp = 1.0;
    if (o->mip) f->comp = f->det0 > 0 ? sqrt(f->det0 / f->det) : 0.0;

    /* projected centre */
    f->mu2[0] = cam->fx * f->t[0] / tz + cam->cx;
    f->mu2[1] = cam->fy * f->t[1] / tz + cam->cy;

    /* Eq. 7-8: conditional law of s = n.(x - mu) given the pixel offset */
    f->nn = sqrt(normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2]);
    f->mode = OR_NORMAL;
    f->wp[0] = f->wp[1] = 0; f->w[0] = f->w[1] = 0; f->k[0] = f->k[1] = 0; f->v = 0; f->var_s = 0;
    if (f->nn < 1e-12) {
        f->mode = OR_HALF;
        f->nh[0] = f->nh[1] = f->nh[2] = 0;
    } else {
        for (int i = 0; i < 3; ++i) f->nh[i] = normal[i] / f->nn;
        double Sn[3];
        for (int i = 0; i < 3; ++i)
            Sn[i] = f->Sw[i][0] * f->nh[0] + f->Sw[i][1] * f->nh[1] + f->Sw[i][2] * f->nh[2];
        f->var_s = f->nh[0] * Sn[0] + f->nh[1] * Sn[1] + f->nh[2] * Sn[2];
        for (int i = 0; i < 2; ++i) f->k[i] = f->M[i][0] * Sn[0] + f->M[i][1] * Sn[1] + f->M[i][2] * Sn[2];
        f->w[0] = f->Q[0] * f->k[0] + f->Q[1] * f->k[1];
        f->w[1] = f->Q[1] * f->k[0] + f->Q[2] * f->k[1];
        f->v = f->var_s - (f->k[0] * f->w[0] + f->k[1] * f->w[1]);
        if (f->v <= 1e-12 * f->var_s) {
            f->mode = OR_STEP;
        } else {
            double s = 1.0 / sqrt(2.0 * f->v);
            f->wp[0] = f->w[0] * s; f->wp[1] = f->w[1] * s;
        }
    }

    /* view-dependent colour from SH (3D-GS prior art, Sec. 3.1) */
    for (int i = 0; i < 3; ++i)
        f->campos[i] = -(Rc[0][i] * tc[0] + Rc[1][i] * tc[1] + Rc[2][i] * tc[2]);
    for (int i = 0; i < 3; ++i) f->dvec[i] = mean[i] - f->campos[i];
    f->dnorm = sqrt(f->dvec[0] * f->dvec[0] + f->dvec[1] * f->dvec[1] + f->dvec[2] * f->dvec[2]);
    for (int i = 0; i < 3; ++i) f->dir[i] = f->dvec[i] / f->dnorm;
    sh_basis(sh_deg, f->dir, f->Y, f->dY);
    int nc = (sh_deg + 1) * (sh_deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0;
        for (int l = 0; l < nc; ++l) acc += sh[3 * l + ch] * f->Y[l];
        f->rgb_raw[ch] = acc + 0.5;
        f->rgb[ch] = f->rgb_raw[ch] < 0 ? 0 : f->rgb_raw[ch];
    }
}

/* P(d): Pr[n.(x-mu) >= 0 | pixel offset d]  (the paper's I(x,y)/2) */
static double half_fraction(const fwd_t *f, double dx, double dy, double *margin)
{
    if (f->mode == OR_HALF) return 0.5;
    if (f->mode == OR_STEP) {
        double z = f->w[0] * dx + f->w[1] * dy;
        double scale = (fabs(f->w[0]) + fabs(f->w[1])) * (fabs(dx) + fabs(dy)) + 1e-300;
        if (margin) { double m = fabs(z) / scale; if (m < *margin) *margin = m; }
        return z > 0 ? 1.0 : (z < 0 ? 0.0 : 0.5);
    }
    return 0.5 * erfc(-(f->wp[0] * dx + f->wp[1] * dy));
}

/* ------------------------------------------------------------------------ */
/* FP32 error model: how far a binary32 evaluation of the pair weight can      */
/* be from the FP64 value.  It decides which threshold decisions of the       */
/* compositing (1/255 floor, 0.99 clamp, 1e-4 stop, step sign) a binary32     */
/* implementation cannot be expected to reproduce (reading B15).              */
/*                                                                            */
/* Shape part.  The screen-space shape terms y = (conic A, B, C, w'x, w'y)    */
/* are modelled as computed backward-stably: the binary32 result is the exact */
/* result for inputs each perturbed by a relative amount of the order of the  */
/* unit roundoff.  The inputs are the 22 values that enter the shape: the     */
/* camera-space mean t (3), the camera rotation (9), the scales (3), the raw  */
/* quaternion (4) and the raw normal (3).  For each input x_k the vector      */
/* v_k = |x_k| dy/dx_k (central differences in FP64) is the change of y per   */
/* unit relative perturbation; E = sum_k v_k v_k^T combines the 22 as         */
/* independent rounding errors (root-sum-square).  Splats whose plane nearly  */
/* contains the ray (v < 1e-3 var_s) have their w' computed in FP64 by a      */
/* binary32 implementation of this design, so only the final rounding of w'   */
/* enters there.                                                              */
/* ------------------------------------------------------------------------ */
#define OR_ERR_DIRS 22
#define OR_U32 5.9604644775390625e-8     /* 2^-24: unit roundoff of binary32       */
#define OR_FP64_GATE 1e-3                /* v / var_s below which w' is FP64       */

/* y = (A, B, C, w'x, w'y) from the inputs x (layout of error_basis_one); returns the
 * mode and writes v / var_s (0 when there is no normal). */
static int shape_terms(const double x[OR_ERR_DIRS], const or_camera *cam, const or_opts *o,
                       double y[5], double *vrel)
{
    const double *t = x, *Rcf = x + 3, *scale = x + 12, *quat = x + 15, *normal = x + 19;
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double qh[4] = {quat[0] / qn, quat[1] / qn, quat[2] / qn, quat[3] / qn};
    double R[3][3], Sw[3][3];
    quat_to_rot(qh, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[i][k] * scale[k] * scale[k] * R[j][k];
            Sw[i][j] = acc;
        }
    double tz = t[2];
    double uxc = t[0] / tz, uyc = t[1] / tz;
    if (o->fov_clamp) {
        double limx = 1.3 * (0.5 * cam->width / cam->fx);
        double limy = 1.3 * (0.5 * cam->height / cam->fy);
        uxc = fmin(fmax(uxc, -limx), limx);
        uyc = fmin(fmax(uyc, -limy), limy);
    }
    double J00 = cam->fx / tz, J02 = -cam->fx * uxc / tz, J11 = cam->fy / tz, J12 = -cam->fy * uyc / tz;
    double M[2][3];
    for (int k = 0; k < 3; ++k) {
        M[0][k] = J00 * Rcf[k] + J02 * Rcf[6 + k];
        M[1][k] = J11 * Rcf[3 + k] + J12 * Rcf[6 + k];
    }
    double MS[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) MS[i][j] = M[i][0] * Sw[0][j] + M[i][1] * Sw[1][j] + M[i][2] * Sw[2][j];
    double a = MS[0][0] * M[0][0] + MS[0][1] * M[0][1] + MS[0][2] * M[0][2] + o->lowpass;
    double b = MS[0][0] * M[1][0] + MS[0][1] * M[1][1] + MS[0][2] * M[1][2];
    double c = MS[1][0] * M[1][0] + MS[1][1] * M[1][1] + MS[1][2] * M[1][2] + o->lowpass;
    double det = a * c - b * b;
    y[0] = c / det; y[1] = -b / det; y[2] = a / det;
    y[3] = y[4] = 0.0;
    *vrel = 0.0;
    double nn = sqrt(normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2]);
    if (nn < 1e-12) return OR_HALF;
    double nh[3] = {normal[0] / nn, normal[1] / nn, normal[2] / nn}, Sn[3];
    for (int i = 0; i < 3; ++i) Sn[i] = Sw[i][0] * nh[0] + Sw[i][1] * nh[1] + Sw[i][2] * nh[2];
    double var_s = nh[0] * Sn[0] + nh[1] * Sn[1] + nh[2] * Sn[2];
    double k0 = M[0][0] * Sn[0] + M[0][1] * Sn[1] + M[0][2] * Sn[2];
    double k1 = M[1][0] * Sn[0] + M[1][1] * Sn[1] + M[1][2] * Sn[2];
    double w0 = y[0] * k0 + y[1] * k1, w1 = y[1] * k0 + y[2] * k1;
    double v = var_s - (k0 * w0 + k1 * w1);
    *vrel = var_s > 0 ? v / var_s : 0.0;
    if (v <= 1e-12 * var_s) return OR_STEP;
    double sc = 1.0 / sqrt(2.0 * v);
    y[3] = w0 * sc; y[4] = w1 * sc;
    return OR_NORMAL;
}

/* The 22 unit-perturbation vectors v_k of one splat (V, optional) and E = sum v v^T
 * (upper triangle, row by row: 00 01 02 03 04 11 12 13 14 22 23 24 33 34 44). */
static void error_basis_one(const double *mean, const double *scale, const double *quat,
                            const double *normal, const or_camera *cam, const or_opts *o,
                            double V[OR_ERR_DIRS][5], double E[15])
{
    const double *W = cam->viewmat;
    double x[OR_ERR_DIRS];
    for (int i = 0; i < 3; ++i) x[i] = W[4 * i] * mean[0] + W[4 * i + 1] * mean[1] + W[4 * i + 2] * mean[2] + W[4 * i + 3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) x[3 + 3 * i + j] = W[4 * i + j];
    for (int k = 0; k < 3; ++k) x[12 + k] = scale[k];
    for (int k = 0; k < 4; ++k) x[15 + k] = quat[k];
    for (int k = 0; k < 3; ++k) x[19 + k] = normal[k];
    double y0[5], vrel0, Vl[OR_ERR_DIRS][5];
    int mode0 = shape_terms(x, cam, o, y0, &vrel0);
    int fp64_w = mode0 != OR_NORMAL || vrel0 < OR_FP64_GATE;
    for (int k = 0; k < OR_ERR_DIRS; ++k) {
        for (int j = 0; j < 5; ++j) Vl[k][j] = 0.0;
        if (x[k] == 0.0) continue;                 /* an exact zero stays exact */
        double h = 1e-6 * fabs(x[k]), xp[OR_ERR_DIRS], xm[OR_ERR_DIRS], yp[5], ym[5], vr;
        memcpy(xp, x, sizeof(x));
        memcpy(xm, x, sizeof(x));
        xp[k] += h;
        xm[k] -= h;
        shape_terms(xp, cam, o, yp, &vr);
        shape_terms(xm, cam, o, ym, &vr);
        for (int j = 0; j < (fp64_w ? 3 : 5); ++j) Vl[k][j] = (yp[j] - ym[j]) / (2.0 * h) * fabs(x[k]);
    }
    int q = 0;
    for (int a = 0; a < 5; ++a)
        for (int b = a; b < 5; ++b) {
            double acc = 0;
            for (int k = 0; k < OR_ERR_DIRS; ++k) acc += Vl[k][a] * Vl[k][b];
            /* FP64 w' (gathered splats): its final rounding to binary32 only */
            if (fp64_w && mode0 == OR_NORMAL && a >= 3 && b >= 3) acc += y0[a] * y0[b];
            E[q++] = acc;
        }
    if (V) memcpy(V, Vl, sizeof(Vl));
}

/* E [n,15] for the splats with sel[i] != 0 (all when sel is NULL) that project (mode
 * != OR_CULLED); zero rows elsewhere.  V (optional) [n,22,5]. */
int or_error_basis(int n, const double *means, const double *scales, const double *quats,
                   const double *normals, const or_camera *cam, const or_opts *o, const int *mode,
                   const unsigned char *sel, double *E, double *V)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < n; ++i) {
        double *Ei = E + 15 * (size_t)i;
        for (int j = 0; j < 15; ++j) Ei[j] = 0.0;
        if (V) for (int j = 0; j < OR_ERR_DIRS * 5; ++j) V[(size_t)i * OR_ERR_DIRS * 5 + j] = 0.0;
        if ((sel && !sel[i]) || mode[i] == OR_CULLED) continue;
        error_basis_one(means + 3 * i, scales + 3 * i, quats + 4 * i, normals + 3 * i, cam, o,
                        V ? (double (*)[5])(V + (size_t)i * OR_ERR_DIRS * 5) : NULL, Ei);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Projection of all splats: canonical binning fields + FP64 continuous ones. */
/* ------------------------------------------------------------------------ */
int or_project(int n, const double *means, const double *scales, const double *quats,
               const double *normals, const double *sh, const double *op1, const double *op2,
               const or_camera *cam, const or_opts *o,
               int *mode, float *depth, float *radius, int *rect, int *tiles,
               float *canon_abc, float *canon_mu,
               double *mu2, double *conic, double *wp, double *rgb, double *var_terms, double *comp)
{
    int nc = (o->sh_degree + 1) * (o->sh_degree + 1);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        canon_t cb;
        canon_bin(means + 3 * i, scales + 3 * i, quats + 4 * i, normals + 3 * i, op1[i], op2[i], cam, o, &cb);
        depth[i] = cb.depth;
        radius[i] = cb.radius;
        for (int j = 0; j < 4; ++j) rect[4 * i + j] = cb.rect[j];
        tiles[i] = cb.culled ? 0 : cb.tiles;
        canon_abc[3 * i] = cb.a; canon_abc[3 * i + 1] = cb.b; canon_abc[3 * i + 2] = cb.c;
        canon_mu[2 * i] = cb.mux; canon_mu[2 * i + 1] = cb.muy;
        if (cb.culled) {
            mode[i] = OR_CULLED;
            continue;
        }
        fwd_t f;
        project_fp64(means + 3 * i, scales + 3 * i, quats + 4 * i, normals + 3 * i,
                     sh + 3 * nc * i, o->sh_degree, cam, o, &f);
        mode[i] = f.mode;
        if (!(f.det > 0)) mode[i] = OR_CULLED;   /* FP64 singular although FP32 was not */
        mu2[2 * i] = f.mu2[0]; mu2[2 * i + 1] = f.mu2[1];
        for (int j = 0; j < 3; ++j) conic[3 * i + j] = f.Q[j];
        wp[2 * i] = f.wp[0]; wp[2 * i + 1] = f.wp[1];
        if (f.mode == OR_STEP) { wp[2 * i] = f.w[0]; wp[2 * i + 1] = f.w[1]; }
        for (int j = 0; j < 3; ++j) rgb[3 * i + j] = f.rgb[j];
        if (var_terms) { var_terms[2 * i] = f.var_s; var_terms[2 * i + 1] = f.v; }
        if (comp) comp[i] = f.comp;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Binning: (tile | depth bits) keys, brute-force lexicographic sort.        */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t id; } pair_t;

static int pair_cmp(const void *pa, const void *pb)
{
    const pair_t *a = (const pair_t *)pa, *b = (const pair_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

static uint32_t float_bits(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
}

/* Returns the pair count; writes keys/ids/ranges only if it fits in `cap`.
 * tile_mask (optional, [tiles]) restricts the emitted pairs to masked tiles;
 * the returned count is then still the full count.                          */
long or_bin(int n, const int *tiles, const int *rect, const float *depth, int tiles_x,
            int n_tiles, const unsigned char *tile_mask, long cap,
            uint64_t *keys, uint32_t *ids, uint32_t *ranges, long *n_emitted)
{
    long total = 0, emit = 0;
    for (int i = 0; i < n; ++i) {
        total += tiles[i];
        if (tiles[i] == 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx)
                if (!tile_mask || tile_mask[ty * tiles_x + tx]) emit++;
    }
    if (n_emitted) *n_emitted = emit;
    if (emit > cap) return total;
    pair_t *pairs = (pair_t *)malloc(sizeof(pair_t) * (emit > 0 ? emit : 1));
    long p = 0;
    for (int i = 0; i < n; ++i) {
        if (tiles[i] == 0) continue;
        uint32_t db = float_bits(depth[i]);
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx) {
                uint64_t tile = (uint64_t)(ty * tiles_x + tx);
                if (tile_mask && !tile_mask[tile]) continue;
                pairs[p].key = (tile << 32) | (uint64_t)db;
                pairs[p].id = (uint32_t)i;
                p++;
            }
    }
    qsort(pairs, (size_t)emit, sizeof(pair_t), pair_cmp);
    for (long j = 0; j < 2L * n_tiles; ++j) ranges[j] = 0;
    for (long j = 0; j < emit; ++j) {
        keys[j] = pairs[j].key;
        ids[j] = pairs[j].id;
        uint32_t tile = (uint32_t)(pairs[j].key >> 32);
        if (j == 0 || (uint32_t)(pairs[j - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)j;
        if (j == emit - 1 || (uint32_t)(pairs[j + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(j + 1);
    }
    free(pairs);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Compositing (Eq. 10 inside front-to-back blending).                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int *mode;
    const double *mu2, *conic, *wp, *rgb, *op1, *op2;
} splats2d_t;

/* per-splat state needed to evaluate it at a pixel */
static void make_fwd_view(const splats2d_t *s, int i, fwd_t *f)
{
    f->mode = s->mode[i];
    f->wp[0] = s->wp[2 * i]; f->wp[1] = s->wp[2 * i + 1];
    f->w[0] = s->wp[2 * i]; f->w[1] = s->wp[2 * i + 1];
}

typedef struct {
    double G, P, A, araw, a;
    int clamped;
} eval_t;

static int eval_splat(const splats2d_t *s, int i, double px, double py, int plain,
                      eval_t *e, double *margin)
{
    double dx = px - s->mu2[2 * i], dy = py - s->mu2[2 * i + 1];
    const double *Q = s->conic + 3 * i;
    double power = -0.5 * (Q[0] * dx * dx + Q[2] * dy * dy) - Q[1] * dx * dy;
    if (power > 0) return 0;
    e->G = exp(power);
    fwd_t f;
    make_fwd_view(s, i, &f);
    double a1 = s->op1[i], a2 = s->op2[i];
    if (plain) {
        e->P = 1.0;
        e->A = a1;
    } else {
        e->P = half_fraction(&f, dx, dy, margin);
        e->A = a2 + (a1 - a2) * e->P;
    }
    e->araw = e->A * e->G;
    e->clamped = e->araw > OR_ALPHA_MAX;
    e->a = e->clamped ? OR_ALPHA_MAX : e->araw;
    return 1;
}


/* Per-pair part of the FP32 error model: a bound on |ln a32 - ln a| for one (pixel,
 * splat) pair, a32 the pair weight of a binary32 evaluation that
 *   - takes the shape terms with the error of E (above; root-sum-square over its
 *     22 inputs, each perturbed by 8 unit roundoffs: the longest chain of rounded
 *     operations from one input to y),
 *   - takes the centre to 2e-7 px (compensated arithmetic, integer anchor plus
 *     fraction) and forms the pixel offset d from tile-local numbers, each rounded
 *     once (u (2|d| + 32) px per axis),
 *   - evaluates the exponent as |U d|^2 with U the Cholesky factor of the conic
 *     (each factor entry within 6 unit roundoffs, each product and sum rounded once),
 *   - evaluates exp with a relative error of 4 ulp (2^-22) and erfc/2 within the
 *     Abramowitz & Stegun 7.1.26 bound (7.5e-8 absolute) plus the rounding of its
 *     polynomial and exponential,
 *   - rounds the opacity mix and the product A G once each (and the mip factor of the
 *     opacities to 16 ulp when mip is on).
 * The sum of these first-order terms is doubled (OR_SAFETY).                         */
#define OR_EX2_REL 2.384185791015625e-7   /* 2^-22 */
#define OR_ERFC_ABS 7.5e-8
#define OR_SAFETY 2.0
#define OR_SHAPE_ULPS 8.0
static double pair_band(const splats2d_t *s, const double *E, int i, double dx, double dy,
                        const eval_t *e, int plain, int mip)
{
    const double u = OR_U32;
    const double *Q = s->conic + 3 * i;
    double A = e->A > 1e-300 ? e->A : 1e-300;
    double d12 = plain ? 0.0 : s->op1[i] - s->op2[i];
    double g[5] = {-0.5 * dx * dx, -dx * dy, -0.5 * dy * dy, 0.0, 0.0};
    double phi = 0.0, z = 0.0, wx = s->wp[2 * i], wy = s->wp[2 * i + 1];
    int normal = !plain && s->mode[i] == OR_NORMAL;
    if (normal) {
        z = wx * dx + wy * dy;
        phi = exp(-z * z) / sqrt(3.14159265358979323846);     /* dP/dz */
        g[3] = d12 * phi * dx / A;
        g[4] = d12 * phi * dy / A;
    }
    double shape = 0.0;
    if (E) {
        const double *Ei = E + 15 * (size_t)i;
        double qf = 0.0;
        int q = 0;
        for (int a = 0; a < 5; ++a)
            for (int b = a; b < 5; ++b, ++q) qf += (a == b ? 1.0 : 2.0) * g[a] * g[b] * Ei[q];
        shape = OR_SHAPE_ULPS * u * sqrt(qf > 0 ? qf : 0.0);
    }
    /* centre and pixel offset */
    double gx = -(Q[0] * dx + Q[1] * dy) + (normal ? d12 * phi * wx / A : 0.0);
    double gy = -(Q[1] * dx + Q[2] * dy) + (normal ? d12 * phi * wy / A : 0.0);
    double pos = fabs(gx) * (2e-7 + u * (2.0 * fabs(dx) + 32.0)) + fabs(gy) * (2e-7 + u * (2.0 * fabs(dy) + 32.0));
    /* the exponent as a sum of two squares */
    double u11 = sqrt(Q[0]), u12 = Q[1] / u11;
    double dq = Q[0] * Q[2] - Q[1] * Q[1];
    double u22 = sqrt(dq > 0 ? dq : 0.0) / u11;
    double s1 = u11 * dx + u12 * dy, s2 = u22 * dy;
    double expo = 6.0 * u * (fabs(s1) * (fabs(u11 * dx) + fabs(u12 * dy)) + s2 * s2) + u * (s1 * s1 + s2 * s2);
    /* approximations and the remaining roundings */
    double mix = 0.0;
    if (normal) {
        double h = 0.5 * erfc(fabs(z));
        double dP = OR_ERFC_ABS + h * (OR_EX2_REL + 8.0 * u) + phi * 2.0 * u * (fabs(wx * dx) + fabs(wy * dy));
        mix = fabs(d12) * dP / A;
    }
    mix += u * (fabs(d12) * e->P / A + 1.0);
    double rnd = OR_EX2_REL + 2.0 * u + (mip ? 16.0 * u : 0.0);
    return OR_SAFETY * (shape + pos + expo + mix + rnd);
}

/* The band pair_band gives each of m (splat, pixel centre) pairs, and the FP64 pair
 * weight a (exported for the model's pins; band -1 where the pair is past the 3-sigma
 * exponent test, power > 0).                                                   */
int or_pair_bands(int n, const int *mode, const double *mu2, const double *conic, const double *wp,
                  const double *op1, const double *op2, const double *errmat, int plain, int mip, int m,
                  const int *ids, const double *px, const double *py, double *band, double *a)
{
    (void)n;
    splats2d_t s = {mode, mu2, conic, wp, NULL, op1, op2};
    for (int j = 0; j < m; ++j) {
        int i = ids[j];
        eval_t e;
        band[j] = -1.0;
        a[j] = 0.0;
        if (!eval_splat(&s, i, px[j], py[j], plain, &e, NULL)) continue;
        a[j] = e.araw;
        band[j] = pair_band(&s, errmat, i, px[j] - mu2[2 * i], py[j] - mu2[2 * i + 1], &e, plain, mip);
    }
    return 0;
}

/* Renders the tiles selected by tile_mask (all if NULL).
 * image [3,H,W], T [H,W], n_contrib [H,W] (1 + list position of the last
 * composited splat, 0 if none), margin [H,W] (smallest relative distance of any
 * threshold decision to its threshold).  Optional outputs (may be NULL), from the
 * FP32 error model (errmat [n,15] from or_error_basis; NULL drops its shape part):
 *   margin_a [H,W]: smallest |a - 1/255| / (a band) over the pixel's evaluated pairs,
 *                   and of the step-sign decisions |z| / (z band);
 *   margin_T [H,W]: the same for the 1e-4 stop, against the accumulated band of T;
 *   margin_c [H,W]: the same for the 0.99 clamp (it bends the gradient, not the image);
 *   n_comp [H,W]:   the number of composited splats;
 *   flip_img, flip_T [H,W]: how much the pixel (any channel) and T may move when every
 *                   decision with margin <= 1 goes the other way: T a (|c| + colour
 *                   behind) for the floor, T |alpha1 - alpha2| G (...) for a step sign,
 *                   T (colour) for the stop;
 *   touched [n]:    1 for every splat with a decision of margin <= 1 in some pixel.
 * A margin <= 1 marks a decision a binary32 evaluation cannot be expected to
 * reproduce.                                                                     */
int or_render_fwd(int n, const int *mode, const double *mu2, const double *conic,
                  const double *wp, const double *rgb, const double *op1, const double *op2,
                  const uint32_t *ids, const uint32_t *ranges, const or_camera *cam,
                  const or_opts *o, const unsigned char *tile_mask,
                  double *image, double *T_out, int *n_contrib, double *margin,
                  double *margin_a, double *margin_T, int *n_comp,
                  const double *errmat, double *margin_c, double *flip_img, double *flip_T,
                  unsigned char *touched, unsigned char *comp)
{
    /* comp (optional, [pairs, tile_w * tile_h], zeroed by the caller): comp[j, q] = 1
     * where list entry j is composited at pixel q (row-major within its tile).      */
    (void)n;
    splats2d_t s = {mode, mu2, conic, wp, rgb, op1, op2};
    int W = cam->width, H = cam->height;
    int tiles_x = (W + o->tile_w - 1) / o->tile_w;
    int tiles_y = (H + o->tile_h - 1) / o->tile_h;
    int n_tiles = tiles_x * tiles_y;
    const double u = OR_U32;
    double bgmax = fmax(fmax(fabs(cam->bg[0]), fabs(cam->bg[1])), fabs(cam->bg[2]));
    /* the FP32 error model only when one of its outputs is wanted */
    const int model = margin_a || margin_T || margin_c || flip_img || flip_T || touched;
#pragma omp parallel for schedule(dynamic, 1)
    for (int tile = 0; tile < n_tiles; ++tile) {
        if (tile_mask && !tile_mask[tile]) continue;
        int tx = tile % tiles_x, ty = tile / tiles_x;
        uint32_t beg = ranges[2 * tile], end = ranges[2 * tile + 1];
        for (int py = ty * o->tile_h; py < (ty + 1) * o->tile_h && py < H; ++py)
            for (int px = tx * o->tile_w; px < (tx + 1) * o->tile_w && px < W; ++px) {
                double pcx = px + 0.5, pcy = py + 0.5;
                double T = 1.0, C[3] = {0, 0, 0}, mg = 1e300, mga = 1e300, mgT = 1e300, mgc = 1e300;
                double step_mg = 1e300, t_err = 0.0;
                double f_own = 0.0, f_wt = 0.0, f_stop = 0.0, f_T = 0.0, cmax = bgmax;
                int last = 0, ncomp = 0;
                for (uint32_t j = beg; j < end; ++j) {
                    int i = (int)ids[j];
                    if (mode[i] == OR_CULLED) continue;
                    eval_t e;
                    if (!eval_splat(&s, i, pcx, pcy, o->plain, &e, &step_mg)) continue;
                    double dx = pcx - mu2[2 * i], dy = pcy - mu2[2 * i + 1];
                    double ci = fmax(fmax(fabs(rgb[3 * i]), fabs(rgb[3 * i + 1])), fabs(rgb[3 * i + 2]));
                    double rel = fabs(e.a - OR_ALPHA_MIN) / OR_ALPHA_MIN;
                    if (rel < mg) mg = rel;
                    double band = -1.0;
                    if (model && (e.a >= OR_ALPHA_MIN || rel < 0.05))
                        band = pair_band(&s, errmat, i, dx, dy, &e, o->plain, o->mip);
                    if (model && rel < 0.05) {
                        double na = rel / band;
                        if (na < mga) mga = na;
                        if (na <= 1.0) {          /* the floor may go either way */
                            f_own += T * e.a * ci;
                            f_wt += T * e.a;
                            t_err += e.a;
                            if (touched) touched[i] = 1;
                        }
                    }
                    if (model && !o->plain && mode[i] == OR_STEP) {
                        /* the sign of w.d decides alpha1 or alpha2 */
                        double z = wp[2 * i] * dx + wp[2 * i + 1] * dy;
                        double zb = fabs(wp[2 * i]) * (2e-7 + u * (2.0 * fabs(dx) + 32.0)) +
                                    fabs(wp[2 * i + 1]) * (2e-7 + u * (2.0 * fabs(dy) + 32.0)) +
                                    2.0 * u * (fabs(wp[2 * i] * dx) + fabs(wp[2 * i + 1] * dy));
                        double ns = fabs(z) / (OR_SAFETY * zb);
                        if (ns < mga) mga = ns;
                        if (ns <= 1.0) {
                            double dw = T * fabs(op1[i] - op2[i]) * e.G;
                            f_own += dw * ci;
                            f_wt += dw;
                            t_err += fabs(op1[i] - op2[i]) * e.G;
                            if (touched) touched[i] = 1;
                        }
                    }
                    if (e.a < OR_ALPHA_MIN) continue;
                    if (margin_c) {
                        double nc = fabs(e.araw - OR_ALPHA_MAX) / OR_ALPHA_MAX / band;
                        if (nc < mgc) mgc = nc;
                        if (nc <= 1.0 && touched) touched[i] = 1;
                    }
                    double Tn = T * (1.0 - e.a);
                    double relT = fabs(Tn - OR_T_MIN) / OR_T_MIN;
                    if (relT < mg) mg = relT;
                    double this_err = model ? e.a / (1.0 - e.a) * band : 0.0;
                    double nT = model ? relT / (t_err + this_err + 2.0 * u * (ncomp + 1)) : 1e300;
                    if (nT < mgT) mgT = nT;
                    if (nT <= 1.0) {              /* the stop may go either way */
                        f_stop += T;
                        f_T += T * e.a;
                        if (ci > cmax) cmax = ci;
                        if (touched) touched[i] = 1;
                    }
                    if (Tn < OR_T_MIN) break;
                    if (comp)
                        comp[(size_t)j * (o->tile_w * o->tile_h) + (py - ty * o->tile_h) * o->tile_w +
                             (px - tx * o->tile_w)] = 1;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * i + ch] * e.a * T;
                    T = Tn;
                    t_err += this_err;
                    if (ci > cmax) cmax = ci;
                    last = (int)(j - beg) + 1;
                    ncomp++;
                }
                if (step_mg < mg) mg = step_mg;
                size_t pix = (size_t)py * W + px;
                for (int ch = 0; ch < 3; ++ch) image[(size_t)ch * W * H + pix] = C[ch] + T * cam->bg[ch];
                T_out[pix] = T;
                n_contrib[pix] = last;
                margin[pix] = mg;
                if (margin_a) margin_a[pix] = mga;
                if (margin_T) margin_T[pix] = mgT;
                if (margin_c) margin_c[pix] = mgc;
                if (n_comp) n_comp[pix] = ncomp;
                if (flip_img) flip_img[pix] = f_own + f_wt * cmax + f_stop * cmax;
                if (flip_T) flip_T[pix] = f_wt + f_T;
            }
    }
    return 0;
}

/* Per-splat screen-space gradients, 12 per splat:
 * [d mu2_x, d mu2_y, d A, d B, d C, d wp_x, d wp_y, d alpha1, d alpha2, d r, d g, d b]
 * where the conic is [[A, B], [B, C]] and B is one scalar parameter.         */
#define G2D 12
/* grad2d_err (optional, [n,12], accumulated): a first-order bound on the error of a
 * binary32 evaluation of each entry, sum over its per-pixel terms t of |t| eps, with
 * eps = 2 band + (the accumulated band of T) + 32 ulp: band (pair_band, with errmat
 * when given) bounds the relative error of the pair weight, which enters each term
 * once through a and once through the quantities derived from it; the transmittance
 * carries the bands of the splats composited in front; 32 ulp cover the term's own
 * products and its share of the summation.  Per-thread accumulators hold only the
 * splats listed in the rendered tiles.                                              */
int or_render_bwd(int n, const int *mode, const double *mu2, const double *conic,
                  const double *wp, const double *rgb, const double *op1, const double *op2,
                  const uint32_t *ids, const uint32_t *ranges, const or_camera *cam,
                  const or_opts *o, const unsigned char *tile_mask,
                  const double *dL_dimage, double *grad2d /* [n,12], accumulated */,
                  const double *errmat, double *grad2d_err)
{
    splats2d_t s = {mode, mu2, conic, wp, rgb, op1, op2};
    int W = cam->width, H = cam->height;
    int tiles_x = (W + o->tile_w - 1) / o->tile_w;
    int tiles_y = (H + o->tile_h - 1) / o->tile_h;
    int n_tiles = tiles_x * tiles_y;
    int nthr = or_num_threads();
    /* compact index of the splats that appear in a rendered tile's list */
    int *slot = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    int *which = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    if (!slot || !which) { free(slot); free(which); return 1; }
    for (int i = 0; i < n; ++i) slot[i] = -1;
    int m_used = 0;
    for (int tile = 0; tile < n_tiles; ++tile) {
        if (tile_mask && !tile_mask[tile]) continue;
        for (uint32_t j = ranges[2 * tile]; j < ranges[2 * tile + 1]; ++j) {
            int i = (int)ids[j];
            if (slot[i] < 0) { slot[i] = m_used; which[m_used++] = i; }
        }
    }
    int nabs = grad2d_err ? 2 : 1;
    double *acc = (double *)calloc((size_t)nthr * nabs * (m_used > 0 ? m_used : 1) * G2D, sizeof(double));
    if (!acc) { free(slot); free(which); return 1; }
#pragma omp parallel
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double *g2c = acc + (size_t)tid * nabs * m_used * G2D;
        double *gac = grad2d_err ? g2c + (size_t)m_used * G2D : NULL;
        int cap = 64;
        int *lst = (int *)malloc(sizeof(int) * cap);
        eval_t *ev = (eval_t *)malloc(sizeof(eval_t) * cap);
        double *Ts = (double *)malloc(sizeof(double) * cap);
        double *eps = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 1)
        for (int tile = 0; tile < n_tiles; ++tile) {
            if (tile_mask && !tile_mask[tile]) continue;
            int tx = tile % tiles_x, ty = tile / tiles_x;
            uint32_t beg = ranges[2 * tile], end = ranges[2 * tile + 1];
            for (int py = ty * o->tile_h; py < (ty + 1) * o->tile_h && py < H; ++py)
                for (int px = tx * o->tile_w; px < (tx + 1) * o->tile_w && px < W; ++px) {
                    double pcx = px + 0.5, pcy = py + 0.5;
                    size_t pix = (size_t)py * W + px;
                    double g[3];
                    for (int ch = 0; ch < 3; ++ch) g[ch] = dL_dimage[(size_t)ch * W * H + pix];
                    /* forward again, remembering the composited splats */
                    int m = 0;
                    double T = 1.0, t_err = 0.0;
                    for (uint32_t j = beg; j < end; ++j) {
                        int i = (int)ids[j];
                        if (mode[i] == OR_CULLED) continue;
                        eval_t e;
                        if (!eval_splat(&s, i, pcx, pcy, o->plain, &e, NULL)) continue;
                        if (e.a < OR_ALPHA_MIN) continue;
                        double Tn = T * (1.0 - e.a);
                        if (Tn < OR_T_MIN) break;
                        if (m == cap) {
                            cap *= 2;
                            lst = (int *)realloc(lst, sizeof(int) * cap);
                            ev = (eval_t *)realloc(ev, sizeof(eval_t) * cap);
                            Ts = (double *)realloc(Ts, sizeof(double) * cap);
                            eps = (double *)realloc(eps, sizeof(double) * cap);
                        }
                        lst[m] = i; ev[m] = e; Ts[m] = T;
                        if (grad2d_err) {
                            double band = pair_band(&s, errmat, i, pcx - mu2[2 * i], pcy - mu2[2 * i + 1], &e,
                                                    o->plain, o->mip);
                            eps[m] = 2.0 * band + t_err + 32.0 * OR_U32;
                            t_err += e.a / (1.0 - e.a) * band;
                        }
                        m++;
                        T = Tn;
                    }
                    double Tfinal = T;
                    double bgg = cam->bg[0] * g[0] + cam->bg[1] * g[1] + cam->bg[2] * g[2];
                    /* reverse sweep: S = colour accumulated behind the current splat */
                    double S[3] = {0, 0, 0};
                    for (int q = m - 1; q >= 0; --q) {
                        int i = lst[q];
                        const eval_t *e = &ev[q];
                        double Ti = Ts[q];
                        double t[G2D] = {0};     /* this pixel's terms */
                        double dLda = 0;
                        for (int ch = 0; ch < 3; ++ch) {
                            t[9 + ch] = e->a * Ti * g[ch];
                            dLda += Ti * (rgb[3 * i + ch] - S[ch]) * g[ch];
                        }
                        dLda -= Tfinal / (1.0 - e->a) * bgg;
                        for (int ch = 0; ch < 3; ++ch) S[ch] = e->a * rgb[3 * i + ch] + (1.0 - e->a) * S[ch];
                        if (!e->clamped) {
                            double dx = pcx - mu2[2 * i], dy = pcy - mu2[2 * i + 1];
                            const double *Qc = conic + 3 * i;
                            double dG = dLda * e->A;
                            double dpow = dG * e->G;
                            t[2] = dpow * (-0.5 * dx * dx);
                            t[3] = dpow * (-dx * dy);
                            t[4] = dpow * (-0.5 * dy * dy);
                            t[0] = dpow * (Qc[0] * dx + Qc[1] * dy);
                            t[1] = dpow * (Qc[1] * dx + Qc[2] * dy);
                            if (o->plain) {
                                t[7] = dLda * e->G;
                            } else {
                                t[7] = dLda * e->P * e->G;
                                t[8] = dLda * (1.0 - e->P) * e->G;
                                if (mode[i] == OR_NORMAL) {
                                    double dP = dLda * (op1[i] - op2[i]) * e->G;
                                    double z = wp[2 * i] * dx + wp[2 * i + 1] * dy;
                                    double dz = dP * exp(-z * z) / sqrt(3.14159265358979323846);
                                    t[5] = dz * dx;
                                    t[6] = dz * dy;
                                    t[0] -= dz * wp[2 * i];
                                    t[1] -= dz * wp[2 * i + 1];
                                }
                            }
                        }
                        double *gi = g2c + (size_t)slot[i] * G2D;
                        for (int f = 0; f < G2D; ++f) gi[f] += t[f];
                        if (gac) {
                            double *ga = gac + (size_t)slot[i] * G2D;
                            for (int f = 0; f < G2D; ++f) ga[f] += fabs(t[f]) * eps[q];
                        }
                    }
                }
        }
        free(lst); free(ev); free(Ts); free(eps);
    }
    for (int t = 0; t < nthr; ++t) {
        const double *g2c = acc + (size_t)t * nabs * m_used * G2D;
        for (int c = 0; c < m_used; ++c)
            for (int f = 0; f < G2D; ++f) {
                grad2d[(size_t)which[c] * G2D + f] += g2c[(size_t)c * G2D + f];
                if (grad2d_err) grad2d_err[(size_t)which[c] * G2D + f] += g2c[((size_t)m_used + c) * G2D + f];
            }
    }
    free(acc); free(slot); free(which);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Projection adjoint.                                                        */
/* ------------------------------------------------------------------------ */
static void rot_vjp(const double q[4], const double gR[3][3], double gq[4])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    /* R entries as functions of (w,x,y,z); each partial written out */
    gq[0] = gR[0][1] * (-2 * z) + gR[0][2] * (2 * y) + gR[1][0] * (2 * z) + gR[1][2] * (-2 * x)
          + gR[2][0] * (-2 * y) + gR[2][1] * (2 * x);
    gq[1] = gR[0][1] * (2 * y) + gR[0][2] * (2 * z) + gR[1][0] * (2 * y) + gR[1][1] * (-4 * x)
          + gR[1][2] * (-2 * w) + gR[2][0] * (2 * z) + gR[2][1] * (2 * w) + gR[2][2] * (-4 * x);
    gq[2] = gR[0][0] * (-4 * y) + gR[0][1] * (2 * x) + gR[0][2] * (2 * w) + gR[1][0] * (2 * x)
          + gR[1][2] * (2 * z) + gR[2][0] * (-2 * w) + gR[2][1] * (2 * z) + gR[2][2] * (-4 * y);
    gq[3] = gR[0][0] * (-4 * z) + gR[0][1] * (-2 * w) + gR[0][2] * (2 * x) + gR[1][0] * (2 * w)
          + gR[1][1] * (-4 * z) + gR[1][2] * (2 * y) + gR[2][0] * (2 * x) + gR[2][1] * (2 * y);
}

int or_project_bwd(int n, const double *means, const double *scales, const double *quats,
                   const double *normals, const double *sh, const double *op1, const double *op2,
                   const or_camera *cam, const or_opts *o, const int *mode_in,
                   const double *grad2d,
                   double *g_means, double *g_scales, double *g_quats, double *g_normals,
                   double *g_op1, double *g_op2, double *g_sh)
{
    int nc = (o->sh_degree + 1) * (o->sh_degree + 1);
    const double *V = cam->viewmat;
    double Rc[3][3] = {{V[0], V[1], V[2]}, {V[4], V[5], V[6]}, {V[8], V[9], V[10]}};
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        if (mode_in[i] == OR_CULLED) continue;
        const double *gg = grad2d + (size_t)G2D * i;
        fwd_t f;
        const double *shi = sh + 3 * nc * i;
        project_fp64(means + 3 * i, scales + 3 * i, quats + 4 * i, normals + 3 * i, shi,
                     o->sh_degree, cam, o, &f);
        /* grad2d[7..8] are taken w.r.t. the opacities the compositing used, comp * op */
        g_op1[i] += f.comp * gg[7];
        g_op2[i] += f.comp * gg[8];
        const double g_comp = op1[i] * gg[7] + op2[i] * gg[8];

        double g_mean[3] = {0, 0, 0};
        /* colour: rgb = max(0, sum sh*Y(dir) + 1/2), dir = (mu - campos)/|mu - campos| */
        double graw[3];
        for (int ch = 0; ch < 3; ++ch) graw[ch] = f.rgb_raw[ch] < 0 ? 0.0 : gg[9 + ch];
        double g_dir[3] = {0, 0, 0};
        for (int l = 0; l < nc; ++l)
            for (int ch = 0; ch < 3; ++ch) {
                g_sh[(size_t)3 * nc * i + 3 * l + ch] += graw[ch] * f.Y[l];
                for (int k = 0; k < 3; ++k) g_dir[k] += graw[ch] * shi[3 * l + ch] * f.dY[l][k];
            }
        double gd = g_dir[0] * f.dir[0] + g_dir[1] * f.dir[1] + g_dir[2] * f.dir[2];
        for (int k = 0; k < 3; ++k) g_mean[k] += (g_dir[k] - gd * f.dir[k]) / f.dnorm;

        /* half-plane terms: wp = w / sqrt(2v), v = var_s - k.w, w = Q k,
           k = M Sigma^w nh, var_s = nh^T Sigma^w nh                           */
        double gQ[3] = {gg[2], gg[3], gg[4]};
        double gM[2][3] = {{0, 0, 0}, {0, 0, 0}};
        double gSw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double g_normal[3] = {0, 0, 0};
        if (f.mode == OR_NORMAL) {
            double s = 1.0 / sqrt(2.0 * f.v);
            double gw[2] = {gg[5] * s, gg[6] * s};
            double gv = -(gg[5] * f.w[0] + gg[6] * f.w[1]) * s * s * s;
            double gvar = gv;
            double gk[2] = {-gv * f.w[0], -gv * f.w[1]};
            gw[0] += -gv * f.k[0];
            gw[1] += -gv * f.k[1];
            gQ[0] += gw[0] * f.k[0];
            gQ[1] += gw[0] * f.k[1] + gw[1] * f.k[0];
            gQ[2] += gw[1] * f.k[1];
            gk[0] += f.Q[0] * gw[0] + f.Q[1] * gw[1];
            gk[1] += f.Q[1] * gw[0] + f.Q[2] * gw[1];
            double Sn[3];
            for (int a = 0; a < 3; ++a) Sn[a] = f.Sw[a][0] * f.nh[0] + f.Sw[a][1] * f.nh[1] + f.Sw[a][2] * f.nh[2];
            double g_nh[3] = {0, 0, 0};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 3; ++b) gM[a][b] += gk[a] * Sn[b];
            /* d(k)/d(Sigma^w): k_a = sum_bc M_ab Sw_bc nh_c */
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) gSw[b][c] += (gk[0] * f.M[0][b] + gk[1] * f.M[1][b]) * f.nh[c];
            double MTgk[3];
            for (int b = 0; b < 3; ++b) MTgk[b] = f.M[0][b] * gk[0] + f.M[1][b] * gk[1];
            for (int c = 0; c < 3; ++c) g_nh[c] += f.Sw[0][c] * MTgk[0] + f.Sw[1][c] * MTgk[1] + f.Sw[2][c] * MTgk[2];
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) gSw[b][c] += gvar * f.nh[b] * f.nh[c];
            for (int c = 0; c < 3; ++c) g_nh[c] += 2.0 * gvar * Sn[c];
            double dd = g_nh[0] * f.nh[0] + g_nh[1] * f.nh[1] + g_nh[2] * f.nh[2];
            for (int c = 0; c < 3; ++c) g_normal[c] = (g_nh[c] - dd * f.nh[c]) / f.nn;
        }

        /* conic Q = hat Sigma^-1: G_Sigma = -Q GQm Q, GQm = [[gA, gB/2],[gB/2, gC]] */
        double Qm[2][2] = {{f.Q[0], f.Q[1]}, {f.Q[1], f.Q[2]}};
        double GQm[2][2] = {{gQ[0], 0.5 * gQ[1]}, {0.5 * gQ[1], gQ[2]}};
        double T1[2][2], Gs[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) T1[a][b] = Qm[a][0] * GQm[0][b] + Qm[a][1] * GQm[1][b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) Gs[a][b] = -(T1[a][0] * Qm[0][b] + T1[a][1] * Qm[1][b]);
        /* mip: comp = sqrt(det S0 / det(S0 + l I)),
           d comp = comp/2 tr((S0^-1 - hat Sigma^-1) dS0), and d hat Sigma = dS0 */
        if (o->mip && f.det0 > 0) {
            const double h = 0.5 * g_comp * f.comp;
            const double I0[2][2] = {{f.S0[2] / f.det0, -f.S0[1] / f.det0}, {-f.S0[1] / f.det0, f.S0[0] / f.det0}};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) Gs[a][b] += h * (I0[a][b] - Qm[a][b]);
        }
        /* hat Sigma = M Sigma^w M^T + l I:  gM += 2 Gs M Sw,  gSw += M^T Gs M */
        double MSw[2][3];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b)
                MSw[a][b] = f.M[a][0] * f.Sw[0][b] + f.M[a][1] * f.Sw[1][b] + f.M[a][2] * f.Sw[2][b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) gM[a][b] += 2.0 * (Gs[a][0] * MSw[0][b] + Gs[a][1] * MSw[1][b]);
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 2; ++a)
                    for (int e = 0; e < 2; ++e) gSw[b][c] += f.M[a][b] * Gs[a][e] * f.M[e][c];

        /* M = J W_rot:  gJ = gM W_rot^T (only the four nonzero entries of J) */
        double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
        for (int k = 0; k < 3; ++k) {
            gJ00 += gM[0][k] * Rc[0][k];
            gJ02 += gM[0][k] * Rc[2][k];
            gJ11 += gM[1][k] * Rc[1][k];
            gJ12 += gM[1][k] * Rc[2][k];
        }
        double tz = f.t[2];
        double gt[3] = {0, 0, 0};
        gt[2] += gJ00 * (-cam->fx / (tz * tz));
        gt[2] += gJ11 * (-cam->fy / (tz * tz));
        if (!f.clampx) {   /* J02 = -fx tx / tz^2 */
            gt[0] += gJ02 * (-cam->fx / (tz * tz));
            gt[2] += gJ02 * (2.0 * cam->fx * f.t[0] / (tz * tz * tz));
        } else {           /* J02 = -fx uxc / tz with uxc fixed */
            gt[2] += gJ02 * (cam->fx * f.uxc / (tz * tz));
        }
        if (!f.clampy) {
            gt[1] += gJ12 * (-cam->fy / (tz * tz));
            gt[2] += gJ12 * (2.0 * cam->fy * f.t[1] / (tz * tz * tz));
        } else {
            gt[2] += gJ12 * (cam->fy * f.uyc / (tz * tz));
        }
        /* projected centre */
        gt[0] += gg[0] * cam->fx / tz;
        gt[2] += -gg[0] * cam->fx * f.t[0] / (tz * tz);
        gt[1] += gg[1] * cam->fy / tz;
        gt[2] += -gg[1] * cam->fy * f.t[1] / (tz * tz);
        /* t = W_rot mu + t_c */
        for (int k = 0; k < 3; ++k) g_mean[k] += Rc[0][k] * gt[0] + Rc[1][k] * gt[1] + Rc[2][k] * gt[2];

        /* Sigma^w = R diag(s^2) R^T.  Symmetrise gSw, then dR and ds. */
        double Gsym[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Gsym[a][b] = gSw[a][b] + gSw[b][a];
        /* Sigma^w = L L^T with L = R diag(s):  gL = (gSw + gSw^T) L */
        double Lm[3][3], gL[3][3];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) Lm[a][k] = f.R[a][k] * scales[3 * i + k];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) gL[a][k] = Gsym[a][0] * Lm[0][k] + Gsym[a][1] * Lm[1][k] + Gsym[a][2] * Lm[2][k];
        double gR[3][3];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) gR[a][k] = gL[a][k] * scales[3 * i + k];
        for (int k = 0; k < 3; ++k)
            g_scales[3 * i + k] += gL[0][k] * f.R[0][k] + gL[1][k] * f.R[1][k] + gL[2][k] * f.R[2][k];
        double gqh[4];
        rot_vjp(f.qh, gR, gqh);
        double dq = gqh[0] * f.qh[0] + gqh[1] * f.qh[1] + gqh[2] * f.qh[2] + gqh[3] * f.qh[3];
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += (gqh[k] - dq * f.qh[k]) / f.qn;
        for (int k = 0; k < 3; ++k) g_means[3 * i + k] += g_mean[k];
        for (int k = 0; k < 3; ++k) g_normals[3 * i + k] += g_normal[k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-splat evaluation helper for the quadrature pins: for splat 0, the   */
/* hat G and P the renderer would use at pixel positions (px, py).            */
/* ------------------------------------------------------------------------ */
int or_eval_splat(const double *mean, const double *scale, const double *quat,
                  const double *normal, const or_camera *cam, const or_opts *o,
                  int npts, const double *px, const double *py, double *G, double *P)
{
    double sh[48] = {0};
    or_opts o2 = *o;
    o2.sh_degree = 0;
    fwd_t f;
    project_fp64(mean, scale, quat, normal, sh, 0, cam, &o2, &f);
    for (int j = 0; j < npts; ++j) {
        double dx = px[j] - f.mu2[0], dy = py[j] - f.mu2[1];
        double power = -0.5 * (f.Q[0] * dx * dx + f.Q[2] * dy * dy) - f.Q[1] * dx * dy;
        G[j] = exp(power);
        P[j] = half_fraction(&f, dx, dy, NULL);
    }
    return f.mode;
}
