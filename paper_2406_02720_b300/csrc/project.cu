// Projection of half-Gaussian pairs to screen-space splats (A1 + A2) and its
// adjoint (A8).
//
// Forward, per (splat, view):
//   Eq. 2      Sigma^w = R S S^T R^T, factored as L L^T with L = R diag(s)
//   Eq. 3-5    hat Sigma = P P^T + l I with P = M L, M = J W (2x3): the top-left
//              2x2 block of J W Sigma^w W^T J^T, plus the 3D-GS low-pass l
//   Eq. 7-8    half-plane fraction P(d) = Pr[n.(x-mu) >= 0 | pixel offset d]
//              = 1/2 erfc(-w'.d) with u = L^T n^, var_s = |u|^2, k = P u,
//              w = hat Sigma^-1 k, v = var_s - k.w, w' = w / sqrt(2 v)
//   Sec. 3.1   view-dependent SH colour
// Both determinants are formed from sums of non-negative terms, so thin splats
// lose no precision to cancellation (p0, p1 are the rows of P):
//   det hat Sigma = |p0 x p1|^2 + l (|p0|^2 + |p1|^2) + l^2
//   v = det C3 / det hat Sigma, C3 the covariance of (s, pixel):
//   det C3 = (u.(p0 x p1))^2 + l (|u x p0|^2 + |u x p1|^2) + l^2 |u|^2
// The conic is stored as its Cholesky factor U (conic = U^T U,
// U = [[sqrt(c/det), -b/sqrt(c det)], [0, 1/sqrt(c)]]), so that the exponent is
// evaluated per pixel as a sum of two squares.
// The binning fields (depth, mu-hat, hat Sigma, 3-sigma radius, tile rect) use a
// fixed FP32 operation order with no fused multiply-add (__f*_rn intrinsics), so
// that the integer decisions they feed are reproducible.  The continuous terms
// are FP32, with FP64 only for near-degenerate splats: in the forward, a splat
// whose plane nearly contains the ray (v < 1e-3 var_s) gets its half-plane terms
// w' recomputed in FP64; in the adjoint, such a splat and a splat whose hat Sigma
// is ill-conditioned (condition number above 150) get their geometry adjoint
// (conic, covariance, half-plane terms to mean, scale, rotation, normal) in FP64.
#include <math.h>

#include "hgs_internal.cuh"

namespace hgs {
namespace {

// Splats per block: 128 in the projection, 64 in its adjoint (at 3M splats, degree 3:
// projection 0.220 / 0.222 / 0.229 ms and adjoint 0.378 / 0.368 / 0.400 ms at
// 128 / 64 / 256, resident threads per SM held equal).
constexpr int kProjBlock = 128;
constexpr int kProjBwdBlock = 64;
enum { MODE_CULLED = 0, MODE_NORMAL = 1, MODE_STEP = 2, MODE_HALF = 3 };

// Degeneracy test that sends a splat's half-plane terms to the FP64 path: the
// splitting plane nearly contains the ray (v < kVRelFp64 * var_s).
constexpr float kVRelFp64 = 1e-3f;
// The projection adjoint also takes the FP64 path for a splat whose hat Sigma has a
// condition number above kCondFp64 (a needle- or disk-like footprint, ~0.9% of the
// splats of the 3M-splat scene): through the conic, dL/d hat Sigma = -conic G conic
// loses about cond x u in binary32, which reached 1e-3..3e-2 of the scale and
// quaternion gradients of such splats (1.2e-3 at a condition number of 242; with the
// cut at 150 instead of 300 the projection adjoint takes 0.347 -> 0.351 ms).
constexpr float kCondFp64 = 150.0f;
constexpr float kCondFp64Test = (1.0f + kCondFp64) * (1.0f + kCondFp64) / kCondFp64;
// Scale applied to w in step mode (v ~ 0): P becomes a step at w.d = 0.
constexpr float kStepScale = 1.2089258196146292e24f;   // 2^80

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }

// Reciprocal and square root of the free-order terms (the conic factor, the half-plane
// terms, the compensated centre's first quotient and the adjoint): the PTX approximations in FP32 (relative error ~1e-7, far
// inside the FP32 parity bars, one instruction instead of an IEEE sequence), the exact
// operations in FP64.  The binning fields never use them.
template <typename T>
__device__ __forceinline__ T rcp_f(T x) { return (T)1 / x; }
template <>
__device__ __forceinline__ float rcp_f<float>(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <typename T>
__device__ __forceinline__ T sqrt_f(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float sqrt_f<float>(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- compensated binary32 arithmetic (value = hi + lo) ---------------------------
// Used for the projected centre, which must be exact to ~1e-7 px although it is
// near 2000 px: t = W mu + t_c, x/z and f x/z + c are formed from error-free
// products (fma) and sums, then split into an integer anchor and a fraction.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_renorm(float hi, float lo) {   // |hi| >= |lo|
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    return df_renorm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_mul(DF a, float b) {
    const DF p = two_prod(a.hi, b);
    return df_renorm(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// a / b with ib ~ 1 / b.hi (a few ulp): the first quotient q1 = a.hi ib, then the
// residual a - q1 b, formed exactly from an error-free product, times ib.  The residual
// absorbs q1's error, so the pair is accurate to ~1e-7 of the residual, far below an ulp
// of q1.
__device__ __forceinline__ DF df_div(DF a, DF b, float ib) {
    const float q1 = __fmul_rn(a.hi, ib);
    const DF p = two_prod(q1, b.hi);
    float r = __fsub_rn(a.hi, p.hi);
    r = __fsub_rn(r, p.lo);
    r = __fadd_rn(r, a.lo);
    r = __fsub_rn(r, __fmul_rn(q1, b.lo));
    return df_renorm(q1, __fmul_rn(r, ib));
}

// Projected centre (anchor = nearest integer, fraction = rest), compensated.
__device__ __forceinline__ void precise_centre(const float m[3], const hgs_camera &cam, float out[4]) {
    const float *V = cam.viewmat;
    DF t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        DF acc = two_prod(V[4 * i], m[0]);
        acc = df_add(acc, two_prod(V[4 * i + 1], m[1]));
        acc = df_add(acc, two_prod(V[4 * i + 2], m[2]));
        t[i] = df_add(acc, DF{V[4 * i + 3], 0.0f});
    }
    const float iz = rcp_f(t[2].hi);
    const DF mx = df_add(df_mul(df_div(t[0], t[2], iz), cam.fx), DF{cam.cx, 0.0f});
    const DF my = df_add(df_mul(df_div(t[1], t[2], iz), cam.fy), DF{cam.cy, 0.0f});
    out[0] = rintf(mx.hi);
    out[1] = rintf(my.hi);
    out[2] = __fadd_rn(__fsub_rn(mx.hi, out[0]), mx.lo);
    out[3] = __fadd_rn(__fsub_rn(my.hi, out[1]), my.lo);
}

struct Canon {
    bool culled;
    float depth, mux, muy, a, b, c, det;
    float L[3][3];
    float P[2][3];
    int rect[4];
    unsigned tiles;
};

// Binning fields in the fixed FP32 order (one IEEE op per step).
__device__ __forceinline__ void canon_project(const float m[3], const float s[3], const float q[4],
                                              const float nrm[3], float op1, float op2,
                                              const hgs_camera &cam, float lp, int fov_clamp,
                                              int tw, int th, int rect_mode, Canon &o) {
    o.culled = true;
    o.tiles = 0;
    o.rect[0] = o.rect[1] = o.rect[2] = o.rect[3] = 0;
    const float *V = cam.viewmat;
    // 1. unit quaternion
    float n2 = fm(q[0], q[0]);
    n2 = fa(n2, fm(q[1], q[1]));
    n2 = fa(n2, fm(q[2], q[2]));
    n2 = fa(n2, fm(q[3], q[3]));
    float qn = __fsqrt_rn(n2);
    const float iq = __frcp_rn(qn);
    float w = fm(q[0], iq), x = fm(q[1], iq), y = fm(q[2], iq), z = fm(q[3], iq);
    // 2. rotation
    float R[3][3];
    R[0][0] = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
    R[0][1] = fm(2.0f, fs(fm(x, y), fm(w, z)));
    R[0][2] = fm(2.0f, fa(fm(x, z), fm(w, y)));
    R[1][0] = fm(2.0f, fa(fm(x, y), fm(w, z)));
    R[1][1] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
    R[1][2] = fm(2.0f, fs(fm(y, z), fm(w, x)));
    R[2][0] = fm(2.0f, fs(fm(x, z), fm(w, y)));
    R[2][1] = fm(2.0f, fa(fm(y, z), fm(w, x)));
    R[2][2] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(y, y))));
    // 3. L = R diag(s)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) o.L[i][k] = fm(R[i][k], s[k]);
    // 4. camera-space mean
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float acc = fm(V[4 * i + 0], m[0]);
        acc = fa(acc, fm(V[4 * i + 1], m[1]));
        acc = fa(acc, fm(V[4 * i + 2], m[2]));
        t[i] = fa(acc, V[4 * i + 3]);
    }
    o.depth = t[2];
    // 5. near-plane cull
    if (!(t[2] > cam.near_plane)) return;
    // 6. clamped x/z, y/z
    const float iz = __frcp_rn(t[2]);
    float ux = fm(t[0], iz), uy = fm(t[1], iz);
    float uxc = ux, uyc = uy;
    if (fov_clamp) {
        float limx = fm(1.3f, fdv(fm(0.5f, (float)cam.width), cam.fx));
        float limy = fm(1.3f, fdv(fm(0.5f, (float)cam.height), cam.fy));
        uxc = fminf(fmaxf(ux, -limx), limx);
        uyc = fminf(fmaxf(uy, -limy), limy);
    }
    // 7. Jacobian
    float j00 = fm(cam.fx, iz);
    float j02 = -fm(fm(cam.fx, uxc), iz);
    float j11 = fm(cam.fy, iz);
    float j12 = -fm(fm(cam.fy, uyc), iz);
    // 8. M = J W
    float M[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        M[0][k] = fa(fm(j00, V[k]), fm(j02, V[8 + k]));
        M[1][k] = fa(fm(j11, V[4 + k]), fm(j12, V[8 + k]));
    }
    // 9. P = M L
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = fm(M[i][0], o.L[0][k]);
            acc = fa(acc, fm(M[i][1], o.L[1][k]));
            o.P[i][k] = fa(acc, fm(M[i][2], o.L[2][k]));
        }
    // 10. hat Sigma (A0, C0: the diagonal before the low-pass)
    float A0 = fm(o.P[0][0], o.P[0][0]);
    A0 = fa(A0, fm(o.P[0][1], o.P[0][1]));
    A0 = fa(A0, fm(o.P[0][2], o.P[0][2]));
    const float a = fa(A0, lp);
    float b = fm(o.P[0][0], o.P[1][0]);
    b = fa(b, fm(o.P[0][1], o.P[1][1]));
    b = fa(b, fm(o.P[0][2], o.P[1][2]));
    float C0 = fm(o.P[1][0], o.P[1][0]);
    C0 = fa(C0, fm(o.P[1][1], o.P[1][1]));
    C0 = fa(C0, fm(o.P[1][2], o.P[1][2]));
    const float c = fa(C0, lp);
    o.a = a; o.b = b; o.c = c;
    // 11. determinant cull
    float det = fs(fm(a, c), fm(b, b));
    o.det = det;
    if (!(det > 0.0f)) return;
    // 12. radius
    float mid = fm(0.5f, fa(a, c));
    float lam = fa(mid, __fsqrt_rn(fmaxf(0.1f, fs(fm(mid, mid), det))));
    float r = ceilf(fm(3.0f, __fsqrt_rn(lam)));
    // 13. centre
    float mux = fa(fm(cam.fx, ux), cam.cx);
    float muy = fa(fm(cam.fy, uy), cam.cy);
    o.mux = mux; o.muy = muy;
    // 14. finiteness
    if (!(isfinite(mux) && isfinite(muy) && isfinite(r))) return;
    // 15. extents towards -x, +x, -y, +y: the 3-sigma radius (3D-GS), or per half
    float ex0 = r, ex1 = r, ey0 = r, ey1 = r;
    if (rect_mode == 1 || rect_mode == 2) {
        // 15a. 1-sigma support of each half under the projection, without the low-pass:
        // the whole ellipse (A0, C0) where the half's outer edge faces that way (sign of
        // k = P L^T n^), else the cut ellipse of the splitting plane (Ar, Cr)
        float K0 = 0.0f, K1 = 0.0f, Ar = A0, Cr = C0;
        float nn = fm(nrm[0], nrm[0]);
        nn = fa(nn, fm(nrm[1], nrm[1]));
        nn = fa(nn, fm(nrm[2], nrm[2]));
        if (nn >= 1e-24f) {
            const float nl = __fsqrt_rn(nn);
            const float h0 = fdv(nrm[0], nl), h1 = fdv(nrm[1], nl), h2 = fdv(nrm[2], nl);
            float u[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float acc = fm(o.L[0][k], h0);
                acc = fa(acc, fm(o.L[1][k], h1));
                u[k] = fa(acc, fm(o.L[2][k], h2));
            }
            float vs = fm(u[0], u[0]);
            vs = fa(vs, fm(u[1], u[1]));
            vs = fa(vs, fm(u[2], u[2]));
            K0 = fm(o.P[0][0], u[0]);
            K0 = fa(K0, fm(o.P[0][1], u[1]));
            K0 = fa(K0, fm(o.P[0][2], u[2]));
            K1 = fm(o.P[1][0], u[0]);
            K1 = fa(K1, fm(o.P[1][1], u[1]));
            K1 = fa(K1, fm(o.P[1][2], u[2]));
            if (vs > 0.0f && rect_mode == 1) {
                Ar = fmaxf(0.0f, fs(A0, fdv(fm(K0, K0), vs)));
                Cr = fmaxf(0.0f, fs(C0, fdv(fm(K1, K1), vs)));
            } else if (vs > 0.0f) {
                // 15a'. Algorithm 1 (Suppl. B.1): basis (v1, v2, n^) of the splitting plane,
                // the covariance in it from the rows L^T v1, L^T v2, u = L^T n^, the in-plane
                // covariance given the normal coordinate (a', b', c'), a third variance
                // min(a', c') / 100 along n^, and the diagonal of M sigma M^T for the
                // flattened covariance sigma in place of the cut ellipse's
                float v1[3], v2[3];
                if (h0 == 0.0f && h1 == 0.0f) {
                    v1[0] = 1.0f; v1[1] = 0.0f; v1[2] = 0.0f;
                    v2[0] = 0.0f; v2[1] = 1.0f; v2[2] = 0.0f;
                } else {
                    const float l1 = __fsqrt_rn(fa(fm(h1, h1), fm(h0, h0)));
                    v1[0] = fdv(h1, l1); v1[1] = -fdv(h0, l1); v1[2] = 0.0f;
                    const float c0 = -fm(h2, v1[1]);      // n^ x v1 with v1[2] = 0
                    const float c1 = fm(h2, v1[0]);
                    const float c2 = fs(fm(h0, v1[1]), fm(h1, v1[0]));
                    float l2 = fm(c0, c0);
                    l2 = fa(l2, fm(c1, c1));
                    l2 = __fsqrt_rn(fa(l2, fm(c2, c2)));
                    v2[0] = fdv(c0, l2); v2[1] = fdv(c1, l2); v2[2] = fdv(c2, l2);
                }
                float g1[3], g2[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float acc = fm(o.L[0][k], v1[0]);
                    acc = fa(acc, fm(o.L[1][k], v1[1]));
                    g1[k] = fa(acc, fm(o.L[2][k], v1[2]));
                    acc = fm(o.L[0][k], v2[0]);
                    acc = fa(acc, fm(o.L[1][k], v2[1]));
                    g2[k] = fa(acc, fm(o.L[2][k], v2[2]));
                }
                float s00 = fm(g1[0], g1[0]), s01 = fm(g1[0], g2[0]), s11 = fm(g2[0], g2[0]);
                float s02 = fm(g1[0], u[0]), s12 = fm(g2[0], u[0]);
#pragma unroll
                for (int k = 1; k < 3; ++k) {
                    s00 = fa(s00, fm(g1[k], g1[k]));
                    s01 = fa(s01, fm(g1[k], g2[k]));
                    s11 = fa(s11, fm(g2[k], g2[k]));
                    s02 = fa(s02, fm(g1[k], u[k]));
                    s12 = fa(s12, fm(g2[k], u[k]));
                }
                const float ap = fs(s00, fdv(fm(s02, s02), vs));
                const float bp = fs(s01, fdv(fm(s02, s12), vs));
                const float cp = fs(s11, fdv(fm(s12, s12), vs));
                const float tt = fdv(fminf(ap, cp), 100.0f);
                float qv[2][3];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    float acc = fm(M[i][0], v1[0]);
                    acc = fa(acc, fm(M[i][1], v1[1]));
                    qv[i][0] = fa(acc, fm(M[i][2], v1[2]));
                    acc = fm(M[i][0], v2[0]);
                    acc = fa(acc, fm(M[i][1], v2[1]));
                    qv[i][1] = fa(acc, fm(M[i][2], v2[2]));
                    acc = fm(M[i][0], h0);
                    acc = fa(acc, fm(M[i][1], h1));
                    qv[i][2] = fa(acc, fm(M[i][2], h2));
                }
                float As = fm(ap, fm(qv[0][0], qv[0][0]));
                As = fa(As, fm(fm(2.0f, bp), fm(qv[0][0], qv[0][1])));
                As = fa(As, fm(cp, fm(qv[0][1], qv[0][1])));
                As = fa(As, fm(tt, fm(qv[0][2], qv[0][2])));
                float Cs = fm(ap, fm(qv[1][0], qv[1][0]));
                Cs = fa(Cs, fm(fm(2.0f, bp), fm(qv[1][0], qv[1][1])));
                Cs = fa(Cs, fm(cp, fm(qv[1][1], qv[1][1])));
                Cs = fa(Cs, fm(tt, fm(qv[1][2], qv[1][2])));
                Ar = fmaxf(0.0f, As);
                Cr = fmaxf(0.0f, Cs);
            }
        }
        // 15b. a half is splatted when its opacity reaches the 1/255 floor
        const float amin = 1.0f / 255.0f;
        const bool keep1 = op1 >= amin, keep2 = op2 >= amin;
        if (!keep1 && !keep2) return;
        float hxp = 0.0f, hxm = 0.0f, hyp = 0.0f, hym = 0.0f;
        if (keep1) {   // side n.(x - mu) >= 0
            hxp = fmaxf(hxp, K0 >= 0.0f ? A0 : Ar);
            hxm = fmaxf(hxm, K0 <= 0.0f ? A0 : Ar);
            hyp = fmaxf(hyp, K1 >= 0.0f ? C0 : Cr);
            hym = fmaxf(hym, K1 <= 0.0f ? C0 : Cr);
        }
        if (keep2) {   // side n.(x - mu) <= 0
            hxp = fmaxf(hxp, K0 <= 0.0f ? A0 : Ar);
            hxm = fmaxf(hxm, K0 >= 0.0f ? A0 : Ar);
            hyp = fmaxf(hyp, K1 <= 0.0f ? C0 : Cr);
            hym = fmaxf(hym, K1 >= 0.0f ? C0 : Cr);
        }
        // 15c. 3-sigma extents with the low-pass in quadrature
        ex1 = fm(3.0f, __fsqrt_rn(fa(hxp, lp)));
        ex0 = fm(3.0f, __fsqrt_rn(fa(hxm, lp)));
        ey1 = fm(3.0f, __fsqrt_rn(fa(hyp, lp)));
        ey0 = fm(3.0f, __fsqrt_rn(fa(hym, lp)));
        if (!(isfinite(ex0) && isfinite(ex1) && isfinite(ey0) && isfinite(ey1))) return;
    }
    // 16. tile rect
    int tiles_x = div_up(cam.width, tw), tiles_y = div_up(cam.height, th);
    // the tile sizes are powers of two, so x * (1/t) rounds to the same value as x / t
    const float itw = __frcp_rn((float)tw), ith = __frcp_rn((float)th);
    float x0 = floorf(fm(fs(mux, ex0), itw));
    float x1 = fa(floorf(fm(fa(mux, ex1), itw)), 1.0f);
    float y0 = floorf(fm(fs(muy, ey0), ith));
    float y1 = fa(floorf(fm(fa(muy, ey1), ith)), 1.0f);
    x0 = fminf(fmaxf(x0, 0.0f), (float)tiles_x);
    x1 = fminf(fmaxf(x1, 0.0f), (float)tiles_x);
    y0 = fminf(fmaxf(y0, 0.0f), (float)tiles_y);
    y1 = fminf(fmaxf(y1, 0.0f), (float)tiles_y);
    o.rect[0] = (int)x0; o.rect[1] = (int)y0; o.rect[2] = (int)x1; o.rect[3] = (int)y1;
    int nx = o.rect[2] - o.rect[0], ny = o.rect[3] - o.rect[1];
    o.tiles = (nx > 0 && ny > 0) ? (unsigned)(nx * ny) : 0u;
    o.culled = false;
}

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Full projection in precision T (FP64 fallback; FP32/FP64 recompute in the
// backward).  Same mathematics as canon_project plus the half-plane terms, with
// free operation order.
template <typename T>
struct Proj {
    T qn, qh[4], R[3][3], L[3][3], t[3], uxc, uyc;
    bool clx, cly;
    T J00, J02, J11, J12, M[2][3], P[2][3], a, b, c, det, Q[3];
    T n0, n1, det0;          // hat Sigma_0 = P P^T (before the low-pass): diagonal, determinant
    T nn, nh[3], u[3], var_s, k[2], w[2], v;
    T lp;                    // the low-pass l
    int mode;

    __device__ __forceinline__ void run(const float *m, const float *s, const float *q,
                                        const float *nrm, const hgs_camera &cam, float lp,
                                        int fov_clamp) {
        const float *V = cam.viewmat;
        this->lp = (T)lp;
        qn = sqrt_f((T)q[0] * q[0] + (T)q[1] * q[1] + (T)q[2] * q[2] + (T)q[3] * q[3]);
        T iq = rcp_f(qn);
#pragma unroll
        for (int i = 0; i < 4; ++i) qh[i] = (T)q[i] * iq;
        const T a0 = qh[0], a1 = qh[1], a2 = qh[2], a3 = qh[3];   // (w, x, y, z)
        R[0][0] = 1 - 2 * (a2 * a2 + a3 * a3); R[0][1] = 2 * (a1 * a2 - a0 * a3); R[0][2] = 2 * (a1 * a3 + a0 * a2);
        R[1][0] = 2 * (a1 * a2 + a0 * a3); R[1][1] = 1 - 2 * (a1 * a1 + a3 * a3); R[1][2] = 2 * (a2 * a3 - a0 * a1);
        R[2][0] = 2 * (a1 * a3 - a0 * a2); R[2][1] = 2 * (a2 * a3 + a0 * a1); R[2][2] = 1 - 2 * (a1 * a1 + a2 * a2);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) L[i][kk] = R[i][kk] * (T)s[kk];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            t[i] = (T)V[4 * i] * m[0] + (T)V[4 * i + 1] * m[1] + (T)V[4 * i + 2] * m[2] + (T)V[4 * i + 3];
        const T itz = rcp_f(t[2]);
        T ux = t[0] * itz, uy = t[1] * itz;
        uxc = ux; uyc = uy; clx = cly = false;
        if (fov_clamp) {
            T limx = (T)1.3 * ((T)0.5 * cam.width * rcp_f((T)cam.fx));
            T limy = (T)1.3 * ((T)0.5 * cam.height * rcp_f((T)cam.fy));
            if (ux > limx) { uxc = limx; clx = true; }
            if (ux < -limx) { uxc = -limx; clx = true; }
            if (uy > limy) { uyc = limy; cly = true; }
            if (uy < -limy) { uyc = -limy; cly = true; }
        }
        J00 = (T)cam.fx * itz; J02 = -(T)cam.fx * uxc * itz;
        J11 = (T)cam.fy * itz; J12 = -(T)cam.fy * uyc * itz;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            M[0][kk] = J00 * V[kk] + J02 * V[8 + kk];
            M[1][kk] = J11 * V[4 + kk] + J12 * V[8 + kk];
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) P[i][kk] = M[i][0] * L[0][kk] + M[i][1] * L[1][kk] + M[i][2] * L[2][kk];
        n0 = P[0][0] * P[0][0] + P[0][1] * P[0][1] + P[0][2] * P[0][2];
        n1 = P[1][0] * P[1][0] + P[1][1] * P[1][1] + P[1][2] * P[1][2];
        a = n0 + (T)lp;
        b = P[0][0] * P[1][0] + P[0][1] * P[1][1] + P[0][2] * P[1][2];
        c = n1 + (T)lp;
        T cr[3];
        cross3(P[0], P[1], cr);
        det0 = dot3(cr, cr);
        det = det0 + (T)lp * (n0 + n1) + (T)lp * (T)lp;
        T id = rcp_f(det);
        Q[0] = c * id; Q[1] = -b * id; Q[2] = a * id;
        nn = sqrt_f((T)nrm[0] * nrm[0] + (T)nrm[1] * nrm[1] + (T)nrm[2] * nrm[2]);
        var_s = v = 0; k[0] = k[1] = w[0] = w[1] = 0;
        u[0] = u[1] = u[2] = nh[0] = nh[1] = nh[2] = 0;
        if (nn < (T)1e-12) { mode = MODE_HALF; return; }
        T in = rcp_f(nn);
#pragma unroll
        for (int i = 0; i < 3; ++i) nh[i] = (T)nrm[i] * in;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) u[kk] = L[0][kk] * nh[0] + L[1][kk] * nh[1] + L[2][kk] * nh[2];
        var_s = dot3(u, u);
        k[0] = dot3(P[0], u);
        k[1] = dot3(P[1], u);
        w[0] = Q[0] * k[0] + Q[1] * k[1];
        w[1] = Q[1] * k[0] + Q[2] * k[1];
        T up0[3], up1[3];
        cross3(u, P[0], up0);
        cross3(u, P[1], up1);
        const T trip = dot3(u, cr);
        v = (trip * trip + (T)lp * (dot3(up0, up0) + dot3(up1, up1)) + (T)lp * (T)lp * var_s) * id;
        mode = (v <= (T)1e-12 * var_s) ? MODE_STEP : MODE_NORMAL;
    }

    __device__ __forceinline__ bool degenerate() const {
        return mode == MODE_NORMAL && v < (T)kVRelFp64 * var_s;
    }

    // hat Sigma ill-conditioned: lambda_max / lambda_min > kCondFp64, tested without a
    // root as tr^2 > (1 + K)^2 / K det (tr^2 / det = (1 + c)^2 / c for condition c).
    __device__ __forceinline__ bool ill_conditioned() const {
        const T tr = a + c;
        return tr * tr > (T)kCondFp64Test * det;
    }

    // Opacity factor of the Mip-Splatting 2D filter: sqrt(det hat Sigma_0 / det hat Sigma).
    __device__ __forceinline__ T mip_factor() const { return det0 > (T)0 ? sqrt_f(det0 * rcp_f(det)) : (T)0; }
};

// ---- real spherical harmonics, degree <= 3 ---------------------------------
// Basis (Condon-Shortley phase, index l*l + l + m):
//   l=0: 1/(2 sqrt(pi))
//   l=1: -c1 y, c1 z, -c1 x                          c1 = sqrt(3/(4 pi))
//   l=2: c2a xy, -c2a yz, c2b (2z^2-x^2-y^2), -c2a xz, c2c (x^2-y^2)
//        c2a = sqrt(15/pi)/2, c2b = sqrt(5/pi)/4, c2c = sqrt(15/pi)/4
//   l=3: -c3a y(3x^2-y^2), c3b xyz, -c3c y(4z^2-x^2-y^2), c3d z(2z^2-3x^2-3y^2),
//        -c3c x(4z^2-x^2-y^2), c3e z(x^2-y^2), -c3a x(x^2-3y^2)
//        c3a = sqrt(70/pi)/8, c3b = sqrt(105/pi)/2, c3c = sqrt(42/pi)/8,
//        c3d = sqrt(7/pi)/4, c3e = sqrt(105/pi)/4
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.48860251190291992f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.54627421529603959f;
constexpr float kC3a = 0.59004358992664352f;
constexpr float kC3b = 2.8906114426405538f;
constexpr float kC3c = 0.45704579946446572f;
constexpr float kC3d = 0.37317633259011540f;
constexpr float kC3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
    Y[0] = kC0;
    if (deg < 1) return;
    Y[1] = -kC1 * y; Y[2] = kC1 * z; Y[3] = -kC1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = -kC2a * y * z;
    Y[6] = kC2b * (2.0f * zz - xx - yy);
    Y[7] = -kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kC3a * y * (3.0f * xx - yy);
    Y[10] = kC3b * x * y * z;
    Y[11] = -kC3c * y * (4.0f * zz - xx - yy);
    Y[12] = kC3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -kC3c * x * (4.0f * zz - xx - yy);
    Y[14] = kC3e * z * (xx - yy);
    Y[15] = -kC3a * x * (xx - 3.0f * yy);
}

// sum_l w_l grad Y_l, with the Cartesian gradient of each basis polynomial.
__device__ __forceinline__ void sh_grad_dot(int deg, float x, float y, float z, const float w[16], float gd[3]) {
    gd[0] = gd[1] = gd[2] = 0.0f;
    if (deg < 1) return;
    gd[0] -= kC1 * w[3];
    gd[1] -= kC1 * w[1];
    gd[2] += kC1 * w[2];
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gd[0] += kC2a * (y * w[4] - z * w[7]) - 2.0f * kC2b * x * w[6] + 2.0f * kC2c * x * w[8];
    gd[1] += kC2a * (x * w[4] - z * w[5]) - 2.0f * kC2b * y * w[6] - 2.0f * kC2c * y * w[8];
    gd[2] += -kC2a * (y * w[5] + x * w[7]) + 4.0f * kC2b * z * w[6];
    if (deg < 3) return;
    gd[0] += -6.0f * kC3a * x * y * w[9] + kC3b * y * z * w[10] + 2.0f * kC3c * x * y * w[11]
             - 6.0f * kC3d * x * z * w[12] - kC3c * (4.0f * zz - 3.0f * xx - yy) * w[13]
             + 2.0f * kC3e * x * z * w[14] - 3.0f * kC3a * (xx - yy) * w[15];
    gd[1] += -3.0f * kC3a * (xx - yy) * w[9] + kC3b * x * z * w[10] - kC3c * (4.0f * zz - xx - 3.0f * yy) * w[11]
             - 6.0f * kC3d * y * z * w[12] + 2.0f * kC3c * x * y * w[13] - 2.0f * kC3e * y * z * w[14]
             + 6.0f * kC3a * x * y * w[15];
    gd[2] += kC3b * x * y * w[10] - 8.0f * kC3c * y * z * w[11] + kC3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12]
             - 8.0f * kC3c * x * z * w[13] + kC3e * (xx - yy) * w[14];
}

__device__ __forceinline__ void camera_centre(const hgs_camera &cam, float c[3]) {
    const float *V = cam.viewmat;
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] = -(V[i] * V[3] + V[4 + i] * V[7] + V[8 + i] * V[11]);
}

// ---- parameter staging -----------------------------------------------------------
// A block projects kProjBlock consecutive splats.  Their parameter rows are
// contiguous in every input array, so the block copies each slice into shared
// memory with 16-byte cp.async copies (bypassing registers), then each thread
// reads its own row.  SH rows of 48 floats are padded to 52 in shared memory so
// that 128-bit reads of consecutive threads fall in distinct banks.
constexpr int kShStride3 = 52;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// rows x row_floats floats from src (16-B aligned) into dst with the given row stride.
__device__ __forceinline__ void stage_rows(const float *__restrict__ src, int rows, int row_floats, float *dst,
                                           int dst_stride) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (row_floats == dst_stride) {
        const int cnt = rows * row_floats, n4 = cnt >> 2;
        for (int j = tid; j < n4; j += nt) cp_async16(dst + 4 * j, src + 4 * j);
        for (int j = 4 * n4 + tid; j < cnt; j += nt) dst[j] = __ldg(src + j);
    } else {                                   // row_floats is a multiple of 4
        const int per = row_floats >> 2, n4 = rows * per;
        for (int j = tid; j < n4; j += nt) {
            const int r = j / per, c = j - r * per;
            cp_async16(dst + r * dst_stride + 4 * c, src + (size_t)r * row_floats + 4 * c);
        }
    }
}

template <int NB>
struct StageSmemN {
    static constexpr int kRows = NB;
    float mean[3 * NB];
    float scale[3 * NB];
    float nrm[3 * NB];
    float quat[4 * NB];
    float o1[NB];
    float o2[NB];
    float sh[kShStride3 * NB];
};
using StageSmem = StageSmemN<kProjBlock>;
using BwdStageSmem = StageSmemN<kProjBwdBlock>;

// Copies the block's parameter rows into shared memory, plus optionally `extra_floats`
// floats per row from `extra` into `extra_dst` in the same batch of asynchronous copies.
// With sh_later the SH rows (three quarters of the bytes at degree 3) are a second
// group of copies still in flight on return, for the caller to overlap with the
// geometry; sh_arrived() (a block barrier) precedes their use.  Measured at 3M splats:
// projection 0.219 vs 0.232 ms.  (Copying each thread's own row instead, so that no
// barrier is needed, was slower: 0.246 ms; so was the adjoint restructured around the
// barrier, hence it stages everything first.)
// SH rows of degree DEG into shared memory at their padded stride.  The row width and
// the block size are compile-time constants, so each 16-byte piece's row and column come
// from a multiply-shift rather than a division (measured: the division made the
// projection issue-bound at ~1,570 instructions per splat).
template <int DEG, int NB>
__device__ __forceinline__ void stage_sh(const float *__restrict__ src, int rows, float *dst) {
    constexpr int nc3 = 3 * (DEG + 1) * (DEG + 1), shs = DEG == 3 ? kShStride3 : nc3;
    if constexpr (nc3 == shs) {
        stage_rows(src, rows, nc3, dst, nc3);
    } else {                                   // nc3 is a multiple of 4
        constexpr int per = nc3 / 4;
        const int n4 = rows * per;
#pragma unroll 4
        for (int j = threadIdx.x; j < n4; j += NB) {
            const int r = j / per, c = j - r * per;
            cp_async16(dst + r * shs + 4 * c, src + (size_t)r * nc3 + 4 * c);
        }
    }
}

template <int DEG, class SM>
__device__ __forceinline__ void stage_params(const hgs_gaussians &g, int base, int rows, SM &sm,
                                             const float *extra = nullptr, int extra_floats = 0,
                                             float *extra_dst = nullptr, bool sh_later = false) {
    constexpr int nc3 = 3 * (DEG + 1) * (DEG + 1);
    if (extra) stage_rows(extra + (size_t)extra_floats * base, rows, extra_floats, extra_dst, extra_floats);
    stage_rows(g.means + 3 * (size_t)base, rows, 3, sm.mean, 3);
    stage_rows(g.scales + 3 * (size_t)base, rows, 3, sm.scale, 3);
    stage_rows(g.normals + 3 * (size_t)base, rows, 3, sm.nrm, 3);
    stage_rows(g.quats + 4 * (size_t)base, rows, 4, sm.quat, 4);
    stage_rows(g.opac1 + base, rows, 1, sm.o1, 1);
    stage_rows(g.opac2 + base, rows, 1, sm.o2, 1);
    if (sh_later) {
        cp_async_commit();
        stage_sh<DEG, SM::kRows>(g.sh + (size_t)nc3 * base, rows, sm.sh);
        cp_async_commit();
        cp_async_wait_prev();
    } else {
        stage_sh<DEG, SM::kRows>(g.sh + (size_t)nc3 * base, rows, sm.sh);
        cp_async_wait_all();
    }
    __syncthreads();
}

__device__ __forceinline__ void sh_arrived() {
    cp_async_wait_all();
    __syncthreads();
}

struct Params {
    float m[3], s[3], q[4], n[3];
};

template <class SM>
__device__ __forceinline__ Params read_params(const SM &sm, int t) {
    Params P;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P.m[k] = sm.mean[3 * t + k];
        P.s[k] = sm.scale[3 * t + k];
        P.n[k] = sm.nrm[3 * t + k];
    }
    const float4 q4 = reinterpret_cast<const float4 *>(sm.quat)[t];
    P.q[0] = q4.x; P.q[1] = q4.y; P.q[2] = q4.z; P.q[3] = q4.w;
    return P;
}

// SH colour (before the clamp) from the staged coefficients of thread t.  Degree 3
// rows (48 floats at stride 52) are read as twelve 128-bit loads, which consecutive
// threads take from distinct banks; entry j of a row is coefficient j / 3 of
// channel j % 3.
template <int DEG, class SM>
__device__ __forceinline__ void sh_colour(const SM &sm, int t, const float Y[16], float out[3]) {
    constexpr int nc = (DEG + 1) * (DEG + 1);
    float acc[3] = {0.0f, 0.0f, 0.0f};
    if (DEG == 3) {
        const float4 *c4 = reinterpret_cast<const float4 *>(sm.sh + t * kShStride3);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float4 c = c4[q];
            acc[(4 * q) % 3] += c.x * Y[(4 * q) / 3];
            acc[(4 * q + 1) % 3] += c.y * Y[(4 * q + 1) / 3];
            acc[(4 * q + 2) % 3] += c.z * Y[(4 * q + 2) / 3];
            acc[(4 * q + 3) % 3] += c.w * Y[(4 * q + 3) / 3];
        }
    } else {
        const float *c = sm.sh + t * (3 * nc);
#pragma unroll
        for (int l = 0; l < nc; ++l) {
            acc[0] += c[3 * l] * Y[l];
            acc[1] += c[3 * l + 1] * Y[l];
            acc[2] += c[3 * l + 2] * Y[l];
        }
    }
    out[0] = acc[0] + 0.5f; out[1] = acc[1] + 0.5f; out[2] = acc[2] + 0.5f;
}

struct HalfPlane {
    int mode;
    float wpx, wpy;
};

// Appends a (view, splat) index to a list [count, entries...] with one atomic per
// warp.  Used to gather the rare near-degenerate splats, so that their FP64 work
// runs in full warps in a follow-up kernel instead of stalling a warp of
// FP32 splats on one lane (FP64 issues at a small fraction of the FP32 rate).
__device__ __forceinline__ void list_append(uint32_t *list, bool want, uint32_t value) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, want);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(list, (uint32_t)__popc(m));
    base = __shfl_sync(act, base, leader);
    if (want) list[1 + base + __popc(m & ((1u << lane) - 1u))] = value;
}

__device__ __forceinline__ Params load_params(const hgs_gaussians &g, int i) {
    Params P;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P.m[k] = g.means[3 * (size_t)i + k];
        P.s[k] = g.scales[3 * (size_t)i + k];
        P.n[k] = g.normals[3 * (size_t)i + k];
    }
    const float4 q4 = reinterpret_cast<const float4 *>(g.quats)[i];
    P.q[0] = q4.x; P.q[1] = q4.y; P.q[2] = q4.z; P.q[3] = q4.w;
    return P;
}

// FP64 recomputation of the half-plane terms of a splat whose plane nearly
// contains the ray.
__device__ __forceinline__ HalfPlane half_plane_fp64(const Params &P, const hgs_camera &cam, float lp, int fov_clamp) {
    Proj<double> d;
    d.run(P.m, P.s, P.q, P.n, cam, lp, fov_clamp);
    HalfPlane h;
    h.mode = d.mode;
    h.wpx = h.wpy = 0.0f;
    if (d.mode == MODE_NORMAL) {
        const double sc = 1.0 / sqrt(2.0 * d.v);
        h.wpx = (float)(d.w[0] * sc);
        h.wpy = (float)(d.w[1] * sc);
    } else if (d.mode == MODE_STEP) {
        h.wpx = (float)d.w[0] * kStepScale;
        h.wpy = (float)d.w[1] * kStepScale;
    }
    return h;
}

// Geometry of one (view, splat): binning fields written out, conic factor and
// half-plane terms kept for the record.  False when the splat is not drawn.
struct Geo {
    float u11, u12, u22, wpx, wpy;
    float comp;              // opacity factor: 1, or the Mip-Splatting 2D filter's
};

__device__ __forceinline__ bool project_geo(const ProjLaunch &p, const Params &P, float o1, float o2, int v,
                                            size_t vi, Geo &out) {
    const hgs_camera &cam = p.cams[v];
    const float lp = p.cfg.lowpass;
    bool defer = false;
    Canon cb;
    canon_project(P.m, P.s, P.q, P.n, o1, o2, cam, lp, p.cfg.fov_clamp, p.cfg.tile_w, p.cfg.tile_h,
                  p.cfg.rect_mode, cb);
    p.out.depth[vi] = cb.depth;
    reinterpret_cast<int4 *>(p.out.rect)[vi] = make_int4(cb.rect[0], cb.rect[1], cb.rect[2], cb.rect[3]);
    p.out.tiles[vi] = cb.culled ? 0u : cb.tiles;
    if (cb.culled || cb.tiles == 0) return false;

    // conic factor and half-plane terms, FP32
    const float n0 = dot3(cb.P[0], cb.P[0]), n1 = dot3(cb.P[1], cb.P[1]);
    float cr[3];
    cross3(cb.P[0], cb.P[1], cr);
    const float det0 = dot3(cr, cr);
    const float det = det0 + lp * (n0 + n1) + lp * lp;
    const float id = rcp_f(det);
    const float a_ = cb.a, b_ = cb.b, c_ = cb.c;
    out.wpx = out.wpy = 0.0f;
    // Mip-Splatting's 2D filter: the low-pass as a normalised convolution scales the
    // footprint by sqrt(det hat Sigma_0 / det hat Sigma), both halves alike (exact
    // operations: with no low-pass the factor is exactly 1)
    out.comp = p.cfg.mip ? sqrtf(det0 / det) : 1.0f;
    const float nn = sqrt_f(dot3(P.n, P.n));
    if (nn >= 1e-12f) {
        const float in = rcp_f(nn);
        const float nh[3] = {P.n[0] * in, P.n[1] * in, P.n[2] * in};
        float u[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) u[k] = cb.L[0][k] * nh[0] + cb.L[1][k] * nh[1] + cb.L[2][k] * nh[2];
        const float var_s = dot3(u, u);
        const float k0 = dot3(cb.P[0], u), k1 = dot3(cb.P[1], u);
        const float wx = (c_ * k0 - b_ * k1) * id;
        const float wy = (a_ * k1 - b_ * k0) * id;
        float up0[3], up1[3];
        cross3(u, cb.P[0], up0);
        cross3(u, cb.P[1], up1);
        const float trip = dot3(u, cr);
        const float vv = (trip * trip + lp * (dot3(up0, up0) + dot3(up1, up1)) + lp * lp * var_s) * id;
        if (vv < kVRelFp64 * var_s) {
            defer = true;          // w' is written by k_project_fp64
        } else {
            const float sc = rsqrtf(2.0f * vv);
            out.wpx = wx * sc;
            out.wpy = wy * sc;
        }
    }
    // Cholesky factor of the conic
    out.u22 = rsqrtf(c_);
    out.u11 = sqrt_f(c_ * id);
    out.u12 = -b_ * rsqrtf(c_ * det);
    list_append(p.out.fp64_list, defer, (uint32_t)vi);
    return true;
}

// SH colour of a drawn (view, splat) and its 64-byte record.
template <int DEG>
__device__ __forceinline__ void project_record(const ProjLaunch &p, const StageSmem &sm, int t, const Params &P,
                                               float o1, float o2, int v, size_t vi, const Geo &g) {
    const hgs_camera &cam = p.cams[v];
    float cpos[3];
    camera_centre(cam, cpos);
    const float dx = P.m[0] - cpos[0], dy = P.m[1] - cpos[1], dz = P.m[2] - cpos[2];
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    float Y[16];
    sh_basis(DEG, dx * il, dy * il, dz * il, Y);
    float rgb[3];
    sh_colour<DEG>(sm, t, Y, rgb);
    float ctr[4];
    precise_centre(P.m, cam, ctr);
    float4 *rec = reinterpret_cast<float4 *>(p.out.rec) + 4 * vi;
    rec[0] = make_float4(ctr[0], ctr[1], ctr[2], ctr[3]);
    rec[1] = make_float4(g.u11, g.u12, g.u22, g.wpx);
    rec[2] = make_float4(g.wpy, o1 * g.comp, o2 * g.comp, fmaxf(rgb[0], 0.0f));
    rec[3] = make_float4(fmaxf(rgb[1], 0.0f), fmaxf(rgb[2], 0.0f), 0.0f, 0.0f);
}

// One thread per splat.  With one view the SH rows are still arriving while the
// geometry is computed (a block barrier separates the two); with several views
// every row is staged first.
template <int DEG, bool ONE_VIEW>
__global__ void __launch_bounds__(kProjBlock, 5) k_project(ProjLaunch p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StageSmem &sm = *reinterpret_cast<StageSmem *>(smem_raw);
    const int n = p.g.n;
    const int base = blockIdx.x * kProjBlock;
    const int rows = min(kProjBlock, n - base);
    stage_params<DEG>(p.g, base, rows, sm, nullptr, 0, nullptr, ONE_VIEW);
    const int t = threadIdx.x;
    const bool live = t < rows;
    const int i = base + t;
    if (ONE_VIEW) {
        Params P;
        float o1 = 0.0f, o2 = 0.0f;
        Geo g;
        bool drawn = false;
        if (live) {
            P = read_params(sm, t);
            o1 = sm.o1[t];
            o2 = sm.o2[t];
            drawn = project_geo(p, P, o1, o2, 0, (size_t)i, g);
        }
        sh_arrived();
        if (drawn) project_record<DEG>(p, sm, t, P, o1, o2, 0, (size_t)i, g);
        return;
    }
    if (!live) return;
    const Params P = read_params(sm, t);
    const float o1 = sm.o1[t], o2 = sm.o2[t];
    for (int v = 0; v < p.n_views; ++v) {
        const size_t vi = (size_t)v * n + i;
        Geo g;
        if (project_geo(p, P, o1, o2, v, vi, g)) project_record<DEG>(p, sm, t, P, o1, o2, v, vi, g);
    }
}

// Half-plane terms of the gathered near-degenerate (view, splat) records, FP64.
// Entry e goes to block e % grid, so that a short list still spreads over all SMs.
__global__ void __launch_bounds__(kProjBlock) k_project_fp64(ProjLaunch p) {
    const uint32_t cnt = min(p.out.fp64_list[0], (uint32_t)p.n_views * (uint32_t)p.g.n);
    for (uint32_t e = blockIdx.x + gridDim.x * threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const uint32_t vi = p.out.fp64_list[1 + e];
        const int v = (int)(vi / (uint32_t)p.g.n), i = (int)(vi - (uint32_t)v * (uint32_t)p.g.n);
        const Params P = load_params(p.g, i);
        const HalfPlane h = half_plane_fp64(P, p.cams[v], p.cfg.lowpass, p.cfg.fov_clamp);
        p.out.rec[16 * (size_t)vi + 7] = h.wpx;
        p.out.rec[16 * (size_t)vi + 8] = h.wpy;
    }
}

// ---- adjoint -------------------------------------------------------------------
struct G2 {
    float v[12];
};

template <typename T>
// g_comp: dL/d(opacity factor) of the Mip-Splatting 2D filter (0 without it).
__device__ __forceinline__ void proj_vjp(const Proj<T> &f, const float *s, const hgs_camera &cam,
                                         const float *g2, float gm[3], float gs[3], float gq[4],
                                         float gn[3], T g_comp = 0) {
    const float *V = cam.viewmat;
    T gA = g2[2], gB = g2[3], gC = g2[4];
    T gk[2] = {0, 0}, gv = 0;
    if (f.mode == MODE_NORMAL) {
        // w' = w / sqrt(2 v) with w = conic k: the w part flows into the conic and k
        T sv = rcp_f(sqrt_f((T)2 * f.v));
        T gw0 = (T)g2[5] * sv, gw1 = (T)g2[6] * sv;
        gv = -((T)g2[5] * f.w[0] + (T)g2[6] * f.w[1]) * sv * sv * sv;
        gA += gw0 * f.k[0]; gB += gw0 * f.k[1] + gw1 * f.k[0]; gC += gw1 * f.k[1];
        gk[0] = f.Q[0] * gw0 + f.Q[1] * gw1;
        gk[1] = f.Q[1] * gw0 + f.Q[2] * gw1;
        // the v part goes to P and u below, through the cancellation-free form of v
    }
    // hat Sigma from the conic: Gs = -Q [[gA, gB/2], [gB/2, gC]] Q
    T hb = (T)0.5 * gB;
    T X00 = f.Q[0] * gA + f.Q[1] * hb, X01 = f.Q[0] * hb + f.Q[1] * gC;
    T X10 = f.Q[1] * gA + f.Q[2] * hb, X11 = f.Q[1] * hb + f.Q[2] * gC;
    T Gs00 = -(X00 * f.Q[0] + X01 * f.Q[1]);
    T Gs01 = -(X00 * f.Q[1] + X01 * f.Q[2]);
    T Gs11 = -(X10 * f.Q[1] + X11 * f.Q[2]);
    // comp = sqrt(det hat Sigma_0 / det hat Sigma):
    // d comp = comp/2 tr((hat Sigma_0^-1 - hat Sigma^-1) d hat Sigma_0), d hat Sigma = d hat Sigma_0
    if (g_comp != (T)0 && f.det0 > (T)0) {
        const T h = (T)0.5 * g_comp * f.mip_factor(), i0 = rcp_f(f.det0);
        Gs00 += h * (f.n1 * i0 - f.Q[0]);
        Gs01 += h * (-f.b * i0 - f.Q[1]);
        Gs11 += h * (f.n0 * i0 - f.Q[2]);
    }
    // hat Sigma = P P^T + l I and k = P u
    T gP[2][3], gu[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        gP[0][kk] = 2 * (Gs00 * f.P[0][kk] + Gs01 * f.P[1][kk]) + gk[0] * f.u[kk];
        gP[1][kk] = 2 * (Gs01 * f.P[0][kk] + Gs11 * f.P[1][kk]) + gk[1] * f.u[kk];
        gu[kk] = f.P[0][kk] * gk[0] + f.P[1][kk] * gk[1];
    }
    // v = N / det with N = (u.(p0 x p1))^2 + l (|u x p0|^2 + |u x p1|^2) + l^2 |u|^2 and
    // det = |p0 x p1|^2 + l (|p0|^2 + |p1|^2) + l^2 (the forward's form).  Differentiated
    // in that form, every term is a product of cross products no larger than the splat's
    // own plane-aligned extent, so nothing cancels when the plane nearly contains the ray;
    // the form var_s - k.w would subtract terms of order var_s / v from one another.
    if (gv != (T)0) {
        const T lp = f.lp;
        T cr[3], up0[3], up1[3], c0[3], c1[3], t0[3], t1[3];
        cross3(f.P[0], f.P[1], cr);
        cross3(f.u, f.P[0], up0);
        cross3(f.u, f.P[1], up1);
        const T trip = dot3(f.u, cr);
        const T g = gv * rcp_f(f.det), two_trip = 2 * trip, two_l = 2 * lp, vv = f.v;
        // d v / d p0 = [2 trip (p1 x u) + 2 l (up0 x u) - v (2 p1 x cr + 2 l p0)] / det
        cross3(f.P[1], f.u, c0);
        cross3(up0, f.u, t0);
        cross3(f.P[1], cr, c1);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            gP[0][kk] += g * (two_trip * c0[kk] + two_l * t0[kk] - vv * (2 * c1[kk] + two_l * f.P[0][kk]));
        // d v / d p1 = [2 trip up0 + 2 l (up1 x u) - v (2 cr x p0 + 2 l p1)] / det
        cross3(up1, f.u, t1);
        cross3(cr, f.P[0], c1);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            gP[1][kk] += g * (two_trip * up0[kk] + two_l * t1[kk] - vv * (2 * c1[kk] + two_l * f.P[1][kk]));
        // d v / d u = [2 trip cr + 2 l (p0 x up0 + p1 x up1) + 2 l^2 u] / det
        cross3(f.P[0], up0, t0);
        cross3(f.P[1], up1, t1);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            gu[kk] += g * (two_trip * cr[kk] + two_l * (t0[kk] + t1[kk]) + two_l * lp * f.u[kk]);
    }
    // P = M L
    T gM[2][3], gL[3][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) gM[i][j] = gP[i][0] * f.L[j][0] + gP[i][1] * f.L[j][1] + gP[i][2] * f.L[j][2];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) gL[j][kk] = f.M[0][j] * gP[0][kk] + f.M[1][j] * gP[1][kk] + f.nh[j] * gu[kk];
    // u = L^T n^, n^ = n / |n|
    if (f.mode != MODE_HALF) {
        T gnh[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) gnh[j] = f.L[j][0] * gu[0] + f.L[j][1] * gu[1] + f.L[j][2] * gu[2];
        T dd = gnh[0] * f.nh[0] + gnh[1] * f.nh[1] + gnh[2] * f.nh[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) gn[j] += (float)((gnh[j] - dd * f.nh[j]) * rcp_f(f.nn));
    }
    // L = R diag(s)
    T gR[3][3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        T acc = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gR[j][kk] = gL[j][kk] * (T)s[kk];
            acc += gL[j][kk] * f.R[j][kk];
        }
        gs[kk] += (float)acc;
    }
    // R(q^), q^ = q / |q|
    T w = f.qh[0], x = f.qh[1], y = f.qh[2], z = f.qh[3];
    T gqh[4];
    gqh[0] = 2 * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    gqh[1] = 2 * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2 * x * gR[1][1] - w * gR[1][2] + z * gR[2][0] +
                  w * gR[2][1] - 2 * x * gR[2][2]);
    gqh[2] = 2 * (-2 * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] +
                  z * gR[2][1] - 2 * y * gR[2][2]);
    gqh[3] = 2 * (-2 * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2 * z * gR[1][1] + y * gR[1][2] +
                  x * gR[2][0] + y * gR[2][1]);
    T dq = gqh[0] * w + gqh[1] * x + gqh[2] * y + gqh[3] * z;
#pragma unroll
    for (int j = 0; j < 4; ++j) gq[j] += (float)((gqh[j] - dq * f.qh[j]) * rcp_f(f.qn));
    // M = J W
    T gJ00 = gM[0][0] * V[0] + gM[0][1] * V[1] + gM[0][2] * V[2];
    T gJ02 = gM[0][0] * V[8] + gM[0][1] * V[9] + gM[0][2] * V[10];
    T gJ11 = gM[1][0] * V[4] + gM[1][1] * V[5] + gM[1][2] * V[6];
    T gJ12 = gM[1][0] * V[8] + gM[1][1] * V[9] + gM[1][2] * V[10];
    T tz = f.t[2], itz = rcp_f(tz), itz2 = itz * itz;
    T fx = cam.fx, fy = cam.fy;
    T gt[3] = {0, 0, 0};
    gt[2] -= (gJ00 * fx + gJ11 * fy) * itz2;
    if (!f.clx) { gt[0] -= gJ02 * fx * itz2; gt[2] += 2 * gJ02 * fx * f.t[0] * itz2 * itz; }
    else { gt[2] += gJ02 * fx * f.uxc * itz2; }
    if (!f.cly) { gt[1] -= gJ12 * fy * itz2; gt[2] += 2 * gJ12 * fy * f.t[1] * itz2 * itz; }
    else { gt[2] += gJ12 * fy * f.uyc * itz2; }
    // mu-hat = (fx tx/tz + cx, fy ty/tz + cy)
    gt[0] += (T)g2[0] * fx * itz;
    gt[1] += (T)g2[1] * fy * itz;
    gt[2] -= ((T)g2[0] * fx * f.t[0] + (T)g2[1] * fy * f.t[1]) * itz2;
    // t = W mu + t_c
#pragma unroll
    for (int j = 0; j < 3; ++j) gm[j] += (float)(V[j] * gt[0] + V[4 + j] * gt[1] + V[8 + j] * gt[2]);
}

struct Grads {
    float m[3], s[3], q[4], n[3];
};

// FP64 adjoint of the projection of one near-degenerate splat.
__device__ __forceinline__ Grads proj_vjp_fp64(const Params &P, const hgs_camera &cam, float lp, int fov_clamp,
                                               const G2 &g2, double g_comp) {
    Proj<double> d;
    d.run(P.m, P.s, P.q, P.n, cam, lp, fov_clamp);
    Grads r;
#pragma unroll
    for (int k = 0; k < 3; ++k) r.m[k] = r.s[k] = r.n[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.q[k] = 0.0f;
    proj_vjp<double>(d, P.s, cam, g2.v, r.m, r.s, r.q, r.n, g_comp);
    return r;
}

// One thread per splat.  SH gradients are gathered in shared rows and written out
// coalesced.  With one view (ONE_VIEW) each thread's gradient row overwrites its
// own coefficient row once the coefficients have been read, which halves the
// shared memory of a block; with several views the rows are separate and summed.
template <int DEG, bool ONE_VIEW>
__global__ void __launch_bounds__(kProjBwdBlock, 8) k_project_bwd(ProjBwdLaunch p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdStageSmem &sm = *reinterpret_cast<BwdStageSmem *>(smem_raw);
    // one view: screen-space gradient rows staged with the parameters; several views:
    // separate SH gradient rows
    float *extra = reinterpret_cast<float *>(smem_raw + sizeof(BwdStageSmem));
    float *gsh_s = ONE_VIEW ? sm.sh : extra;
    const int n = p.g.n;
    const int base = blockIdx.x * kProjBwdBlock;
    const int rows = min(kProjBwdBlock, n - base);
    constexpr int nc = (DEG + 1) * (DEG + 1), nc3 = 3 * nc, shs = DEG == 3 ? kShStride3 : nc3;
    if (!ONE_VIEW)
        for (int j = threadIdx.x; j < kProjBwdBlock * shs; j += blockDim.x) gsh_s[j] = 0.0f;
    if (ONE_VIEW)
        stage_params<DEG>(p.g, base, rows, sm, p.grad2d, 12, extra);
    else
        stage_params<DEG>(p.g, base, rows, sm);
    const int t = threadIdx.x;
    const float lp = p.cfg.lowpass;
    float gm[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gn[3] = {0, 0, 0};
    float go1 = 0.0f, go2 = 0.0f;
    if (t < rows) {
        const int i = base + t;
        const Params P = read_params(sm, t);
        float *gsh = gsh_s + t * shs;
        const float *shc = sm.sh + t * shs;
        bool wrote = false;
        for (int v = 0; v < p.n_views; ++v) {
            const size_t vi = (size_t)v * n + i;
            const float4 *g4 = ONE_VIEW ? reinterpret_cast<const float4 *>(extra) + 3 * t
                                        : reinterpret_cast<const float4 *>(p.grad2d) + 3 * vi;
            const float4 a = g4[0], b = g4[1], c = g4[2];
            G2 g2;
            g2.v[0] = a.x; g2.v[1] = a.y; g2.v[2] = a.z; g2.v[3] = a.w;
            g2.v[4] = b.x; g2.v[5] = b.y; g2.v[6] = b.z; g2.v[7] = b.w;
            g2.v[8] = c.x; g2.v[9] = c.y; g2.v[10] = c.z; g2.v[11] = c.w;
            bool any = false;
#pragma unroll
            for (int j = 0; j < 12; ++j) any |= (g2.v[j] != 0.0f);
            if (!any) continue;
            const hgs_camera &cam = p.cams[v];
            Proj<float> f;
            f.run(P.m, P.s, P.q, P.n, cam, lp, p.cfg.fov_clamp);
            // grad2d[7..8] are w.r.t. the opacities the compositing used (x comp with mip)
            const bool mip = p.cfg.mip != 0;
            const float comp = mip ? f.mip_factor() : 1.0f;
            go1 += comp * g2.v[7];
            go2 += comp * g2.v[8];
            const float g_comp = mip ? sm.o1[t] * g2.v[7] + sm.o2[t] * g2.v[8] : 0.0f;
            // geometry adjoint by k_project_bwd_fp64
            const bool defer = f.degenerate() || f.ill_conditioned();
            list_append(p.fp64_list, defer, (uint32_t)vi);
            if (!defer) proj_vjp<float>(f, P.s, cam, g2.v, gm, gs, gq, gn, g_comp);
            // SH colour: rgb = max(0, sum c Y(dir) + 1/2), dir = unit(mu - camera centre)
            float cpos[3];
            camera_centre(cam, cpos);
            const float dv[3] = {P.m[0] - cpos[0], P.m[1] - cpos[1], P.m[2] - cpos[2]};
            const float il = rsqrtf(dot3(dv, dv));
            const float dir[3] = {dv[0] * il, dv[1] * il, dv[2] * il};
            float Y[16];
            sh_basis(DEG, dir[0], dir[1], dir[2], Y);
            float raw[3];
            sh_colour<DEG>(sm, t, Y, raw);
            float graw[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) graw[ch] = raw[ch] < 0.0f ? 0.0f : g2.v[9 + ch];
            // d rgb / d coefficient (l, ch) = Y_l (into the shared row), and
            // wl[l] = sum_ch graw[ch] c[l][ch] for the direction gradient
            float wl[16];
#pragma unroll
            for (int l = 0; l < 16; ++l) wl[l] = 0.0f;
            wrote = true;
            if (DEG == 3) {
                float4 *g4s = reinterpret_cast<float4 *>(gsh);
                const float4 *c4 = reinterpret_cast<const float4 *>(shc);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const float4 c = c4[q];                     // read before an in-place overwrite
                    float4 a = ONE_VIEW ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : g4s[q];
                    a.x += graw[(4 * q) % 3] * Y[(4 * q) / 3];
                    a.y += graw[(4 * q + 1) % 3] * Y[(4 * q + 1) / 3];
                    a.z += graw[(4 * q + 2) % 3] * Y[(4 * q + 2) / 3];
                    a.w += graw[(4 * q + 3) % 3] * Y[(4 * q + 3) / 3];
                    g4s[q] = a;
                    wl[(4 * q) / 3] += graw[(4 * q) % 3] * c.x;
                    wl[(4 * q + 1) / 3] += graw[(4 * q + 1) % 3] * c.y;
                    wl[(4 * q + 2) / 3] += graw[(4 * q + 2) % 3] * c.z;
                    wl[(4 * q + 3) / 3] += graw[(4 * q + 3) % 3] * c.w;
                }
            } else {
#pragma unroll
                for (int l = 0; l < nc; ++l) {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float c = shc[3 * l + ch];
                        wl[l] += graw[ch] * c;
                        gsh[3 * l + ch] = (ONE_VIEW ? 0.0f : gsh[3 * l + ch]) + graw[ch] * Y[l];
                    }
                }
            }
            float gd[3];
            sh_grad_dot(DEG, dir[0], dir[1], dir[2], wl, gd);
            const float dd = dot3(gd, dir);
#pragma unroll
            for (int k = 0; k < 3; ++k) gm[k] += (gd[k] - dd * dir[k]) * il;
        }
        if (ONE_VIEW && !wrote)
            for (int j = 0; j < nc3; ++j) gsh[j] = 0.0f;
        const bool acc = p.cfg.accumulate != 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const size_t o = 3 * (size_t)i + k;
            p.out.means[o] = acc ? p.out.means[o] + gm[k] : gm[k];
            p.out.scales[o] = acc ? p.out.scales[o] + gs[k] : gs[k];
            p.out.normals[o] = acc ? p.out.normals[o] + gn[k] : gn[k];
        }
        float4 q4 = make_float4(gq[0], gq[1], gq[2], gq[3]);
        if (acc) {
            const float4 o4 = reinterpret_cast<const float4 *>(p.out.quats)[i];
            q4.x += o4.x; q4.y += o4.y; q4.z += o4.z; q4.w += o4.w;
        }
        reinterpret_cast<float4 *>(p.out.quats)[i] = q4;
        p.out.opac1[i] = acc ? p.out.opac1[i] + go1 : go1;
        p.out.opac2[i] = acc ? p.out.opac2[i] + go2 : go2;
    }
    __syncthreads();
    // SH gradients: shared rows -> contiguous global slice, coalesced
    float *dst = p.out.sh + (size_t)nc3 * base;
    const bool acc = p.cfg.accumulate != 0;
    for (int j = threadIdx.x; j < rows * nc3; j += blockDim.x) {
        const int r = j / nc3, c = j - r * nc3;
        dst[j] = acc ? dst[j] + gsh_s[r * shs + c] : gsh_s[r * shs + c];
    }
}

// Geometry adjoint (mean, scale, quaternion, normal) of the gathered near-degenerate
// (view, splat) pairs in FP64, added to what k_project_bwd wrote.  Atomic adds,
// since one splat can be listed for several views.
__global__ void __launch_bounds__(kProjBlock) k_project_bwd_fp64(ProjBwdLaunch p) {
    const uint32_t cnt = min(p.fp64_list[0], (uint32_t)p.n_views * (uint32_t)p.g.n);
    for (uint32_t e = blockIdx.x + gridDim.x * threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const uint32_t vi = p.fp64_list[1 + e];
        const int v = (int)(vi / (uint32_t)p.g.n), i = (int)(vi - (uint32_t)v * (uint32_t)p.g.n);
        const Params P = load_params(p.g, i);
        G2 g2;
        const float4 *g4 = reinterpret_cast<const float4 *>(p.grad2d) + 3 * (size_t)vi;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float4 a = g4[j];
            g2.v[4 * j] = a.x; g2.v[4 * j + 1] = a.y; g2.v[4 * j + 2] = a.z; g2.v[4 * j + 3] = a.w;
        }
        const double g_comp = p.cfg.mip ? (double)p.g.opac1[i] * g2.v[7] + (double)p.g.opac2[i] * g2.v[8] : 0.0;
        const Grads r = proj_vjp_fp64(P, p.cams[v], p.cfg.lowpass, p.cfg.fov_clamp, g2, g_comp);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicAdd(p.out.means + 3 * (size_t)i + k, r.m[k]);
            atomicAdd(p.out.scales + 3 * (size_t)i + k, r.s[k]);
            atomicAdd(p.out.normals + 3 * (size_t)i + k, r.n[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(p.out.quats + 4 * (size_t)i + k, r.q[k]);
    }
}

}  // namespace

// Dynamic shared memory of a projection kernel: the staged parameters, plus for the
// adjoint either the screen-space gradient rows (one view) or SH gradient rows.
size_t project_smem_bytes(bool bwd, bool one_view) {
    if (!bwd) return sizeof(StageSmem);
    return sizeof(BwdStageSmem) + sizeof(float) * (one_view ? 12 : kShStride3) * kProjBwdBlock;
}

// Grid of the FP64 follow-up kernels: the list length is known only on the device,
// so a fixed grid strides over it (one thread per entry while it is short).
constexpr int kFp64Blocks = 148;

template <int DEG, bool ONE_VIEW>
cudaError_t launch_project_deg(const ProjLaunch &p, cudaStream_t s) {
    const size_t smem = project_smem_bytes(false, true);
    cudaError_t e = cudaFuncSetAttribute(k_project<DEG, ONE_VIEW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_project<DEG, ONE_VIEW><<<div_up(p.g.n, kProjBlock), kProjBlock, smem, s>>>(p);
    return cudaGetLastError();
}

template <int DEG>
cudaError_t launch_project_views(const ProjLaunch &p, cudaStream_t s) {
    return p.n_views == 1 ? launch_project_deg<DEG, true>(p, s) : launch_project_deg<DEG, false>(p, s);
}

template <int DEG, bool ONE_VIEW>
cudaError_t launch_project_bwd_deg(const ProjBwdLaunch &p, cudaStream_t s) {
    const size_t smem = project_smem_bytes(true, ONE_VIEW);
    cudaError_t e = cudaFuncSetAttribute(k_project_bwd<DEG, ONE_VIEW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_project_bwd<DEG, ONE_VIEW><<<div_up(p.g.n, kProjBwdBlock), kProjBwdBlock, smem, s>>>(p);
    return cudaGetLastError();
}

template <int DEG>
cudaError_t launch_project_bwd_views(const ProjBwdLaunch &p, cudaStream_t s) {
    return p.n_views == 1 ? launch_project_bwd_deg<DEG, true>(p, s) : launch_project_bwd_deg<DEG, false>(p, s);
}

cudaError_t launch_project(const ProjLaunch &p, cudaStream_t s) {
    if (p.g.n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.out.fp64_list, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    switch (p.g.sh_degree) {
        case 0: e = launch_project_views<0>(p, s); break;
        case 1: e = launch_project_views<1>(p, s); break;
        case 2: e = launch_project_views<2>(p, s); break;
        default: e = launch_project_views<3>(p, s); break;
    }
    if (e != cudaSuccess) return e;
    k_project_fp64<<<kFp64Blocks, kProjBlock, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const ProjBwdLaunch &p, cudaStream_t s) {
    if (p.g.n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.fp64_list, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    switch (p.g.sh_degree) {
        case 0: e = launch_project_bwd_views<0>(p, s); break;
        case 1: e = launch_project_bwd_views<1>(p, s); break;
        case 2: e = launch_project_bwd_views<2>(p, s); break;
        default: e = launch_project_bwd_views<3>(p, s); break;
    }
    if (e != cudaSuccess) return e;
    k_project_bwd_fp64<<<kFp64Blocks, kProjBlock, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace hgs
