// cvp_device.cuh -- device-side geometry of the cutting voxel projector (FP32).
//
// Kulvait & Rose, arXiv 2110.09841. Notation of the paper: voxel (i,j,k) with centre
// x^(i,j,k) (Sec. II-A), pixel (u,v) = (n,m) with unit-square extent in detector index
// units (Sec. II-B), source s, cut V^(i,j,k)_(m,n) of the voxel with all rays to the pixel
// (Eq. extinction), weights of Eq. vox.
//
// Geometry of one view in the frame of the source (Sec. III-A, III-C). With the detector
// rows along x_3 and rectangular pixels, a point X has depth t = w.(X - s) along the
// horizontal principal direction w, lateral offset xi = h.(X - s) along h = (-w_y, w_x),
// height zeta = X_3 - s_3, and
//     u = cu + gu * xi / t ,     v = cv + gv * zeta / t .
// Column boundaries u = n +- 1/2 are vertical planes through s, row boundaries
// v = m +- 1/2 are planes through the horizontal line {t = 0, zeta = 0}, so in a voxel
// (local coordinates t', xi', zeta' around its centre)
//   * the column cut of the voxel base, H_n, is the base square clipped by two lines;
//   * the x_3 extent of a row over a base point depends on t' only (Eq.
//     columnprojectionidentity and the row-plane pencil).
//
// Near-exact pair (exact variant). H_n is clipped directly between the two column lines.
// For a row boundary V, h_V(t') = clamp(p0 + p1 t', 0, a3) is the height of the part of the
// voxel column above base point t' that projects to v < V. The cut of pixel (n, m) is
//     int_{H_n} (h_{m+1/2} - h_{m-1/2}) (1, D.x') dA     (volume and first moment along D).
// When both planes stay inside the voxel over the base the integrand is linear in t' and
// the pair is a closed form of the moments of H_n (weights 1, t', t'^2, lambda, lambda t',
// lambda = t_c t' + xi_c xi'). A plane that leaves the voxel through a face needs the
// moments of H_n ∩ {t' < tau}: the chord of H_n at depth t' is linear in t' between vertex
// depths, so each moment is a cubic in tau there, evaluated exactly from a per-column
// depth profile of H_n (depth_profile, profile_cut).
// The weight is W = V / |c - s|^2 with c the centre of mass of the cut:
//     |c - s|^2 = |D + M/V|^2 ~ (V |D|^2 + 2 D.M) / V       (D = x_vox - s),
// the dropped |M/V|^2 / |D|^2 <= 3/4 (a / r)^2 being below the FP32 resolution of r^2 for
// the voxel sizes and distances of cone-beam CT (e.g. 3e-7 for 0.25 mm voxels at 400 mm).
//
// Relaxed pair (relaxed variant, Sec. III-A, Eq. cutvolume): A_n = |H_n|, CM_n its centre of
// mass, d = h_{m+1/2}(t'_CM) - h_{m-1/2}(t'_CM), W = A_n d / |D|^2.
#pragma once

#include <cmath>
#include <cstdint>

// geometry functions compile for host and device (the host copy serves debugging tools)
#define KCT_HD __host__ __device__ __forceinline__

namespace kct {

// Per-view parameters, FP32 (wx, wy, aw carry a low-order part for a compensated sum).
struct View {
    float wx, wy, wx_lo, wy_lo;  // unit horizontal principal direction (hi + lo)
    float aw, aw_lo;             // -w . s  (depth of the origin, hi + lo)
    float ah;                    // -h . s  (lateral offset of the origin)
    float sz;                    // source height s_3
    float cu, gu, cv, gv;        // u = cu + gu xi/t,  v = cv + gv zeta/t
    float igu, igv;              // 1/gu, 1/gv
    float inv_agv;               // 1/|gv|
    float sgv;                   // sign(gv)
    float fcos;                  // |gu gv| = f^2 / (pixel area)
    float sq_t[4], sq_x[4];      // voxel base square vertices (t', xi'), counter-clockwise
    float sx, sy;                // source s_1, s_2 (used by the ray-driven comparator only)
    float cv_lo, inv_agv_lo;     // low-order parts of cv and 1/|gv|
    float sz_lo;                 // low-order part of s_3
};

struct Grid {
    int nx, ny, nz, nu, nv, nviews;
    float ax, ay, az;
    float x0, y0, z0;            // centre of voxel (0, 0, 0)
    double axd, ayd, azd;        // the same in double precision (exact geometry of faces and columns)
    double x0d, y0d, z0d;
};

constexpr int KCT_CB = 8;        // column boundaries handled per pass (7 columns)
constexpr int KCT_MAX_SPAN = 4096;   // larger footprints are reported as errors

// ----------------------------------------------------------------------------------------
// Pixel factors (Sec. III-C second phase)
// ----------------------------------------------------------------------------------------

// Eq. cvp at the pixel centre: f^2 / (a cos^3 theta) = |gu gv| (1 + alpha^2 + beta^2)^{3/2}
KCT_HD float factor_cos(const View& V, int n, int m) {
    float al = ((float)n - V.cu) * V.igu;
    float be = ((float)m - V.cv) * V.igv;
    float q = fmaf(al, al, fmaf(be, be, 1.0f));
    return V.fcos * q * sqrtf(q);
}

// Eq. cvpus: 1 / solid angle of the pixel. The pixel is the rectangle [a0,a1] x [b0,b1] on
// the plane t = 1 of the source frame; its solid angle is the sum over the two triangles
// (P00, P10, P11), (P00, P11, P01) of the Van Oosterom-Strackee expression
// tan(Omega/2) = |[a b c]| / (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|), where the
// triple product of either triangle equals (a1 - a0)(b1 - b0) exactly.
KCT_HD float factor_exact(const View& V, int n, int m) {
    float a0 = ((float)n - 0.5f - V.cu) * V.igu, a1 = ((float)n + 0.5f - V.cu) * V.igu;
    float b0 = ((float)m - 0.5f - V.cv) * V.igv, b1 = ((float)m + 0.5f - V.cv) * V.igv;
    float num = fabsf(V.igu * V.igv);
    float l00 = sqrtf(fmaf(a0, a0, fmaf(b0, b0, 1.f)));
    float l10 = sqrtf(fmaf(a1, a1, fmaf(b0, b0, 1.f)));
    float l11 = sqrtf(fmaf(a1, a1, fmaf(b1, b1, 1.f)));
    float l01 = sqrtf(fmaf(a0, a0, fmaf(b1, b1, 1.f)));
    float d00_10 = fmaf(a0, a1, fmaf(b0, b0, 1.f));
    float d00_11 = fmaf(a0, a1, fmaf(b0, b1, 1.f));
    float d10_11 = fmaf(a1, a1, fmaf(b0, b1, 1.f));
    float d00_01 = fmaf(a0, a0, fmaf(b0, b1, 1.f));
    float d11_01 = fmaf(a1, a0, fmaf(b1, b1, 1.f));
    float D1 = l00 * l10 * l11 + d00_10 * l11 + d00_11 * l10 + d10_11 * l00;
    float D2 = l00 * l11 * l01 + d00_11 * l01 + d00_01 * l11 + d11_01 * l00;
    float omega = 2.f * (atan2f(num, D1) + atan2f(num, D2));
    return 1.0f / omega;
}

template <int SCALING>
KCT_HD float pixel_factor(const View& V, int n, int m) {
    if (SCALING == 1) return factor_exact(V, n, m);
    return factor_cos(V, n, m);
}

// ----------------------------------------------------------------------------------------
// Green's theorem over the directed edges of a polygon in the (t', xi') plane
// ----------------------------------------------------------------------------------------

struct Green2 {
    float a, t;   // sums of c and c (t0 + t1), c = t0 x1 - t1 x0: twice the area, six times the t' moment
};

KCT_HD void seg_acc(Green2& m, float pt, float px, float qt, float qx) {
    const float c = pt * qx - qt * px;
    m.a += c;
    m.t = fmaf(c, pt + qt, m.t);
}

// 1/x to about 2 ulp (the hardware reciprocal on the device) for 2^-126 < |x| < 2^126
KCT_HD float rcp_fast(float x) {
#ifdef __CUDA_ARCH__
    return __fdividef(1.f, x);
#else
    return 1.f / x;
#endif
}

// p / (p - q) for p, q of opposite signs (where a segment crosses a line), in [0, 1]
KCT_HD float cross_frac(float p, float q) { return fminf(fmaxf(p * rcp_fast(p - q), 0.f), 1.f); }

// restrict the parameter interval [s0, s1] of a segment to {L < 0}; L linear along it
KCT_HD void clip_param(float Lp, float Lq, float& s0, float& s1) {
    bool pin = Lp < 0.f, qin = Lq < 0.f;
    if (pin != qin) {
        float ss = cross_frac(Lp, Lq);
        if (pin) s1 = fminf(s1, ss);
        else s0 = fmaxf(s0, ss);
    } else if (!pin) {
        s1 = -1.f;
    }
}

// A half-plane {at t' + ax xi' - c < 0} of the (t', xi') plane. Line{0, 0, 1} is the
// whole plane (inactive).
struct Line {
    float at, ax, c;
};

KCT_HD Line line_none() { return Line{0.f, 0.f, 1.f}; }

KCT_HD float line_eval(const Line& l, float t, float x) { return fmaf(l.at, t, fmaf(l.ax, x, -l.c)); }

// The points that square edge e contributes to the square clipped by two half-planes: its
// start vertex when inside both, then, in order along the edge, the points where it crosses
// a line while inside the other half-plane (ot, ox)[0 .. n), n <= 3.
KCT_HD int clip_square_edge(const View& V, const Line& l0, const Line& l1, int e, float (&ot)[3], float (&ox)[3]) {
    const int f = (e + 1) & 3;
    const float at = V.sq_t[e], ax = V.sq_x[e], bt = V.sq_t[f], bx = V.sq_x[f];
    const float A0 = line_eval(l0, at, ax), B0 = line_eval(l0, bt, bx);
    const float A1 = line_eval(l1, at, ax), B1 = line_eval(l1, bt, bx);
    const bool sv = A0 < 0.f && A1 < 0.f;
    // inside parameter intervals of the edge for each line
    float a0 = 0.f, b0 = 1.f, a1 = 0.f, b1 = 1.f;
    clip_param(A0, B0, a0, b0);
    clip_param(A1, B1, a1, b1);
    const float s0 = cross_frac(A0, B0), s1 = cross_frac(A1, B1);
    const bool h0 = ((A0 < 0.f) != (B0 < 0.f)) && s0 >= a1 && s0 <= b1;
    const bool h1 = ((A1 < 0.f) != (B1 < 0.f)) && s1 >= a0 && s1 <= b0;
    const float sa = h0 ? (h1 ? fminf(s0, s1) : s0) : s1, sb = fmaxf(s0, s1);
    const float cat = fmaf(sa, bt - at, at), cax = fmaf(sa, bx - ax, ax);
    const float cbt = fmaf(sb, bt - at, at), cbx = fmaf(sb, bx - ax, ax);
    ot[0] = sv ? at : cat;
    ox[0] = sv ? ax : cax;
    ot[1] = sv ? cat : cbt;
    ox[1] = sv ? cax : cbx;
    ot[2] = cbt;
    ox[2] = cbx;
    return (int)sv + (int)h0 + (int)h1;
}

// Vertices (counter-clockwise) of the square clipped by two half-planes, edge by edge
// (clip_square_edge); at most 8 are kept.
KCT_HD int clip_square(const View& V, const Line& l0, const Line& l1, float* pt, float* px) {
    int nv = 0;
    for (int e = 0; e < 4; ++e) {
        float ot[3], ox[3];
        const int n = clip_square_edge(V, l0, l1, e, ot, ox);
        for (int q = 0; q < n; ++q) {
            if (nv < 8) {
                pt[nv] = ot[q];
                px[nv] = ox[q];
                ++nv;
            }
        }
    }
    return nv;
}

// ----------------------------------------------------------------------------------------
// Depth profile of a convex polygon: the moments of its part below a depth t' = tau
// ----------------------------------------------------------------------------------------

constexpr int KCT_IV = 7;        // depth intervals of H_n (its at most 8 vertices give at most 7)

// Between two consecutive vertex depths T_j < T_(j+1) the chord of a convex polygon at depth
// t' joins the same two edges, so its length w and midpoint c are linear in t'. The moments
// (1, t', t'^2, xi', t' xi') of the part below tau then grow by the integrals of w, w t',
// w t'^2, w c and w c t' from T_j to tau: polynomials of degree <= 3 in t', which Simpson's
// rule integrates exactly. simpson5 adds them for [t0, t1], s = t1 - t0, with the chord at t0
// (w0, c0) and its change over the interval (dw, dc) taken at the fraction lam of it.
KCT_HD void simpson5(float t0, float t1, float s, float lam, float w0, float dw, float c0, float dc, float& A,
                     float& T, float& TT, float& X, float& TX) {
    const float hl = 0.5f * lam;
    const float wm4 = 4.f * fmaf(hl, dw, w0), w1 = fmaf(lam, dw, w0);
    const float cm = fmaf(hl, dc, c0), c1 = fmaf(lam, dc, c0);
    const float tm = fmaf(0.5f, s, t0);
    const float a0t = w0 * t0, amt = wm4 * tm, a1t = w1 * t1;
    const float a0c = w0 * c0, amc = wm4 * cm, a1c = w1 * c1;
    const float h6 = s * (1.f / 6.f);
    A = fmaf(h6, w0 + wm4 + w1, A);
    T = fmaf(h6, a0t + amt + a1t, T);
    TT = fmaf(h6, fmaf(a0t, t0, fmaf(amt, tm, a1t * t1)), TT);
    X = fmaf(h6, a0c + amc + a1c, X);
    TX = fmaf(h6, fmaf(a0c, t0, fmaf(amc, tm, a1c * t1)), TX);
}

// The profile of the convex polygon (pt, px)[0 .. nv) (vertices in order, either sense):
// the interval starts st[j] = T_j (st[K .. 7] = +inf) and per depth interval j,
// a[j] = (1 / (T_(j+1) - T_j), w(T_j), w(T_(j+1)) - w(T_j), c(T_j)),
// b[j] = (c(T_(j+1)) - c(T_j), the area, t' and t'^2 moments of the part below T_j) and
// m[j] = its xi' and t' xi' moments. The two chains from the lowest to the highest vertex
// are walked together; w and c at an interval's ends come from the two edges that span it.
// Returns the number of intervals (0 for a degenerate polygon); the moments of the whole
// polygon go to full and its depth range to tlo, thi.
KCT_HD int depth_profile(const float* pt, const float* px, int nv, float* st, float4* a, float4* b, float2* m,
                         float (&full)[5], float& tlo, float& thi) {
    float A = 0.f, T = 0.f, TT = 0.f, X = 0.f, TX = 0.f;
    int imin = 0, imax = 0;
    for (int e = 1; e < nv; ++e) {
        if (pt[e] < pt[imin]) imin = e;
        if (pt[e] > pt[imax]) imax = e;
    }
    tlo = nv > 0 ? pt[imin] : 0.f;
    thi = nv > 0 ? pt[imax] : 0.f;
    int K = 0;
    if (nv >= 3) {
        int ia = imin, ib = imin;      // the chains forward and backward from the lowest vertex
        float Tc = tlo;
        for (int it = 0; it < KCT_IV && Tc < thi; ++it) {
            // pass the vertices at depth <= Tc (neither chain can pass the highest vertex)
            for (int q = 0; q < nv; ++q) {
                const int na = ia + 1 == nv ? 0 : ia + 1;
                if (pt[na] > Tc) break;
                ia = na;
            }
            for (int q = 0; q < nv; ++q) {
                const int nb = ib == 0 ? nv - 1 : ib - 1;
                if (pt[nb] > Tc) break;
                ib = nb;
            }
            const int na = ia + 1 == nv ? 0 : ia + 1, nb = ib == 0 ? nv - 1 : ib - 1;
            const float Tn = fminf(fminf(pt[na], pt[nb]), thi);
            // both edges span [Tc, Tn]: pt[ia], pt[ib] <= Tc < Tn <= pt[na], pt[nb]
            const float ra = rcp_fast(pt[na] - pt[ia]), rb = rcp_fast(pt[nb] - pt[ib]);
            const float dxa = px[na] - px[ia], dxb = px[nb] - px[ib];
            const float xa0 = fmaf((Tc - pt[ia]) * ra, dxa, px[ia]), xa1 = fmaf((Tn - pt[ia]) * ra, dxa, px[ia]);
            const float xb0 = fmaf((Tc - pt[ib]) * rb, dxb, px[ib]), xb1 = fmaf((Tn - pt[ib]) * rb, dxb, px[ib]);
            const float w0 = fabsf(xb0 - xa0), w1 = fabsf(xb1 - xa1);
            const float c0 = 0.5f * (xa0 + xb0), c1 = 0.5f * (xa1 + xb1);
            st[K] = Tc;
            a[K] = make_float4(rcp_fast(Tn - Tc), w0, w1 - w0, c0);
            b[K] = make_float4(c1 - c0, A, T, TT);
            m[K] = make_float2(X, TX);
            simpson5(Tc, Tn, Tn - Tc, 1.f, w0, w1 - w0, c0, c1 - c0, A, T, TT, X, TX);
            ++K;
            Tc = Tn;
        }
    }
    for (int j = K; j < KCT_IV + 1; ++j) st[j] = 3.0e38f;
    full[0] = A;
    full[1] = T;
    full[2] = TT;
    full[3] = X;
    full[4] = TX;
    return K;
}

// Moments (1, t', t'^2, xi', t' xi') of the part below tau of a polygon with profile
// (st, a, b, m), for T_0 <= tau <= T_K: the interval holding tau is the number of interval
// starts T_1 .. T_7 at or below it (two vector loads, the same for every thread of a column).
KCT_HD void profile_cut(const float* st, const float4* a, const float4* b, const float2* m, float tau, float& A,
                        float& T, float& TT, float& X, float& TX) {
    const float4 s0 = reinterpret_cast<const float4*>(st)[0], s1 = reinterpret_cast<const float4*>(st)[1];
    const int j = (tau >= s0.y) + (tau >= s0.z) + (tau >= s0.w) + (tau >= s1.x) + (tau >= s1.y) + (tau >= s1.z) +
                  (tau >= s1.w);
    const float4 aj = a[j], bj = b[j];
    const float2 mj = m[j];
    const float t0 = st[j];
    A = bj.y;
    T = bj.z;
    TT = bj.w;
    X = mj.x;
    TX = mj.y;
    const float s = tau - t0;
    simpson5(t0, tau, s, s * aj.x, aj.y, aj.z, aj.w, bj.x, A, T, TT, X, TX);
}

// ----------------------------------------------------------------------------------------
// Column setup: the voxel column (i, j) in one view
// ----------------------------------------------------------------------------------------

// A float pair (hi, lo) holding hi + lo to about twice float precision (used where a small
// height is the difference of two large coordinates).
struct F2 {
    float hi, lo;
};

KCT_HD F2 f2_of(double d) {
    const float h = (float)d;
    return F2{h, (float)(d - (double)h)};
}

// a + b c for an integer-valued float b: the product split exactly by an FMA, the sum by
// Knuth's two-sum
KCT_HD F2 f2_axpy(F2 a, float b, F2 c) {
    const float p = b * c.hi;
    const float pe = fmaf(b, c.hi, -p);
    const float s = a.hi + p;
    const float z = s - a.hi;
    const float e = (a.hi - (s - z)) + (p - z);
    return F2{s, a.lo + fmaf(b, c.lo, pe + e)};
}

// (a - b) rounded to float; the large parts cancel exactly when a and b are close
KCT_HD float f2_diff(F2 a, F2 b) { return (a.hi - b.hi) + (a.lo - b.lo); }

struct Column {
    float tc, xc;        // depth and lateral offset of the column centre
    float itc;           // 1 / tc
    float alc;           // xi_c / t_c
    float gxi;           // gu / tc
    float umin, umax;    // u range of the base square
    int n_first, n_last; // detector columns touched (clipped), n_first > n_last if none
    F2 da;               // tc / |gv|: height per detector row at the column centre depth (two floats)
};

KCT_HD bool column_setup(const View& V, const Grid& G, int i, int j, Column& C) {
    float x = fmaf((float)i, G.ax, G.x0);
    float y = fmaf((float)j, G.ay, G.y0);
    // compensated t = w.x + aw and xi = h.x + ah with w = (wx, wy), h = (-wy, wx)
    float tlo = fmaf(V.wx_lo, x, fmaf(V.wy_lo, y, V.aw_lo));
    float tc = fmaf(V.wx, x, fmaf(V.wy, y, V.aw + tlo));
    float xlo = fmaf(-V.wy_lo, x, V.wx_lo * y);
    float xc = fmaf(-V.wy, x, fmaf(V.wx, y, V.ah + xlo));
    C.tc = tc;
    C.xc = xc;
    C.itc = 1.0f / tc;
    C.alc = xc * C.itc;
    C.gxi = V.gu * C.itc;
    float umin = 3.0e38f, umax = -3.0e38f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float u = fmaf(V.gu, (xc + V.sq_x[e]) / (tc + V.sq_t[e]), V.cu);
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
    }
    C.umin = umin;
    C.umax = umax;
    int n0 = (int)floorf(umin + 0.5f), n1 = (int)floorf(umax + 0.5f);
    C.n_first = max(n0, 0);
    C.n_last = min(n1, G.nu - 1);
    // tc in two floats: the products w x exactly split by FMAs (x, y are exact voxel
    // coordinates), summed with the low-order parts; then da = tc / |gv| = tc inv_agv
    const float p1 = V.wx * x, e1 = fmaf(V.wx, x, -p1);
    const float p2 = V.wy * y, e2 = fmaf(V.wy, y, -p2);
    const float s1 = p1 + p2, z1 = s1 - p1, f1 = (p1 - (s1 - z1)) + (p2 - z1);
    const float s2 = s1 + V.aw, z2 = s2 - s1, f2 = (s1 - (s2 - z2)) + (V.aw - z2);
    const float tlo2 = e1 + e2 + f1 + f2 + tlo;
    const float th = s2 + tlo2, tl = tlo2 - (th - s2);
    const float dh = th * V.inv_agv;
    C.da = F2{dh, fmaf(th, V.inv_agv, -dh) + fmaf(th, V.inv_agv_lo, tl * V.inv_agv)};
    return C.n_first <= C.n_last;
}

// ----------------------------------------------------------------------------------------
// Column cuts and their moments
// ----------------------------------------------------------------------------------------

// moments of a part of H_n: 1, t', t'^2, lambda, lambda t'
struct Mom {
    float m1, mt, mtt, ml, mlt;
};

KCT_HD Mom mom_sub(const Mom& a, const Mom& b) {
    return Mom{a.m1 - b.m1, a.mt - b.mt, a.mtt - b.mtt, a.ml - b.ml, a.mlt - b.mlt};
}

// The two boundary lines of detector column n on the voxel base: H_n = base ∩ lo ∩ hi with
//   u > n - 1/2  (lo)  and  u < n + 1/2  (hi);   u < U  <=>  gu xi' + (cu - U) t' + tc (u_c - U) < 0.
// A line that does not cut the base is made inactive.
KCT_HD void column_lines(const View& V, const Column& C, int n, Line& lo, Line& hi) {
    const float Ul = (float)n - 0.5f, Uh = (float)n + 0.5f;
    if (Ul > C.umin) lo = Line{-(V.cu - Ul) * C.itc, -C.gxi, fmaf(V.gu, C.alc, V.cu - Ul)};
    else lo = line_none();
    if (Uh < C.umax) hi = Line{(V.cu - Uh) * C.itc, C.gxi, -fmaf(V.gu, C.alc, V.cu - Uh)};
    else hi = line_none();
}

}  // namespace kct
