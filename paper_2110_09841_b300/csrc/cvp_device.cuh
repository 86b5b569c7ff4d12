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
// Near-exact pair (exact variant). Let P_U = base square ∩ {u < U}, and for a row
// boundary V let h_V(t') = clamp(p0 + p1 t', 0, a3) be the height of the part of the voxel
// column above a base point that projects to v < V. Then
//     G(U, V) = int_{P_U} (1, D.x') h_V dA      (volume and first moment along D)
// is the 2D cumulative distribution of the voxel over the detector, and the cut of pixel
// (n, m) follows by inclusion-exclusion of G at its four corners. G needs, for the
// polygon P_U, the moments of weights 1, t', t'^2, lambda, lambda t' (lambda = t_c t' +
// xi_c xi') over P_U ∩ {t' < tau} at the two depths tau where the row plane leaves the
// voxel through its bottom and top faces. They are integrated exactly by Green's theorem
// over the boundary of the convex polygon square ∩ {L1 < 0} ∩ {t' < tau}.
// The weight is W = V / |c - s|^2 with c the centre of mass of the cut:
//     |c - s|^2 = |D + M/V|^2 ~ (V |D|^2 + 2 D.M) / V       (D = x_vox - s),
// the dropped |M/V|^2 / |D|^2 <= 3/4 (a / r)^2 being below the FP32 resolution of r^2 for
// the voxel sizes and distances of cone-beam CT (e.g. 3e-7 for 0.25 mm voxels at 400 mm).
//
// Relaxed pair (relaxed variant, Sec. III-A, Eq. cutvolume): A_n = |H_n|, CM_n its centre of
// mass, d = h_{m+1/2}(t'_CM) - h_{m-1/2}(t'_CM), W = A_n d / |D|^2.
#pragma once

#include <cstdint>

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
    float tmin_sq, tmax_sq;      // t' range of the square
    float sq_tt, sq_tx;          // Green sums of the full square for t'^2 and t' xi'
    float pad[2];
};

struct Grid {
    int nx, ny, nz, nu, nv, nviews;
    float ax, ay, az;
    float x0, y0, z0;            // centre of voxel (0, 0, 0)
};

constexpr int KCT_CB = 8;        // column boundaries handled per pass (7 columns)
constexpr int KCT_MAX_SPAN = 4096;   // larger footprints are reported as errors

// ----------------------------------------------------------------------------------------
// Pixel factors (Sec. III-C second phase)
// ----------------------------------------------------------------------------------------

// Eq. cvp at the pixel centre: f^2 / (a cos^3 theta) = |gu gv| (1 + alpha^2 + beta^2)^{3/2}
__device__ __forceinline__ float factor_cos(const View& V, int n, int m) {
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
__device__ __forceinline__ float factor_exact(const View& V, int n, int m) {
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
__device__ __forceinline__ float pixel_factor(const View& V, int n, int m) {
    if (SCALING == 1) return factor_exact(V, n, m);
    return factor_cos(V, n, m);
}

// ----------------------------------------------------------------------------------------
// Green's theorem sums over directed segments in the (t', xi') plane
// ----------------------------------------------------------------------------------------

struct Mom5 {
    float a, t, x, tt, tx;   // sums of c, c(t0+t1), c(x0+x1), c(t0^2+t0 t1+t1^2), c(2t0x0+t0x1+t1x0+2t1x1)
};

__device__ __forceinline__ Mom5 mom_zero() { return Mom5{0.f, 0.f, 0.f, 0.f, 0.f}; }

template <bool FULL>
__device__ __forceinline__ void seg_acc(Mom5& m, float pt, float px, float qt, float qx) {
    float c = pt * qx - qt * px;
    m.a += c;
    m.t = fmaf(c, pt + qt, m.t);
    if (FULL) {
        m.x = fmaf(c, px + qx, m.x);
        m.tt = fmaf(c, fmaf(pt, pt, fmaf(pt, qt, qt * qt)), m.tt);
        m.tx = fmaf(c, fmaf(2.f * pt, px, fmaf(pt, qx, fmaf(qt, px, 2.f * qt * qx))), m.tx);
    }
}

// restrict the parameter interval [s0, s1] of a segment to {L < 0}; L linear along it
__device__ __forceinline__ void clip_param(float Lp, float Lq, float& s0, float& s1) {
    bool pin = Lp < 0.f, qin = Lq < 0.f;
    if (pin != qin) {
        float ss = Lp / (Lp - Lq);
        if (pin) s1 = fminf(s1, ss);
        else s0 = fmaxf(s0, ss);
    } else if (!pin) {
        s1 = -1.f;
    }
}

// accumulate the part [s0, s1] of segment p -> q
template <bool FULL>
__device__ __forceinline__ void seg_part(Mom5& m, float pt, float px, float qt, float qx, float s0, float s1) {
    if (s1 > s0) {
        float dt = qt - pt, dx = qx - px;
        float at = fmaf(s0, dt, pt), ax = fmaf(s0, dx, px);
        float bt = fmaf(-(1.f - s1), dt, qt), bx = fmaf(-(1.f - s1), dx, qx);
        seg_acc<FULL>(m, at, ax, bt, bx);
    }
}

// Green sums of  square ∩ {L1 < 0} ∩ {t' < tau},  L1 = l1t t' + l1x xi' - l1c.
// The boundary of an intersection of convex sets is the union of each set's boundary
// restricted to the others: square edges clipped by both half-planes, plus the segment of
// each line inside the square clipped by the other half-plane, oriented counter-clockwise.
template <bool USE1, bool USE2, bool FULL>
__device__ __forceinline__ Mom5 region(const View& V, float l1t, float l1x, float l1c, float tau) {
    Mom5 m = mom_zero();
    float L1[4], L2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        L1[e] = USE1 ? fmaf(l1t, V.sq_t[e], fmaf(l1x, V.sq_x[e], -l1c)) : -1.f;
        L2[e] = USE2 ? V.sq_t[e] - tau : -1.f;
    }
    float x1t = 0.f, x1x = 0.f, n1t = 0.f, n1x = 0.f;   // exit / entry of line 1
    float x2t = 0.f, x2x = 0.f, n2t = 0.f, n2x = 0.f;   // exit / entry of line 2
    bool hx1 = false, hn1 = false, hx2 = false, hn2 = false;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int f = (e + 1) & 3;
        float pt = V.sq_t[e], px = V.sq_x[e], qt = V.sq_t[f], qx = V.sq_x[f];
        float s0 = 0.f, s1 = 1.f;
        if (USE1) clip_param(L1[e], L1[f], s0, s1);
        if (USE2) clip_param(L2[e], L2[f], s0, s1);
        seg_part<FULL>(m, pt, px, qt, qx, s0, s1);
        if (USE1) {
            if ((L1[e] < 0.f) != (L1[f] < 0.f)) {
                float ss = L1[e] / (L1[e] - L1[f]);
                float ct = fmaf(ss, qt - pt, pt), cx = fmaf(ss, qx - px, px);
                if (L1[e] < 0.f) { x1t = ct; x1x = cx; hx1 = true; }
                else { n1t = ct; n1x = cx; hn1 = true; }
            }
        }
        if (USE2) {
            if ((L2[e] < 0.f) != (L2[f] < 0.f)) {
                float ss = L2[e] / (L2[e] - L2[f]);
                float ct = fmaf(ss, qt - pt, pt), cx = fmaf(ss, qx - px, px);
                if (L2[e] < 0.f) { x2t = ct; x2x = cx; hx2 = true; }
                else { n2t = ct; n2x = cx; hn2 = true; }
            }
        }
    }
    if (USE1 && hx1 && hn1) {     // along line 1 from its exit to its entry, inside {t' < tau}
        float s0 = 0.f, s1 = 1.f;
        if (USE2) clip_param(x1t - tau, n1t - tau, s0, s1);
        seg_part<FULL>(m, x1t, x1x, n1t, n1x, s0, s1);
    }
    if (USE2 && hx2 && hn2) {     // along line 2 (t' = tau) inside {L1 < 0}
        float s0 = 0.f, s1 = 1.f;
        if (USE1) clip_param(fmaf(l1t, x2t, fmaf(l1x, x2x, -l1c)), fmaf(l1t, n2t, fmaf(l1x, n2x, -l1c)), s0, s1);
        seg_part<FULL>(m, x2t, x2x, n2t, n2x, s0, s1);
    }
    return m;
}

// ----------------------------------------------------------------------------------------
// Column setup: the voxel column (i, j) in one view
// ----------------------------------------------------------------------------------------

struct Column {
    float tc, xc;        // depth and lateral offset of the column centre
    float itc;           // 1 / tc
    float alc;           // xi_c / t_c
    float gxi;           // gu / tc
    float umin, umax;    // u range of the base square
    int n_first, n_last; // detector columns touched (clipped), n_first > n_last if none
};

__device__ __forceinline__ bool column_setup(const View& V, const Grid& G, int i, int j, Column& C) {
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
    return C.n_first <= C.n_last;
}

// Voxel k of the column: height zeta_c of its centre, projected centre beta_c, row range.
struct Slice {
    float zc;            // zeta of the voxel centre
    float bc;            // zeta_c / t_c
    float vmin, vmax;
    int m_first, m_last;
};

__device__ __forceinline__ bool slice_setup(const View& V, const Grid& G, const Column& C, int k, Slice& S) {
    float z = fmaf((float)k, G.az, G.z0);
    float zc = z - V.sz;
    S.zc = zc;
    S.bc = zc * C.itc;
    float it0 = 1.0f / (C.tc + V.tmin_sq), it1 = 1.0f / (C.tc + V.tmax_sq);
    float zl = zc - 0.5f * G.az, zh = zc + 0.5f * G.az;
    float b00 = zl * it0, b01 = zl * it1, b10 = zh * it0, b11 = zh * it1;
    float bmin = fminf(fminf(b00, b01), fminf(b10, b11));
    float bmax = fmaxf(fmaxf(b00, b01), fmaxf(b10, b11));
    float va = fmaf(V.gv, bmin, V.cv), vb = fmaf(V.gv, bmax, V.cv);
    S.vmin = fminf(va, vb);
    S.vmax = fmaxf(va, vb);
    int m0 = (int)floorf(S.vmin + 0.5f), m1 = (int)floorf(S.vmax + 0.5f);
    S.m_first = max(m0, 0);
    S.m_last = min(m1, G.nv - 1);
    return S.m_first <= S.m_last;
}

// Row boundary V in the voxel: h(t') = clamp(p0 + p1 t', 0, az) is the height of the part
// of the column above base point t' that projects to v < V.
__device__ __forceinline__ void row_plane(const View& V, const Grid& G, const Column& C, const Slice& S,
                                          float Vb, float& p0, float& p1) {
    // V - v_c with v_c = cv + gv beta_c, evaluated as one fused operation
    float dv = -fmaf(V.gv, S.bc, V.cv - Vb);
    p0 = fmaf(C.tc * dv, V.inv_agv, 0.5f * G.az);
    p1 = (Vb - V.cv) * V.inv_agv;
}

// ----------------------------------------------------------------------------------------
// Exact variant: enumerate (k, n, m, W) for voxels k0 <= k < k1 of column (i, j)
// ----------------------------------------------------------------------------------------

// normalised moments of a Green-sum record: 1, t', t'^2, lambda, lambda t'
struct Mom {
    float m1, mt, mtt, ml, mlt;
};

__device__ __forceinline__ Mom normalise(const Mom5& g, float tc, float xc) {
    Mom r;
    r.m1 = 0.5f * g.a;
    r.mt = g.t * (1.f / 6.f);
    float mx = g.x * (1.f / 6.f);
    r.mtt = g.tt * (1.f / 12.f);
    float mtx = g.tx * (1.f / 24.f);
    r.ml = fmaf(tc, r.mt, xc * mx);
    r.mlt = fmaf(tc, r.mtt, xc * mtx);
    return r;
}

__device__ __forceinline__ Mom mom_sub(const Mom& a, const Mom& b) {
    return Mom{a.m1 - b.m1, a.mt - b.mt, a.mtt - b.mtt, a.ml - b.ml, a.mlt - b.mlt};
}

enum { KIND_EMPTY = 0, KIND_GEN = 1, KIND_FULL = 2 };

// moments over P_c ∩ {t' < tau}
__device__ __forceinline__ Mom cpm(const View& V, const Column& C, int kind, float l1t, float l1c,
                                   const Mom& full, float tau) {
    if (tau <= V.tmin_sq || kind == KIND_EMPTY) return Mom{0.f, 0.f, 0.f, 0.f, 0.f};
    if (tau >= V.tmax_sq) return full;
    Mom5 g = (kind == KIND_GEN) ? region<true, true, true>(V, l1t, C.gxi, l1c, tau)
                                : region<false, true, true>(V, 0.f, 0.f, 0.f, tau);
    return normalise(g, C.tc, C.xc);
}

}  // namespace kct
