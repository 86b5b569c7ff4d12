/*
 * oracle.c -- plain, slow FP64 CPU reference of the cutting voxel projector (CVP).
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the package smoke check and the CPU
 * baseline leg of the benchmark call it; the product path never links or calls it,
 * and it shares no source with the CUDA library.
 *
 * Method: Kulvait & Rose, "Cutting Voxel Projector: a New Approach to Construct 3D
 * Cone Beam CT Operator" (arXiv 2110.09841).
 *
 *  - Voxel grid centred at the origin, voxel (i,j,k) centre x0 + (i a1, j a2, k a3),
 *    x0 = (-l + a)/2 (Sec. II-A). Volume layout [nz][ny][nx].
 *  - Pixel (u,v) is the open square of side 1 around index coordinates (u,v); the
 *    projection matrix P maps homogeneous world points to (u,v,1) (Sec. II-B, III-C).
 *    Projection layout [view][nv][nu].
 *  - The cut V_(m,n)^(i,j,k) is the voxel intersected with the pyramid of all rays from
 *    the source to the pixel (Eq. extinction). Here it is obtained by generic convex
 *    polytope clipping: the voxel box is clipped by the four half-spaces of the pixel
 *    pyramid, then volume and centre of mass follow from a tetrahedral decomposition.
 *  - Near-exact pair weight (Eq. vox with r taken at the centre of mass of the cut):
 *        W = |V_cut| / |c_cut - s|^2.
 *  - Relaxed pair weight (Sec. III-A, Eq. cutvolume; r at the voxel centre, Eq. vox):
 *        W = A_n * d / |x_vox - s|^2, A_n the area of the column cut H_n, d the x_3 length
 *        of the voxel part of the vertical line through the centre of mass of H_n whose
 *        points project into the pixel row.
 *  - Pixel factors (Sec. II-D, "second phase" of Sec. III-C):
 *        cos scaling   F = f^2 / (a cos^3 theta)  at the pixel centre (Eq. cvp),
 *        exact scaling F = 1 / abar, abar the spherical-excess area of the pixel on the
 *                      unit sphere (Eq. cvpus and the formula above it).
 *  - Projector  b[view,v,u] = F(u,v) * sum_vox mu_vox W(vox,pix)   (Eq. cvpsu)
 *    Adjoint    x[vox] = sum_view sum_pix W(vox,pix) F(u,v) y[view,v,u]   (Eq. fundament).
 *  - Truth integral J = int_cut r^-2 dV (Eq. intcut) by the divergence theorem,
 *    div((x-s)/|x-s|^2) = |x-s|^-2, with a degree-5 triangle rule on each face.
 *  - Ray integration (Eq. discreteextinction, the SiddonK construction of Sec. II-C):
 *    the average over K x K equally spaced points of the pixel of the exact path-length
 *    weighted line integral, optionally weighted by the solid angle element.
 *
 * Candidate pixels of a voxel are those in the bounding box of the projections of its
 * eight corners; pixels outside the detector are dropped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXV 32
#define OR_MAXF 16

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double norm(v3 a) { return sqrt(dot(a, a)); }

/* ------------------------------------------------------------------------------------ */
/* Convex polytopes as face lists                                                        */
/* ------------------------------------------------------------------------------------ */

typedef struct { int nv; v3 v[OR_MAXV]; } face_t;          /* CCW seen from outside */
typedef struct { int nf; face_t f[OR_MAXF]; double scale; } ptope_t;

/* axis-aligned box [lo, hi] with outward-oriented faces */
static void box_ptope(ptope_t *P, const double lo[3], const double hi[3]) {
    v3 c[8];
    for (int n = 0; n < 8; ++n)
        c[n] = mk((n & 1) ? hi[0] : lo[0], (n & 2) ? hi[1] : lo[1], (n & 4) ? hi[2] : lo[2]);
    /* corner index bits: 1 = +x, 2 = +y, 4 = +z */
    static const int F[6][4] = {
        {0, 4, 6, 2},   /* -x */
        {1, 3, 7, 5},   /* +x */
        {0, 1, 5, 4},   /* -y */
        {2, 6, 7, 3},   /* +y */
        {0, 2, 3, 1},   /* -z */
        {4, 5, 7, 6},   /* +z */
    };
    P->nf = 6;
    for (int f = 0; f < 6; ++f) {
        P->f[f].nv = 4;
        for (int k = 0; k < 4; ++k) P->f[f].v[k] = c[F[f][k]];
    }
    double e = fmax(fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    P->scale = e;
}

/* Keep the part where dot(n, x) + d >= 0. Returns the number of faces left. */
static int clip_ptope(ptope_t *P, v3 n, double d) {
    /* A plane that only touches the polytope (or contains one of its faces) keeps it
     * whole or removes it whole; otherwise it cuts through the interior and no face
     * lies in it. */
    double gmin = INFINITY, gmax = -INFINITY;
    for (int f = 0; f < P->nf; ++f)
        for (int k = 0; k < P->f[f].nv; ++k) {
            double g = dot(n, P->f[f].v[k]) + d;
            gmin = fmin(gmin, g);
            gmax = fmax(gmax, g);
        }
    double tol = 1e-13 * norm(n) * P->scale;
    if (P->nf == 0) return 0;
    if (gmin >= -tol) return P->nf;
    if (gmax <= tol) { P->nf = 0; return 0; }
    ptope_t out;
    out.nf = 0;
    out.scale = P->scale;
    v3 cap[OR_MAXV * 2];
    int ncap = 0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t *F = &P->f[f];
        face_t G;
        G.nv = 0;
        for (int k = 0; k < F->nv; ++k) {
            v3 a = F->v[k], b = F->v[(k + 1) % F->nv];
            double ga = dot(n, a) + d, gb = dot(n, b) + d;
            if (ga >= 0.0 && G.nv < OR_MAXV) G.v[G.nv++] = a;
            if ((ga >= 0.0) != (gb >= 0.0)) {
                double t = ga / (ga - gb);
                v3 p = add(a, scl(sub(b, a), t));
                if (G.nv < OR_MAXV) G.v[G.nv++] = p;
                if (ncap < OR_MAXV * 2) cap[ncap++] = p;
            } else if (ga == 0.0 && ncap < OR_MAXV * 2) {
                cap[ncap++] = a;
            }
        }
        if (G.nv >= 3 && out.nf < OR_MAXF) out.f[out.nf++] = G;
    }
    /* cap face on the plane, outward normal -n */
    if (ncap >= 3 && out.nf < OR_MAXF) {
        double tol = 1e-12 * P->scale;
        v3 u[OR_MAXV * 2];
        int nu = 0;
        for (int k = 0; k < ncap; ++k) {
            int dup = 0;
            for (int q = 0; q < nu; ++q)
                if (norm(sub(cap[k], u[q])) <= tol) { dup = 1; break; }
            if (!dup) u[nu++] = cap[k];
        }
        if (nu >= 3 && nu <= OR_MAXV) {
            v3 c = mk(0, 0, 0);
            for (int k = 0; k < nu; ++k) c = add(c, u[k]);
            c = scl(c, 1.0 / nu);
            v3 m = scl(n, -1.0 / norm(n));              /* outward normal of the cap */
            v3 e1 = sub(u[0], c);
            e1 = scl(e1, 1.0 / norm(e1));
            v3 e2 = cross(m, e1);                        /* (e1, e2, m) right-handed */
            double ang[OR_MAXV * 2];
            for (int k = 0; k < nu; ++k) {
                v3 r = sub(u[k], c);
                ang[k] = atan2(dot(r, e2), dot(r, e1));
            }
            /* insertion sort by angle: CCW around m */
            for (int a = 1; a < nu; ++a) {
                double ta = ang[a];
                v3 va = u[a];
                int b = a - 1;
                while (b >= 0 && ang[b] > ta) { ang[b + 1] = ang[b]; u[b + 1] = u[b]; --b; }
                ang[b + 1] = ta;
                u[b + 1] = va;
            }
            face_t G;
            G.nv = nu;
            for (int k = 0; k < nu; ++k) G.v[k] = u[k];
            out.f[out.nf++] = G;
        }
    }
    *P = out;
    return P->nf;
}

/* volume and centre of mass by tetrahedra from an interior reference point */
static double ptope_volume(const ptope_t *P, v3 *centroid) {
    if (P->nf < 4) { if (centroid) *centroid = mk(0, 0, 0); return 0.0; }
    v3 o = mk(0, 0, 0);
    int cnt = 0;
    for (int f = 0; f < P->nf; ++f)
        for (int k = 0; k < P->f[f].nv; ++k) { o = add(o, P->f[f].v[k]); ++cnt; }
    o = scl(o, 1.0 / cnt);
    double V = 0.0;
    v3 M = mk(0, 0, 0);
    for (int f = 0; f < P->nf; ++f) {
        const face_t *F = &P->f[f];
        for (int k = 1; k + 1 < F->nv; ++k) {
            v3 a = sub(F->v[0], o), b = sub(F->v[k], o), c = sub(F->v[k + 1], o);
            double vt = dot(a, cross(b, c)) / 6.0;
            V += vt;
            M = add(M, scl(add(add(a, b), c), vt / 4.0));
        }
    }
    if (centroid) *centroid = (V > 0.0) ? add(o, scl(M, 1.0 / V)) : o;
    return V > 0.0 ? V : 0.0;
}

/* 7-point degree-5 rule on the triangle (Radon): barycentric points and weights */
static void tri_rule(double bary[7][3], double w[7]) {
    const double r15 = sqrt(15.0);
    double b1 = (6.0 - r15) / 21.0, a1 = 1.0 - 2.0 * b1;
    double b2 = (6.0 + r15) / 21.0, a2 = 1.0 - 2.0 * b2;
    double w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
    double B[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a1, b1, b1}, {b1, a1, b1}, {b1, b1, a1},
                      {a2, b2, b2}, {b2, a2, b2}, {b2, b2, a2}};
    double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    memcpy(bary, B, sizeof(B));
    memcpy(w, W, sizeof(W));
}

/* int_T |x - s|^-2 dA over triangle T, split into 4^level sub-triangles */
static double tri_inv_r2(v3 a, v3 b, v3 c, v3 s, int level) {
    if (level > 0) {
        v3 ab = scl(add(a, b), 0.5), bc = scl(add(b, c), 0.5), ca = scl(add(c, a), 0.5);
        return tri_inv_r2(a, ab, ca, s, level - 1) + tri_inv_r2(ab, b, bc, s, level - 1) +
               tri_inv_r2(ca, bc, c, s, level - 1) + tri_inv_r2(ab, bc, ca, s, level - 1);
    }
    double B[7][3], w[7];
    tri_rule(B, w);
    double area = 0.5 * norm(cross(sub(b, a), sub(c, a)));
    double acc = 0.0;
    for (int q = 0; q < 7; ++q) {
        v3 p = add(add(scl(a, B[q][0]), scl(b, B[q][1])), scl(c, B[q][2]));
        v3 r = sub(p, s);
        acc += w[q] / dot(r, r);
    }
    return acc * area;
}

/* J = int_P |x - s|^-2 dV = sum_faces h_F int_F |x - s|^-2 dA,  h_F = (x - s).n_F */
static double ptope_inv_r2(const ptope_t *P, v3 s, int level) {
    double J = 0.0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t *F = &P->f[f];
        v3 nrm = mk(0, 0, 0);
        for (int k = 1; k + 1 < F->nv; ++k)
            nrm = add(nrm, cross(sub(F->v[k], F->v[0]), sub(F->v[k + 1], F->v[0])));
        double ln = norm(nrm);
        if (ln <= 0.0) continue;
        nrm = scl(nrm, 1.0 / ln);
        double h = dot(sub(F->v[0], s), nrm);
        for (int k = 1; k + 1 < F->nv; ++k)
            J += h * tri_inv_r2(F->v[0], F->v[k], F->v[k + 1], s, level);
    }
    return J;
}

/* int_T |x - s| / |m2 . (x - s)|^3 dA over triangle T, split into 4^level sub-triangles */
static double tri_area_kernel(v3 a, v3 b, v3 c, v3 s, v3 m2, int level) {
    if (level > 0) {
        v3 ab = scl(add(a, b), 0.5), bc = scl(add(b, c), 0.5), ca = scl(add(c, a), 0.5);
        return tri_area_kernel(a, ab, ca, s, m2, level - 1) + tri_area_kernel(ab, b, bc, s, m2, level - 1) +
               tri_area_kernel(ca, bc, c, s, m2, level - 1) + tri_area_kernel(ab, bc, ca, s, m2, level - 1);
    }
    double B[7][3], w[7];
    tri_rule(B, w);
    double area = 0.5 * norm(cross(sub(b, a), sub(c, a)));
    double acc = 0.0;
    for (int q = 0; q < 7; ++q) {
        v3 p = add(add(scl(a, B[q][0]), scl(b, B[q][1])), scl(c, B[q][2]));
        v3 r = sub(p, s);
        double t = fabs(dot(m2, r));
        acc += w[q] * norm(r) / (t * t * t);
    }
    return acc * area;
}

/* int_P |x - s| / |m2 . (x - s)|^3 dV = sum_faces h_F int_F |x - s| / |m2 . (x - s)|^3 dA: the
 * field (x - s) |x - s| / |m2 . (x - s)|^3 is homogeneous of degree -2 about s, so its
 * divergence is the integrand, as for |x - s|^-2 above. */
static double ptope_area_kernel(const ptope_t *P, v3 s, v3 m2, int level) {
    double K = 0.0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t *F = &P->f[f];
        v3 nrm = mk(0, 0, 0);
        for (int k = 1; k + 1 < F->nv; ++k)
            nrm = add(nrm, cross(sub(F->v[k], F->v[0]), sub(F->v[k + 1], F->v[0])));
        double ln = norm(nrm);
        if (ln <= 0.0) continue;
        nrm = scl(nrm, 1.0 / ln);
        double h = dot(sub(F->v[0], s), nrm);
        for (int k = 1; k + 1 < F->nv; ++k)
            K += h * tri_area_kernel(F->v[0], F->v[k], F->v[k + 1], s, m2, level);
    }
    return K;
}

/* ------------------------------------------------------------------------------------ */
/* Geometry from the projection matrix                                                   */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double P[3][4];
    double Minv[3][3];
    double detM;
    v3 s;            /* source = -M^{-1} p4 */
    double sigma;    /* sign making sigma * (P2 . X) > 0 in front of the source */
} view_t;

static int view_setup(view_t *V, const double *P12) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) V->P[r][c] = P12[r * 4 + c];
    double (*M)[4] = V->P;
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(fabs(det) > 0.0) || !isfinite(det)) return -1;
    V->detM = det;
    double id = 1.0 / det;
    V->Minv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) * id;
    V->Minv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * id;
    V->Minv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * id;
    V->Minv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) * id;
    V->Minv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * id;
    V->Minv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * id;
    V->Minv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) * id;
    V->Minv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) * id;
    V->Minv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * id;
    double p4[3] = {M[0][3], M[1][3], M[2][3]};
    V->s = mk(-(V->Minv[0][0] * p4[0] + V->Minv[0][1] * p4[1] + V->Minv[0][2] * p4[2]),
              -(V->Minv[1][0] * p4[0] + V->Minv[1][1] * p4[1] + V->Minv[1][2] * p4[2]),
              -(V->Minv[2][0] * p4[0] + V->Minv[2][1] * p4[1] + V->Minv[2][2] * p4[2]));
    /* points in front of the source: the origin (centre of the volume) is assumed in front */
    double w0 = M[2][3];
    V->sigma = (w0 >= 0.0) ? 1.0 : -1.0;
    return 0;
}

static double prow(const view_t *V, int r, v3 x) {
    return V->P[r][0] * x.x + V->P[r][1] * x.y + V->P[r][2] * x.z + V->P[r][3];
}

static void project_point(const view_t *V, v3 x, double *u, double *v) {
    double w = prow(V, 2, x);
    *u = prow(V, 0, x) / w;
    *v = prow(V, 1, x) / w;
}

/* ray direction from the source through detector index point (u, v) */
static v3 ray_dir(const view_t *V, double u, double v) {
    double q[3] = {u, v, 1.0};
    v3 d = mk(V->Minv[0][0] * q[0] + V->Minv[0][1] * q[1] + V->Minv[0][2] * q[2],
              V->Minv[1][0] * q[0] + V->Minv[1][1] * q[1] + V->Minv[1][2] * q[2],
              V->Minv[2][0] * q[0] + V->Minv[2][1] * q[1] + V->Minv[2][2] * q[2]);
    /* orient towards the detector: sigma * P2 . (s + d) > 0  <=>  sigma * (M2 . d) > 0 */
    double m2d = V->P[2][0] * d.x + V->P[2][1] * d.y + V->P[2][2] * d.z;
    if (V->sigma * m2d < 0.0) d = scl(d, -1.0);
    return d;
}

/* half-space sigma * (A - c P2) . X >= 0 as (n, d) with A = P row r */
static void pyramid_plane(const view_t *V, int r, double c, double sgn, v3 *n, double *d) {
    double s = V->sigma * sgn;
    *n = mk(s * (V->P[r][0] - c * V->P[2][0]), s * (V->P[r][1] - c * V->P[2][1]),
            s * (V->P[r][2] - c * V->P[2][2]));
    *d = s * (V->P[r][3] - c * V->P[2][3]);
}

/* ------------------------------------------------------------------------------------ */
/* Pixel factors                                                                         */
/* ------------------------------------------------------------------------------------ */

/* cos scaling, Eq. cvp: f^2 / (a cos^3 theta) at the pixel centre.  In detector index
 * units the matrix is M = lambda K R with K = [[f/p1, s, c1], [0, f/p2, c2], [0, 0, 1]],
 * so f^2 / a = f^2 / (p1 p2) = |det M| / |M_2|^3 (M_2 = third row), and theta is the
 * angle between the ray to the pixel centre and the detector normal M_2. */
static double factor_cos(const view_t *V, double u, double v) {
    v3 m2 = mk(V->P[2][0], V->P[2][1], V->P[2][2]);
    double lm2 = norm(m2);
    double f2_over_a = fabs(V->detM) / (lm2 * lm2 * lm2);
    v3 d = ray_dir(V, u, v);
    double cth = fabs(dot(d, m2)) / (norm(d) * lm2);
    return f2_over_a / (cth * cth * cth);
}

/* exact scaling, Eq. cvpus: 1 / abar with abar = 2 pi - sum_i arccos(...) over the
 * four corner directions t_0..t_3 in cyclic order (spherical excess of the pixel). */
static double pixel_solid_angle(const view_t *V, double u, double v) {
    v3 t[4];
    t[0] = ray_dir(V, u - 0.5, v - 0.5);
    t[1] = ray_dir(V, u + 0.5, v - 0.5);
    t[2] = ray_dir(V, u + 0.5, v + 0.5);
    t[3] = ray_dir(V, u - 0.5, v + 0.5);
    for (int i = 0; i < 4; ++i) t[i] = scl(t[i], 1.0 / norm(t[i]));
    double sum = 0.0;
    for (int i = 0; i < 4; ++i) {
        v3 a = cross(t[i], t[(i + 1) % 4]);
        v3 b = cross(t[(i + 1) % 4], t[(i + 2) % 4]);
        double c = dot(a, b) / (norm(a) * norm(b));
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        sum += acos(c);
    }
    return 2.0 * M_PI - sum;
}

static double factor_exact(const view_t *V, double u, double v) {
    return 1.0 / pixel_solid_angle(V, u, v);
}

static double pixel_factor(const view_t *V, double u, double v, int scaling) {
    return scaling == 1 ? factor_exact(V, u, v) : factor_cos(V, u, v);
}

/* ------------------------------------------------------------------------------------ */
/* Pair weights                                                                          */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    double a[3];
    double x0[3];
    int nu, nv;
} grid_t;

static void grid_setup(grid_t *G, int nx, int ny, int nz, double ax, double ay, double az, int nu, int nv) {
    G->nx = nx; G->ny = ny; G->nz = nz;
    G->a[0] = ax; G->a[1] = ay; G->a[2] = az;
    G->x0[0] = (-nx * ax + ax) / 2.0;
    G->x0[1] = (-ny * ay + ay) / 2.0;
    G->x0[2] = (-nz * az + az) / 2.0;
    G->nu = nu; G->nv = nv;
}

static v3 voxel_centre(const grid_t *G, int i, int j, int k) {
    return mk(G->x0[0] + i * G->a[0], G->x0[1] + j * G->a[1], G->x0[2] + k * G->a[2]);
}

/* pair quantities for a box and a pixel */
typedef struct { double V, cx, cy, cz, W, J, Wrel; } pair_t;

static void box_pixel_pair(const view_t *Vw, const double lo[3], const double hi[3],
                           double u, double v, int want_J, pair_t *out) {
    ptope_t P;
    box_ptope(&P, lo, hi);
    v3 n; double d;
    pyramid_plane(Vw, 0, u - 0.5, +1.0, &n, &d); clip_ptope(&P, n, d);   /* u(X) >= u - 1/2 */
    pyramid_plane(Vw, 0, u + 0.5, -1.0, &n, &d); clip_ptope(&P, n, d);   /* u(X) <= u + 1/2 */
    /* relaxed variant needs the column cut only */
    ptope_t Pc = P;
    pyramid_plane(Vw, 1, v - 0.5, +1.0, &n, &d); clip_ptope(&P, n, d);   /* v(X) >= v - 1/2 */
    pyramid_plane(Vw, 1, v + 0.5, -1.0, &n, &d); clip_ptope(&P, n, d);   /* v(X) <= v + 1/2 */
    v3 c;
    double Vol = ptope_volume(&P, &c);
    out->V = Vol;
    out->cx = c.x; out->cy = c.y; out->cz = c.z;
    v3 r = sub(c, Vw->s);
    out->W = Vol > 0.0 ? Vol / dot(r, r) : 0.0;
    out->J = (want_J && Vol > 0.0) ? ptope_inv_r2(&P, Vw->s, want_J - 1) : 0.0;

    /* relaxed: A_n = |column cut| / a3, centre of mass CM of the column cut in x1 x2,
     * d = |[z0, z1] intersected with {x3 : v(CM, x3) in (v - 1/2, v + 1/2)}| */
    v3 cm;
    double Vc = ptope_volume(&Pc, &cm);
    double a3 = hi[2] - lo[2];
    double A = Vc / a3;
    double Wrel = 0.0;
    if (Vc > 0.0) {
        /* v(x3) = (q1 + P12 x3) / q2 along the vertical line through CM (P22 = 0) */
        double q1 = Vw->P[1][0] * cm.x + Vw->P[1][1] * cm.y + Vw->P[1][3];
        double q2 = Vw->P[2][0] * cm.x + Vw->P[2][1] * cm.y + Vw->P[2][3];
        double p12 = Vw->P[1][2];
        double za = ((v - 0.5) * q2 - q1) / p12, zb = ((v + 0.5) * q2 - q1) / p12;
        double zl = fmin(za, zb), zh = fmax(za, zb);
        double dlen = fmin(zh, hi[2]) - fmax(zl, lo[2]);
        if (dlen > 0.0) {
            v3 xc = mk(0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2]));
            v3 rv = sub(xc, Vw->s);
            Wrel = A * dlen / dot(rv, rv);
        }
    }
    out->Wrel = Wrel;
}

/* Truth of the area-averaged pixel value for one pair (Eq. integ with Eq. voxat): the area
 * average over pixel (u, v) of the voxel's chord lengths. The detector-index area element
 * per solid angle at a ray through x is |det M| (|x - s| / |w|)^3 with w = P2 . (x, 1), and
 * dV = r^2 dr dOmega, so the average is |det M| int_cut |x - s| / |w|^3 dV; P2 . (x, 1) =
 * M2 . (x - s) since M s + p4 = 0. */
static double box_pixel_area_truth(const view_t *Vw, const double lo[3], const double hi[3], double u, double v) {
    ptope_t P;
    box_ptope(&P, lo, hi);
    v3 n; double d;
    pyramid_plane(Vw, 0, u - 0.5, +1.0, &n, &d); clip_ptope(&P, n, d);
    pyramid_plane(Vw, 0, u + 0.5, -1.0, &n, &d); clip_ptope(&P, n, d);
    pyramid_plane(Vw, 1, v - 0.5, +1.0, &n, &d); clip_ptope(&P, n, d);
    pyramid_plane(Vw, 1, v + 0.5, -1.0, &n, &d); clip_ptope(&P, n, d);
    if (!(ptope_volume(&P, NULL) > 0.0)) return 0.0;
    v3 m2 = mk(Vw->P[2][0], Vw->P[2][1], Vw->P[2][2]);
    return fabs(Vw->detM) * ptope_area_kernel(&P, Vw->s, m2, 0);
}

static void voxel_box(const grid_t *G, int i, int j, int k, double lo[3], double hi[3]) {
    v3 c = voxel_centre(G, i, j, k);
    lo[0] = c.x - 0.5 * G->a[0]; hi[0] = c.x + 0.5 * G->a[0];
    lo[1] = c.y - 0.5 * G->a[1]; hi[1] = c.y + 0.5 * G->a[1];
    lo[2] = c.z - 0.5 * G->a[2]; hi[2] = c.z + 0.5 * G->a[2];
}

/* bounding box of the corner projections -> candidate pixel index ranges (clipped) */
static int voxel_footprint(const view_t *V, const grid_t *G, const double lo[3], const double hi[3],
                           int *u0, int *u1, int *v0, int *v1) {
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int n = 0; n < 8; ++n) {
        v3 x = mk((n & 1) ? hi[0] : lo[0], (n & 2) ? hi[1] : lo[1], (n & 4) ? hi[2] : lo[2]);
        double u, v;
        project_point(V, x, &u, &v);
        umin = fmin(umin, u); umax = fmax(umax, u);
        vmin = fmin(vmin, v); vmax = fmax(vmax, v);
    }
    *u0 = (int)floor(umin + 0.5); *u1 = (int)floor(umax + 0.5);
    *v0 = (int)floor(vmin + 0.5); *v1 = (int)floor(vmax + 0.5);
    if (*u0 < 0) *u0 = 0;
    if (*v0 < 0) *v0 = 0;
    if (*u1 > G->nu - 1) *u1 = G->nu - 1;
    if (*v1 > G->nv - 1) *v1 = G->nv - 1;
    return (*u0 <= *u1) && (*v0 <= *v1);
}

static double pair_weight(const pair_t *p, int variant) { return variant == 1 ? p->Wrel : p->W; }

/* ------------------------------------------------------------------------------------ */
/* Exported entry points (ctypes)                                                        */
/* ------------------------------------------------------------------------------------ */

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Source position of a view; returns 0 on success. */
int or_source(const double *P12, double *s_out) {
    view_t V;
    if (view_setup(&V, P12)) return -1;
    s_out[0] = V.s.x; s_out[1] = V.s.y; s_out[2] = V.s.z;
    return 0;
}

/* Pair quantities for an arbitrary box and pixel:
 * out = [V, cx, cy, cz, W_exact, J, W_relaxed].  quad_level < 0 skips J. */
int or_box_pixel(const double *P12, const double *lo, const double *hi, double u, double v,
                 int quad_level, double *out) {
    view_t V;
    if (view_setup(&V, P12)) return -1;
    pair_t p;
    box_pixel_pair(&V, lo, hi, u, v, quad_level >= 0 ? quad_level + 1 : 0, &p);
    out[0] = p.V; out[1] = p.cx; out[2] = p.cy; out[3] = p.cz;
    out[4] = p.W; out[5] = p.J; out[6] = p.Wrel;
    return 0;
}

/* Volume and centroid of a box clipped by nplanes half-spaces n.x + d >= 0
 * (planes: [nplanes][4] = nx, ny, nz, d). out = [V, cx, cy, cz]. */
int or_box_clip(const double *lo, const double *hi, const double *planes, int nplanes, double *out) {
    ptope_t P;
    box_ptope(&P, lo, hi);
    for (int q = 0; q < nplanes; ++q)
        clip_ptope(&P, mk(planes[4 * q], planes[4 * q + 1], planes[4 * q + 2]), planes[4 * q + 3]);
    v3 c;
    out[0] = ptope_volume(&P, &c);
    out[1] = c.x; out[2] = c.y; out[3] = c.z;
    return 0;
}

/* int_box |x - s|^-2 dV by the face formula (used to check it against volume quadrature) */
double or_box_inv_r2(const double *lo, const double *hi, const double *s, int level) {
    ptope_t P;
    box_ptope(&P, lo, hi);
    return ptope_inv_r2(&P, mk(s[0], s[1], s[2]), level);
}

/* Pixel factor F(u, v) of a view. scaling 0 = cos, 1 = exact. */
double or_pixel_factor(const double *P12, double u, double v, int scaling) {
    view_t V;
    if (view_setup(&V, P12)) return NAN;
    return pixel_factor(&V, u, v, scaling);
}

double or_pixel_solid_angle(const double *P12, double u, double v) {
    view_t V;
    if (view_setup(&V, P12)) return NAN;
    return pixel_solid_angle(&V, u, v);
}

/* Forward projection b = F (W x).  x: [nz][ny][nx], b: [nviews][nv][nu]. */
int or_project(int nx, int ny, int nz, double ax, double ay, double az, int nu, int nv,
               const double *pmats, int nviews, int variant, int scaling,
               const double *x, double *b) {
    grid_t G;
    grid_setup(&G, nx, ny, nz, ax, ay, az, nu, nv);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int view = 0; view < nviews; ++view) {
        view_t V;
        if (view_setup(&V, pmats + 12 * view)) { err |= 1; continue; }
        double *S = b + (size_t)view * nu * nv;
        for (size_t q = 0; q < (size_t)nu * nv; ++q) S[q] = 0.0;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double mu = x[((size_t)k * ny + j) * nx + i];
                    if (mu == 0.0) continue;
                    double lo[3], hi[3];
                    voxel_box(&G, i, j, k, lo, hi);
                    int u0, u1, v0, v1;
                    if (!voxel_footprint(&V, &G, lo, hi, &u0, &u1, &v0, &v1)) continue;
                    for (int pv = v0; pv <= v1; ++pv)
                        for (int pu = u0; pu <= u1; ++pu) {
                            pair_t p;
                            box_pixel_pair(&V, lo, hi, pu, pv, 0, &p);
                            S[(size_t)pv * nu + pu] += mu * pair_weight(&p, variant);
                        }
                }
        for (int pv = 0; pv < nv; ++pv)
            for (int pu = 0; pu < nu; ++pu) S[(size_t)pv * nu + pu] *= pixel_factor(&V, pu, pv, scaling);
    }
    return err ? -1 : 0;
}

/* one voxel of the adjoint: sum over views and footprint pixels of W F y */
static double backproject_voxel(const grid_t *G, const view_t *views, int nviews, int variant, int scaling,
                                const double *y, int i, int j, int k) {
    double lo[3], hi[3];
    voxel_box(G, i, j, k, lo, hi);
    double acc = 0.0;
    for (int view = 0; view < nviews; ++view) {
        const view_t *V = &views[view];
        int u0, u1, v0, v1;
        if (!voxel_footprint(V, G, lo, hi, &u0, &u1, &v0, &v1)) continue;
        const double *Y = y + (size_t)view * G->nu * G->nv;
        for (int pv = v0; pv <= v1; ++pv)
            for (int pu = u0; pu <= u1; ++pu) {
                pair_t p;
                box_pixel_pair(V, lo, hi, pu, pv, 0, &p);
                double w = pair_weight(&p, variant);
                if (w != 0.0) acc += w * pixel_factor(V, pu, pv, scaling) * Y[(size_t)pv * G->nu + pu];
            }
    }
    return acc;
}

/* Adjoint x = W^T (F y).  y: [nviews][nv][nu], x: [nz][ny][nx]. */
int or_backproject(int nx, int ny, int nz, double ax, double ay, double az, int nu, int nv,
                   const double *pmats, int nviews, int variant, int scaling,
                   const double *y, double *x) {
    grid_t G;
    grid_setup(&G, nx, ny, nz, ax, ay, az, nu, nv);
    view_t *views = (view_t *)malloc(sizeof(view_t) * (size_t)(nviews > 0 ? nviews : 1));
    if (!views) return -2;
    for (int q = 0; q < nviews; ++q)
        if (view_setup(&views[q], pmats + 12 * q)) { free(views); return -1; }
    long total = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 16)
    for (long idx = 0; idx < total; ++idx) {
        int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((long)nx * ny));
        x[idx] = backproject_voxel(&G, views, nviews, variant, scaling, y, i, j, k);
    }
    free(views);
    return 0;
}

/* Adjoint on selected voxels only. vox: [count][3] = (k, j, i). */
int or_backproject_voxels(int nx, int ny, int nz, double ax, double ay, double az, int nu, int nv,
                          const double *pmats, int nviews, int variant, int scaling,
                          const double *y, const int32_t *vox, int count, double *out) {
    grid_t G;
    grid_setup(&G, nx, ny, nz, ax, ay, az, nu, nv);
    view_t *views = (view_t *)malloc(sizeof(view_t) * (size_t)(nviews > 0 ? nviews : 1));
    if (!views) return -2;
    for (int q = 0; q < nviews; ++q)
        if (view_setup(&views[q], pmats + 12 * q)) { free(views); return -1; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < count; ++q)
        out[q] = backproject_voxel(&G, views, nviews, variant, scaling, y, vox[3 * q + 2], vox[3 * q + 1], vox[3 * q]);
    free(views);
    return 0;
}

/* Forward projection of selected pixels only. pix: [count][3] = (view, v, u).
 * Candidate voxels: columns (i, j) whose base square is not entirely outside one of
 * the two column planes of the pixel, and for those the slices k that meet the z-range
 * of the row slab over the column's four vertical edges.
 * variant 0 / 1: the near-exact / relaxed pair weights W. variant 2: the truth the scaled
 * projection approximates, with no sampling of rays: for the exact scaling the solid-angle
 * average over the pixel of the line integrals of the voxel volume (Eq. integub), the
 * truth integral J = int_cut r^-2 dV of every pair (Eq. intcut) times 1 / abar; for the cos
 * scaling their area average over the pixel (Eq. integ), box_pixel_area_truth per pair. */
int or_project_pixels(int nx, int ny, int nz, double ax, double ay, double az, int nu, int nv,
                      const double *pmats, int nviews, int variant, int scaling,
                      const double *x, const int32_t *pix, int count, double *out) {
    grid_t G;
    grid_setup(&G, nx, ny, nz, ax, ay, az, nu, nv);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int q = 0; q < count; ++q) {
        int view = pix[3 * q], pv = pix[3 * q + 1], pu = pix[3 * q + 2];
        view_t V;
        if (view < 0 || view >= nviews || view_setup(&V, pmats + 12 * view)) { err |= 1; out[q] = NAN; continue; }
        v3 n1, n2, n3, n4; double d1, d2, d3, d4;
        pyramid_plane(&V, 0, pu - 0.5, +1.0, &n1, &d1);
        pyramid_plane(&V, 0, pu + 0.5, -1.0, &n2, &d2);
        pyramid_plane(&V, 1, pv - 0.5, +1.0, &n3, &d3);
        pyramid_plane(&V, 1, pv + 0.5, -1.0, &n4, &d4);
        double acc = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                v3 c = voxel_centre(&G, i, j, 0);
                double xs[2] = {c.x - 0.5 * ax, c.x + 0.5 * ax}, ys[2] = {c.y - 0.5 * ay, c.y + 0.5 * ay};
                int out1 = 1, out2 = 1;
                for (int e = 0; e < 4; ++e) {
                    v3 p = mk(xs[e & 1], ys[e >> 1], 0.0);   /* column planes are vertical */
                    if (dot(n1, p) + d1 >= 0.0) out1 = 0;
                    if (dot(n2, p) + d2 >= 0.0) out2 = 0;
                }
                if (out1 || out2) continue;
                /* z where each row plane meets each vertical edge */
                double zmin = INFINITY, zmax = -INFINITY;
                for (int e = 0; e < 4; ++e) {
                    v3 p = mk(xs[e & 1], ys[e >> 1], 0.0);
                    double za = -(n3.x * p.x + n3.y * p.y + d3) / n3.z;
                    double zb = -(n4.x * p.x + n4.y * p.y + d4) / n4.z;
                    zmin = fmin(zmin, fmin(za, zb));
                    zmax = fmax(zmax, fmax(za, zb));
                }
                int k0 = (int)floor((zmin - (G.x0[2] - 0.5 * az)) / az) - 1;
                int k1 = (int)floor((zmax - (G.x0[2] - 0.5 * az)) / az) + 1;
                if (k0 < 0) k0 = 0;
                if (k1 > nz - 1) k1 = nz - 1;
                for (int k = k0; k <= k1; ++k) {
                    double mu = x[((size_t)k * ny + j) * nx + i];
                    if (mu == 0.0) continue;
                    double lo[3], hi[3];
                    voxel_box(&G, i, j, k, lo, hi);
                    pair_t p;
                    if (variant == 2 && scaling == 0) {
                        acc += mu * box_pixel_area_truth(&V, lo, hi, pu, pv);
                        continue;
                    }
                    box_pixel_pair(&V, lo, hi, pu, pv, variant == 2 ? 1 : 0, &p);
                    acc += mu * (variant == 2 ? p.J : pair_weight(&p, variant));
                }
            }
        out[q] = (variant == 2 && scaling == 0) ? acc : acc * pixel_factor(&V, pu, pv, scaling);
    }
    return err ? -1 : 0;
}

/* length of the segment s + t d, t in (0, inf), inside box [lo, hi] (slab method) */
static double ray_box_length(v3 s, v3 d, const double lo[3], const double hi[3]) {
    double t0 = 0.0, t1 = INFINITY;
    double S[3] = {s.x, s.y, s.z}, D[3] = {d.x, d.y, d.z};
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.0) {
            if (S[a] <= lo[a] || S[a] >= hi[a]) return 0.0;
        } else {
            double ta = (lo[a] - S[a]) / D[a], tb = (hi[a] - S[a]) / D[a];
            if (ta > tb) { double t = ta; ta = tb; tb = t; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        }
    }
    return (t1 > t0) ? (t1 - t0) * norm(d) : 0.0;
}

/* Ray-integration value of one pixel: average over K x K equally spaced points of the
 * line integral sum_vox mu |vox ∩ ray| (exact path lengths, every voxel tested).
 * weighting 0: equal weights (area average, Eq. integ); 1: solid-angle element weights
 * (unit-sphere average, Eq. integub). */
double or_ray_pixel(int nx, int ny, int nz, double ax, double ay, double az,
                    const double *P12, const double *x, double u, double v, int K, int weighting) {
    grid_t G;
    grid_setup(&G, nx, ny, nz, ax, ay, az, 1, 1);
    view_t V;
    if (view_setup(&V, P12)) return NAN;
    double num = 0.0, den = 0.0;
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            double uu = u - 0.5 + (a + 0.5) / K, vv = v - 0.5 + (b + 0.5) / K;
            v3 d = ray_dir(&V, uu, vv);
            double line = 0.0;
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        double mu = x[((size_t)k * ny + j) * nx + i];
                        if (mu == 0.0) continue;
                        double lo[3], hi[3];
                        voxel_box(&G, i, j, k, lo, hi);
                        line += mu * ray_box_length(V.s, d, lo, hi);
                    }
            double w = 1.0;
            if (weighting == 1) {
                /* dOmega = |det M^{-1}| / |d|^3 du dv for d = M^{-1}(u, v, 1) */
                double q[3] = {uu, vv, 1.0};
                v3 dd = mk(V.Minv[0][0] * q[0] + V.Minv[0][1] * q[1] + V.Minv[0][2] * q[2],
                           V.Minv[1][0] * q[0] + V.Minv[1][1] * q[1] + V.Minv[1][2] * q[2],
                           V.Minv[2][0] * q[0] + V.Minv[2][1] * q[1] + V.Minv[2][2] * q[2]);
                double ln = norm(dd);
                w = 1.0 / (ln * ln * ln);
            }
            num += w * line;
            den += w;
        }
    return num / den;
}
