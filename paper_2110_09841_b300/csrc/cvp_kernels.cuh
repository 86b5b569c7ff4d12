// cvp_kernels.cuh -- brick-tiled CUDA kernels of the cutting voxel projector (sm_103a).
//
// A thread block owns a brick of BX x BY voxel columns and SEG = 64 voxels along x_3.
//  * Forward: the brick's attenuation values are staged in shared memory once; for each view
//    of the block's chunk, the voxel-pixel weights are accumulated into a shared-memory
//    detector tile that covers the brick's footprint, then the tile is added to the global
//    sums with coalesced float atomics (the paper's two rounds of atomic addition, Sec.
//    III-C, with a tile per brick instead of per voxel cube).
//  * Adjoint: for each view the brick's footprint of the pixel-scaled projection is staged
//    in shared memory; every voxel gathers its weights times those values (no atomics) and
//    the block writes each voxel once at the end.
// Inside a block, a warp processes one voxel column at a time, lane l owning voxels
// kbase + l + 32 p (p < KPL). The column cuts H_n of the voxel base are the same for every
// voxel of the column (Sec. III-A, Eq. columnprojectionidentity): lane c computes H_n for
// n = cstart + c and the warp shares the moments through shared memory. Each lane then
// walks the rows of its own voxel. A row whose two planes stay inside the voxel over the
// whole base gives its pairs in closed form from the moments of H_n; a plane that leaves the
// voxel through its top or bottom face ("crossing") needs the moments of H_n cut at a depth
// tau. Crossing planes are queued per warp and evaluated by all 32 lanes together, one
// (event, column) task per lane, so the clipping never runs with most of the warp idle.
// Forward projection and adjoint enumerate the same pairs with the same code, so
// <A x, y> = <x, A^T y> holds to float rounding.
#pragma once

#include "cvp_device.cuh"

namespace kct {

constexpr int KPL = 2;             // voxels per lane in a column segment
constexpr int SEG = 32 * KPL;      // voxels of a column in a brick
constexpr int BX = 8, BY = 8;      // voxel columns of a brick
constexpr int NCOLS = BX * BY;
constexpr int NWARP = 8;           // warps per block
constexpr int NTHREADS = 32 * NWARP;
constexpr int EV_CAP = 64;         // crossing events queued per warp and round
constexpr int KCT_ROWS = 32;       // row boundaries of one voxel (its footprint spans <= 31 rows)
constexpr int TILE_CAP = 8192;     // floats of the shared detector tile
constexpr int VIEW_CHUNK = 16;     // views per forward block
constexpr unsigned FULLMASK = 0xffffffffu;

struct WarpSmem {
    Column C;                      // the warp's current column
    float4 fa[KCT_CB];             // moments of H_n: m1, mt, mtt, ml
    float fb[KCT_CB];              // mlt
    float ev_p0[EV_CAP], ev_p1[EV_CAP], ev_zs[EV_CAP];
    float res_v[EV_CAP][KCT_CB];
    float res_q[EV_CAP][KCT_CB];
};

struct Tile {                      // detector window covered by a brick in one view
    int u0, v0, w, h, ok;
};

struct BlockSmem {
    View V;
    Tile T;
    WarpSmem ws[NWARP];
};

// Row-boundary classes (in the sense of the region v < V_b)
enum { ROW_ZERO = 0, ROW_FULL = 1, ROW_LIN = 2, ROW_CROSS = 3 };

// Height of {v < V_b} over base point t' is clamp(p0 + p1 t', 0, az), measured from the face
// on which that region sits ("bottom frame"). The complementary region {v > V_b} has height
// clamp(pt0 - p1 t', 0, az), pt0 = az - p0, measured from the opposite face ("top frame").
struct RowPlane {
    int cls;
    float p0, p1, pt0;
};

KCT_HD RowPlane row_boundary(const View& V, const Grid& G, const Column& C, const Slice& S, float Vb) {
    RowPlane r;
    r.p0 = r.p1 = 0.f;
    r.pt0 = G.az;
    if (Vb <= S.vmin) { r.cls = ROW_ZERO; return r; }
    if (Vb >= S.vmax) { r.cls = ROW_FULL; r.p0 = G.az; r.pt0 = 0.f; return r; }
    const float dv = -fmaf(V.gv, S.bc, V.cv - Vb);        // V_b - v_c
    const float off = C.tc * dv * V.inv_agv;
    r.p0 = 0.5f * G.az + off;
    r.pt0 = 0.5f * G.az - off;
    r.p1 = (Vb - V.cv) * V.inv_agv;
    // does the plane leave the voxel through a horizontal face inside the base's depth range?
    const float h_lo = fmaf(r.p1, V.tmin_sq, r.p0), h_hi = fmaf(r.p1, V.tmax_sq, r.p0);
    r.cls = (fminf(h_lo, h_hi) < 0.f || fmaxf(h_lo, h_hi) > G.az) ? ROW_CROSS : ROW_LIN;
    return r;
}

// Moments (1, t', t'^2, lambda, lambda t') of H_n ∩ {t' < tau}; tau = +inf for all of H_n.
// Not inlined: the polygon clipping exists once in the code and its callers stay small.
__device__ __noinline__ Mom cut_moments_call(const View* V, const Column* C, int n, float tau) {
    if (tau <= V->tmin_sq) return Mom{0.f, 0.f, 0.f, 0.f, 0.f};
    Line lo, hi;
    column_lines(*V, *C, n, lo, hi);
    const Line lt = (tau < V->tmax_sq) ? Line{1.f, 0.f, tau} : line_none();
    return normalise(region3<true>(*V, lo, hi, lt), C->tc, C->xc);
}

// Volume and first moment along D of {(t', xi') in H_n, 0 < height < clamp(p0 + p1 t', 0, az)}
// (height from the frame's face; zs = zeta_c * sign(gv), negated in the top frame) for a
// plane that leaves the voxel through a face: h = 0 at tau0 and h = az at tau1.
KCT_HD void g_cross_from(float az, const Mom& c0, const Mom& c1, const Mom& full, float p0, float p1, float p1s,
                         float zs, float& gv, float& gq) {
    Mom lin, fu;
    if (p1s > 0.f) { lin = mom_sub(c1, c0); fu = mom_sub(full, c1); }
    else { lin = mom_sub(c0, c1); fu = c1; }
    const float Vg = fmaf(p0, lin.m1, fmaf(p1, lin.mt, az * fu.m1));
    const float Sl = fmaf(p0, lin.ml, fmaf(p1, lin.mlt, az * fu.ml));
    const float Sh2 = fmaf(p0 * p0, lin.m1, fmaf(2.f * p0 * p1, lin.mt, fmaf(p1 * p1, lin.mtt, az * az * fu.m1)));
    gv = Vg;
    gq = fmaf(zs, fmaf(0.5f, Sh2, -0.5f * az * Vg), Sl);
}

// the same quantity for a plane that stays inside the voxel over the whole base
KCT_HD void g_lin(float az, float p0, float p1, float zs, float f1, float ft, float ftt, float fl, float flt,
                  float& gv, float& gq) {
    const float Vg = fmaf(p0, f1, p1 * ft);
    const float Sl = fmaf(p0, fl, p1 * flt);
    const float Sh2 = fmaf(p0 * p0, f1, fmaf(2.f * p0 * p1, ft, p1 * p1 * ftt));
    gv = Vg;
    gq = fmaf(zs, fmaf(0.5f, Sh2, -0.5f * az * Vg), Sl);
}

__device__ __forceinline__ float pair_weight(float pv, float pq, float D2) {
    return __fdividef(pv * pv, fmaf(pv, D2, 2.f * pq));
}

// Near-exact pairs of voxels kbase + lane + 32 p of the warp's column, columns
// n = cstart .. cstart + ncol - 1. Each pair (n, m) is the integral over H_n of the height
// between the two row planes of row m. When both planes stay inside the voxel this height
// is linear in t' and the pair is a closed form of the moments of H_n. Otherwise it is the
// difference of the cuts below (or above) the two planes, measured from the nearer face
// (bottom frame for the lower half of the voxel's rows, top frame for the upper half), so
// that no pair is a small difference of two near-full voxel volumes.
template <class Sink>
__device__ __forceinline__ void exact_voxels(const View& V, const Grid& G, const Column& C, int cstart, int ncol,
                                             int kbase, int lane, WarpSmem* ws, Sink& sink, int* err) {
    const float az = G.az;
    const float dp0 = C.tc * V.inv_agv, dp1 = V.inv_agv;   // change of p0, p1 from one row boundary to the next
    const float vtiny = 1e-9f * G.ax * G.ay * az;
    for (int pass = 0; pass < KPL; ++pass) {
        const int k = kbase + pass * 32 + lane;
        Slice S;
        bool act = (k < G.nz) && slice_setup(V, G, C, k, S);
        if (act && S.m_last - S.m_first + 2 > KCT_ROWS) { atomicOr(err, 1); act = false; }
        const int R = act ? S.m_last - S.m_first + 1 : 0;      // rows of this voxel
        const int rb = (R + 1) >> 1;                            // rows r < rb use the bottom frame
        const float zs = act ? S.zc * V.sgv : 0.f;
        // crossing boundaries: bottom-frame events for b <= rb, top-frame events for b >= rb
        unsigned cross = 0u;
        for (int b = 0; b <= R && act; ++b)
            if (row_boundary(V, G, C, S, (float)(S.m_first + b) - 0.5f).cls == ROW_CROSS) cross |= 1u << b;
        const unsigned mbot = cross & ((2u << rb) - 1u);
        const unsigned mtop = cross & ~((1u << rb) - 1u);
        const int nbot = __popc(mbot);
        const int nev = nbot + __popc(mtop);
        int incl = nev;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULLMASK, incl, o);
            if (lane >= o) incl += t;
        }
        const int base = incl - nev;
        // lanes are served in contiguous groups whose events fit the queue (a lane has at most
        // KCT_ROWS + 1 <= EV_CAP events, so every group makes progress)
        for (int lo_lane = 0; lo_lane < 32;) {
            const int base_lo = __shfl_sync(FULLMASK, base, lo_lane);
            const unsigned fit = __ballot_sync(FULLMASK, lane >= lo_lane && incl - base_lo <= EV_CAP);
            const int hi_lane = 32 - __clz(fit);
            const bool mine = lane >= lo_lane && lane < hi_lane;
            const int ne = __shfl_sync(FULLMASK, incl, hi_lane - 1) - base_lo;
            const int e0 = base - base_lo;
            // 1) queue the group's crossing planes (frame-transformed parameters)
            if (mine && nev) {
                for (int b = 0; b <= R; ++b) {
                    if (!((cross >> b) & 1u)) continue;
                    const RowPlane rp = row_boundary(V, G, C, S, (float)(S.m_first + b) - 0.5f);
                    if (b <= rb) {
                        const int q = e0 + __popc(mbot & ((1u << b) - 1u));
                        ws->ev_p0[q] = rp.p0;
                        ws->ev_p1[q] = rp.p1;
                        ws->ev_zs[q] = zs;
                    }
                    if (b >= rb) {
                        const int q = e0 + nbot + __popc(mtop & ((1u << b) - 1u));
                        ws->ev_p0[q] = rp.pt0;
                        ws->ev_p1[q] = -rp.p1;
                        ws->ev_zs[q] = -zs;
                    }
                }
            }
            __syncwarp();
            // 2) the whole warp evaluates (event, column) tasks
            for (int t = lane; t < ne * ncol; t += 32) {
                const int e = t / ncol, c = t - e * ncol;
                const float p0 = ws->ev_p0[e], p1 = ws->ev_p1[e];
                const float p1s = (fabsf(p1) < 1e-30f) ? copysignf(1e-30f, p1) : p1;
                const float4 a = ws->fa[c];
                const Mom full = Mom{a.x, a.y, a.z, a.w, ws->fb[c]};
                const Mom c0 = cut_moments_call(&V, &ws->C, cstart + c, -p0 / p1s);
                const Mom c1 = cut_moments_call(&V, &ws->C, cstart + c, (az - p0) / p1s);
                float gv, gq;
                g_cross_from(az, c0, c1, full, p0, p1, p1s, ws->ev_zs[e], gv, gq);
                ws->res_v[e][c] = gv;
                ws->res_q[e][c] = gq;
            }
            __syncwarp();
            // 3) pairs of the group's voxels
            if (mine && act) {
                sink.begin(pass, k);
                const float D2 = fmaf(C.tc, C.tc, fmaf(C.xc, C.xc, S.zc * S.zc));
                // the crossing decision is taken once (the mask): a plane that touches a face
                // to within rounding must not be classified differently here
                RowPlane rlo = row_boundary(V, G, C, S, (float)S.m_first - 0.5f);
                if (rlo.cls >= ROW_LIN) rlo.cls = (cross & 1u) ? ROW_CROSS : ROW_LIN;
                for (int r = 0; r < R; ++r) {
                    const int m = S.m_first + r;
                    RowPlane rhi = row_boundary(V, G, C, S, (float)m + 0.5f);
                    if (rhi.cls >= ROW_LIN) rhi.cls = ((cross >> (r + 1)) & 1u) ? ROW_CROSS : ROW_LIN;
                    if (rlo.cls == ROW_LIN && rhi.cls == ROW_LIN) {
                        // height between the planes: dp0 + dp1 t', centred at s0 + s1 t'
                        const float s0 = C.tc * (-fmaf(V.gv, S.bc, V.cv - (float)m)) * V.inv_agv;
                        const float s1 = ((float)m - V.cv) * V.inv_agv;
                        const float a0 = zs * dp0 * s0, a1 = zs * fmaf(dp0, s1, dp1 * s0), a2 = zs * dp1 * s1;
#pragma unroll 1
                        for (int c = 0; c < ncol; ++c) {
                            const float4 f = ws->fa[c];
                            const float pv = fmaf(dp0, f.x, dp1 * f.y);
                            const float pq = fmaf(dp0, f.w, fmaf(dp1, ws->fb[c], fmaf(a0, f.x, fmaf(a1, f.y, a2 * f.z))));
                            if (pv > vtiny) sink.pair(pass, cstart + c, m, pair_weight(pv, pq, D2));
                        }
                    } else {
                        const bool top = r >= rb;
                        const int ql = rlo.cls == ROW_CROSS ? (top ? e0 + nbot + __popc(mtop & ((1u << r) - 1u))
                                                                   : e0 + __popc(mbot & ((1u << r) - 1u))) : -1;
                        const int qh = rhi.cls == ROW_CROSS ? (top ? e0 + nbot + __popc(mtop & ((1u << (r + 1)) - 1u))
                                                                   : e0 + __popc(mbot & ((1u << (r + 1)) - 1u))) : -1;
                        const float lp0 = top ? rlo.pt0 : rlo.p0, lp1 = top ? -rlo.p1 : rlo.p1;
                        const float hp0 = top ? rhi.pt0 : rhi.p0, hp1 = top ? -rhi.p1 : rhi.p1;
                        const float fz = top ? -zs : zs;
#pragma unroll 1
                        for (int c = 0; c < ncol; ++c) {
                            const float4 f = ws->fa[c];
                            const float fb = ws->fb[c];
                            float gvl, gql, gvh, gqh;
                            if (ql >= 0) { gvl = ws->res_v[ql][c]; gql = ws->res_q[ql][c]; }
                            else g_lin(az, lp0, lp1, fz, f.x, f.y, f.z, f.w, fb, gvl, gql);
                            if (qh >= 0) { gvh = ws->res_v[qh][c]; gqh = ws->res_q[qh][c]; }
                            else g_lin(az, hp0, hp1, fz, f.x, f.y, f.z, f.w, fb, gvh, gqh);
                            const float pv = top ? gvl - gvh : gvh - gvl;
                            const float pq = top ? gql - gqh : gqh - gql;
                            if (pv > vtiny) sink.pair(pass, cstart + c, m, pair_weight(pv, pq, D2));
                        }
                    }
                    rlo = rhi;
                }
                sink.end(pass, k);
            }
            __syncwarp();
            lo_lane = hi_lane;
        }
    }
}

// Relaxed pairs: W = A_n d / |D|^2 with d the x_3 length of row m along the vertical line
// through the centre of mass of H_n (Sec. III-A, Eq. cutvolume). fa[c] = (A_n, t'_CM, ., .).
template <class Sink>
__device__ __forceinline__ void relaxed_voxels(const View& V, const Grid& G, const Column& C, int cstart, int ncol,
                                               int kbase, int lane, WarpSmem* ws, Sink& sink, int* err) {
    const float az = G.az;
    const float atiny = 1e-9f * G.ax * G.ay;
    const float dp0 = C.tc * V.inv_agv, dp1 = V.inv_agv;
    for (int pass = 0; pass < KPL; ++pass) {
        const int k = kbase + pass * 32 + lane;
        Slice S;
        bool act = (k < G.nz) && slice_setup(V, G, C, k, S);
        if (act && S.m_last - S.m_first + 2 > KCT_ROWS) { atomicOr(err, 1); act = false; }
        if (!act) continue;
        sink.begin(pass, k);
        const float iD2 = 1.0f / fmaf(C.tc, C.tc, fmaf(C.xc, C.xc, S.zc * S.zc));
        const int R = S.m_last - S.m_first + 1;
        const int rb = (R + 1) >> 1;
        RowPlane rlo = row_boundary(V, G, C, S, (float)S.m_first - 0.5f);
        for (int r = 0; r < R; ++r) {
            const int m = S.m_first + r;
            const RowPlane rhi = row_boundary(V, G, C, S, (float)m + 0.5f);
            const bool top = r >= rb;
#pragma unroll 1
            for (int c = 0; c < ncol; ++c) {
                const float4 f = ws->fa[c];
                const float A = f.x, T = f.y;
                const float hl = fmaf(rlo.p1, T, rlo.p0), hh = fmaf(rhi.p1, T, rhi.p0);
                float d;
                if (hl > 0.f && hl < az && hh > 0.f && hh < az) d = fmaf(dp1, T, dp0);
                else if (top) d = fminf(fmaxf(fmaf(-rlo.p1, T, rlo.pt0), 0.f), az) -
                                  fminf(fmaxf(fmaf(-rhi.p1, T, rhi.pt0), 0.f), az);
                else d = fminf(fmaxf(hh, 0.f), az) - fminf(fmaxf(hl, 0.f), az);
                if (A > atiny && d > 0.f) sink.pair(pass, cstart + c, m, A * d * iD2);
            }
            rlo = rhi;
        }
        sink.end(pass, k);
    }
}

// All pairs of voxels kbase .. kbase + SEG - 1 of column (i, j) in view V (in shared memory).
// Called by all 32 lanes of a warp with the same arguments.
template <int VARIANT, class Sink>
__device__ __forceinline__ void warp_column(const View& V, const Grid& G, int i, int j, int kbase, int lane,
                                            WarpSmem* ws, Sink& sink, int* err) {
    Column C;
    if (!column_setup(V, G, i, j, C)) return;
    if (C.n_last - C.n_first + 2 > KCT_MAX_SPAN) {
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    __syncwarp();                  // the previous column's readers of ws are done
    if (lane == 0) ws->C = C;
    for (int cstart = C.n_first; cstart <= C.n_last; cstart += KCT_CB) {
        const int ncol = min(KCT_CB, C.n_last - cstart + 1);
        __syncwarp();
        if (lane < ncol) {
            const Mom f = cut_moments_call(&V, &ws->C, cstart + lane, 3.0e38f);
            if (VARIANT == 1) ws->fa[lane] = make_float4(f.m1, f.m1 > 0.f ? f.mt / f.m1 : 0.f, 0.f, 0.f);
            else {
                ws->fa[lane] = make_float4(f.m1, f.mt, f.mtt, f.ml);
                ws->fb[lane] = f.mlt;
            }
        }
        __syncwarp();
        if (VARIANT == 1) relaxed_voxels(V, G, C, cstart, ncol, kbase, lane, ws, sink, err);
        else exact_voxels(V, G, C, cstart, ncol, kbase, lane, ws, sink, err);
    }
}

// Detector window covered by the brick [i0, i0+BX) x [j0, j0+BY) x [k0, k0+SEG) in view V:
// the bounding box of the projected corners (u does not depend on x_3), one pixel of margin.
__device__ __forceinline__ Tile brick_tile(const View& V, const Grid& G, int i0, int j0, int k0) {
    const float xs[2] = {G.x0 + (i0 - 0.5f) * G.ax, G.x0 + (min(i0 + BX, G.nx) - 0.5f) * G.ax};
    const float ys[2] = {G.y0 + (j0 - 0.5f) * G.ay, G.y0 + (min(j0 + BY, G.ny) - 0.5f) * G.ay};
    const float zs[2] = {G.z0 + (k0 - 0.5f) * G.az - V.sz, G.z0 + (min(k0 + SEG, G.nz) - 0.5f) * G.az - V.sz};
    float umin = 3e38f, umax = -3e38f, vmin = 3e38f, vmax = -3e38f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float x = xs[c & 1], y = ys[c >> 1];
        const float t = fmaf(V.wx, x, fmaf(V.wy, y, V.aw));
        const float xi = fmaf(-V.wy, x, fmaf(V.wx, y, V.ah));
        const float u = fmaf(V.gu, xi / t, V.cu);
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float v = fmaf(V.gv, zs[h] / t, V.cv);
            vmin = fminf(vmin, v);
            vmax = fmaxf(vmax, v);
        }
    }
    Tile T;
    T.u0 = max((int)floorf(umin + 0.5f) - 1, 0);
    T.v0 = max((int)floorf(vmin + 0.5f) - 1, 0);
    const int u1 = min((int)floorf(umax + 0.5f) + 1, G.nu - 1);
    const int v1 = min((int)floorf(vmax + 0.5f) + 1, G.nv - 1);
    T.w = u1 - T.u0 + 1;
    T.h = v1 - T.v0 + 1;
    if (T.w <= 0 || T.h <= 0) T.w = T.h = 0;
    T.ok = (T.w > 0 && (long)T.w * T.h <= TILE_CAP) ? 1 : 0;
    return T;
}

// ---------------------------------------------------------------------------------------
// Sinks
// ---------------------------------------------------------------------------------------

struct FwdSink {      // tile[m][n] += mu * W  (unscaled sums of Eq. cvpsu)
    const float* mu_s;             // brick attenuation values, [SEG][BY][BX] in shared memory
    float* tile;
    Tile T;
    float* __restrict__ Sg;        // global sums of the view (used where the tile does not reach)
    int nu, col, kbase;
    float mu;
    __device__ __forceinline__ void begin(int, int k) { mu = mu_s[(k - kbase) * NCOLS + col]; }
    __device__ __forceinline__ void end(int, int) {}
    __device__ __forceinline__ void pair(int, int n, int m, float W) {
        if (mu == 0.f) return;
        const int du = n - T.u0, dv = m - T.v0;
        if (T.ok && (unsigned)du < (unsigned)T.w && (unsigned)dv < (unsigned)T.h) atomicAdd(&tile[dv * T.w + du], mu * W);
        else atomicAdd(&Sg[(size_t)m * nu + n], mu * W);
    }
};

struct BwdSink {      // acc += W * (F y)[m][n]
    const float* tile;
    Tile T;
    const float* __restrict__ yg;
    int nu;
    float acc[KPL];
    __device__ __forceinline__ void begin(int, int) {}
    __device__ __forceinline__ void end(int, int) {}
    __device__ __forceinline__ void pair(int p, int n, int m, float W) {
        const int du = n - T.u0, dv = m - T.v0;
        const float y = (T.ok && (unsigned)du < (unsigned)T.w && (unsigned)dv < (unsigned)T.h)
                            ? tile[dv * T.w + du] : __ldg(&yg[(size_t)m * nu + n]);
#pragma unroll
        for (int q = 0; q < KPL; ++q)
            if (q == p) acc[q] = fmaf(W, y, acc[q]);
    }
};

struct CountSink {
    unsigned long long n;
    __device__ __forceinline__ void begin(int, int) {}
    __device__ __forceinline__ void end(int, int) {}
    __device__ __forceinline__ void pair(int, int, int, float W) { n += (W > 0.f) ? 1ull : 0ull; }
};

__device__ __forceinline__ void brick_origin(const Grid& G, int& i0, int& j0) {
    const int nbx = (G.nx + BX - 1) / BX;
    i0 = (blockIdx.x % nbx) * BX;
    j0 = (blockIdx.x / nbx) * BY;
}

// ---------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------

// grid: (bricks in x1 x2, segments along x3, view chunks); S receives the unscaled sums.
// Dynamic shared memory: SEG * NCOLS + TILE_CAP floats.
template <int VARIANT>
__global__ void __launch_bounds__(NTHREADS, 2) fwd_kernel(const View* __restrict__ views, Grid G,
                                                          const float* __restrict__ vol, float* __restrict__ S,
                                                          int* err) {
    extern __shared__ float dyn[];
    __shared__ BlockSmem bs;
    float* mu_s = dyn;
    float* tile = dyn + SEG * NCOLS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, j0;
    brick_origin(G, i0, j0);
    const int kbase = blockIdx.y * SEG;
    for (int q = threadIdx.x; q < SEG * NCOLS; q += NTHREADS) {
        const int kk = q / NCOLS, c = q % NCOLS;
        const int i = i0 + c % BX, j = j0 + c / BX, k = kbase + kk;
        mu_s[q] = (i < G.nx && j < G.ny && k < G.nz) ? __ldg(&vol[((size_t)k * G.ny + j) * G.nx + i]) : 0.f;
    }
    const int v_end = min((int)(blockIdx.z + 1) * VIEW_CHUNK, G.nviews);
    for (int view = blockIdx.z * VIEW_CHUNK; view < v_end; ++view) {
        __syncthreads();
        if (threadIdx.x == 0) {
            bs.V = views[view];
            bs.T = brick_tile(bs.V, G, i0, j0, kbase);
        }
        __syncthreads();
        const Tile T = bs.T;
        if (T.ok)
            for (int q = threadIdx.x; q < T.w * T.h; q += NTHREADS) tile[q] = 0.f;
        __syncthreads();
        float* Sv = S + (size_t)view * G.nu * G.nv;
        for (int c = warp; c < NCOLS; c += NWARP) {
            const int i = i0 + c % BX, j = j0 + c / BX;
            if (i >= G.nx || j >= G.ny) continue;
            FwdSink s{mu_s, tile, T, Sv, G.nu, c, kbase, 0.f};
            warp_column<VARIANT>(bs.V, G, i, j, kbase, lane, &bs.ws[warp], s, err);
        }
        __syncthreads();
        if (T.ok)
            for (int q = threadIdx.x; q < T.w * T.h; q += NTHREADS) {
                const float v = tile[q];
                if (v != 0.f) atomicAdd(&Sv[(size_t)(T.v0 + q / T.w) * G.nu + T.u0 + q % T.w], v);
            }
    }
}

// grid: (bricks in x1 x2, segments along x3); every block loops over all views.
// Dynamic shared memory: SEG * NCOLS + TILE_CAP floats.
template <int VARIANT>
__global__ void __launch_bounds__(NTHREADS, 2) bwd_kernel(const View* __restrict__ views, Grid G,
                                                          const float* __restrict__ yF, float* __restrict__ vol,
                                                          int accumulate, int* err) {
    extern __shared__ float dyn[];
    __shared__ BlockSmem bs;
    float* acc_s = dyn;                 // [NCOLS][SEG]
    float* tile = dyn + SEG * NCOLS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, j0;
    brick_origin(G, i0, j0);
    const int kbase = blockIdx.y * SEG;
    for (int q = threadIdx.x; q < SEG * NCOLS; q += NTHREADS) acc_s[q] = 0.f;
    for (int view = 0; view < G.nviews; ++view) {
        __syncthreads();
        if (threadIdx.x == 0) {
            bs.V = views[view];
            bs.T = brick_tile(bs.V, G, i0, j0, kbase);
        }
        __syncthreads();
        const Tile T = bs.T;
        const float* yv = yF + (size_t)view * G.nu * G.nv;
        if (T.ok)
            for (int q = threadIdx.x; q < T.w * T.h; q += NTHREADS)
                tile[q] = __ldg(&yv[(size_t)(T.v0 + q / T.w) * G.nu + T.u0 + q % T.w]);
        __syncthreads();
        for (int c = warp; c < NCOLS; c += NWARP) {
            const int i = i0 + c % BX, j = j0 + c / BX;
            if (i >= G.nx || j >= G.ny) continue;
            BwdSink s{tile, T, yv, G.nu, {}};
#pragma unroll
            for (int p = 0; p < KPL; ++p) s.acc[p] = 0.f;
            warp_column<VARIANT>(bs.V, G, i, j, kbase, lane, &bs.ws[warp], s, err);
#pragma unroll
            for (int p = 0; p < KPL; ++p) acc_s[c * SEG + p * 32 + lane] += s.acc[p];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SEG * NCOLS; q += NTHREADS) {
        const int c = q / SEG, kk = q % SEG;
        const int i = i0 + c % BX, j = j0 + c / BX, k = kbase + kk;
        if (i < G.nx && j < G.ny && k < G.nz) {
            const size_t idx = ((size_t)k * G.ny + j) * G.nx + i;
            vol[idx] = accumulate ? vol[idx] + acc_s[q] : acc_s[q];
        }
    }
}

// grid: (bricks, segments, views)
template <int VARIANT>
__global__ void __launch_bounds__(NTHREADS, 2) count_kernel(const View* __restrict__ views, Grid G,
                                                            unsigned long long* count, int* err) {
    __shared__ BlockSmem bs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, j0;
    brick_origin(G, i0, j0);
    const int kbase = blockIdx.y * SEG;
    if (threadIdx.x == 0) bs.V = views[blockIdx.z];
    __syncthreads();
    CountSink s{0ull};
    for (int c = warp; c < NCOLS; c += NWARP) {
        const int i = i0 + c % BX, j = j0 + c / BX;
        if (i >= G.nx || j >= G.ny) continue;
        warp_column<VARIANT>(bs.V, G, i, j, kbase, lane, &bs.ws[warp], s, err);
    }
    unsigned long long v = s.n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
    if (lane == 0 && v) atomicAdd(count, v);
}

// out[view][m][n] = F(n, m) * in[view][m][n] (+ out when accumulate); grid (pixels, views)
template <int SCALING>
__global__ void scale_kernel(const View* __restrict__ views, Grid G, const float* __restrict__ in,
                             float* __restrict__ out, int accumulate) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)G.nu * G.nv) return;
    const View V = views[blockIdx.y];
    const int n = (int)(q % G.nu), m = (int)(q / G.nu);
    const size_t idx = (size_t)blockIdx.y * G.nu * G.nv + q;
    const float v = pixel_factor<SCALING>(V, n, m) * in[idx];
    out[idx] = accumulate ? out[idx] + v : v;
}

template <int SCALING>
__global__ void factor_kernel(const View* __restrict__ views, Grid G, float* __restrict__ out) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)G.nu * G.nv) return;
    const View V = views[blockIdx.y];
    const int n = (int)(q % G.nu), m = (int)(q / G.nu);
    out[(size_t)blockIdx.y * G.nu * G.nv + q] = pixel_factor<SCALING>(V, n, m);
}

}  // namespace kct
