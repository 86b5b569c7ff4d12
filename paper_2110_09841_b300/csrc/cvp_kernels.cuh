// cvp_kernels.cuh -- warp-cooperative CUDA kernels of the cutting voxel projector (sm_103a).
//
// Work unit: one warp, one voxel column (i, j) of the volume, SEG = 32 * KPL consecutive
// voxels along x_3 (lane l owns voxels kbase + l + 32 p, p < KPL), one view.
//  * The column cuts H_n of the voxel base are the same for every voxel of the column
//    (Sec. III-A, Eq. columnprojectionidentity), so they are computed once per warp: lane c
//    clips the base to detector column n = cstart + c and the warp shares the moments of
//    H_n with shuffles.
//  * Each lane then walks the rows of its own voxel. A row whose two planes stay inside the
//    voxel over the whole base gives its pairs in closed form from the moments of H_n; a
//    plane that leaves the voxel through its top or bottom face ("crossing") needs the
//    moments of H_n cut at a depth tau. Crossing planes are queued per warp and evaluated
//    by all 32 lanes together, one (event, column) task per lane, so the clipping never
//    runs with most of the warp idle.
// Forward projection and adjoint enumerate the same pairs with the same code, so
// <A x, y> = <x, A^T y> holds to float rounding.
#pragma once

#include "cvp_device.cuh"

namespace kct {

constexpr int KPL = 2;             // voxels per lane in a column segment
constexpr int SEG = 32 * KPL;      // voxels per warp segment
constexpr int EV_CAP = 64;         // crossing events queued per warp and round
constexpr int KCT_ROWS = 32;       // row boundaries of one voxel (its footprint spans <= 31 rows)
constexpr int WARPS = 4;           // warps per block (a 2 x 2 patch of columns)
constexpr unsigned FULLMASK = 0xffffffffu;

struct WarpSmem {
    float fm[5][KCT_CB];           // moments of H_n: m1, mt, mtt, ml, mlt
    float ev_p0[EV_CAP], ev_p1[EV_CAP], ev_zs[EV_CAP];
    float res_v[EV_CAP][KCT_CB];
    float res_q[EV_CAP][KCT_CB];
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

KCT_HD RowPlane row_boundary(const View& V, const Grid& G, const Column& C, const Slice& S,
                                                 float Vb) {
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

// Volume and first moment along D of {(t', xi') in H_n, 0 < height < clamp(p0 + p1 t', 0, az)}
// (height from the frame's face; zs = zeta_c * sign(gv), negated in the top frame),
// for a plane that leaves the voxel through a face: h = 0 at tau0, h = az at tau1.
KCT_HD void g_cross(const View& V, const Grid& G, const Column& C, const Line& lo, const Line& hi,
                                        const Mom& full, float p0, float p1, float zs, float& gv, float& gq) {
    const float az = G.az;
    const float p1s = (fabsf(p1) < 1e-30f) ? copysignf(1e-30f, p1) : p1;
    const float tau0 = -p0 / p1s, tau1 = (az - p0) / p1s;
    const Mom c0 = cut_moments(V, C, lo, hi, full, tau0);
    const Mom c1 = cut_moments(V, C, lo, hi, full, tau1);
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
KCT_HD void g_lin(float az, float p0, float p1, float zs, float f1, float ft, float ftt, float fl,
                                      float flt, float& gv, float& gq) {
    const float Vg = fmaf(p0, f1, p1 * ft);
    const float Sl = fmaf(p0, fl, p1 * flt);
    const float Sh2 = fmaf(p0 * p0, f1, fmaf(2.f * p0 * p1, ft, p1 * p1 * ftt));
    gv = Vg;
    gq = fmaf(zs, fmaf(0.5f, Sh2, -0.5f * az * Vg), Sl);
}

// Near-exact pairs of one column segment. Columns n = cstart .. cstart + ncol - 1.
// Each pair (n, m) is the integral over the column cut H_n of the height between the two
// row planes of row m. When both planes stay inside the voxel this height is linear in t'
// and the pair follows directly from the moments of H_n. Otherwise it is the difference of
// the cut below the upper plane and the cut below the lower one, both measured from the
// nearer face (bottom frame for the lower half of the voxel's rows, top frame for the upper
// half), so that no pair is a small difference of two near-full voxel volumes.
template <class Sink>
__device__ __forceinline__ void exact_segment(const View& V, const Grid& G, const Column& C, int cstart, int ncol,
                                              int kbase, int lane, WarpSmem* ws, Sink& sink, int* err) {
    const float az = G.az;
    Mom my = Mom{0.f, 0.f, 0.f, 0.f, 0.f};
    if (lane < ncol) {
        Line lo, hi;
        column_lines(V, C, cstart + lane, lo, hi);
        my = normalise(region3<true>(V, lo, hi, line_none()), C.tc, C.xc);
    }
    if (lane < KCT_CB) {
        ws->fm[0][lane] = my.m1;
        ws->fm[1][lane] = my.mt;
        ws->fm[2][lane] = my.mtt;
        ws->fm[3][lane] = my.ml;
        ws->fm[4][lane] = my.mlt;
    }
    float f1[KCT_CB], ft[KCT_CB], ftt[KCT_CB], fl[KCT_CB], flt[KCT_CB];
#pragma unroll
    for (int c = 0; c < KCT_CB; ++c) {
        f1[c] = __shfl_sync(FULLMASK, my.m1, c);
        ft[c] = __shfl_sync(FULLMASK, my.mt, c);
        ftt[c] = __shfl_sync(FULLMASK, my.mtt, c);
        fl[c] = __shfl_sync(FULLMASK, my.ml, c);
        flt[c] = __shfl_sync(FULLMASK, my.mlt, c);
    }
    __syncwarp();
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
        if (act)
            for (int b = 0; b <= R; ++b)
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
            // 1) queue the group's crossing boundaries (frame-transformed plane parameters)
            if (mine && nev) {
                int e = e0;
                for (int b = 0; b <= R; ++b) {
                    if (!((cross >> b) & 1u)) continue;
                    const RowPlane rp = row_boundary(V, G, C, S, (float)(S.m_first + b) - 0.5f);
                    if (b <= rb) {
                        ws->ev_p0[e + __popc(mbot & ((1u << b) - 1u))] = rp.p0;
                        ws->ev_p1[e + __popc(mbot & ((1u << b) - 1u))] = rp.p1;
                        ws->ev_zs[e + __popc(mbot & ((1u << b) - 1u))] = zs;
                    }
                    if (b >= rb) {
                        const int q = e + nbot + __popc(mtop & ((1u << b) - 1u));
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
                Line lo, hi;
                column_lines(V, C, cstart + c, lo, hi);
                const Mom full = Mom{ws->fm[0][c], ws->fm[1][c], ws->fm[2][c], ws->fm[3][c], ws->fm[4][c]};
                float gv, gq;
                g_cross(V, G, C, lo, hi, full, ws->ev_p0[e], ws->ev_p1[e], ws->ev_zs[e], gv, gq);
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
                    float pv[KCT_CB], pq[KCT_CB];
                    if (rlo.cls == ROW_LIN && rhi.cls == ROW_LIN) {
                        // height between the planes: dp0 + dp1 t', centred at s0 + s1 t'
                        const float s0 = C.tc * (-fmaf(V.gv, S.bc, V.cv - (float)m)) * V.inv_agv;
                        const float s1 = ((float)m - V.cv) * V.inv_agv;
                        const float a0 = zs * dp0 * s0, a1 = zs * fmaf(dp0, s1, dp1 * s0), a2 = zs * dp1 * s1;
#pragma unroll
                        for (int c = 0; c < KCT_CB; ++c) {
                            pv[c] = fmaf(dp0, f1[c], dp1 * ft[c]);
                            pq[c] = fmaf(dp0, fl[c], fmaf(dp1, flt[c], fmaf(a0, f1[c], fmaf(a1, ft[c], a2 * ftt[c]))));
                        }
                    } else {
                        const bool top = r >= rb;
                        const int bl = r, bh = r + 1;
#pragma unroll
                        for (int c = 0; c < KCT_CB; ++c) {
                            float gvl, gql, gvh, gqh;
                            // lower plane
                            if (rlo.cls == ROW_CROSS) {
                                const int q = top ? e0 + nbot + __popc(mtop & ((1u << bl) - 1u))
                                                  : e0 + __popc(mbot & ((1u << bl) - 1u));
                                gvl = ws->res_v[q][c];
                                gql = ws->res_q[q][c];
                            } else if (top) {
                                g_lin(az, rlo.pt0, -rlo.p1, -zs, f1[c], ft[c], ftt[c], fl[c], flt[c], gvl, gql);
                            } else {
                                g_lin(az, rlo.p0, rlo.p1, zs, f1[c], ft[c], ftt[c], fl[c], flt[c], gvl, gql);
                            }
                            // upper plane
                            if (rhi.cls == ROW_CROSS) {
                                const int q = top ? e0 + nbot + __popc(mtop & ((1u << bh) - 1u))
                                                  : e0 + __popc(mbot & ((1u << bh) - 1u));
                                gvh = ws->res_v[q][c];
                                gqh = ws->res_q[q][c];
                            } else if (top) {
                                g_lin(az, rhi.pt0, -rhi.p1, -zs, f1[c], ft[c], ftt[c], fl[c], flt[c], gvh, gqh);
                            } else {
                                g_lin(az, rhi.p0, rhi.p1, zs, f1[c], ft[c], ftt[c], fl[c], flt[c], gvh, gqh);
                            }
                            pv[c] = top ? gvl - gvh : gvh - gvl;
                            pq[c] = top ? gql - gqh : gqh - gql;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < KCT_CB; ++c)
                        if (c < ncol && pv[c] > vtiny) sink.pair(pass, cstart + c, m, pv[c] * pv[c] / fmaf(pv[c], D2, 2.f * pq[c]));
                    rlo = rhi;
                }
            }
            __syncwarp();
            lo_lane = hi_lane;
        }
    }
}

// Relaxed pairs: W = A_n d / |D|^2 with d the x_3 length of row m along the vertical line
// through the centre of mass of H_n (Sec. III-A, Eq. cutvolume).
template <class Sink>
__device__ __forceinline__ void relaxed_segment(const View& V, const Grid& G, const Column& C, int cstart, int ncol,
                                                int kbase, int lane, Sink& sink, int* err) {
    const float az = G.az;
    float A = 0.f, T = 0.f;       // area and centre-of-mass depth of H_n, n = cstart + lane
    if (lane < ncol) {
        Line lo, hi;
        column_lines(V, C, cstart + lane, lo, hi);
        Mom5 g = region3<false>(V, lo, hi, line_none());
        A = 0.5f * g.a;
        T = (A > 0.f) ? g.t * (1.f / 6.f) / A : 0.f;
    }
    float An[KCT_CB], Tn[KCT_CB];
#pragma unroll
    for (int c = 0; c < KCT_CB; ++c) {
        An[c] = __shfl_sync(FULLMASK, A, c);
        Tn[c] = __shfl_sync(FULLMASK, T, c);
    }
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
#pragma unroll
            for (int c = 0; c < KCT_CB; ++c) {
                const float hl = fmaf(rlo.p1, Tn[c], rlo.p0), hh = fmaf(rhi.p1, Tn[c], rhi.p0);
                float d;
                if (hl > 0.f && hl < az && hh > 0.f && hh < az) d = fmaf(dp1, Tn[c], dp0);
                else if (top) d = fminf(fmaxf(fmaf(-rlo.p1, Tn[c], rlo.pt0), 0.f), az) -
                                  fminf(fmaxf(fmaf(-rhi.p1, Tn[c], rhi.pt0), 0.f), az);
                else d = fminf(fmaxf(hh, 0.f), az) - fminf(fmaxf(hl, 0.f), az);
                if (c < ncol && An[c] > atiny && d > 0.f) sink.pair(pass, cstart + c, m, An[c] * d * iD2);
            }
            rlo = rhi;
        }
    }
}

// All pairs of one column segment in one view. Called by all 32 lanes of a warp with the
// same (i, j, kbase, view).
template <int VARIANT, class Sink>
__device__ __forceinline__ void warp_column(const View& V, const Grid& G, int i, int j, int kbase, int lane,
                                            WarpSmem* ws, Sink& sink, int* err) {
    Column C;
    if (!column_setup(V, G, i, j, C)) return;
    if (C.n_last - C.n_first + 2 > KCT_MAX_SPAN) {
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    for (int cstart = C.n_first; cstart <= C.n_last; cstart += KCT_CB) {
        const int ncol = min(KCT_CB, C.n_last - cstart + 1);
        if (VARIANT == 1) relaxed_segment(V, G, C, cstart, ncol, kbase, lane, sink, err);
        else exact_segment(V, G, C, cstart, ncol, kbase, lane, ws, sink, err);
    }
}

// block -> 2 x 2 patch of columns, warp -> one column
__device__ __forceinline__ bool warp_column_index(const Grid& G, int bx, int warp, int& i, int& j) {
    const int px = (G.nx + 1) >> 1;
    i = 2 * (bx % px) + (warp & 1);
    j = 2 * (bx / px) + (warp >> 1);
    return i < G.nx && j < G.ny;
}

// ---------------------------------------------------------------------------------------
// Sinks
// ---------------------------------------------------------------------------------------

struct FwdSink {      // S[m][n] += mu * W  (unscaled sums of Eq. cvpsu)
    const float* __restrict__ vol;
    float* __restrict__ S;
    int nx, ny, nu, i, j;
    float mu;
    __device__ __forceinline__ void begin(int, int k) { mu = __ldg(&vol[((size_t)k * ny + j) * nx + i]); }
    __device__ __forceinline__ void pair(int, int n, int m, float W) {
        if (mu != 0.f) atomicAdd(&S[(size_t)m * nu + n], mu * W);
    }
};

struct BwdSink {      // acc[p] += W * (F y)[m][n]
    const float* __restrict__ yF;
    int nu;
    float acc[KPL];
    __device__ __forceinline__ void begin(int, int) {}
    __device__ __forceinline__ void pair(int p, int n, int m, float W) {
        float y = __ldg(&yF[(size_t)m * nu + n]);
#pragma unroll
        for (int q = 0; q < KPL; ++q)
            if (q == p) acc[q] = fmaf(W, y, acc[q]);
    }
};

struct CountSink {
    unsigned long long n;
    __device__ __forceinline__ void begin(int, int) {}
    __device__ __forceinline__ void pair(int, int, int, float W) { n += (W > 0.f) ? 1ull : 0ull; }
};

// ---------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------

// grid: (column patches, views, segments); S receives the unscaled sums
template <int VARIANT>
__global__ void __launch_bounds__(32 * WARPS) fwd_kernel(const View* __restrict__ views, Grid G,
                                                         const float* __restrict__ vol, float* __restrict__ S,
                                                         int* err) {
    __shared__ WarpSmem wsm[WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i, j;
    if (!warp_column_index(G, blockIdx.x, warp, i, j)) return;
    const View V = views[blockIdx.y];
    FwdSink s{vol, S + (size_t)blockIdx.y * G.nu * G.nv, G.nx, G.ny, G.nu, i, j, 0.f};
    warp_column<VARIANT>(V, G, i, j, blockIdx.z * SEG, lane, &wsm[warp], s, err);
}

// grid: (column patches, segments); every warp loops over all views
template <int VARIANT>
__global__ void __launch_bounds__(32 * WARPS) bwd_kernel(const View* __restrict__ views, Grid G,
                                                         const float* __restrict__ yF, float* __restrict__ vol,
                                                         int accumulate, int* err) {
    __shared__ WarpSmem wsm[WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i, j;
    if (!warp_column_index(G, blockIdx.x, warp, i, j)) return;
    const int kbase = blockIdx.y * SEG;
    BwdSink s{nullptr, G.nu, {}};
#pragma unroll
    for (int q = 0; q < KPL; ++q) s.acc[q] = 0.f;
    for (int view = 0; view < G.nviews; ++view) {
        const View V = views[view];
        s.yF = yF + (size_t)view * G.nu * G.nv;
        warp_column<VARIANT>(V, G, i, j, kbase, lane, &wsm[warp], s, err);
    }
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const int k = kbase + q * 32 + lane;
        if (k < G.nz) {
            const size_t idx = ((size_t)k * G.ny + j) * G.nx + i;
            vol[idx] = accumulate ? vol[idx] + s.acc[q] : s.acc[q];
        }
    }
}

template <int VARIANT>
__global__ void __launch_bounds__(32 * WARPS) count_kernel(const View* __restrict__ views, Grid G,
                                                           unsigned long long* count, int* err) {
    __shared__ WarpSmem wsm[WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i, j;
    if (!warp_column_index(G, blockIdx.x, warp, i, j)) return;
    CountSink s{0ull};
    warp_column<VARIANT>(views[blockIdx.y], G, i, j, blockIdx.z * SEG, lane, &wsm[warp], s, err);
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
