// cvp_kernels.cuh -- warp-cooperative CUDA kernels of the cutting voxel projector (sm_103a).
//
// Work unit: one warp, one voxel column (i, j) of the volume, SEG = 32 * KPL consecutive
// voxels along x_3 (lane l owns voxels kbase + l + 32 p, p < KPL), one view.
//  * The column cuts of the voxel base are the same for every voxel of the column (Sec.
//    III-A, Eq. columnprojectionidentity), so they are computed once per warp: lane c
//    computes the polygon P_c = base ∩ {u < U_c} of column boundary c and the warp shares
//    its moments with shuffles.
//  * Each lane then walks the row boundaries of its own voxel. A row plane whose height
//    stays inside the voxel over the whole base gives the cumulative cut in closed form
//    from the polygon moments; a plane that leaves the voxel through its top or bottom
//    face ("crossing") needs the moments of P_c cut at a depth tau. Crossing boundaries
//    are queued per warp and evaluated by all 32 lanes together, one (event, column
//    boundary) task per lane, so the clipping never runs with most of the warp idle.
// Forward projection and adjoint enumerate the same pairs with the same code, so
// <A x, y> = <x, A^T y> holds to float rounding.
#pragma once

#include "cvp_device.cuh"

namespace kct {

constexpr int KPL = 2;             // voxels per lane in a column segment
constexpr int SEG = 32 * KPL;      // voxels per warp segment
constexpr int EV_CAP = 64;         // crossing boundaries queued per warp and round
constexpr int KCT_ROWS = 32;       // row boundaries of one voxel (its footprint spans <= 31 rows)
constexpr int WARPS = 4;           // warps per block (a 2 x 2 patch of columns)
constexpr unsigned FULLMASK = 0xffffffffu;

struct WarpSmem {
    float fm[5][KCT_CB];           // moments of P_c: m1, mt, mtt, ml, mlt
    float ev_p0[EV_CAP], ev_p1[EV_CAP], ev_zs[EV_CAP];
    float res_v[EV_CAP][KCT_CB];
    float res_q[EV_CAP][KCT_CB];
};

__device__ __forceinline__ int boundary_kind(float U, const Column& C) {
    return (U <= C.umin) ? KIND_EMPTY : ((U >= C.umax) ? KIND_FULL : KIND_GEN);
}

// Cumulative cut G(U_c, V_b) = (volume, first moment along D) for a crossing boundary:
// h(t') = clamp(p0 + p1 t', 0, az) changes form at tau0 (h = 0) and tau1 (h = az).
__device__ __forceinline__ void g_cross(const View& V, const Grid& G, const Column& C, int kind, float l1t,
                                        float l1c, const Mom& full, float p0, float p1, float zs,
                                        float& gv, float& gq) {
    const float az = G.az;
    if (kind == KIND_EMPTY) { gv = 0.f; gq = 0.f; return; }
    float p1s = (fabsf(p1) < 1e-30f) ? copysignf(1e-30f, p1) : p1;
    float tau0 = -p0 / p1s, tau1 = (az - p0) / p1s;
    Mom c0 = cpm(V, C, kind, l1t, l1c, full, tau0);
    Mom c1 = cpm(V, C, kind, l1t, l1c, full, tau1);
    Mom lin, fu;
    if (p1s > 0.f) { lin = mom_sub(c1, c0); fu = mom_sub(full, c1); }
    else { lin = mom_sub(c0, c1); fu = c1; }
    float Vg = fmaf(p0, lin.m1, fmaf(p1, lin.mt, az * fu.m1));
    float Sl = fmaf(p0, lin.ml, fmaf(p1, lin.mlt, az * fu.ml));
    float Sh2 = fmaf(p0 * p0, lin.m1, fmaf(2.f * p0 * p1, lin.mt, fmaf(p1 * p1, lin.mtt, az * az * fu.m1)));
    gv = Vg;
    gq = fmaf(zs, fmaf(0.5f, Sh2, -0.5f * az * Vg), Sl);
}

// Row-boundary classes of the exact variant
enum { ROW_ZERO = 0, ROW_FULL = 1, ROW_LIN = 2, ROW_CROSS = 3 };

__device__ __forceinline__ int classify_row(const View& V, const Grid& G, const Column& C, const Slice& S,
                                            float Vb, float& p0, float& p1) {
    if (Vb <= S.vmin) return ROW_ZERO;
    if (Vb >= S.vmax) return ROW_FULL;
    row_plane(V, G, C, S, Vb, p0, p1);
    // does the plane leave the voxel through a horizontal face inside the base's depth range?
    float h_lo = fmaf(p1, V.tmin_sq, p0), h_hi = fmaf(p1, V.tmax_sq, p0);
    float hmin = fminf(h_lo, h_hi), hmax = fmaxf(h_lo, h_hi);
    return (hmin < 0.f || hmax > G.az) ? ROW_CROSS : ROW_LIN;
}

template <class Sink>
__device__ __forceinline__ void exact_segment(const View& V, const Grid& G, const Column& C, int cstart, int nb,
                                              int kbase, int lane, WarpSmem* ws, Sink& sink, int* err) {
    const float az = G.az;
    // moments of P_c for this lane's boundary c = lane, then shared
    Mom my = Mom{0.f, 0.f, 0.f, 0.f, 0.f};
    if (lane < nb) {
        float U = (float)(cstart + lane) - 0.5f;
        int kind = boundary_kind(U, C);
        if (kind == KIND_FULL) {
            my.m1 = G.ax * G.ay;
            my.mtt = V.sq_tt * (1.f / 12.f);
            my.mlt = fmaf(C.tc, my.mtt, C.xc * (V.sq_tx * (1.f / 24.f)));
        } else if (kind == KIND_GEN) {
            float l1t = (V.cu - U) * C.itc;
            float l1c = -fmaf(V.gu, C.alc, V.cu - U);
            my = normalise(region<true, false, true>(V, l1t, C.gxi, l1c, 0.f), C.tc, C.xc);
        }
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

    for (int pass = 0; pass < KPL; ++pass) {
        const int k = kbase + pass * 32 + lane;
        Slice S;
        bool act = (k < G.nz) && slice_setup(V, G, C, k, S);
        if (act && S.m_last - S.m_first + 2 > KCT_ROWS) { atomicOr(err, 1); act = false; }
        const int R = act ? S.m_last - S.m_first + 1 : -1;
        const float zs = act ? S.zc * V.sgv : 0.f;
        // crossing boundaries of this lane's voxel (at most KCT_ROWS <= EV_CAP)
        int nev = 0;
        for (int b = 0; b <= R; ++b) {
            float p0, p1;
            if (classify_row(V, G, C, S, (float)(S.m_first + b) - 0.5f, p0, p1) == ROW_CROSS) ++nev;
        }
        int incl = nev;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULLMASK, incl, o);
            if (lane >= o) incl += t;
        }
        const int base = incl - nev;
        // lanes are served in contiguous groups whose events fit the queue
        for (int lo = 0; lo < 32;) {
            const int base_lo = __shfl_sync(FULLMASK, base, lo);
            const unsigned fit = __ballot_sync(FULLMASK, lane >= lo && incl - base_lo <= EV_CAP);
            const int hi = 32 - __clz(fit);
            const bool mine = lane >= lo && lane < hi;
            const int ne = __shfl_sync(FULLMASK, incl, hi - 1) - base_lo;
            // 1) queue the group's crossing boundaries
            if (mine) {
                int e = base - base_lo;
                for (int b = 0; b <= R; ++b) {
                    float p0, p1;
                    if (classify_row(V, G, C, S, (float)(S.m_first + b) - 0.5f, p0, p1) == ROW_CROSS) {
                        ws->ev_p0[e] = p0;
                        ws->ev_p1[e] = p1;
                        ws->ev_zs[e] = zs;
                        ++e;
                    }
                }
            }
            __syncwarp();
            // 2) the whole warp evaluates (event, column boundary) tasks
            for (int t = lane; t < ne * nb; t += 32) {
                const int e = t / nb, c = t - e * nb;
                float U = (float)(cstart + c) - 0.5f;
                float l1t = (V.cu - U) * C.itc;
                float l1c = -fmaf(V.gu, C.alc, V.cu - U);
                Mom full = Mom{ws->fm[0][c], ws->fm[1][c], ws->fm[2][c], ws->fm[3][c], ws->fm[4][c]};
                float gv, gq;
                g_cross(V, G, C, boundary_kind(U, C), l1t, l1c, full, ws->ev_p0[e], ws->ev_p1[e], ws->ev_zs[e],
                        gv, gq);
                ws->res_v[e][c] = gv;
                ws->res_q[e][c] = gq;
            }
            __syncwarp();
            // 3) pairs of the group's voxels
            if (mine && act) {
                sink.begin(pass, k);
                const float D2 = fmaf(C.tc, C.tc, fmaf(C.xc, C.xc, S.zc * S.zc));
                const float vtiny = 1e-9f * G.ax * G.ay * az;
                float pV[KCT_CB], pQ[KCT_CB];
#pragma unroll
                for (int c = 0; c < KCT_CB; ++c) { pV[c] = 0.f; pQ[c] = 0.f; }
                int e = base - base_lo;
                for (int b = 0; b <= R; ++b) {
                    float p0 = 0.f, p1 = 0.f;
                    const int cls = classify_row(V, G, C, S, (float)(S.m_first + b) - 0.5f, p0, p1);
                    float gV[KCT_CB], gQ[KCT_CB];
                    if (cls == ROW_ZERO) {
#pragma unroll
                        for (int c = 0; c < KCT_CB; ++c) { gV[c] = 0.f; gQ[c] = 0.f; }
                    } else if (cls == ROW_FULL) {
#pragma unroll
                        for (int c = 0; c < KCT_CB; ++c) { gV[c] = az * f1[c]; gQ[c] = az * fl[c]; }
                    } else if (cls == ROW_LIN) {
                        const float p00 = p0 * p0, p01 = 2.f * p0 * p1, p11 = p1 * p1;
#pragma unroll
                        for (int c = 0; c < KCT_CB; ++c) {
                            float Vg = fmaf(p0, f1[c], p1 * ft[c]);
                            float Sl = fmaf(p0, fl[c], p1 * flt[c]);
                            float Sh2 = fmaf(p00, f1[c], fmaf(p01, ft[c], p11 * ftt[c]));
                            gV[c] = Vg;
                            gQ[c] = fmaf(zs, fmaf(0.5f, Sh2, -0.5f * az * Vg), Sl);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < KCT_CB; ++c) { gV[c] = ws->res_v[e][c]; gQ[c] = ws->res_q[e][c]; }
                        ++e;
                    }
                    if (b > 0) {
                        const int m = S.m_first + b - 1;
#pragma unroll
                        for (int c = 0; c + 1 < KCT_CB; ++c) {
                            if (c + 1 < nb) {
                                float Vp = (gV[c + 1] - gV[c]) - (pV[c + 1] - pV[c]);
                                float Qp = (gQ[c + 1] - gQ[c]) - (pQ[c + 1] - pQ[c]);
                                if (Vp > vtiny) sink.pair(pass, cstart + c, m, Vp * Vp / fmaf(Vp, D2, 2.f * Qp));
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < KCT_CB; ++c) { pV[c] = gV[c]; pQ[c] = gQ[c]; }
                }
            }
            __syncwarp();
            lo = hi;
        }
    }
}

template <class Sink>
__device__ __forceinline__ void relaxed_segment(const View& V, const Grid& G, const Column& C, int cstart, int nb,
                                                int kbase, int lane, Sink& sink, int* err) {
    const float az = G.az;
    float A = 0.f, T = 0.f;       // area and t'-moment of P_c, c = lane
    if (lane < nb) {
        float U = (float)(cstart + lane) - 0.5f;
        int kind = boundary_kind(U, C);
        if (kind == KIND_FULL) A = G.ax * G.ay;
        else if (kind == KIND_GEN) {
            float l1t = (V.cu - U) * C.itc;
            float l1c = -fmaf(V.gu, C.alc, V.cu - U);
            Mom5 g = region<true, false, false>(V, l1t, C.gxi, l1c, 0.f);
            A = 0.5f * g.a;
            T = g.t * (1.f / 6.f);
        }
    }
    float An[KCT_CB - 1], Tn[KCT_CB - 1];    // area and centre-of-mass depth of H_n
    {
        float Ap = __shfl_sync(FULLMASK, A, 0), Tp = __shfl_sync(FULLMASK, T, 0);
#pragma unroll
        for (int c = 0; c + 1 < KCT_CB; ++c) {
            float Aq = __shfl_sync(FULLMASK, A, c + 1), Tq = __shfl_sync(FULLMASK, T, c + 1);
            An[c] = Aq - Ap;
            Tn[c] = (An[c] > 0.f) ? (Tq - Tp) / An[c] : 0.f;
            Ap = Aq;
            Tp = Tq;
        }
    }
    const float atiny = 1e-9f * G.ax * G.ay;
    for (int pass = 0; pass < KPL; ++pass) {
        const int k = kbase + pass * 32 + lane;
        Slice S;
        bool act = (k < G.nz) && slice_setup(V, G, C, k, S);
        if (act && S.m_last - S.m_first + 2 > KCT_ROWS) { atomicOr(err, 1); act = false; }
        if (!act) continue;
        sink.begin(pass, k);
        const float iD2 = 1.0f / fmaf(C.tc, C.tc, fmaf(C.xc, C.xc, S.zc * S.zc));
        float ph[KCT_CB - 1];
#pragma unroll
        for (int c = 0; c + 1 < KCT_CB; ++c) ph[c] = 0.f;
        const int R = S.m_last - S.m_first + 1;
        for (int b = 0; b <= R; ++b) {
            float p0, p1;
            row_plane(V, G, C, S, (float)(S.m_first + b) - 0.5f, p0, p1);
#pragma unroll
            for (int c = 0; c + 1 < KCT_CB; ++c) {
                float h = fminf(fmaxf(fmaf(p1, Tn[c], p0), 0.f), az);
                if (b > 0 && c + 1 < nb && An[c] > atiny) {
                    float d = h - ph[c];
                    if (d > 0.f) sink.pair(pass, cstart + c, S.m_first + b - 1, An[c] * d * iD2);
                }
                ph[c] = h;
            }
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
    for (int cstart = C.n_first; cstart <= C.n_last; cstart += KCT_CB - 1) {
        const int nb = min(KCT_CB - 1, C.n_last - cstart + 1) + 1;
        if (VARIANT == 1) relaxed_segment(V, G, C, cstart, nb, kbase, lane, sink, err);
        else exact_segment(V, G, C, cstart, nb, kbase, lane, ws, sink, err);
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
