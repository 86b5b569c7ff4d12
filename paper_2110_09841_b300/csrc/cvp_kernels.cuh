// cvp_kernels.cuh -- brick-tiled CUDA kernels of the cutting voxel projector (sm_103a).
//
// A thread block owns a brick of BX x BY voxel columns and Brick<VARIANT>::Z voxels along x_3
// (one or two runs of SEG = 64).
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
// voxel of the column (Sec. III-A, Eq. columnprojectionidentity): the warp builds them
// together (a few lanes per column) and shares their moments through shared memory. Each
// lane then walks the rows of its own voxel. A row whose two planes stay inside the voxel
// over the whole base gives its pairs in closed form from the moments of H_n; a plane that
// leaves the voxel through its top or bottom face ("crossing") needs the moments of H_n cut
// at a depth tau. The warp's crossing planes ("events") are numbered by a prefix sum over
// the lanes and evaluated one per lane, each lane reading its event's plane from the owning
// lane's registers, so the cuts never run with most of the warp idle.
// Forward projection and adjoint enumerate the same pairs with the same code, so
// <A x, y> = <x, A^T y> holds to float rounding.
#pragma once

#include <type_traits>

#include "cvp_device.cuh"

namespace kct {

constexpr int KPL = 2;             // voxels per lane in a column segment
constexpr int SEG = 32 * KPL;      // voxels of a column in a brick
constexpr int BX = 8, BY = 8;      // voxel columns of a brick
constexpr int NCOLS = BX * BY;
constexpr int NWARP = 8;           // warps per block
constexpr int NTHREADS = 32 * NWARP;
// Blocks per SM: 2 for the near-exact kernels (their register need), 3 for the relaxed ones
// (measured 21 % faster than with 2); the shared memory of a block (static part +
// Brick::DYN_FLOATS floats) is sized accordingly.
constexpr int EV_CAP = 64;         // crossing events evaluated per warp and round (>= KPL * KCT_ROWS)
constexpr int KCT_ROWS = 32;       // row boundaries of one voxel (its footprint spans <= 31 rows)

// Brick height along x_3: two runs of SEG voxels per column-cut build (the build is a large
// part of the per-voxel work). The relaxed adjoint takes one or two runs (RUNS_ = 1 or 2), as
// the plan chooses from the geometry: two runs share each build along more voxels but overflow
// the shared tile where a brick's footprint is tall, and its fallback reads y from global memory.
// Detector tile: 12288 floats for the near-exact kernels (2 blocks per SM), 8192 for the
// relaxed ones (3 blocks per SM, small static shared memory).
template <int VARIANT, bool FWD = true, int RUNS_ = 0>
struct Brick {
    static constexpr int RUNS = RUNS_ ? RUNS_ : ((VARIANT == 0 || FWD) ? 2 : 1);
    static constexpr int Z = SEG * RUNS;                       // voxels along x_3
    static constexpr int TILE = VARIANT == 0 ? 12288 : 8192;   // floats of the detector tile
    static constexpr int DYN_FLOATS = Z * NCOLS + TILE;        // dynamic shared memory
};
constexpr int VIEW_CHUNK = 16;     // default views per forward block (a plan may tune it)
constexpr int MAX_VIEW_CHUNK = 64; // largest views per forward block a plan accepts
constexpr int TUNE_VIEWS = 64;     // views the forward tuning launches cover
constexpr unsigned FULLMASK = 0xffffffffu;

struct WarpSmem {
    Column C;                      // the warp's current column
    alignas(16) float ivs[KCT_CB][KCT_IV + 1];   // exact: depth profile of H_n, n = cstart + c (depth_profile)
    float4 iva[KCT_CB][KCT_IV];
    float4 ivb[KCT_CB][KCT_IV];
    float2 ivm[KCT_CB][KCT_IV];
    float4 fa[KCT_CB];             // exact: moments of H_n m1, mt, mtt, ml; relaxed: A_n, t_n, 1/t_n, -
    float4 fb[KCT_CB];             // exact: mlt, t'-range of H_n (lo, hi), -
    float2 fr[KCT_CB];             // exact: 1 / depth at the two ends of that range
    float res_v[EV_CAP], res_q[EV_CAP];   // exact: the crossing planes' region values (volume, moment)
    float sc_t[KCT_CB * 8], sc_x[KCT_CB * 8];   // exact: vertices of H_n while the cuts are built
    int sc_n[KCT_CB];
};

// The relaxed kernels keep only the column cuts' areas and depth centroids, so that their
// blocks stay small.
struct WarpSmemRelaxed {
    Column C;
    float pt[KCT_CB][8], px[KCT_CB][8];   // vertices of H_n (build scratch)
    float4 fa[KCT_CB];             // A_n t_n / |gv|, t'_CM / t_n, 1/t_n, half the voxel's projected row extent
};

struct Tile {                      // detector window covered by a brick in one view
    int u0, v0, w, h, ok;
};

template <class WS>
struct BlockSmemOf {
    View V;
    Tile T;
    WS ws[NWARP];
};

template <int VARIANT>
using BlockSmem = BlockSmemOf<typename std::conditional<VARIANT == 0, WarpSmem, WarpSmemRelaxed>::type>;

// Moments (1, t', t'^2, lambda, lambda t') of H_n ∩ {t' < tau}, tlo <= tau <= thi, from the
// depth profile of H_n in slot c: one interval's closed form, the same work for every tau.
__device__ __forceinline__ Mom cut_moments(const WarpSmem* ws, int c, float tau, float tc, float xc) {
    float A, T, TT, X, TX;
    profile_cut(ws->ivs[c], ws->iva[c], ws->ivb[c], ws->ivm[c], tau, A, T, TT, X, TX);
    return Mom{A, T, TT, fmaf(tc, T, xc * X), fmaf(tc, TT, xc * TX)};
}

// the same, not inlined, for the rare second cut of a plane that crosses both faces
__device__ __noinline__ Mom cut_moments_call(const WarpSmem* ws, int c, float tau, float tc, float xc) {
    return cut_moments(ws, c, tau, tc, xc);
}

// position of set bit j (from 0, counted from the lowest) of m; j < popc(m)
__device__ __forceinline__ int nth_bit(unsigned m, int j) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));   // set bits in the low half of the window
        const bool up = j >= c;
        j -= up ? c : 0;
        m >>= up ? w : 0;
        pos += up ? w : 0;
    }
    return pos;
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

// the same quantity for a plane that stays inside the voxel over the whole base, with paired
// FP32 instructions (two independent FMAs per issue)
__device__ __forceinline__ void g_lin2(float az, float p0, float p1, float zs, float f1, float ft, float ftt, float fl,
                                       float flt, float& gv, float& gq) {
    const float2 vs = __ffma2_rn(make_float2(p0, p0), make_float2(f1, fl), __fmul2_rn(make_float2(p1, p1), make_float2(ft, flt)));
    const float2 sq = __fmul2_rn(make_float2(p0, p1), make_float2(p0, p1));
    const float Sh2 = fmaf(sq.x, f1, fmaf(2.f * p0 * p1, ft, sq.y * ftt));
    gv = vs.x;
    gq = fmaf(zs, fmaf(0.5f, Sh2, -0.5f * az * vs.x), vs.y);
}

__device__ __forceinline__ float pair_weight(float pv, float pq, float D2) {
    return __fdividef(pv * pv, fmaf(pv, D2, 2.f * pq));
}

// Per-column constants of the row geometry in two floats: the voxel centre k projects at row
// cv + vc_k at the column centre depth, vc_k = gv zeta_k / tc = sign(gv) zeta_k / da; with
// B_k = -cv - vc_k = B0 + k dB, the distance of row boundary m - 1/2 from that projection is
// (m - 1/2) + B_k: a small difference of large row coordinates, which thin slivers need to
// float precision (the plain float sum loses up to ulp(cv + vc) rows).
__device__ __forceinline__ void row_frame(const View& V, const Grid& G, const Column& C, F2& B0, F2& dB) {
    const float ida = __fdividef(1.0f, C.da.hi);
    const F2 z0s = f2_of(G.z0d - ((double)V.sz + (double)V.sz_lo)), azF = f2_of(G.azd);
    const float q0 = z0s.hi * ida, q1 = (fmaf(-q0, C.da.hi, z0s.hi) + fmaf(-q0, C.da.lo, z0s.lo)) * ida;
    const float r0 = azF.hi * ida, r1 = (fmaf(-r0, C.da.hi, azF.hi) + fmaf(-r0, C.da.lo, azF.lo)) * ida;
    const float vch = V.sgv * q0;
    const float bs = -V.cv - vch, bz = bs + V.cv;
    B0 = F2{bs, ((-V.cv - (bs - bz)) + (-vch - bz)) - V.cv_lo - V.sgv * q1};
    dB = F2{-V.sgv * r0, -V.sgv * r1};
}

// bit index of floor(x) / ceil(x) for a plane index bound x, clamped to [-1, 32]
__device__ __forceinline__ int floor_bit(float x) { return (int)floorf(fminf(fmaxf(x, -1.f), 32.f)); }
__device__ __forceinline__ int ceil_bit(float x) { return (int)ceilf(fminf(fmaxf(x, -1.f), 32.f)); }

// bits lo .. hi of a 32-bit word (lo, hi clamped to 0 .. 31; empty if lo > hi)
__device__ __forceinline__ unsigned range_bits(int lo, int hi) {
    lo = max(lo, 0);
    hi = min(hi, 31);
    return lo > hi ? 0u : ((2u << hi) - (1u << lo));
}

// Near-exact pairs of voxels kbase + lane + 32 p of the warp's column with detector
// columns n = cstart .. cstart + ncol - 1, one detector column at a time. Each pair (n, m)
// is the integral over H_n of the height between the two row planes of row m. When both
// planes stay inside the voxel over the depth range of H_n this height is linear in t'
// and the pair is a closed form of the moments of H_n. Otherwise it is the difference of
// the cuts below (or above) the two planes, measured from the nearer face (bottom frame
// for the lower half of the rows, top frame for the upper half), so that no pair is a
// small difference of two near-full voxel volumes.
template <class Sink>
__device__ __forceinline__ void exact_voxels(const View& V, const Grid& G, const Column& C, int cstart, int ncol,
                                             int kbase, int lane, WarpSmem* ws, Sink& sink, int* err) {
    const float az = G.az, agv = fabsf(V.gv);
    const float dp0 = C.tc * V.inv_agv, dp1 = V.inv_agv;   // change of p0, p1 from one row boundary to the next
    const float idp0 = agv * C.itc;                         // 1 / dp0
    // Rows r < rb take the bottom frame, the others the top frame. Plane rb is the one nearest
    // the voxel's mid-height at the column centre (p0 = az/2): its value passes from one frame
    // to the other as the complement az (m1, ml) - g, which loses nothing there, and every
    // other plane is evaluated in the frame of the face it is nearer to.
    auto frame_split = [&](float off0, int R) { return max(1, min(R, __float2int_rn(-off0 * idp0))); };
    const float vtiny = 1e-9f * G.ax * G.ay * az;
    // Height offset of row boundary m - 1/2 over the centre of voxel k at the column centre depth,
    // tc (m - 1/2 - v_c) / |gv| = ((m - 1/2) + B_k) da (row_frame): the row distance is formed in
    // two floats and is small, so the offset keeps float precision; a plane b rows higher is
    // then az/2 + b dp0 + offset (small terms, plain float).
    F2 B0, dB;
    row_frame(V, G, C, B0, dB);
    auto row_offset = [&](int k, int m) -> float {
        const F2 Bk = f2_axpy(B0, (float)k, dB);
        return ((((float)m - 0.5f) + Bk.hi) + Bk.lo) * C.da.hi;
    };
    // the lane's voxels kbase + lane + 32 p; their crossing planes share one evaluation round
#pragma unroll
    for (int p = 0; p < KPL; ++p) {
        const int k = kbase + p * 32 + lane;
        if (k < G.nz) sink.begin(p, k);
    }
#pragma unroll 1
    for (int c = 0; c < ncol; ++c) {
        const float4 fa = ws->fa[c], fb = ws->fb[c];
        const float tlo = fb.y, thi = fb.z;
        const float2 fr = ws->fr[c];
        int m_first[KPL], R[KPL];
        float off0p[KPL];
        unsigned cross[KPL], zero[KPL], full[KPL];
        int nev[KPL];
#pragma unroll
        for (int p = 0; p < KPL; ++p) {
            const int k = kbase + p * 32 + lane;
            const float zc = fmaf((float)k, az, G.z0) - V.sz;     // zeta of the voxel centre
            // rows touched by this voxel over the depth range of H_n
            m_first[p] = 0;
            R[p] = 0;
            if (k < G.nz && fa.x > 0.f) {
                const float zl = zc - 0.5f * az, zh = zc + 0.5f * az;
                const float b0 = fminf(fminf(zl * fr.x, zl * fr.y), fminf(zh * fr.x, zh * fr.y));
                const float b1 = fmaxf(fmaxf(zl * fr.x, zl * fr.y), fmaxf(zh * fr.x, zh * fr.y));
                const float va = fmaf(V.gv, b0, V.cv), vb = fmaf(V.gv, b1, V.cv);
                m_first[p] = max((int)floorf(fminf(va, vb) + 0.5f), 0);
                const int m_last = min((int)floorf(fmaxf(va, vb) + 0.5f), G.nv - 1);
                R[p] = m_last - m_first[p] + 1;
                if (R[p] + 1 > KCT_ROWS) { atomicOr(err, 1); R[p] = 0; }
                if (R[p] < 0) R[p] = 0;
            }
            // height of {v < V_b} over t' is p0 + p1 t', p0 = az/2 + tc (V_b - v_c)/|gv|, p1 = (V_b - cv)/|gv|
            const float off0 = row_offset(k, m_first[p]);
            off0p[p] = off0;
            const float p1_0 = ((float)m_first[p] - 0.5f - V.cv) * V.inv_agv;
            // classes of the boundaries b = 0 .. R (0 / az for planes under / over the voxel, inside,
            // crossing a face), in closed form: at the two ends of the depth range of H_n the height
            // of plane b is H0 + b S0 and H1 + b S1 with S0, S1 = (tc + t') / |gv| > 0, so the planes
            // under the voxel, over it and inside it are three ranges of b, and the rest cross a face
            const float iS0 = agv * fr.x, iS1 = agv * fr.y;            // 1 / S0, 1 / S1
            const float c0 = fmaf(0.5f, az, off0);
            const float H0 = fmaf(p1_0, tlo, c0), H1 = fmaf(p1_0, thi, c0);
            const float n0 = -H0 * iS0, n1 = -H1 * iS1;                 // b where an end height is 0
            const float a0 = (az - H0) * iS0, a1 = (az - H1) * iS1;     // ... where it is az
            const unsigned all = (2u << R[p]) - 1u;
            const unsigned ze = range_bits(-1, floor_bit(fminf(n0, n1))) & all;
            const unsigned fu = range_bits(ceil_bit(fmaxf(a0, a1)), 32) & all & ~ze;
            const unsigned in = range_bits(ceil_bit(fmaxf(n0, n1)), floor_bit(fminf(a0, a1))) & all & ~ze & ~fu;
            const unsigned cr = all & ~(ze | fu | in);
            cross[p] = cr;
            zero[p] = ze;
            full[p] = fu;
            // planes b <= rb give a bottom-frame event, b > rb a top-frame one
            nev[p] = __popc(cr);
        }
        int nl = 0;
#pragma unroll
        for (int p = 0; p < KPL; ++p) nl += nev[p];
        int base = 0, total = 0;
        if (__any_sync(FULLMASK, nl > 0)) {
            int incl = nl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(FULLMASK, incl, o);
                if (lane >= o) incl += t;
            }
            base = incl - nl;
            total = __shfl_sync(FULLMASK, incl, 31);
        }
        // lanes are served in contiguous groups whose events fit the result slots (a lane has at
        // most KPL * KCT_ROWS <= EV_CAP events, so every group makes progress)
        for (int lo_lane = 0; lo_lane < 32;) {
            int hi_lane = 32, e0 = 0;
            if (total > 0) {
                const int incl = base + nl;
                const int base_lo = __shfl_sync(FULLMASK, base, lo_lane);
                const unsigned fit = __ballot_sync(FULLMASK, lane >= lo_lane && incl - base_lo <= EV_CAP);
                hi_lane = 32 - __clz(fit);
                const int ne = __shfl_sync(FULLMASK, incl, hi_lane - 1) - base_lo;
                e0 = base - base_lo;
                static_assert(KPL == 2, "the event decoding below reads the state of two voxels per lane");
                // 1) lane e of the warp evaluates event e of the group (cut moments at the
                // crossing depths): it is event j of lane s, the last lane whose events start
                // at or before it, and its plane comes from that lane's state. A lane's events
                // are, per voxel p, its crossing planes b <= rb in the bottom frame, then those
                // b > rb in the top frame.
                const Mom full_m = Mom{fa.x, fa.y, fa.z, fa.w, fb.x};
                const Mom zero_m = Mom{0.f, 0.f, 0.f, 0.f, 0.f};
                for (int er = 0; er < ne; er += 32) {
                    const int e = er + lane, target = base_lo + e;
                    int src = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1)
                        if (__shfl_sync(FULLMASK, base, src + step) <= target) src += step;
                    int j = target - __shfl_sync(FULLMASK, base, src);
                    const unsigned cm0 = __shfl_sync(FULLMASK, cross[0], src), cm1 = __shfl_sync(FULLMASK, cross[1], src);
                    const int rr0 = __shfl_sync(FULLMASK, R[0], src), rr1 = __shfl_sync(FULLMASK, R[1], src);
                    const int mf0 = __shfl_sync(FULLMASK, m_first[0], src), mf1 = __shfl_sync(FULLMASK, m_first[1], src);
                    const float of0 = __shfl_sync(FULLMASK, off0p[0], src), of1 = __shfl_sync(FULLMASK, off0p[1], src);
                    if (e >= ne) continue;
                    // the event's voxel p, frame and plane b
                    const int rb0 = frame_split(of0, rr0), rb1 = frame_split(of1, rr1);
                    const unsigned mb0 = cm0 & ((2u << rb0) - 1u), mt0 = cm0 & ~((2u << rb0) - 1u);
                    const unsigned mb1 = cm1 & ((2u << rb1) - 1u), mt1 = cm1 & ~((2u << rb1) - 1u);
                    const int n0 = __popc(mb0), n1 = n0 + __popc(mt0), n2 = n1 + __popc(mb1);
                    const bool p1v = j >= n1, top = (j >= n0 && j < n1) || j >= n2;
                    const unsigned msk = j < n0 ? mb0 : j < n1 ? mt0 : j < n2 ? mb1 : mt1;
                    const int jj = j - (j < n0 ? 0 : j < n1 ? n0 : j < n2 ? n1 : n2);
                    const int b = nth_bit(msk, jj);
                    const int k = kbase + (p1v ? 32 : 0) + src;
                    const float zc = fmaf((float)k, az, G.z0) - V.sz;
                    const float zs0 = zc * V.sgv;
                    const float p1_0 = ((float)(p1v ? mf1 : mf0) - 0.5f - V.cv) * V.inv_agv;
                    const float q0 = fmaf(0.5f, az, fmaf((float)b, dp0, p1v ? of1 : of0)), q1 = fmaf((float)b, dp1, p1_0);
                    const float p0 = top ? az - q0 : q0, p1 = top ? -q1 : q1, zs = top ? -zs0 : zs0;
                    const float p1s = (fabsf(p1) < 1e-30f) ? copysignf(1e-30f, p1) : p1;
                    const float ip1 = rcp_fast(p1s);
                    const float tau0 = -p0 * ip1, tau1 = (az - p0) * ip1;
                    // A plane usually leaves through one face only, so one of the two depths
                    // lies inside H_n's depth range: one call site serves every lane (a
                    // second one only for planes that cross both faces within H_n).
                    const bool in0 = tau0 > tlo && tau0 < thi, in1 = tau1 > tlo && tau1 < thi;
                    Mom ca = zero_m, cb = zero_m;
                    if (in0 || in1) ca = cut_moments(ws, c, in0 ? tau0 : tau1, C.tc, C.xc);
                    if (in0 && in1) cb = cut_moments_call(ws, c, tau1, C.tc, C.xc);
                    const Mom c0 = in0 ? ca : (tau0 <= tlo) ? zero_m : full_m;
                    const Mom c1 = in1 ? (in0 ? cb : ca) : (tau1 <= tlo) ? zero_m : full_m;
                    float gv, gq;
                    g_cross_from(az, c0, c1, full_m, p0, p1, p1s, zs, gv, gq);
                    ws->res_v[e] = gv;
                    ws->res_q[e] = gq;
                }
                __syncwarp();
            }
            // 3) pairs of the group's voxels with detector column n
            if (lane >= lo_lane && lane < hi_lane) {
                const int n = cstart + c;
                int ep = e0;
#pragma unroll
                for (int p = 0; p < KPL; ++p) {
                    const int k = kbase + p * 32 + lane;
                    const float zc = fmaf((float)k, az, G.z0) - V.sz;
                    const float zs = zc * V.sgv;
                    const float D2 = fmaf(C.tc, C.tc, fmaf(C.xc, C.xc, zc * zc));
                    const float p1_0 = ((float)m_first[p] - 0.5f - V.cv) * V.inv_agv;
                    const int rb = frame_split(off0p[p], R[p]);
                    const unsigned mbot = cross[p] & ((2u << rb) - 1u), mtop = cross[p] & ~((2u << rb) - 1u);
                    const int nbot = __popc(mbot);
                    // Every row is the difference of its two planes' region values in the row's frame
                    // (bottom for r < rb, top after), so all lanes take the same path whatever the
                    // planes' classes; the upper plane's value is carried to the next row, whose
                    // lower plane it is (complemented where the frame changes).
                    float carry_v = 0.f, carry_q = 0.f;
#pragma unroll 1
                    for (int r = 0; r < R[p]; ++r) {
                        const int m = m_first[p] + r;
                        float pv, pq;
                        {
                            const bool top = r >= rb;
                            float g[2][2];
                            const bool reuse = r > 0;
                            // plane rb changes frame: its value from the other face
                            g[0][0] = r == rb ? fmaf(az, fa.x, -carry_v) : carry_v;
                            g[0][1] = r == rb ? fmaf(az, fa.w, -carry_q) : carry_q;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                if (h == 0 && reuse) continue;
                                const int b = r + h;
                                const unsigned bit = 1u << b;
                                const float2 pp = __ffma2_rn(make_float2((float)b, (float)b), make_float2(dp0, dp1),
                                                             make_float2(off0p[p], p1_0));
                                float p0 = pp.x + 0.5f * az, p1 = pp.y;
                                if (zero[p] & bit) { p0 = 0.f; p1 = 0.f; }
                                if (full[p] & bit) { p0 = az; p1 = 0.f; }
                                g_lin2(az, top ? az - p0 : p0, top ? -p1 : p1, top ? -zs : zs, fa.x, fa.y, fa.z, fa.w, fb.x,
                                       g[h][0], g[h][1]);
                                if (cross[p] & bit) {
                                    const int q = top ? ep + nbot + __popc(mtop & (bit - 1u)) : ep + __popc(mbot & (bit - 1u));
                                    g[h][0] = ws->res_v[q];
                                    g[h][1] = ws->res_q[q];
                                }
                            }
                            pv = top ? g[0][0] - g[1][0] : g[1][0] - g[0][0];
                            pq = top ? g[0][1] - g[1][1] : g[1][1] - g[0][1];
                            carry_v = g[1][0];
                            carry_q = g[1][1];
                        }
                        if (pv > vtiny) sink.pair(p, n, m, pair_weight(pv, pq, D2));
                    }
                    ep += nev[p];
                }
            }
            if (total > 0) __syncwarp();
            lo_lane = hi_lane;
        }
    }
#pragma unroll
    for (int p = 0; p < KPL; ++p) {
        const int k = kbase + p * 32 + lane;
        if (k < G.nz) sink.end(p, k);
    }
}

// Relaxed pairs: W = A_n d / |D|^2 with d the x_3 length of row m along the vertical line
// through the centre of mass of H_n (Sec. III-A, Eq. cutvolume, voxel-centre r). At the
// depth t_n = t_c + t'_CM of that line the voxel spans v_n -+ hv in detector rows, v_n =
// cv + gv zeta_c / t_n, hv = |gv| az / (2 t_n), and d = (overlap with [m - 1/2, m + 1/2]) t_n / |gv|;
// the overlap is evaluated relative to v_n so that no large row index enters a difference.
template <class Sink>
__device__ __forceinline__ void relaxed_voxels(const View& V, const Grid& G, const Column& C, int cstart, int ncol,
                                               int kbase, int lane, const WarpSmemRelaxed* ws, Sink& sink,
                                               int* err) {
    const float az = G.az;
    // distance of row boundary m from the voxel centre's projection at the column centre depth,
    // (m + B_k) with B_k = -cv - vc_k in two floats (row_frame); at the centroid depth t_n of H_n
    // it is m + B_k + vc_k delta, delta = t'_CM / t_n
    F2 B0, dB;
    row_frame(V, G, C, B0, dB);
    for (int pass = 0; pass < KPL; ++pass) {
        const int k = kbase + pass * 32 + lane;
        if (k >= G.nz) continue;
        sink.begin(pass, k);
        const float zc = fmaf((float)k, az, G.z0) - V.sz;
        const float iD2 = rcp_fast(fmaf(C.tc, C.tc, fmaf(C.xc, C.xc, zc * zc)));
        const float gz = V.gv * zc;
        const F2 Bk = f2_axpy(B0, (float)k, dB);
        const float bs = Bk.hi, bl = Bk.lo, vch = -(bs + V.cv);
        for (int c = 0; c < ncol; ++c) {
            const float4 fa = ws->fa[c];           // A_n t_n / |gv|, t'_CM / t_n, 1/t_n, hv
            if (!(fa.x > 0.f)) continue;
            const float hv = fa.w;
            const float vn = fmaf(gz, fa.z, V.cv);
            const int m_first = max((int)floorf(vn - hv + 0.5f), 0);
            const int m_last = min((int)floorf(vn + hv + 0.5f), G.nv - 1);
            if (m_last - m_first + 2 > KCT_ROWS) { atomicOr(err, 1); continue; }
            const float w = fa.x * iD2;
            float e = ((float)m_first + bs) + fmaf(vch, fa.y, bl);   // m_first - v_n
            const int n = cstart + c;
            for (int m = m_first; m <= m_last; ++m, e += 1.0f) {
                const float d = fminf(hv, e + 0.5f) - fmaxf(-hv, e - 0.5f);
                if (d > 0.f) sink.pair(pass, n, m, w * d);
            }
        }
        sink.end(pass, k);
    }
}

// The column cuts H_n, n = cstart + c (c < ncol <= KCT_CB), of one voxel column in one view
// are built by the whole warp.
//
// Polygons: lanes 4c .. 4c + 3 clip the base square for column n, lane 4c + e taking square
// edge e (clip_square_edge); the points are compacted, in the order of clip_square, into
// (pts, pxs)[8c ..]. Each lane keeps its own points and returns whether its column exists.
struct EdgePoints {
    float t[3], x[3];
    int n, first, nv;              // its points, their index in the polygon, the polygon's size
};

__device__ __forceinline__ bool clip_lanes(const View& V, const Column& C, int cstart, int ncol, int lane, float* pts,
                                           float* pxs, EdgePoints& r) {
    const int c = lane >> 2, e = lane & 3;
    const bool act = c < ncol;
    Line lo, hi;
    column_lines(V, C, cstart + c, lo, hi);
    r.n = act ? clip_square_edge(V, lo, hi, e, r.t, r.x) : 0;
    int incl = r.n;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const int t = __shfl_up_sync(FULLMASK, incl, o, 4);
        if (e >= o) incl += t;
    }
    r.first = incl - r.n;
    r.nv = min(__shfl_sync(FULLMASK, incl, 3, 4), 8);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q < r.n && r.first + q < 8) {
            pts[8 * c + r.first + q] = r.t[q];
            pxs[8 * c + r.first + q] = r.x[q];
        }
    }
    return act;
}

// Relaxed variant: the area of H_n and its depth centroid into slot c, the Green's-theorem
// sums of each lane's edges added over the column's four lanes. Not inlined: it runs once
// per column and view.
__device__ __noinline__ void build_cuts(const View* Vp, const Column* Cp, float az, int cstart, int ncol, int lane,
                                        WarpSmemRelaxed* ws) {
    const View& V = *Vp;
    const Column& C = *Cp;
    EdgePoints r;
    const bool act = clip_lanes(V, C, cstart, ncol, lane, &ws->pt[0][0], &ws->px[0][0], r);
    __syncwarp();
    const int c = lane >> 2;
    Green2 g{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = r.first + q;
        if (q < r.n && i < r.nv) {
            const int nx = i + 1 < r.nv ? i + 1 : 0;
            seg_acc(g, r.t[q], r.x[q], ws->pt[c][nx], ws->px[c][nx]);
        }
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        g.a += __shfl_xor_sync(FULLMASK, g.a, o, 4);
        g.t += __shfl_xor_sync(FULLMASK, g.t, o, 4);
    }
    if (act && (lane & 3) == 0) {
        const float m1 = 0.5f * g.a, mt = g.t * (1.f / 6.f);
        const float tcm = m1 > 0.f ? mt * rcp_fast(m1) : 0.f;  // t' of the centre of mass of H_n
        const float tn = C.tc + tcm, itn = rcp_fast(tn);
        ws->fa[c] = make_float4(m1 * tn * V.inv_agv, tcm * itn, itn, 0.5f * az * fabsf(V.gv) * itn);
    }
}

// Near-exact variant: the depth profile of H_n (as depth_profile computes it serially), its
// moments and depth range into slot c. After the polygons, lanes 8c' .. 8c' + 7 take column
// c = c0 + c' and lane 8c' + v its vertex v: the chord of H_n at that vertex's depth T_v
// (from every edge that spans it), and if the vertex is the first at the depth and below the
// top, the interval from T_v to the next vertex depth (chord there from the lane of that
// vertex) and its integral; the moments below T_v are the sum of the integrals of the
// intervals below it, and the interval's index is their number. Not inlined: it runs once per
// column and view.
__device__ __noinline__ void build_cuts(const View* Vp, const Column* Cp, float az, int cstart, int ncol, int lane,
                                        WarpSmem* ws) {
    const View& V = *Vp;
    const Column& C = *Cp;
    int* nvs = ws->sc_n;
    {
        EdgePoints r;
        const bool act = clip_lanes(V, C, cstart, ncol, lane, ws->sc_t, ws->sc_x, r);
        if (act && (lane & 3) == 0) nvs[lane >> 2] = r.nv;
    }
    __syncwarp();
    const int v = lane & 7, seg = lane & ~7;
#pragma unroll 1
    for (int c0 = 0; c0 < ncol; c0 += 4) {
        const int c = c0 + (lane >> 3);
        const bool colok = c < ncol;
        const int nv = colok ? nvs[c] : 0;
        const float* pt = ws->sc_t + 8 * c;
        const float* px = ws->sc_x + 8 * c;
        float T[8], X[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            T[u] = pt[u];          // slots u >= nv are not used
            X[u] = px[u];
        }
        float tlo = 0.f, thi = 0.f;
        if (nv > 0) {
            tlo = 3.0e38f;
            thi = -3.0e38f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (u < nv) {
                    tlo = fminf(tlo, T[u]);
                    thi = fmaxf(thi, T[u]);
                }
            }
        }
        const bool vert = v < nv;
        const float Tv = vert ? pt[v] : 3.0e38f;
        bool first = vert && nv >= 3;
        float Tn = 3.0e38f;
        int un = v;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (u < nv) {
                if (u < v && T[u] == Tv) first = false;
                if (T[u] > Tv && T[u] < Tn) {
                    Tn = T[u];
                    un = u;
                }
            }
        }
        // the chord at depth Tv (an edge along t' = Tv gives both of its ends)
        float xl = 3.0e38f, xr = -3.0e38f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (u < nv) {
                const bool wrap = u + 1 >= nv;
                const float ta = T[u], xa = X[u], tb = wrap ? T[0] : T[(u + 1) & 7], xb = wrap ? X[0] : X[(u + 1) & 7];
                if (fminf(ta, tb) <= Tv && Tv <= fmaxf(ta, tb)) {
                    float x0 = xa, x1 = xb;
                    if (ta != tb) x0 = x1 = fmaf((Tv - ta) * rcp_fast(tb - ta), xb - xa, xa);
                    xl = fminf(xl, fminf(x0, x1));
                    xr = fmaxf(xr, fmaxf(x0, x1));
                }
            }
        }
        const float w = vert ? fmaxf(xr - xl, 0.f) : 0.f, cm = vert ? 0.5f * (xl + xr) : 0.f;
        const float wn = __shfl_sync(FULLMASK, w, seg + un), cn = __shfl_sync(FULLMASK, cm, seg + un);
        const bool own = first && Tv < thi;   // the interval [Tv, Tn] is this lane's
        float I[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (own) simpson5(Tv, Tn, Tn - Tv, 1.f, w, wn - w, cm, cn - cm, I[0], I[1], I[2], I[3], I[4]);
        const unsigned ownm = (__ballot_sync(FULLMASK, own) >> seg) & 0xffu;
        float B[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        int rank = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float Iu[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) Iu[k] = __shfl_sync(FULLMASK, I[k], seg + u);
            if ((ownm >> u) & 1u) {
                const bool below = T[u] < Tv;
                rank += below ? 1 : 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    S[k] += Iu[k];
                    if (below) B[k] += Iu[k];
                }
            }
        }
        if (colok) {
            if (own) {
                ws->ivs[c][rank] = Tv;
                ws->iva[c][rank] = make_float4(rcp_fast(Tn - Tv), w, wn - w, cm);
                ws->ivb[c][rank] = make_float4(cn - cm, B[0], B[1], B[2]);
                ws->ivm[c][rank] = make_float2(B[3], B[4]);
            }
            if (v >= __popc(ownm)) ws->ivs[c][v] = 3.0e38f;
            if (v == 0) {
                ws->fa[c] = make_float4(S[0], S[1], S[2], fmaf(C.tc, S[1], C.xc * S[3]));
                ws->fb[c] = make_float4(fmaf(C.tc, S[2], C.xc * S[4]), tlo, thi, 0.f);
                ws->fr[c] = make_float2(1.0f / (C.tc + tlo), 1.0f / (C.tc + thi));
            }
        }
    }
}

// All pairs of voxels kbase .. kbase + runs * SEG - 1 of column (i, j) in view V (in shared
// memory): each column cut is built once and used by `runs` runs of SEG voxels; the sink is
// told when a run ends. Called by all 32 lanes of a warp with the same arguments.
template <int VARIANT, class Sink, class WS>
__device__ __forceinline__ void warp_column(const View& V, const Grid& G, int i, int j, int kbase, int runs,
                                            int lane, WS* ws, Sink& sink, int* err) {
    Column C;
    if (!column_setup(V, G, i, j, C)) return;
    if (C.n_last - C.n_first + 2 > KCT_MAX_SPAN) {
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    for (int cstart = C.n_first; cstart <= C.n_last; cstart += KCT_CB) {
        const int ncol = min(KCT_CB, C.n_last - cstart + 1);
        __syncwarp();              // the previous readers of ws are done
        build_cuts(&V, &C, G.az, cstart, ncol, lane, ws);
        __syncwarp();
#pragma unroll 1
        for (int r = 0; r < runs; ++r) {
            const int kb = kbase + r * SEG;
            if (kb >= G.nz) break;
            if constexpr (VARIANT == 1) relaxed_voxels(V, G, C, cstart, ncol, kb, lane, ws, sink, err);
            else exact_voxels(V, G, C, cstart, ncol, kb, lane, ws, sink, err);
            sink.end_run(r);
        }
    }
}

// Detector window covered by the brick [i0, i0+BX) x [j0, j0+BY) x [k0, k0+bz) in view V:
// the bounding box of the projected corners (u does not depend on x_3), one pixel of margin,
// if it holds at most `cap` pixels.
__device__ __forceinline__ Tile brick_tile(const View& V, const Grid& G, int i0, int j0, int k0, int bz, int cap) {
    const float xs[2] = {G.x0 + (i0 - 0.5f) * G.ax, G.x0 + (min(i0 + BX, G.nx) - 0.5f) * G.ax};
    const float ys[2] = {G.y0 + (j0 - 0.5f) * G.ay, G.y0 + (min(j0 + BY, G.ny) - 0.5f) * G.ay};
    const float zs[2] = {G.z0 + (k0 - 0.5f) * G.az - V.sz, G.z0 + (min(k0 + bz, G.nz) - 0.5f) * G.az - V.sz};
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
    T.ok = (T.w > 0 && (long)T.w * T.h <= cap) ? 1 : 0;
    return T;
}

// ---------------------------------------------------------------------------------------
// Sinks
// ---------------------------------------------------------------------------------------

// Forward sink: tile[m][n] += mu * W (sums of Eq. cvpsu). Pairs that fall outside the
// brick's tile go straight to the global output, multiplied by the pixel factor when the
// kernel applies it (SCALING >= 0); SCALING < 0 leaves the sums unscaled.
template <int SCALING>
struct FwdSink {
    const View* V;
    const float* mu_s;             // brick attenuation values, [Brick::Z][BY][BX] in shared memory
    float* tile;
    Tile T;
    float* __restrict__ Sg;        // global output of the view
    int nu, col, kbase;
    float mu[KPL];
    __device__ __forceinline__ void begin(int p, int k) {
#pragma unroll
        for (int q = 0; q < KPL; ++q)
            if (q == p) mu[q] = mu_s[(k - kbase) * NCOLS + col];
    }
    __device__ __forceinline__ void end(int, int) {}
    __device__ __forceinline__ void end_run(int) {}
    __device__ __forceinline__ void pair(int p, int n, int m, float W) {
        float mp = 0.f;
#pragma unroll
        for (int q = 0; q < KPL; ++q)
            if (q == p) mp = mu[q];
        if (mp == 0.f) return;
        const int du = n - T.u0, dv = m - T.v0;
        if (T.ok && (unsigned)du < (unsigned)T.w && (unsigned)dv < (unsigned)T.h) atomicAdd(&tile[dv * T.w + du], mp * W);
        else atomicAdd(&Sg[(size_t)m * nu + n], SCALING >= 0 ? mp * W * pixel_factor<(SCALING > 0)>(*V, n, m) : mp * W);
    }
};

// Adjoint sink: acc += W * F y. The staged tile already holds F y; pairs outside it read y
// and apply F here.
template <int SCALING>
struct BwdSink {
    const View* V;
    const float* tile;
    Tile T;
    const float* __restrict__ yg;
    int nu;
    float* acc_col;                // the column's accumulators in shared memory, one per voxel of the brick
    int lane;
    float acc[KPL];
    __device__ __forceinline__ void begin(int, int) {}
    __device__ __forceinline__ void end(int, int) {}
    // voxel kbase + r * SEG + p * 32 + lane of the brick
    __device__ __forceinline__ void end_run(int r) {
#pragma unroll
        for (int p = 0; p < KPL; ++p) {
            acc_col[r * SEG + p * 32 + lane] += acc[p];
            acc[p] = 0.f;
        }
    }
    __device__ __forceinline__ void pair(int p, int n, int m, float W) {
        const int du = n - T.u0, dv = m - T.v0;
        const float y = (T.ok && (unsigned)du < (unsigned)T.w && (unsigned)dv < (unsigned)T.h)
                            ? tile[dv * T.w + du]
                            : __ldg(&yg[(size_t)m * nu + n]) * pixel_factor<SCALING>(*V, n, m);
#pragma unroll
        for (int q = 0; q < KPL; ++q)
            if (q == p) acc[q] = fmaf(W, y, acc[q]);
    }
};

struct CountSink {
    unsigned long long n;
    __device__ __forceinline__ void begin(int, int) {}
    __device__ __forceinline__ void end(int, int) {}
    __device__ __forceinline__ void end_run(int) {}
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

// Forward projection. grid: (bricks in x1 x2, segments along x3, view chunks x batch), a
// chunk being view_chunk consecutive views.
// Volume b of the batch starts at vol + b * vstride, its projections at out + b * pstride.
// SCALING 0 / 1 multiplies by the cos / exact pixel factor while the tile is flushed;
// SCALING < 0 leaves the unscaled sums of Eq. cvpsu. out must be zeroed (or hold the values
// to add to) before the launch.
// Dynamic shared memory: Brick<VARIANT>::DYN_FLOATS floats.
template <int VARIANT, int SCALING>
__global__ void __launch_bounds__(NTHREADS, VARIANT == 1 ? 3 : 2) fwd_kernel(const View* __restrict__ views, Grid G,
                                                          const float* __restrict__ vol, float* __restrict__ out,
                                                          long long vstride, long long pstride, int view_chunk,
                                                          int* err) {
    extern __shared__ float dyn[];
    __shared__ BlockSmem<VARIANT> bs;
    using B = Brick<VARIANT>;
    float* mu_s = dyn;
    float* tile = dyn + B::Z * NCOLS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, j0;
    brick_origin(G, i0, j0);
    const int kbase = blockIdx.y * B::Z;
    const int nchunk = (G.nviews + view_chunk - 1) / view_chunk;
    const int chunk = blockIdx.z % nchunk, batch = blockIdx.z / nchunk;
    vol += batch * vstride;
    out += batch * pstride;
    for (int q = threadIdx.x; q < B::Z * NCOLS; q += NTHREADS) {
        const int kk = q / NCOLS, c = q % NCOLS;
        const int i = i0 + c % BX, j = j0 + c / BX, k = kbase + kk;
        mu_s[q] = (i < G.nx && j < G.ny && k < G.nz) ? __ldg(&vol[((size_t)k * G.ny + j) * G.nx + i]) : 0.f;
    }
    const int v_end = min((chunk + 1) * view_chunk, G.nviews);
    for (int view = chunk * view_chunk; view < v_end; ++view) {
        __syncthreads();
        if (threadIdx.x == 0) {
            bs.V = views[view];
            bs.T = brick_tile(bs.V, G, i0, j0, kbase, B::Z, B::TILE);
        }
        __syncthreads();
        const Tile T = bs.T;
        if (T.ok)
            for (int q = threadIdx.x; q < T.w * T.h; q += NTHREADS) tile[q] = 0.f;
        __syncthreads();
        float* Sv = out + (size_t)view * G.nu * G.nv;
        for (int c = warp; c < NCOLS; c += NWARP) {
            const int i = i0 + c % BX, j = j0 + c / BX;
            if (i >= G.nx || j >= G.ny) continue;
            FwdSink<SCALING> s{&bs.V, mu_s, tile, T, Sv, G.nu, c, kbase, 0.f};
            warp_column<VARIANT>(bs.V, G, i, j, kbase, B::RUNS, lane, &bs.ws[warp], s, err);
        }
        __syncthreads();
        if (T.ok)
            for (int q = threadIdx.x; q < T.w * T.h; q += NTHREADS) {
                const float v = tile[q];
                if (v != 0.f) {
                    const int n = T.u0 + q % T.w, m = T.v0 + q / T.w;
                    atomicAdd(&Sv[(size_t)m * G.nu + n], SCALING >= 0 ? v * pixel_factor<(SCALING > 0)>(bs.V, n, m) : v);
                }
            }
    }
}

// Adjoint. grid: (bricks in x1 x2, segments along x3, batch); every block loops over all
// views, staging F y of the brick's footprint in shared memory per view.
// Dynamic shared memory: Brick<VARIANT, false, RUNS_>::DYN_FLOATS floats.
template <int VARIANT, int SCALING, int RUNS_ = 0>
__global__ void __launch_bounds__(NTHREADS, VARIANT == 1 ? 3 : 2) bwd_kernel(const View* __restrict__ views, Grid G,
                                                          const float* __restrict__ y, float* __restrict__ vol,
                                                          long long vstride, long long pstride, int accumulate,
                                                          int* err) {
    extern __shared__ float dyn[];
    __shared__ BlockSmem<VARIANT> bs;
    using B = Brick<VARIANT, false, RUNS_>;
    float* acc_s = dyn;                 // [NCOLS][B::Z]
    float* tile = dyn + B::Z * NCOLS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, j0;
    brick_origin(G, i0, j0);
    const int kbase = blockIdx.y * B::Z;
    vol += blockIdx.z * vstride;
    y += blockIdx.z * pstride;
    for (int q = threadIdx.x; q < B::Z * NCOLS; q += NTHREADS) acc_s[q] = 0.f;
    for (int view = 0; view < G.nviews; ++view) {
        __syncthreads();
        if (threadIdx.x == 0) {
            bs.V = views[view];
            bs.T = brick_tile(bs.V, G, i0, j0, kbase, B::Z, B::TILE);
        }
        __syncthreads();
        const Tile T = bs.T;
        const float* yv = y + (size_t)view * G.nu * G.nv;
        if (T.ok)
            for (int q = threadIdx.x; q < T.w * T.h; q += NTHREADS) {
                const int n = T.u0 + q % T.w, m = T.v0 + q / T.w;
                tile[q] = __ldg(&yv[(size_t)m * G.nu + n]) * pixel_factor<SCALING>(bs.V, n, m);
            }
        __syncthreads();
        for (int c = warp; c < NCOLS; c += NWARP) {
            const int i = i0 + c % BX, j = j0 + c / BX;
            if (i >= G.nx || j >= G.ny) continue;
            BwdSink<SCALING> s{&bs.V, tile, T, yv, G.nu, acc_s + c * B::Z, lane, {}};
#pragma unroll
            for (int p = 0; p < KPL; ++p) s.acc[p] = 0.f;
            warp_column<VARIANT>(bs.V, G, i, j, kbase, B::RUNS, lane, &bs.ws[warp], s, err);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < B::Z * NCOLS; q += NTHREADS) {
        const int c = q / B::Z, kk = q % B::Z;
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
    __shared__ BlockSmem<VARIANT> bs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, j0;
    brick_origin(G, i0, j0);
    const int kbase = blockIdx.y * Brick<VARIANT>::Z;
    if (threadIdx.x == 0) bs.V = views[blockIdx.z];
    __syncthreads();
    CountSink s{0ull};
    for (int c = warp; c < NCOLS; c += NWARP) {
        const int i = i0 + c % BX, j = j0 + c / BX;
        if (i >= G.nx || j >= G.ny) continue;
        warp_column<VARIANT>(bs.V, G, i, j, kbase, Brick<VARIANT>::RUNS, lane, &bs.ws[warp], s, err);
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
