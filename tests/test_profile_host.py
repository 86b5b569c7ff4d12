"""Host check of the near-exact kernels' column-cut moments (the depth profile of H_n).

The moments (1, t', t'^2, xi', t' xi') of H_n ∩ {t' < tau} that a row plane crossing a
voxel face needs (Sec. III-C, the cut of the voxel with the pixel's rays) are evaluated in
the kernels from a per-column depth profile of the convex polygon H_n. The same helpers
compile for the host; here they run on voxel bases (rotated squares) clipped by two column
lines, and are compared with the polygon clipped at tau in double precision and summed by
Green's theorem. No GPU: the helpers are built with nvcc as host code.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2110_09841_b300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include <random>
#include "cvp_device.cuh"
using namespace kct;

// the polygon clipped to t' < tau (one pass of Sutherland-Hodgman), then Green's theorem
static void clipped_moments(const float* pt, const float* px, int nv, double tau, double out[5]) {
    double ct[32], cx[32];
    int n = 0;
    for (int e = 0; e < nv; ++e) {
        const int f = (e + 1) % nv;
        const double at = pt[e], ax = px[e], bt = pt[f], bx = px[f];
        const bool ain = at < tau, bin = bt < tau;
        if (ain) { ct[n] = at; cx[n] = ax; ++n; }
        if (ain != bin) {
            const double s = (tau - at) / (bt - at);
            ct[n] = at + s * (bt - at); cx[n] = ax + s * (bx - ax); ++n;
        }
    }
    double a = 0, t = 0, x = 0, tt = 0, tx = 0;
    for (int e = 0; e < n; ++e) {
        const int f = (e + 1) % n;
        const double p = ct[e], q = cx[e], r = ct[f], s = cx[f], c = p * s - r * q;
        a += c; t += c * (p + r); x += c * (q + s);
        tt += c * (p * p + p * r + r * r);
        tx += c * (2 * p * q + p * s + r * q + 2 * r * s);
    }
    out[0] = a / 2; out[1] = t / 6; out[2] = tt / 12; out[3] = x / 6; out[4] = tx / 24;
}

int main() {
    std::mt19937 rng(20211019);
    std::uniform_real_distribution<float> U(0.f, 1.f);
    double worst = 0.0;
    long cases = 0, bad_layout = 0;
    int maxK = 0;
    for (int it = 0; it < 40000; ++it) {
        View V{};
        // axis-aligned views (edges parallel to the depth axis) and random angles
        const float ang = (it % 7 == 0) ? 0.f : (it % 7 == 1 ? 1.5707963f : U(rng) * 6.2831853f);
        const float hx = 0.5f * (0.2f + U(rng)), hy = 0.5f * (0.2f + U(rng));
        const float c = cosf(ang), s = sinf(ang);
        const float lx[4] = {-hx, hx, hx, -hx}, ly[4] = {-hy, -hy, hy, hy};
        for (int e = 0; e < 4; ++e) { V.sq_t[e] = c * lx[e] - s * ly[e]; V.sq_x[e] = s * lx[e] + c * ly[e]; }
        auto line = [&](float sign) {
            const float k = 0.3f * (U(rng) - 0.5f), x0 = (U(rng) - 0.5f) * 1.2f;
            return Line{-k * sign, sign, x0 * sign};
        };
        const Line l0 = (it % 5 == 0) ? line_none() : line(1.f), l1 = (it % 3 == 0) ? line_none() : line(-1.f);
        float pt[8], px[8];
        const int nv = clip_square(V, l0, l1, pt, px);
        alignas(16) float st[KCT_IV + 1];
        float4 a[KCT_IV], b[KCT_IV];
        float2 m[KCT_IV];
        float full[5], tlo, thi;
        const int K = depth_profile(pt, px, nv, st, a, b, m, full, tlo, thi);
        maxK = K > maxK ? K : maxK;
        for (int j = 0; j < KCT_IV + 1; ++j) {
            if (j >= K && st[j] < 1e38f) ++bad_layout;
            if (j > 0 && j < K && !(st[j] > st[j - 1])) ++bad_layout;
        }
        if (nv < 3) continue;
        double whole[5];
        clipped_moments(pt, px, nv, 1e30, whole);
        if (whole[0] <= 1e-6) continue;
        double ts = 0, xs = 0;
        for (int e = 0; e < nv; ++e) { ts = fmax(ts, fabs(pt[e])); xs = fmax(xs, fabs(px[e])); }
        for (int q = 0; q < 10; ++q) {
            // whole polygon, interior depths, depths just above the lowest vertex
            const float tau = q == 0 ? thi : tlo + (thi - tlo) * (q < 8 ? U(rng) : 1e-4f * U(rng));
            double ref[5];
            clipped_moments(pt, px, nv, tau, ref);
            float P[5];
            if (q == 0) for (int k = 0; k < 5; ++k) P[k] = full[k];
            else profile_cut(st, a, b, m, tau, P[0], P[1], P[2], P[3], P[4]);
            // relative to the cut's own size (floored at 1e-6 of the polygon)
            const double cs = fabs(ref[0]) + 1e-6 * whole[0];
            const double scale[5] = {cs, cs * ts, cs * ts * ts, cs * xs, cs * ts * xs};
            for (int k = 0; k < 5; ++k) worst = fmax(worst, fabs(P[k] - ref[k]) / scale[k]);
            ++cases;
        }
    }
    printf("%ld %d %ld %.6e\n", cases, maxK, bad_layout, worst);
    return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_profile_cut_matches_exact_clipping(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "profile_host.cu"
    exe = tmp_path / "profile_host"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(src)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    cases, max_k, bad_layout, worst = int(out[0]), int(out[1]), int(out[2]), float(out[3])
    assert cases > 200000
    assert max_k <= 7 and bad_layout == 0
    # float arithmetic on coordinates of O(1): a few 1e-5 of the cut's own moments at worst
    assert worst < 2e-4, worst
