// siddon.cuh -- ray-driven comparator: the average over K x K rays per pixel of the line
// integral of the voxel volume, with exact path lengths through the voxel grid (Siddon's
// method in the incremental form of Amanatides and Woo). The paper compares the CVP with
// such multi-ray projectors (Sec. IV, "Siddon8"); here it serves the accuracy study, where
// the CVP values are measured against a supersampled ray integration. Not part of A.
//
// One warp per pixel: lane l traces rays l, l + 32, ... of the K x K sub-pixel grid (rays of
// one pixel visit almost the same voxels, so the lanes stay together), then the warp adds.
// Ray (a, b) through sub-pixel point (u', v') leaves the source s along
// d = w + a h + b e_3 with a = (u' - cu) / gu, b = (v' - cv) / gv (the view frame of the
// projector), so |d| = sqrt(1 + a^2 + b^2) and the solid-angle weight of the ray is |d|^-3.
#pragma once

#include "cvp_device.cuh"

namespace kct {

// Integral of the volume along p(l) = q + l d, l in [0, lmax] (q inside the grid box or on its
// boundary), in units of l.
__device__ __forceinline__ float trace_grid(const Grid& G, const float* __restrict__ vol, float qx, float qy,
                                            float qz, float dx, float dy, float dz, float lmax) {
    const float bx = G.x0 - 0.5f * G.ax, by = G.y0 - 0.5f * G.ay, bz = G.z0 - 0.5f * G.az;
    int ix = min(max((int)floorf((qx - bx) / G.ax), 0), G.nx - 1);
    int iy = min(max((int)floorf((qy - by) / G.ay), 0), G.ny - 1);
    int iz = min(max((int)floorf((qz - bz) / G.az), 0), G.nz - 1);
    const int sx = dx > 0.f ? 1 : -1, sy = dy > 0.f ? 1 : -1, sz = dz > 0.f ? 1 : -1;
    const float inf = 3.0e38f;
    const float tdx = dx != 0.f ? G.ax / fabsf(dx) : inf;
    const float tdy = dy != 0.f ? G.ay / fabsf(dy) : inf;
    const float tdz = dz != 0.f ? G.az / fabsf(dz) : inf;
    float tx = dx != 0.f ? (bx + (ix + (sx > 0)) * G.ax - qx) / dx : inf;
    float ty = dy != 0.f ? (by + (iy + (sy > 0)) * G.ay - qy) / dy : inf;
    float tz = dz != 0.f ? (bz + (iz + (sz > 0)) * G.az - qz) / dz : inf;
    float l = 0.f, acc = 0.f;
    const size_t sxy = (size_t)G.nx * G.ny;
    for (int guard = G.nx + G.ny + G.nz + 3; guard > 0 && l < lmax; --guard) {
        const float next = fminf(fminf(tx, ty), fminf(tz, lmax));
        acc = fmaf(next - l, __ldg(&vol[(size_t)iz * sxy + (size_t)iy * G.nx + ix]), acc);
        l = next;
        if (next >= lmax) break;
        if (tx <= ty && tx <= tz) {
            ix += sx;
            tx += tdx;
            if ((unsigned)ix >= (unsigned)G.nx) break;
        } else if (ty <= tz) {
            iy += sy;
            ty += tdy;
            if ((unsigned)iy >= (unsigned)G.ny) break;
        } else {
            iz += sz;
            tz += tdz;
            if ((unsigned)iz >= (unsigned)G.nz) break;
        }
    }
    return acc;
}

// line integral (mm x mm^-1) of the ray through detector point (u', v') of view V
__device__ __forceinline__ float ray_line_integral(const View& V, const Grid& G, const float* __restrict__ vol,
                                                   float a, float b) {
    const float dx = V.wx - a * V.wy, dy = V.wy + a * V.wx, dz = b;
    // entry and exit of the grid box along s + l d (slab method)
    const float lo[3] = {G.x0 - 0.5f * G.ax, G.y0 - 0.5f * G.ay, G.z0 - 0.5f * G.az};
    const float hi[3] = {lo[0] + G.nx * G.ax, lo[1] + G.ny * G.ay, lo[2] + G.nz * G.az};
    const float S[3] = {V.sx, V.sy, V.sz}, D[3] = {dx, dy, dz};
    float l0 = 0.f, l1 = 3.0e38f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (D[q] == 0.f) {
            if (S[q] <= lo[q] || S[q] >= hi[q]) return 0.f;
        } else {
            float ta = (lo[q] - S[q]) / D[q], tb = (hi[q] - S[q]) / D[q];
            if (ta > tb) { const float t = ta; ta = tb; tb = t; }
            l0 = fmaxf(l0, ta);
            l1 = fminf(l1, tb);
        }
    }
    if (!(l1 > l0)) return 0.f;
    // trace from the entry point, so that the traversal works with distances inside the box
    const float L = trace_grid(G, vol, fmaf(l0, dx, V.sx), fmaf(l0, dy, V.sy), fmaf(l0, dz, V.sz), dx, dy, dz, l1 - l0);
    return L * sqrtf(fmaf(a, a, fmaf(b, b, 1.0f)));
}

template <int WEIGHTED>
__global__ void __launch_bounds__(256) siddon_kernel(const View* __restrict__ views, Grid G,
                                                     const float* __restrict__ vol, float* __restrict__ out, int K) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long pix = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const int view = blockIdx.y;
    if (pix >= (long long)G.nu * G.nv) return;
    const int n = (int)(pix % G.nu), m = (int)(pix / G.nu);
    const View V = views[view];
    float num = 0.f, den = 0.f;
    const float inv_k = 1.0f / (float)K;
    for (int r = lane; r < K * K; r += 32) {
        const float uu = (float)n - 0.5f + ((float)(r % K) + 0.5f) * inv_k;
        const float vv = (float)m - 0.5f + ((float)(r / K) + 0.5f) * inv_k;
        const float a = (uu - V.cu) * V.igu, b = (vv - V.cv) * V.igv;
        const float line = ray_line_integral(V, G, vol, a, b);
        float w = 1.f;
        if (WEIGHTED) {
            const float d2 = fmaf(a, a, fmaf(b, b, 1.0f));
            w = 1.0f / (d2 * sqrtf(d2));
        }
        num = fmaf(w, line, num);
        den += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane == 0) out[((size_t)view * G.nv + m) * G.nu + n] = num / den;
}

}  // namespace kct
