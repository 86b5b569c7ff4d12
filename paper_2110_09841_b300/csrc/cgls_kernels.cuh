// Vector kernels of CGLS (conjugate gradients on the normal equations, the reconstruction
// that drives the projector timings of Sec. IV-A). Each CGLS step is one forward
// projection, one backprojection and the four kernels below; all of them stream their
// arrays once from HBM, so they are written as grid-stride float4 loops over a grid of a
// few blocks per SM.
//
// Reductions are deterministic: every block writes its partial sum (FP64) to a slot of a
// partials array, and the consumer kernel re-adds the partials in a fixed order. Scalars
// (alpha, beta, the residual norms) never leave the device during a step.
#pragma once

#include <cstdint>

namespace kct {

constexpr int VEC_THREADS = 256;
constexpr int VEC_MAX_BLOCKS = 2048;   // capacity of each partials array

// sum over the block; the result is valid in thread 0. `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// the sum of `n` partials, in a fixed order, returned to every thread of the block
__device__ __forceinline__ double sum_partials(const double* part, int n, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    v = sh[32];
    __syncthreads();
    return v;
}

__device__ __forceinline__ float sq4(float4 a) { return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w; }

// part[block] = sum of a[i]^2 over the block's share of [0, n)
__global__ void __launch_bounds__(VEC_THREADS) sumsq_kernel(const float* __restrict__ a, long long n,
                                                           double* __restrict__ part) {
    __shared__ double sh[33];
    const long long n4 = n >> 2, stride = (long long)gridDim.x * blockDim.x;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        acc += (double)sq4(__ldcs(a4 + i));
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
        const float t = a[4 * n4 + threadIdx.x];
        acc += (double)t * t;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// dst = sum of the partials (one block)
__global__ void store_sum_kernel(const double* __restrict__ part, int nb, double* __restrict__ dst) {
    __shared__ double sh[33];
    const double v = sum_partials(part, nb, sh);
    if (threadIdx.x == 0) *dst = v;
}

// r = b - q and part_rr[block] = sum r^2 (the residual of a warm start)
__global__ void __launch_bounds__(VEC_THREADS) residual_kernel(const float* __restrict__ b, const float* __restrict__ q,
                                                              float* __restrict__ r, long long n,
                                                              double* __restrict__ part_rr) {
    __shared__ double sh[33];
    const long long n4 = n >> 2, stride = (long long)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 bv = __ldcs(reinterpret_cast<const float4*>(b) + i);
        const float4 qv = __ldcs(reinterpret_cast<const float4*>(q) + i);
        const float4 rv = make_float4(bv.x - qv.x, bv.y - qv.y, bv.z - qv.z, bv.w - qv.w);
        reinterpret_cast<float4*>(r)[i] = rv;
        acc += (double)sq4(rv);
    }
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
        const long long i = 4 * n4 + threadIdx.x;
        const float t = b[i] - q[i];
        r[i] = t;
        acc += (double)t * t;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = acc;
}

// One half of a CGLS step, after q = A p:
//   alpha = gamma / |q|^2 (|q|^2 from part_qq);  x += alpha p;  r -= alpha q;
//   part_rr[block] = sum of the new r^2.
__global__ void __launch_bounds__(VEC_THREADS) cgls_xr_kernel(float* __restrict__ x, const float* __restrict__ p, long long nvol,
                                                             float* __restrict__ r, const float* __restrict__ q, long long nproj,
                                                             const double* __restrict__ part_qq, int nb,
                                                             const double* __restrict__ gamma,
                                                             double* __restrict__ part_rr) {
    __shared__ double sh[33];
    const double qq = sum_partials(part_qq, nb, sh);
    const float alpha = qq > 0.0 ? (float)(*gamma / qq) : 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long v4 = nvol >> 2;
    for (long long i = t0; i < v4; i += stride) {
        float4 xv = reinterpret_cast<float4*>(x)[i];
        const float4 pv = __ldcs(reinterpret_cast<const float4*>(p) + i);
        xv.x = fmaf(alpha, pv.x, xv.x);
        xv.y = fmaf(alpha, pv.y, xv.y);
        xv.z = fmaf(alpha, pv.z, xv.z);
        xv.w = fmaf(alpha, pv.w, xv.w);
        reinterpret_cast<float4*>(x)[i] = xv;
    }
    if (blockIdx.x == 0 && threadIdx.x < (nvol & 3)) {
        const long long i = 4 * v4 + threadIdx.x;
        x[i] = fmaf(alpha, p[i], x[i]);
    }
    const long long p4 = nproj >> 2;
    double acc = 0.0;
    for (long long i = t0; i < p4; i += stride) {
        float4 rv = reinterpret_cast<float4*>(r)[i];
        const float4 qv = __ldcs(reinterpret_cast<const float4*>(q) + i);
        rv.x = fmaf(-alpha, qv.x, rv.x);
        rv.y = fmaf(-alpha, qv.y, rv.y);
        rv.z = fmaf(-alpha, qv.z, rv.z);
        rv.w = fmaf(-alpha, qv.w, rv.w);
        reinterpret_cast<float4*>(r)[i] = rv;
        acc += (double)sq4(rv);
    }
    if (blockIdx.x == 0 && threadIdx.x < (nproj & 3)) {
        const long long i = 4 * p4 + threadIdx.x;
        const float t = fmaf(-alpha, q[i], r[i]);
        r[i] = t;
        acc += (double)t * t;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = acc;
}

// Per-step scalars kept on the device (FP64).
struct CglsScalars {
    double gamma[2];   // |s|^2 of the current and the next step (ping-pong)
    double atb2;       // |A^T b|^2
    double bb2;        // |b|^2
    double normal;     // |A^T r| / |A^T b| after the step
    double data;       // |r| / |b| after the step
    double pad[2];
};

// Other half of the step, after s = A^T r:
//   gamma' = |s|^2 (from part_ss); beta = gamma' / gamma (0 at the start); p = s + beta p;
//   block 0 stores gamma' and the two residuals (|r|^2 from part_rr).
__global__ void __launch_bounds__(VEC_THREADS) cgls_p_kernel(const float* __restrict__ s, float* __restrict__ p, long long nvol,
                                                            const double* __restrict__ part_ss,
                                                            const double* __restrict__ part_rr, int nb,
                                                            const double* __restrict__ gamma_old,
                                                            double* __restrict__ gamma_new,
                                                            CglsScalars* __restrict__ sc) {
    __shared__ double sh[33];
    const double ss = sum_partials(part_ss, nb, sh);
    const double go = gamma_old ? *gamma_old : 0.0;
    const float beta = go > 0.0 ? (float)(ss / go) : 0.0f;
    // at the start p holds whatever the workspace held (possibly NaN): p = s without reading it
    const bool keep = beta != 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long v4 = nvol >> 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < v4; i += stride) {
        const float4 sv = __ldcs(reinterpret_cast<const float4*>(s) + i);
        float4 pv = sv;
        if (keep) {
            pv = reinterpret_cast<float4*>(p)[i];
            pv.x = fmaf(beta, pv.x, sv.x);
            pv.y = fmaf(beta, pv.y, sv.y);
            pv.z = fmaf(beta, pv.z, sv.z);
            pv.w = fmaf(beta, pv.w, sv.w);
        }
        reinterpret_cast<float4*>(p)[i] = pv;
    }
    if (blockIdx.x == 0 && threadIdx.x < (nvol & 3)) {
        const long long i = 4 * v4 + threadIdx.x;
        p[i] = keep ? fmaf(beta, p[i], s[i]) : s[i];
    }
    if (blockIdx.x == 0) {
        const double rr = sum_partials(part_rr, nb, sh);
        if (threadIdx.x == 0) {
            *gamma_new = ss;
            sc->normal = sc->atb2 > 0.0 ? sqrt(ss / sc->atb2) : 0.0;
            sc->data = sc->bb2 > 0.0 ? sqrt(rr / sc->bb2) : 0.0;
        }
    }
}

}  // namespace kct
