// cvp_kernels.cuh -- CUDA kernels of the cutting voxel projector (sm_103a).
//
// Forward projection (Eq. cvpsu then the pixel factor) and its adjoint. Both enumerate
// the same voxel-pixel pairs with the same device function, column by column (all voxels
// of a column (i, j) share the column cuts of Sec. III-A), so <A x, y> = <x, A^T y> holds up
// to float rounding.
#pragma once

#include "cvp_device.cuh"

namespace kct {

// ---------------------------------------------------------------------------------------
// forward: scatter mu * W * F into the projections with float atomics
// ---------------------------------------------------------------------------------------

template <int SCALING>
struct FwdEmit {
    const View& V;
    const float* __restrict__ vol;
    float* __restrict__ proj;
    int nx, ny, nu, i, j;
    float mu;
    __device__ __forceinline__ void begin(int k) { mu = __ldg(&vol[((size_t)k * ny + j) * nx + i]); }
    __device__ __forceinline__ void end(int) {}
    __device__ __forceinline__ void pair(int, int n, int m, float W) {
        if (mu != 0.f) atomicAdd(&proj[(size_t)m * nu + n], mu * W * pixel_factor<SCALING>(V, n, m));
    }
};

template <int VARIANT, int SCALING>
__global__ void __launch_bounds__(128) fwd_atomic_kernel(const View* __restrict__ views, Grid G,
                                                         const float* __restrict__ vol, float* __restrict__ proj,
                                                         int kchunk, int* err) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= G.nx * G.ny) return;
    const int i = col % G.nx, j = col / G.nx;
    const int view = blockIdx.y;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, G.nz);
    const View V = views[view];
    FwdEmit<SCALING> e{V, vol, proj + (size_t)view * G.nu * G.nv, G.nx, G.ny, G.nu, i, j, 0.f};
    column_pairs<VARIANT>(V, G, i, j, k0, k1, e, err);
}

// ---------------------------------------------------------------------------------------
// adjoint: gather W * F * y over all views, one thread per voxel, no atomics
// ---------------------------------------------------------------------------------------

template <int SCALING>
struct BwdEmit {
    const View& V;
    const float* __restrict__ y;
    int nu;
    float acc;
    __device__ __forceinline__ void begin(int) {}
    __device__ __forceinline__ void end(int) {}
    __device__ __forceinline__ void pair(int, int n, int m, float W) {
        acc = fmaf(W * pixel_factor<SCALING>(V, n, m), __ldg(&y[(size_t)m * nu + n]), acc);
    }
};

template <int VARIANT, int SCALING>
__global__ void __launch_bounds__(128) bwd_gather_kernel(const View* __restrict__ views, Grid G,
                                                         const float* __restrict__ proj, float* __restrict__ vol,
                                                         int accumulate, int* err) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nvox = (long)G.nx * G.ny * G.nz;
    if (idx >= nvox) return;
    const int i = (int)(idx % G.nx);
    const int j = (int)((idx / G.nx) % G.ny);
    const int k = (int)(idx / ((long)G.nx * G.ny));
    float acc = 0.f;
    for (int view = 0; view < G.nviews; ++view) {
        const View V = views[view];
        BwdEmit<SCALING> e{V, proj + (size_t)view * G.nu * G.nv, G.nu, 0.f};
        column_pairs<VARIANT>(V, G, i, j, k, k + 1, e, err);
        acc += e.acc;
    }
    vol[idx] = accumulate ? vol[idx] + acc : acc;
}

// ---------------------------------------------------------------------------------------
// number of nonzero pairs
// ---------------------------------------------------------------------------------------

struct CountEmit {
    unsigned long long n;
    __device__ __forceinline__ void begin(int) {}
    __device__ __forceinline__ void end(int) {}
    __device__ __forceinline__ void pair(int, int, int, float W) { n += (W > 0.f) ? 1ull : 0ull; }
};

template <int VARIANT>
__global__ void __launch_bounds__(128) count_kernel(const View* __restrict__ views, Grid G, int kchunk,
                                                   unsigned long long* count, int* err) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    CountEmit e{0ull};
    if (col < G.nx * G.ny) {
        const int i = col % G.nx, j = col / G.nx;
        const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, G.nz);
        const View V = views[blockIdx.y];
        column_pairs<VARIANT>(V, G, i, j, k0, k1, e, err);
    }
    unsigned long long v = e.n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(count, v);
}

// ---------------------------------------------------------------------------------------
// pixel factors of every view
// ---------------------------------------------------------------------------------------

template <int SCALING>
__global__ void factor_kernel(const View* __restrict__ views, Grid G, float* __restrict__ out) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)G.nu * G.nv) return;
    const View V = views[blockIdx.y];
    const int n = (int)(q % G.nu), m = (int)(q / G.nu);
    out[(size_t)blockIdx.y * G.nu * G.nv + q] = pixel_factor<SCALING>(V, n, m);
}

}  // namespace kct
