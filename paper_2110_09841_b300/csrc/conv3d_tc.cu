// conv3d_tc.cu -- 3x3x3 convolutions (stride 1, zero padding 1) on the 5th-generation tensor
// cores of sm_103a: BF16 operands staged in shared memory by TMA, FP32 accumulators in
// tensor memory (tcgen05.mma issued by one thread), read back with tcgen05.ld.
//
// These are the contractions of the 3D U-Net that maps a backprojection to a CGLS warm
// start. Layouts are channels-last: activations [n][z][y][x][c] bf16, weights
// [cout][tap][cin] bf16 with tap = (dz * 3 + dy) * 3 + dx.
//
// Forward / input gradient (kct_conv3d_fwd): implicit GEMM with M = 128 output voxels (a
// WB x HB patch of one z-slice), N = cout, K = 27 taps x cin. For every (tap, channel chunk)
// TMA loads the shifted input patch (out-of-range voxels are filled with zeros, which is
// the padding) and the weight slice; the input gradient is the same kernel with the
// weights flipped in the taps and transposed in the channels.
//
// Weight gradient (kct_conv3d_wgrad): dW[co][t][ci] = sum_v g[v][co] x[v + t][ci], a GEMM
// with K = voxels. Operands are channels-first copies (g^T [co][v], and x^T shifted along x
// by -1, 0, +1) so that both tiles are K-major. Taps are stacked along M: one A tile holds
// 128 / cin taps of x (cin rows each), B is the g^T tile (N = cout), so one MMA yields dW^T
// for several taps; a block keeps a few tap groups in TMEM, loads each g^T tile once for all
// of them, and its voxel range is reduced into dW with float atomics.
//
// Every wait on an mbarrier is bounded: on timeout the kernel sets an error word, waits
// (bounded) for its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>

#include "kct.h"
#include "kct_conv.h"

namespace {

thread_local std::string g_conv_error;

int conv_fail(int status, const std::string& why) {
    g_conv_error = why;
    return status;
}

// ------------------------------------------------------------------------------------------
// PTX wrappers
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // a pipeline wait longer than 1 s is a failure

// true if the phase with the given parity completed within the time bound
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, kind::f16 (BF16 in, FP32 accumulate)
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on `bar` once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 consecutive FP32 columns: thread t gets lane (lane_base + t), columns col..col+15
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor of a K-major tile whose rows are `row_bytes` (32, 64 or
// 128) long and swizzled by TMA in the same span: 8-row core groups `8 * row_bytes` apart.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t row_bytes) {
    const uint64_t layout = row_bytes == 128 ? 2ull : row_bytes == 64 ? 4ull : 6ull;   // SW128 / SW64 / SW32
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);                 // start address
    d |= (uint64_t)1 << 16;                                   // leading byte offset (unused when swizzled)
    d |= (uint64_t)(((8u * row_bytes) & 0x3FFFFu) >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;                                   // descriptor version
    d |= layout << 61;
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// ------------------------------------------------------------------------------------------
// Forward (and input-gradient) kernel
// ------------------------------------------------------------------------------------------

constexpr int kStages = 4;
constexpr int kThreads = 192;            // warp 0 TMA, warp 1 MMA + TMEM owner, warps 2..5 epilogue

struct ConvDims {
    int n, d, h, w, cin, cout;
    int wb, hb;                          // output patch of a tile: wb x hb voxels of one slice (= 128)
    int tiles_x, tiles_y;
};

template <int KC, int COUT>
struct FwdCfg {
    static constexpr int A_BYTES = 128 * KC * 2;
    static constexpr int B_BYTES = COUT * KC * 2;
    static constexpr int STAGE = ((A_BYTES + B_BYTES) + 1023) / 1024 * 1024;
    static constexpr int TMEM_COLS = COUT <= 32 ? 32 : COUT <= 64 ? 64 : 128;
    static constexpr int SMEM = 1024 + kStages * STAGE + 1024;   // alignment slack + stages + barriers
};

template <int KC, int COUT>
__global__ void __launch_bounds__(kThreads, 1) conv_fwd_kernel(const __grid_constant__ CUtensorMap tm_x,
                                                               const __grid_constant__ CUtensorMap tm_w, ConvDims D,
                                                               const float* __restrict__ bias,
                                                               __nv_bfloat16* __restrict__ y, int relu, int* err) {
    using C = FwdCfg<KC, COUT>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + kStages * C::STAGE);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int t = blockIdx.x;
    const int tx = t % D.tiles_x; t /= D.tiles_x;
    const int ty = t % D.tiles_y; t /= D.tiles_y;
    const int z = t % D.d;
    const int nb = t / D.d;
    const int x0 = tx * D.wb, y0 = ty * D.hb;
    const int chunks = D.cin / KC;
    const int iters = 27 * chunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            bool ok = true;
            for (int it = 0; it < iters && ok; ++it) {
                const int s = it % kStages;
                const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
                const int tap = it / chunks, ch = it % chunks;
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                uint8_t* a = smem + s * C::STAGE;
                uint8_t* b = a + C::A_BYTES;
                mbar_expect_tx(&full[s], C::A_BYTES + C::B_BYTES);
                tma_load_5d(a, &tm_x, ch * KC, x0 + dx - 1, y0 + dy - 1, z + dz - 1, nb, &full[s]);
                tma_load_2d(b, &tm_w, tap * D.cin + ch * KC, 0, &full[s]);
                ++issued;
            }
            if (!ok) {
                atomicExch(err, 1);
                // let the copies already in flight land before the block exits
                for (int it = issued - kStages < 0 ? 0 : issued - kStages; it < issued; ++it)
                    mbar_wait(&full[it % kStages], (uint32_t)(it / kStages) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, COUT);
            bool ok = true;
            for (int it = 0; it < iters; ++it) {
                const int s = it % kStages;
                const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                if (!mbar_wait(&full[s], ph)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a = smem_u32(smem + s * C::STAGE);
                const uint32_t b = a + C::A_BYTES;
#pragma unroll
                for (int k = 0; k < KC / 16; ++k)
                    umma_bf16(tmem, kmajor_desc(a + 32 * k, KC * 2), kmajor_desc(b + 32 * k, KC * 2), idesc,
                              (it > 0 || k > 0) ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            if (!ok) atomicExch(err, 1);
            umma_commit(acc_full);       // also fires after a failed wait: nothing then is pending
        }
    } else {
        // epilogue: TMEM lanes 32 * (warp % 4) .. + 31 are output voxels of the tile
        const int row = 32 * (warp & 3) + lane;
        const bool ok = mbar_wait(acc_full, 0);
        tc_fence_after();
        if (!ok) {
            if (lane == 0) atomicExch(err, 1);
        } else {
            const int xv = x0 + row % D.wb, yv = y0 + row / D.wb;
            __nv_bfloat16* out = y + ((((size_t)nb * D.d + z) * D.h + yv) * D.w + xv) * COUT;
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    v[q] += bias ? __ldg(&bias[c0 + q]) : 0.f;
                    if (relu) v[q] = fmaxf(v[q], 0.f);
                }
                uint4 p0, p1;
                p0.x = pack_bf16(v[0], v[1]);
                p0.y = pack_bf16(v[2], v[3]);
                p0.z = pack_bf16(v[4], v[5]);
                p0.w = pack_bf16(v[6], v[7]);
                p1.x = pack_bf16(v[8], v[9]);
                p1.y = pack_bf16(v[10], v[11]);
                p1.z = pack_bf16(v[12], v[13]);
                p1.w = pack_bf16(v[14], v[15]);
                reinterpret_cast<uint4*>(out + c0)[0] = p0;
                reinterpret_cast<uint4*>(out + c0)[1] = p1;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// ------------------------------------------------------------------------------------------
// Weight-gradient kernel
// ------------------------------------------------------------------------------------------

struct WgradDims {
    int n, d, h, w, cin, cout;
    int kb;                              // voxels of one K chunk (a row segment along x)
    int chunks_x;                        // w / kb
    long long nchunks;                   // n * d * h * chunks_x
    int tap_sets;                        // blocks along the taps (each takes up to GMAX tap groups)
    int splits;                          // voxel splits (gridDim.x = tap_sets * splits)
};

constexpr int kWgStages = 2;

constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int pow2_at_least(int v) { return v <= 32 ? 32 : v <= 64 ? 64 : v <= 128 ? 128 : v <= 256 ? 256 : 512; }

// Taps are stacked along M: an A tile holds P = 128 / CI taps of x (CI rows each), so one MMA
// gives dW^T for P taps at once (M = 128 rows of (tap, ci), N = CO columns of cout).
template <int KB, int CI, int CO>
struct WgCfg {
    static constexpr int P = 128 / CI;                         // taps per A tile
    static constexpr int GROUPS = (27 + P - 1) / P;            // tap groups in all
    static constexpr int A_BYTES = 128 * KB * 2;
    static constexpr int B_BYTES = CO * KB * 2;
    static constexpr int GMAX = cmin(cmin(GROUPS, 512 / CO), (96 * 1024 - B_BYTES) / A_BYTES);   // groups per block
    static constexpr int STAGE = ((GMAX * A_BYTES + B_BYTES) + 1023) / 1024 * 1024;
    static constexpr int TMEM_COLS = pow2_at_least(GMAX * CO);
    static constexpr int SMEM = 1024 + kWgStages * STAGE + 1024;
};

template <int KB, int CI, int CO>
__global__ void __launch_bounds__(kThreads, 1) conv_wgrad_kernel(const __grid_constant__ CUtensorMap tm_g,
                                                                 const __grid_constant__ CUtensorMap tm_x0,
                                                                 const __grid_constant__ CUtensorMap tm_x1,
                                                                 const __grid_constant__ CUtensorMap tm_x2, WgradDims D,
                                                                 float* __restrict__ gw, int* err) {
    using C = WgCfg<KB, CI, CO>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + kWgStages * C::STAGE);
    uint64_t* empty = full + kWgStages;
    uint64_t* acc_full = empty + kWgStages;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int set = blockIdx.x % D.tap_sets, split = blockIdx.x / D.tap_sets;
    const int g0 = set * C::GMAX;                              // first tap group of this block
    const int ng = min(C::GMAX, C::GROUPS - g0);
    const int tap0 = g0 * C::P;
    const int ntap = min(ng * C::P, 27 - tap0);                // taps of this block
    const long long c_begin = D.nchunks * split / D.splits, c_end = D.nchunks * (split + 1) / D.splits;
    const long long iters = c_end - c_begin;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long long issued = 0;
            bool ok = true;
            const uint32_t bytes = C::B_BYTES + (uint32_t)ntap * CI * KB * 2;
            for (long long it = 0; it < iters; ++it) {
                const int s = (int)(it % kWgStages);
                const uint32_t ph = (uint32_t)(it / kWgStages) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
                long long c = c_begin + it;
                const int cx = (int)(c % D.chunks_x);
                c /= D.chunks_x;
                const int yv = (int)(c % D.h);
                c /= D.h;
                const int zv = (int)(c % D.d);
                const int nb = (int)(c / D.d);
                uint8_t* b = smem + s * C::STAGE;
                uint8_t* a = b + C::B_BYTES;
                mbar_expect_tx(&full[s], bytes);
                // g^T [n][co][z][y][x]: dims (x, y, z, co, n), CO rows
                tma_load_5d(b, &tm_g, cx * KB, yv, zv, 0, nb, &full[s]);
                for (int j = 0; j < ntap; ++j) {
                    const int tap = tap0 + j;
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                    const CUtensorMap* tx = dx == 0 ? &tm_x0 : dx == 1 ? &tm_x1 : &tm_x2;
                    uint8_t* dst = a + (j / C::P) * C::A_BYTES + (j % C::P) * CI * KB * 2;
                    tma_load_5d(dst, tx, cx * KB, yv + dy - 1, zv + dz - 1, 0, nb, &full[s]);
                }
                ++issued;
            }
            if (!ok) {
                atomicExch(err, 1);
                for (long long it = issued - kWgStages < 0 ? 0 : issued - kWgStages; it < issued; ++it)
                    mbar_wait(&full[it % kWgStages], (uint32_t)(it / kWgStages) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, CO);
            bool ok = true;
            for (long long it = 0; it < iters; ++it) {
                const int s = (int)(it % kWgStages);
                const uint32_t ph = (uint32_t)(it / kWgStages) & 1u;
                if (!mbar_wait(&full[s], ph)) { ok = false; break; }
                tc_fence_after();
                const uint32_t b = smem_u32(smem + s * C::STAGE);
                const uint32_t a = b + C::B_BYTES;
                for (int g = 0; g < ng; ++g) {
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k)
                        umma_bf16(tmem + (uint32_t)(g * CO), kmajor_desc(a + g * C::A_BYTES + 32 * k, KB * 2),
                                  kmajor_desc(b + 32 * k, KB * 2), idesc, (it > 0 || k > 0) ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            if (!ok) atomicExch(err, 1);
            umma_commit(acc_full);
        }
    } else {
        // TMEM lane r of group g holds tap tap0 + g * P + r / CI, input channel r % CI
        const int row = 32 * (warp & 3) + lane;
        const bool ok = mbar_wait(acc_full, 0);
        tc_fence_after();
        if (!ok) {
            if (lane == 0) atomicExch(err, 1);
        } else if (iters > 0) {
            for (int g = 0; g < ng; ++g) {
                const int j = g * C::P + row / CI;
                const bool valid = row / CI < C::P && j < ntap;
                const int ci = row % CI;
#pragma unroll
                for (int c0 = 0; c0 < CO; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(g * CO + c0), v);
                    if (valid) {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (c0 + q < D.cout) atomicAdd(gw + ((size_t)(c0 + q) * 27 + (tap0 + j)) * D.cin + ci, v[q]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

CUtensorMapSwizzle swizzle_for(int row_bytes) {
    return row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                            : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

// bf16 tensor map: dims[0] innermost; strides in bytes for dims 1..rank-1
int make_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
             const uint32_t* box, int row_bytes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return conv_fail(KCT_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    cuuint64_t gd[5], gs[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) gs[i] = strides[i];
    }
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(row_bytes), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return conv_fail(KCT_ERR_INVALID_ARG, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return KCT_OK;
}

template <class K>
cudaError_t allow_smem(K kernel, int bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Dynamic shared memory of a launch: at least the kernel's own need, and enough that no more
// CTAs share an SM than its tensor memory (512 columns) can hold at once.
int smem_request(int need, int tmem_cols) {
    const int max_ctas = 512 / tmem_cols;
    const int floor_bytes = max_ctas >= 8 ? 0 : (227 * 1024) / max_ctas - 2048;
    return need > floor_bytes ? need : floor_bytes;
}

template <int KC, int COUT>
int launch_fwd(const CUtensorMap& tx, const CUtensorMap& tw, const ConvDims& D, const float* bias, void* y, int relu,
               int* err, cudaStream_t st) {
    using C = FwdCfg<KC, COUT>;
    const int smem = smem_request(C::SMEM, C::TMEM_COLS);
    cudaError_t e = allow_smem(conv_fwd_kernel<KC, COUT>, smem);
    if (e != cudaSuccess) return conv_fail(KCT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    const long long tiles = (long long)D.n * D.d * D.tiles_y * D.tiles_x;
    conv_fwd_kernel<KC, COUT><<<(unsigned)tiles, kThreads, smem, st>>>(tx, tw, D, bias, (__nv_bfloat16*)y, relu, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return conv_fail(KCT_ERR_CUDA, std::string("conv forward launch: ") + cudaGetErrorString(e));
    return KCT_OK;
}

template <int KC>
int dispatch_fwd_cout(const CUtensorMap& tx, const CUtensorMap& tw, const ConvDims& D, const float* bias, void* y,
                      int relu, int* err, cudaStream_t st) {
    switch (D.cout) {
        case 16: return launch_fwd<KC, 16>(tx, tw, D, bias, y, relu, err, st);
        case 32: return launch_fwd<KC, 32>(tx, tw, D, bias, y, relu, err, st);
        case 48: return launch_fwd<KC, 48>(tx, tw, D, bias, y, relu, err, st);
        case 64: return launch_fwd<KC, 64>(tx, tw, D, bias, y, relu, err, st);
        case 96: return launch_fwd<KC, 96>(tx, tw, D, bias, y, relu, err, st);
        case 128: return launch_fwd<KC, 128>(tx, tw, D, bias, y, relu, err, st);
    }
    return conv_fail(KCT_ERR_UNSUPPORTED, "cout must be 16, 32, 48, 64, 96 or 128");
}

template <int KB, int CI, int CO>
int launch_wgrad(const CUtensorMap& tg, const CUtensorMap* tx, WgradDims D, float* gw, int* err, int sms,
                 cudaStream_t st) {
    using C = WgCfg<KB, CI, CO>;
    D.tap_sets = (C::GROUPS + C::GMAX - 1) / C::GMAX;
    long long splits = (2LL * sms + D.tap_sets - 1) / D.tap_sets;
    if (splits > D.nchunks) splits = D.nchunks;
    if (splits < 1) splits = 1;
    D.splits = (int)splits;
    const int smem = smem_request(C::SMEM, C::TMEM_COLS);
    cudaError_t e = allow_smem(conv_wgrad_kernel<KB, CI, CO>, smem);
    if (e != cudaSuccess) return conv_fail(KCT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    conv_wgrad_kernel<KB, CI, CO><<<(unsigned)(D.tap_sets * D.splits), kThreads, smem, st>>>(tg, tx[0], tx[1], tx[2],
                                                                                           D, gw, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return conv_fail(KCT_ERR_CUDA, std::string("conv weight-gradient launch: ") + cudaGetErrorString(e));
    return KCT_OK;
}

template <int KB, int CI>
int dispatch_wgrad_co(const CUtensorMap& tg, const CUtensorMap* tx, const WgradDims& D, float* gw, int* err, int sms,
                      cudaStream_t st) {
    switch (D.cout) {
        case 16: return launch_wgrad<KB, CI, 16>(tg, tx, D, gw, err, sms, st);
        case 32: return launch_wgrad<KB, CI, 32>(tg, tx, D, gw, err, sms, st);
        case 48: return launch_wgrad<KB, CI, 48>(tg, tx, D, gw, err, sms, st);
        case 64: return launch_wgrad<KB, CI, 64>(tg, tx, D, gw, err, sms, st);
        case 96: return launch_wgrad<KB, CI, 96>(tg, tx, D, gw, err, sms, st);
        case 128: return launch_wgrad<KB, CI, 128>(tg, tx, D, gw, err, sms, st);
    }
    return conv_fail(KCT_ERR_UNSUPPORTED, "cout must be 16, 32, 48, 64, 96 or 128");
}

template <int KB>
int dispatch_wgrad_ci(const CUtensorMap& tg, const CUtensorMap* tx, const WgradDims& D, float* gw, int* err, int sms,
                      cudaStream_t st) {
    switch (D.cin) {
        case 16: return dispatch_wgrad_co<KB, 16>(tg, tx, D, gw, err, sms, st);
        case 32: return dispatch_wgrad_co<KB, 32>(tg, tx, D, gw, err, sms, st);
        case 48: return dispatch_wgrad_co<KB, 48>(tg, tx, D, gw, err, sms, st);
        case 64: return dispatch_wgrad_co<KB, 64>(tg, tx, D, gw, err, sms, st);
        case 96: return dispatch_wgrad_co<KB, 96>(tg, tx, D, gw, err, sms, st);
        case 128: return dispatch_wgrad_co<KB, 128>(tg, tx, D, gw, err, sms, st);
    }
    return conv_fail(KCT_ERR_UNSUPPORTED, "cin must be 16, 32, 48, 64, 96 or 128");
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int check_desc(const kct_conv_desc* c) {
    if (!c) return conv_fail(KCT_ERR_INVALID_ARG, "null descriptor");
    if (c->n < 1 || c->d < 1 || c->h < 1 || c->w < 1) return conv_fail(KCT_ERR_INVALID_ARG, "sizes must be positive");
    if (c->cin % 16 || c->cout % 16 || c->cin < 16 || c->cout < 16 || c->cin > 128 || c->cout > 128)
        return conv_fail(KCT_ERR_UNSUPPORTED, "channels must be multiples of 16 in [16, 128]");
    if (c->w < 16 || c->w % 16) return conv_fail(KCT_ERR_UNSUPPORTED, "w must be a multiple of 16");
    return KCT_OK;
}

}  // namespace

extern "C" {

const char* kct_conv_last_error(void) { return g_conv_error.c_str(); }

int kct_conv3d_fwd(const kct_conv_desc* c, const void* d_x, const void* d_w, const float* d_bias, void* d_y,
                   int32_t relu, int32_t* d_err, void* stream) {
    int s = check_desc(c);
    if (s != KCT_OK) return s;
    if (!d_x || !d_w || !d_y || !d_err) return conv_fail(KCT_ERR_INVALID_ARG, "null pointer");
    if (!aligned16(d_x) || !aligned16(d_w) || !aligned16(d_y)) return conv_fail(KCT_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    ConvDims D;
    D.n = c->n; D.d = c->d; D.h = c->h; D.w = c->w; D.cin = c->cin; D.cout = c->cout;
    // the widest divisor of 128 that also divides w (16 always qualifies: w % 16 == 0)
    D.wb = c->w < 128 ? c->w : 128;
    while (128 % D.wb || c->w % D.wb) D.wb -= 16;
    D.hb = 128 / D.wb;
    if (c->h % D.hb) return conv_fail(KCT_ERR_UNSUPPORTED, "h must be a multiple of 128 / min(w, 128)");
    D.tiles_x = c->w / D.wb;
    D.tiles_y = c->h / D.hb;
    const int kc = c->cin % 64 == 0 ? 64 : c->cin % 32 == 0 ? 32 : 16;
    // x: dims (c, x, y, z, n)
    const uint64_t xd[5] = {(uint64_t)c->cin, (uint64_t)c->w, (uint64_t)c->h, (uint64_t)c->d, (uint64_t)c->n};
    const uint64_t xs[4] = {(uint64_t)c->cin * 2, (uint64_t)c->cin * 2 * c->w, (uint64_t)c->cin * 2 * c->w * c->h,
                            (uint64_t)c->cin * 2 * c->w * c->h * c->d};
    const uint32_t xb[5] = {(uint32_t)kc, (uint32_t)D.wb, (uint32_t)D.hb, 1, 1};
    // w: dims (27 cin, cout)
    const uint64_t wd[2] = {(uint64_t)27 * c->cin, (uint64_t)c->cout};
    const uint64_t ws[1] = {(uint64_t)27 * c->cin * 2};
    const uint32_t wbx[2] = {(uint32_t)kc, (uint32_t)c->cout};
    CUtensorMap tx, tw;
    if ((s = make_map(&tx, d_x, 5, xd, xs, xb, kc * 2)) != KCT_OK) return s;
    if ((s = make_map(&tw, d_w, 2, wd, ws, wbx, kc * 2)) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (kc == 64) return dispatch_fwd_cout<64>(tx, tw, D, d_bias, d_y, relu, d_err, st);
    if (kc == 32) return dispatch_fwd_cout<32>(tx, tw, D, d_bias, d_y, relu, d_err, st);
    return dispatch_fwd_cout<16>(tx, tw, D, d_bias, d_y, relu, d_err, st);
}

int kct_conv3d_wgrad(const kct_conv_desc* c, const void* d_gt, const void* d_xt0, const void* d_xt1, const void* d_xt2,
                     float* d_gw, int32_t* d_err, void* stream) {
    int s = check_desc(c);
    if (s != KCT_OK) return s;
    if (!d_gt || !d_xt0 || !d_xt1 || !d_xt2 || !d_gw || !d_err) return conv_fail(KCT_ERR_INVALID_ARG, "null pointer");
    if (!aligned16(d_gt) || !aligned16(d_xt0) || !aligned16(d_xt1) || !aligned16(d_xt2))
        return conv_fail(KCT_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    WgradDims D;
    D.n = c->n; D.d = c->d; D.h = c->h; D.w = c->w; D.cin = c->cin; D.cout = c->cout;
    D.kb = c->w % 64 == 0 ? 64 : c->w % 32 == 0 ? 32 : 16;
    D.chunks_x = c->w / D.kb;
    D.nchunks = (long long)c->n * c->d * c->h * D.chunks_x;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // channels-first tensors: dims (x, y, z, c, n)
    auto cf_map = [&](CUtensorMap* m, const void* p, int ch, int rows) {
        const uint64_t dd[5] = {(uint64_t)c->w, (uint64_t)c->h, (uint64_t)c->d, (uint64_t)ch, (uint64_t)c->n};
        const uint64_t ss[4] = {(uint64_t)c->w * 2, (uint64_t)c->w * 2 * c->h, (uint64_t)c->w * 2 * c->h * c->d,
                                (uint64_t)c->w * 2 * c->h * c->d * ch};
        const uint32_t bb[5] = {(uint32_t)D.kb, 1, 1, (uint32_t)rows, 1};
        return make_map(m, p, 5, dd, ss, bb, D.kb * 2);
    };
    CUtensorMap tg, tx[3];
    if ((s = cf_map(&tg, d_gt, c->cout, c->cout)) != KCT_OK) return s;
    if ((s = cf_map(&tx[0], d_xt0, c->cin, c->cin)) != KCT_OK) return s;
    if ((s = cf_map(&tx[1], d_xt1, c->cin, c->cin)) != KCT_OK) return s;
    if ((s = cf_map(&tx[2], d_xt2, c->cin, c->cin)) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_gw, 0, sizeof(float) * (size_t)c->cout * 27 * c->cin, st);
    if (e != cudaSuccess) return conv_fail(KCT_ERR_CUDA, "cudaMemsetAsync");
    if (D.kb == 64) return dispatch_wgrad_ci<64>(tg, tx, D, d_gw, d_err, sms, st);
    if (D.kb == 32) return dispatch_wgrad_ci<32>(tg, tx, D, d_gw, d_err, sms, st);
    return dispatch_wgrad_ci<16>(tg, tx, D, d_gw, d_err, sms, st);
}

}  // extern "C"
