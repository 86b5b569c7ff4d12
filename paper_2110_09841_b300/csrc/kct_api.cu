// kct_api.cu -- C ABI of the cutting voxel projector: plan creation, geometry validation,
// kernel launches. See include/kct.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kct.h"
#include "cvp_device.cuh"
#include "cvp_kernels.cuh"
#include "cgls_kernels.cuh"
#include "siddon.cuh"

using kct::Grid;
using kct::View;

struct kct_plan {
    int device;
    kct_volume_desc vol;
    kct_detector_desc det;
    int32_t nviews;
    kct_variant variant;
    kct_scaling scaling;
    Grid grid;
    std::vector<View> h_views;
    View* d_views;
    int* d_err;
    unsigned long long* d_count;
    int fwd_chunk;                 // views per forward block (kct_plan_autotune may change it)
    int bwd_runs;                  // relaxed adjoint: runs of 64 voxels per brick (1 or 2)
};

namespace {

thread_local std::string g_last_error;

kct_status fail(kct_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

kct_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return KCT_ERR_CUDA;
}

bool finite_all(const double* p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

void split(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Convert one 3x4 projection matrix into the kernel's per-view parameters.
// Returns an empty string on success, else the reason it violates the arrangement the
// projector needs (Sec. III-A): u independent of x_3, rows along x_3, volume in front.
std::string setup_view(const double* P, const kct_volume_desc& vol, View& V) {
    if (!finite_all(P, 12)) return "non-finite matrix entry";
    double M[3][3], p4[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) M[r][c] = P[4 * r + c];
        p4[r] = P[4 * r + 3];
    }
    double n0 = std::sqrt(M[0][0] * M[0][0] + M[0][1] * M[0][1] + M[0][2] * M[0][2]);
    double n1 = std::sqrt(M[1][0] * M[1][0] + M[1][1] * M[1][1] + M[1][2] * M[1][2]);
    double n2 = std::sqrt(M[2][0] * M[2][0] + M[2][1] * M[2][1] + M[2][2] * M[2][2]);
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(std::fabs(det) > 1e-12 * n0 * n1 * n2)) return "singular 3x3 part";
    if (std::fabs(M[0][2]) > 1e-9 * n0) return "detector column depends on x3 (P[0][2] != 0)";
    if (std::fabs(M[2][2]) > 1e-9 * n2) return "principal axis not horizontal (P[2][2] != 0)";
    // source s = -M^{-1} p4
    double inv[3][3];
    double id = 1.0 / det;
    inv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) * id;
    inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * id;
    inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * id;
    inv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) * id;
    inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * id;
    inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * id;
    inv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) * id;
    inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) * id;
    inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * id;
    double s[3];
    for (int r = 0; r < 3; ++r) s[r] = -(inv[r][0] * p4[0] + inv[r][1] * p4[1] + inv[r][2] * p4[2]);
    // orientation: the volume centre (origin) must be in front of the source
    if (p4[2] == 0.0) return "volume centre on the source plane";
    double sigma = p4[2] > 0.0 ? 1.0 : -1.0;
    double m2h = std::sqrt(M[2][0] * M[2][0] + M[2][1] * M[2][1]);
    double wx = sigma * M[2][0] / m2h, wy = sigma * M[2][1] / m2h;
    double hx = -wy, hy = wx;
    // rectangular pixels with rows along x3: horizontal part of row 1 parallel to row 2
    double m1h_h = M[1][0] * hx + M[1][1] * hy;
    if (std::fabs(m1h_h) > 1e-9 * n1) return "detector rows not along x3 (skewed pixel grid)";
    if (!(std::fabs(M[1][2]) > 1e-12 * n1)) return "detector row index independent of x3";
    double den = sigma * m2h;
    double cu = (M[0][0] * wx + M[0][1] * wy) / den;
    double gu = (M[0][0] * hx + M[0][1] * hy) / den;
    double cv = (M[1][0] * wx + M[1][1] * wy) / den;
    double gv = M[1][2] / den;
    if (!(std::fabs(gu) > 0.0) || !(std::fabs(gv) > 0.0)) return "degenerate detector scale";
    // whole volume in front of the source: depth t = w.(X - s) > 0 at all eight corners
    double lx = 0.5 * vol.nx * vol.ax, ly = 0.5 * vol.ny * vol.ay;
    double tmin = 1e300;
    for (int c = 0; c < 4; ++c) {
        double X = (c & 1) ? lx : -lx, Y = (c & 2) ? ly : -ly;
        tmin = std::fmin(tmin, wx * (X - s[0]) + wy * (Y - s[1]));
    }
    double diag = std::sqrt(vol.ax * vol.ax + vol.ay * vol.ay);
    if (!(tmin > diag)) return "source inside or too close to the volume";
    // rows spanned by one voxel: |gv| * (range of zeta / t over the voxel) + 2
    double zabs = std::fmax(std::fabs(0.5 * vol.nz * vol.az - s[2]), std::fabs(-0.5 * vol.nz * vol.az - s[2]));
    double tnear = tmin - 0.5 * diag;
    double rows = std::fabs(gv) * (vol.az / tnear + zabs * diag / (tnear * tnear)) + 2.0;
    if (rows > kct::KCT_ROWS - 2) return "unsupported: a voxel would span more than 30 detector rows";
    split(wx, V.wx, V.wx_lo);
    split(wy, V.wy, V.wy_lo);
    split(-(wx * s[0] + wy * s[1]), V.aw, V.aw_lo);
    V.ah = (float)(-(hx * s[0] + hy * s[1]));
    V.sz = (float)s[2];
    V.cu = (float)cu;
    V.gu = (float)gu;
    V.cv = (float)cv;
    V.gv = (float)gv;
    V.igu = (float)(1.0 / gu);
    V.igv = (float)(1.0 / gv);
    V.inv_agv = (float)(1.0 / std::fabs(gv));
    V.sgv = gv > 0.0 ? 1.0f : -1.0f;
    V.fcos = (float)std::fabs(gu * gv);
    // base square of a voxel, counter-clockwise in (x1, x2); (t', xi') = (w.q, h.q)
    const double qx[4] = {-0.5 * vol.ax, 0.5 * vol.ax, 0.5 * vol.ax, -0.5 * vol.ax};
    const double qy[4] = {-0.5 * vol.ay, -0.5 * vol.ay, 0.5 * vol.ay, 0.5 * vol.ay};
    double tt[4], xx[4];
    for (int e = 0; e < 4; ++e) {
        tt[e] = wx * qx[e] + wy * qy[e];
        xx[e] = hx * qx[e] + hy * qy[e];
        V.sq_t[e] = (float)tt[e];
        V.sq_x[e] = (float)xx[e];
    }
    V.sx = (float)s[0];
    V.sy = (float)s[1];
    V.cv_lo = (float)(cv - (double)V.cv);
    V.inv_agv_lo = (float)(1.0 / std::fabs(gv) - (double)V.inv_agv);
    V.sz_lo = (float)(s[2] - (double)V.sz);
    return std::string();
}

void set_grid_doubles(Grid& G, const kct_volume_desc& vol) {
    G.axd = vol.ax;
    G.ayd = vol.ay;
    G.azd = vol.az;
    G.x0d = 0.5 * (1 - vol.nx) * vol.ax;
    G.y0d = 0.5 * (1 - vol.ny) * vol.ay;
    G.z0d = 0.5 * (1 - vol.nz) * vol.az;
}

unsigned bricks(const Grid& G) {
    return (unsigned)(((G.nx + kct::BX - 1) / kct::BX) * ((G.ny + kct::BY - 1) / kct::BY));
}

template <int VARIANT, bool FWD = true, int RUNS = 0>
unsigned segments(const Grid& G) {
    return (unsigned)((G.nz + kct::Brick<VARIANT, FWD, RUNS>::Z - 1) / kct::Brick<VARIANT, FWD, RUNS>::Z);
}

template <int VARIANT, bool FWD = true, int RUNS = 0>
constexpr size_t brick_dyn_smem() { return sizeof(float) * kct::Brick<VARIANT, FWD, RUNS>::DYN_FLOATS; }

// Fraction of the bricks of bz voxels along x_3 whose detector window (the bounding box of the
// projected brick corners plus one pixel, clipped to the detector, as the kernels compute it)
// holds more than `cap` pixels, over up to 8 evenly spaced views and up to 4096 bricks per view.
double brick_overflow(const double* pmats, int nviews, const kct_volume_desc& vol, const kct_detector_desc& det,
                      int bz, int cap) {
    const int nbx = (vol.nx + kct::BX - 1) / kct::BX, nby = (vol.ny + kct::BY - 1) / kct::BY;
    const int nbz = (vol.nz + bz - 1) / bz;
    const long long nb = (long long)nbx * nby * nbz;
    const long long step = nb > 4096 ? nb / 4096 : 1;
    const int vstep = nviews > 8 ? nviews / 8 : 1;
    long long over = 0, count = 0;
    for (int q = 0; q < nviews; q += vstep) {
        const double* P = pmats + 12 * (size_t)q;
        for (long long b = 0; b < nb; b += step) {
            const int bi = (int)(b % nbx), bj = (int)((b / nbx) % nby), bk = (int)(b / ((long long)nbx * nby));
            const int i0 = bi * kct::BX, j0 = bj * kct::BY, k0 = bk * bz;
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            for (int c = 0; c < 8; ++c) {
                const int ii = (c & 1) ? std::min(i0 + kct::BX, vol.nx) : i0;
                const int jj = (c & 2) ? std::min(j0 + kct::BY, vol.ny) : j0;
                const int kk = (c & 4) ? std::min(k0 + bz, vol.nz) : k0;
                const double X = (ii - 0.5 * vol.nx) * vol.ax, Y = (jj - 0.5 * vol.ny) * vol.ay, Z = (kk - 0.5 * vol.nz) * vol.az;
                const double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
                const double u = (P[0] * X + P[1] * Y + P[2] * Z + P[3]) / w;
                const double v = (P[4] * X + P[5] * Y + P[6] * Z + P[7]) / w;
                umin = std::fmin(umin, u);
                umax = std::fmax(umax, u);
                vmin = std::fmin(vmin, v);
                vmax = std::fmax(vmax, v);
            }
            const long long u0 = std::max((long long)std::floor(umin + 0.5) - 1, 0LL);
            const long long u1 = std::min((long long)std::floor(umax + 0.5) + 1, (long long)det.nu - 1);
            const long long v0 = std::max((long long)std::floor(vmin + 0.5) - 1, 0LL);
            const long long v1 = std::min((long long)std::floor(vmax + 0.5) + 1, (long long)det.nv - 1);
            const long long area = (u1 >= u0 && v1 >= v0) ? (u1 - u0 + 1) * (v1 - v0 + 1) : 0;
            over += area > cap ? 1 : 0;
            ++count;
        }
    }
    return count ? (double)over / count : 0.0;
}

constexpr int kMaxDevices = 64;

// opt in to more than 48 KB of shared memory per block (once per device: the attribute
// belongs to the kernel on the current device)
template <class K>
cudaError_t set_dyn(K kernel, size_t bytes, cudaError_t e) {
    return e == cudaSuccess ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) : e;
}

cudaError_t brick_kernel_attributes() {
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        e = set_dyn(kct::fwd_kernel<0, 0>, brick_dyn_smem<0>(), e);
        e = set_dyn(kct::fwd_kernel<0, 1>, brick_dyn_smem<0>(), e);
        e = set_dyn(kct::fwd_kernel<1, 0>, brick_dyn_smem<1>(), e);
        e = set_dyn(kct::fwd_kernel<1, 1>, brick_dyn_smem<1>(), e);
        e = set_dyn(kct::fwd_kernel<0, -1>, brick_dyn_smem<0>(), e);
        e = set_dyn(kct::fwd_kernel<1, -1>, brick_dyn_smem<1>(), e);
        e = set_dyn(kct::bwd_kernel<0, 0>, brick_dyn_smem<0, false>(), e);
        e = set_dyn(kct::bwd_kernel<0, 1>, brick_dyn_smem<0, false>(), e);
        e = set_dyn(kct::bwd_kernel<1, 0>, brick_dyn_smem<1, false>(), e);
        e = set_dyn(kct::bwd_kernel<1, 1>, brick_dyn_smem<1, false>(), e);
        e = set_dyn(kct::bwd_kernel<1, 0, 2>, brick_dyn_smem<1, false, 2>(), e);
        e = set_dyn(kct::bwd_kernel<1, 1, 2>, brick_dyn_smem<1, false, 2>(), e);
        done[dev] = e == cudaSuccess;
    }
    return e;
}

unsigned view_chunks(const Grid& G, int chunk) { return (unsigned)((G.nviews + chunk - 1) / chunk); }

// Forward launch over the views of G (the plan's grid, or the same grid cut to its first
// views when tuning) with `chunk` views per block.
template <int VARIANT, int SCALING>
void launch_fwd_grid(const kct_plan* p, const Grid& G, int chunk, const float* vol, float* out, int nbatch,
                     cudaStream_t st) {
    dim3 grid(bricks(G), segments<VARIANT>(G), view_chunks(G, chunk) * (unsigned)nbatch);
    const long long vs = (long long)G.nx * G.ny * G.nz, ps = (long long)G.nu * G.nv * G.nviews;
    kct::fwd_kernel<VARIANT, SCALING><<<grid, kct::NTHREADS, brick_dyn_smem<VARIANT>(), st>>>(
        p->d_views, G, vol, out, vs, ps, chunk, p->d_err);
}

template <int VARIANT, int SCALING>
void launch_fwd(const kct_plan* p, const float* vol, float* out, int nbatch, cudaStream_t st) {
    launch_fwd_grid<VARIANT, SCALING>(p, p->grid, p->fwd_chunk, vol, out, nbatch, st);
}

void launch_fwd_any(const kct_plan* p, const Grid& G, int chunk, const float* vol, float* out, cudaStream_t st) {
    const int key = (p->variant == KCT_CVP_RELAXED ? 2 : 0) + (p->scaling == KCT_SCALE_EXACT ? 1 : 0);
    switch (key) {
        case 0: launch_fwd_grid<0, 0>(p, G, chunk, vol, out, 1, st); break;
        case 1: launch_fwd_grid<0, 1>(p, G, chunk, vol, out, 1, st); break;
        case 2: launch_fwd_grid<1, 0>(p, G, chunk, vol, out, 1, st); break;
        default: launch_fwd_grid<1, 1>(p, G, chunk, vol, out, 1, st); break;
    }
}

template <int VARIANT, int SCALING, int RUNS = 0>
void launch_bwd_runs(const kct_plan* p, const float* y, float* vol, int nbatch, int accumulate, cudaStream_t st) {
    const Grid& G = p->grid;
    dim3 grid(bricks(G), segments<VARIANT, false, RUNS>(G), (unsigned)nbatch);
    const long long vs = (long long)G.nx * G.ny * G.nz, ps = (long long)G.nu * G.nv * G.nviews;
    kct::bwd_kernel<VARIANT, SCALING, RUNS><<<grid, kct::NTHREADS, brick_dyn_smem<VARIANT, false, RUNS>(), st>>>(
        p->d_views, G, y, vol, vs, ps, accumulate, p->d_err);
}

template <int VARIANT, int SCALING>
void launch_bwd(const kct_plan* p, const float* y, float* vol, int nbatch, int accumulate, cudaStream_t st) {
    if (VARIANT == 1 && p->bwd_runs == 2) launch_bwd_runs<VARIANT, SCALING, 2>(p, y, vol, nbatch, accumulate, st);
    else launch_bwd_runs<VARIANT, SCALING>(p, y, vol, nbatch, accumulate, st);
}

template <int VARIANT>
void launch_count(const kct_plan* p, cudaStream_t st) {
    const Grid& G = p->grid;
    dim3 grid(bricks(G), segments<VARIANT>(G), (unsigned)G.nviews);
    kct::count_kernel<VARIANT><<<grid, kct::NTHREADS, 0, st>>>(p->d_views, G, p->d_count, p->d_err);
}

kct_status check_plan(const kct_plan* p) {
    if (!p) return fail(KCT_ERR_INVALID_ARG, "null plan");
    return KCT_OK;
}

// Makes the plan's device current for the duration of one call and gives the calling thread
// its previous device back on return (the work enqueued stays on its stream).
class DeviceScope {
  public:
    explicit DeviceScope(int dev) {
        err_ = cudaGetDevice(&prev_);
        if (err_ == cudaSuccess && prev_ != dev) {
            err_ = cudaSetDevice(dev);
            switched_ = err_ == cudaSuccess;
        }
    }
    ~DeviceScope() {
        if (switched_) cudaSetDevice(prev_);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
    kct_status status() const { return err_ == cudaSuccess ? KCT_OK : cuda_fail(err_, "selecting the plan's device"); }

  private:
    int prev_ = -1;
    bool switched_ = false;
    cudaError_t err_ = cudaSuccess;
};

}  // namespace

extern "C" {

int32_t kct_version(void) { return KCT_VERSION; }

const char* kct_status_string(kct_status s) {
    switch (s) {
        case KCT_OK: return "ok";
        case KCT_ERR_INVALID_ARG: return "invalid argument";
        case KCT_ERR_GEOMETRY: return "geometry outside the projector's arrangement";
        case KCT_ERR_CUDA: return "CUDA error";
        case KCT_ERR_OOM: return "out of memory";
        case KCT_ERR_DEVICE_CHECK: return "device-side check failed";
        case KCT_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char* kct_last_error_message(void) { return g_last_error.c_str(); }

kct_status kct_plan_create(kct_plan** out, const kct_volume_desc* vol, const kct_detector_desc* det,
                           const double* pmats, int32_t nviews, kct_variant variant, kct_scaling scaling) {
    g_last_error.clear();
    if (!out) return fail(KCT_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (!vol || !det || !pmats) return fail(KCT_ERR_INVALID_ARG, "null descriptor or matrix pointer");
    if (vol->nx <= 0 || vol->ny <= 0 || vol->nz <= 0) return fail(KCT_ERR_INVALID_ARG, "volume sizes must be positive");
    if (!(vol->ax > 0.0) || !(vol->ay > 0.0) || !(vol->az > 0.0) || !std::isfinite(vol->ax) ||
        !std::isfinite(vol->ay) || !std::isfinite(vol->az))
        return fail(KCT_ERR_INVALID_ARG, "voxel sizes must be positive and finite");
    if (det->nu <= 0 || det->nv <= 0) return fail(KCT_ERR_INVALID_ARG, "detector sizes must be positive");
    if (!(det->pu > 0.0) || !(det->pv > 0.0)) return fail(KCT_ERR_INVALID_ARG, "pixel pitch must be positive");
    if (nviews <= 0 || nviews > 65535) return fail(KCT_ERR_INVALID_ARG, "nviews must be in [1, 65535]");
    if (variant != KCT_CVP_EXACT && variant != KCT_CVP_RELAXED) return fail(KCT_ERR_INVALID_ARG, "unknown variant");
    if (scaling != KCT_SCALE_COS && scaling != KCT_SCALE_EXACT) return fail(KCT_ERR_INVALID_ARG, "unknown scaling");
    long long nvox = (long long)vol->nx * vol->ny * vol->nz;
    long long npix = (long long)det->nu * det->nv * nviews;
    if (nvox > (1LL << 31) - 1 || npix > (1LL << 40)) return fail(KCT_ERR_UNSUPPORTED, "problem too large for 32-bit voxel indexing");
    if ((long long)vol->nx * vol->ny > (1LL << 31) - 1) return fail(KCT_ERR_UNSUPPORTED, "volume slice too large");

    kct_plan* p = new (std::nothrow) kct_plan();
    if (!p) return fail(KCT_ERR_OOM, "host allocation of the plan");
    p->vol = *vol;
    p->det = *det;
    p->nviews = nviews;
    p->variant = variant;
    p->scaling = scaling;
    p->d_views = nullptr;
    p->d_err = nullptr;
    p->d_count = nullptr;
    p->fwd_chunk = kct::VIEW_CHUNK;
    p->h_views.resize(nviews);
    for (int q = 0; q < nviews; ++q) {
        std::string why = setup_view(pmats + 12 * q, *vol, p->h_views[q]);
        if (!why.empty()) {
            delete p;
            char buf[64];
            std::snprintf(buf, sizeof buf, "view %d: ", q);
            bool unsup = why.compare(0, 12, "unsupported:") == 0;
            return fail(unsup ? KCT_ERR_UNSUPPORTED : KCT_ERR_GEOMETRY, buf + why);
        }
    }
    // relaxed adjoint: two runs per brick where (almost) every brick's footprint fits the tile
    // (after the views are validated: the whole volume is then in front of the source)
    p->bwd_runs = (variant == KCT_CVP_RELAXED &&
                   brick_overflow(pmats, nviews, *vol, *det, kct::Brick<1, false, 2>::Z, kct::Brick<1, false, 2>::TILE) <= 0.02)
                      ? 2 : 1;
    Grid& G = p->grid;
    G.nx = vol->nx; G.ny = vol->ny; G.nz = vol->nz;
    G.nu = det->nu; G.nv = det->nv; G.nviews = nviews;
    G.ax = (float)vol->ax; G.ay = (float)vol->ay; G.az = (float)vol->az;
    G.x0 = (float)(0.5 * (1 - vol->nx) * vol->ax);
    G.y0 = (float)(0.5 * (1 - vol->ny) * vol->ay);
    G.z0 = (float)(0.5 * (1 - vol->nz) * vol->az);
    set_grid_doubles(G, *vol);

    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    e = brick_kernel_attributes();
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaFuncSetAttribute"); }
    e = cudaMalloc(&p->d_views, sizeof(View) * nviews);
    if (e != cudaSuccess) { delete p; return fail(KCT_ERR_OOM, std::string("cudaMalloc views: ") + cudaGetErrorString(e)); }
    e = cudaMalloc(&p->d_err, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_count, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(p->d_views);
        cudaFree(p->d_err);
        cudaFree(p->d_count);
        delete p;
        return fail(KCT_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(p->d_views, p->h_views.data(), sizeof(View) * nviews, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int) * 4);
    if (e != cudaSuccess) {
        cudaFree(p->d_views); cudaFree(p->d_err); cudaFree(p->d_count);
        delete p;
        return cuda_fail(e, "uploading view parameters");
    }
    *out = p;
    return KCT_OK;
}

kct_status kct_plan_destroy(kct_plan* p) {
    if (!p) return KCT_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaFree(p->d_views);
    cudaFree(p->d_err);
    cudaFree(p->d_count);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
    return KCT_OK;
}

static kct_status project_impl(const kct_plan* p, const float* d_vol, float* d_proj, int32_t nbatch,
                               int32_t accumulate, void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!d_vol || !d_proj) return fail(KCT_ERR_INVALID_ARG, "null data pointer");
    if (nbatch <= 0) return fail(KCT_ERR_INVALID_ARG, "nbatch must be positive");
    const Grid& G = p->grid;
    if ((long long)view_chunks(G, p->fwd_chunk) * nbatch > 65535)
        return fail(KCT_ERR_UNSUPPORTED, "batch too large for one launch");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    size_t pbytes = sizeof(float) * (size_t)G.nu * G.nv * G.nviews * nbatch;
    cudaError_t e;
    if (!accumulate) {
        e = cudaMemsetAsync(d_proj, 0, pbytes, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    const int key = (p->variant == KCT_CVP_RELAXED ? 2 : 0) + (p->scaling == KCT_SCALE_EXACT ? 1 : 0);
    switch (key) {
        case 0: launch_fwd<0, 0>(p, d_vol, d_proj, nbatch, st); break;
        case 1: launch_fwd<0, 1>(p, d_vol, d_proj, nbatch, st); break;
        case 2: launch_fwd<1, 0>(p, d_vol, d_proj, nbatch, st); break;
        default: launch_fwd<1, 1>(p, d_vol, d_proj, nbatch, st); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "forward projection launch");
    return KCT_OK;
}

static kct_status backproject_impl(const kct_plan* p, const float* d_proj, float* d_vol, int32_t nbatch,
                                   int32_t accumulate, void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!d_vol || !d_proj) return fail(KCT_ERR_INVALID_ARG, "null data pointer");
    if (nbatch <= 0 || nbatch > 65535) return fail(KCT_ERR_INVALID_ARG, "nbatch must be in [1, 65535]");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int key = (p->variant == KCT_CVP_RELAXED ? 2 : 0) + (p->scaling == KCT_SCALE_EXACT ? 1 : 0);
    const int acc = accumulate ? 1 : 0;
    switch (key) {
        case 0: launch_bwd<0, 0>(p, d_proj, d_vol, nbatch, acc, st); break;
        case 1: launch_bwd<0, 1>(p, d_proj, d_vol, nbatch, acc, st); break;
        case 2: launch_bwd<1, 0>(p, d_proj, d_vol, nbatch, acc, st); break;
        default: launch_bwd<1, 1>(p, d_proj, d_vol, nbatch, acc, st); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "backprojection launch");
    return KCT_OK;
}

kct_status kct_project(const kct_plan* p, const float* d_vol, float* d_proj, int32_t accumulate, void* stream) {
    return project_impl(p, d_vol, d_proj, 1, accumulate, stream);
}

kct_status kct_backproject(const kct_plan* p, const float* d_proj, float* d_vol, int32_t accumulate, void* stream) {
    return backproject_impl(p, d_proj, d_vol, 1, accumulate, stream);
}

kct_status kct_project_batch(const kct_plan* p, const float* d_vol, int32_t nbatch, float* d_proj,
                             int32_t accumulate, void* stream) {
    return project_impl(p, d_vol, d_proj, nbatch, accumulate, stream);
}

kct_status kct_backproject_batch(const kct_plan* p, const float* d_proj, int32_t nbatch, float* d_vol,
                                 int32_t accumulate, void* stream) {
    return backproject_impl(p, d_proj, d_vol, nbatch, accumulate, stream);
}

kct_status kct_plan_set_view_chunk(kct_plan* p, int32_t chunk) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (chunk < 1 || chunk > kct::MAX_VIEW_CHUNK) return fail(KCT_ERR_INVALID_ARG, "view chunk outside [1, 64]");
    p->fwd_chunk = chunk;
    return KCT_OK;
}

kct_status kct_plan_get_view_chunk(const kct_plan* p, int32_t* chunk) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!chunk) return fail(KCT_ERR_INVALID_ARG, "null output pointer");
    *chunk = p->fwd_chunk;
    return KCT_OK;
}

kct_status kct_plan_autotune(kct_plan* p, const float* d_vol, float* d_proj, int32_t* chunk, float* ms,
                             void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!d_vol || !d_proj) return fail(KCT_ERR_INVALID_ARG, "null data pointer");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Grid G = p->grid;
    G.nviews = std::min(G.nviews, kct::TUNE_VIEWS);
    const size_t pbytes = sizeof(float) * (size_t)G.nu * G.nv * G.nviews;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    static const int kCand[] = {1, 2, 4, 8, 16, 32, 64};
    int best = p->fwd_chunk;
    float best_ms = -1.f;
    for (int ci = 0; ci < 7 && e == cudaSuccess; ++ci) {
        const int c = kCand[ci];
        if (c > kct::MAX_VIEW_CHUNK || (c > G.nviews && c != 1)) break;
        float t = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run is a warm-up
            e = cudaMemsetAsync(d_proj, 0, pbytes, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) launch_fwd_any(p, G, c, d_vol, d_proj, st);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        }
        if (e == cudaSuccess && (best_ms < 0.f || t < best_ms)) {
            best_ms = t;
            best = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    p->fwd_chunk = best;
    if (chunk) *chunk = best;
    if (ms) *ms = best_ms;
    return KCT_OK;
}

kct_status kct_siddon_project(const kct_plan* p, const float* d_vol, float* d_proj, int32_t K, int32_t weighting,
                              void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!d_vol || !d_proj) return fail(KCT_ERR_INVALID_ARG, "null data pointer");
    if (K < 1 || K > 64) return fail(KCT_ERR_INVALID_ARG, "K must be in [1, 64]");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    const Grid& G = p->grid;
    const long long npix = (long long)G.nu * G.nv;
    dim3 grid((unsigned)((npix + 7) / 8), (unsigned)G.nviews);
    if (weighting) kct::siddon_kernel<1><<<grid, 256, 0, (cudaStream_t)stream>>>(p->d_views, G, d_vol, d_proj, K);
    else kct::siddon_kernel<0><<<grid, 256, 0, (cudaStream_t)stream>>>(p->d_views, G, d_vol, d_proj, K);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ray-driven comparator launch");
    return KCT_OK;
}

kct_status kct_pixel_factors(const kct_plan* p, float* d_out, void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!d_out) return fail(KCT_ERR_INVALID_ARG, "null output pointer");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    const Grid& G = p->grid;
    long n = (long)G.nu * G.nv;
    dim3 grid((unsigned)((n + 255) / 256), G.nviews);
    if (p->scaling == KCT_SCALE_EXACT)
        kct::factor_kernel<1><<<grid, 256, 0, (cudaStream_t)stream>>>(p->d_views, G, d_out);
    else
        kct::factor_kernel<0><<<grid, 256, 0, (cudaStream_t)stream>>>(p->d_views, G, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pixel factor launch");
    return KCT_OK;
}

kct_status kct_count_pairs(const kct_plan* p, uint64_t* count, void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!count) return fail(KCT_ERR_INVALID_ARG, "null output pointer");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(p->d_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (p->variant == KCT_CVP_RELAXED) launch_count<1>(p, st);
    else launch_count<0>(p, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pair count launch");
    unsigned long long h = 0;
    e = cudaMemcpyAsync(&h, p->d_count, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the pair count");
    *count = (uint64_t)h;
    return KCT_OK;
}

kct_status kct_last_device_error(const kct_plan* p, int32_t* code, void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!code) return fail(KCT_ERR_INVALID_ARG, "null output pointer");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    *code = h;
    return KCT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// CGLS
// ---------------------------------------------------------------------------------------

namespace {

struct CglsLayout {
    size_t r, q, s, p, part, sc, total;
};

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

CglsLayout cgls_layout(const Grid& G) {
    const size_t nproj = (size_t)G.nu * G.nv * G.nviews, nvol = (size_t)G.nx * G.ny * G.nz;
    CglsLayout L;
    L.r = 0;
    L.q = L.r + align256(nproj * sizeof(float));
    L.s = L.q + align256(nproj * sizeof(float));
    L.p = L.s + align256(nvol * sizeof(float));
    L.part = L.p + align256(nvol * sizeof(float));
    L.sc = L.part + align256(3 * kct::VEC_MAX_BLOCKS * sizeof(double));
    L.total = L.sc + align256(sizeof(kct::CglsScalars));
    return L;
}

}  // namespace

extern "C" {

size_t kct_cgls_workspace_bytes(const kct_plan* p) { return p ? cgls_layout(p->grid).total : 0; }

kct_status kct_cgls(const kct_plan* p, const float* d_b, float* d_x, const float* d_atb, int32_t warm_start,
                    int32_t max_iter, double tol, void* d_work, size_t work_bytes, double* h_normal, double* h_data,
                    kct_cgls_report* report, void* stream) {
    kct_status s = check_plan(p);
    if (s != KCT_OK) return s;
    if (!d_b || !d_x || !d_work) return fail(KCT_ERR_INVALID_ARG, "null data pointer");
    if (max_iter < 0 || !(tol >= 0.0)) return fail(KCT_ERR_INVALID_ARG, "max_iter and tol must be >= 0");
    const Grid& G = p->grid;
    const CglsLayout L = cgls_layout(G);
    if (work_bytes < L.total) return fail(KCT_ERR_INVALID_ARG, "workspace smaller than kct_cgls_workspace_bytes");
    if (((uintptr_t)d_work & 255) || ((uintptr_t)d_b & 15) || ((uintptr_t)d_x & 15) || ((uintptr_t)d_atb & 15))
        return fail(KCT_ERR_INVALID_ARG, "d_work must be 256-byte and d_b, d_x, d_atb 16-byte aligned");
    DeviceScope scope(p->device);
    if ((s = scope.status()) != KCT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const int nb = std::min(kct::VEC_MAX_BLOCKS, std::max(1, 8 * sms));
    const long long nproj = (long long)G.nu * G.nv * G.nviews, nvol = (long long)G.nx * G.ny * G.nz;
    unsigned char* w = (unsigned char*)d_work;
    float* r = (float*)(w + L.r);
    float* q = (float*)(w + L.q);
    float* sv = (float*)(w + L.s);
    float* pv = (float*)(w + L.p);
    double* part_qq = (double*)(w + L.part);
    double* part_ss = part_qq + kct::VEC_MAX_BLOCKS;
    double* part_rr = part_ss + kct::VEC_MAX_BLOCKS;
    kct::CglsScalars* sc = (kct::CglsScalars*)(w + L.sc);
    const int T = kct::VEC_THREADS;

    // start: r = b - A x0, s = A^T r, p = s, gamma_0 = |s|^2, plus |b|^2 and |A^T b|^2
    kct::sumsq_kernel<<<nb, T, 0, st>>>(d_b, nproj, part_rr);
    kct::store_sum_kernel<<<1, T, 0, st>>>(part_rr, nb, &sc->bb2);
    if (warm_start) {
        // |A^T b|, the denominator of the stopping rule, from the caller's A^T b if given
        if (d_atb) {
            kct::sumsq_kernel<<<nb, T, 0, st>>>(d_atb, nvol, part_ss);
        } else {
            if ((s = backproject_impl(p, d_b, sv, 1, 0, st)) != KCT_OK) return s;
            kct::sumsq_kernel<<<nb, T, 0, st>>>(sv, nvol, part_ss);
        }
        kct::store_sum_kernel<<<1, T, 0, st>>>(part_ss, nb, &sc->atb2);
        if ((s = project_impl(p, d_x, q, 1, 0, st)) != KCT_OK) return s;
        kct::residual_kernel<<<nb, T, 0, st>>>(d_b, q, r, nproj, part_rr);
        if ((s = backproject_impl(p, r, sv, 1, 0, st)) != KCT_OK) return s;
        kct::sumsq_kernel<<<nb, T, 0, st>>>(sv, nvol, part_ss);
    } else {
        e = cudaMemsetAsync(d_x, 0, sizeof(float) * nvol, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r, d_b, sizeof(float) * nproj, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && d_atb) e = cudaMemcpyAsync(sv, d_atb, sizeof(float) * nvol, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "CGLS start");
        if (!d_atb && (s = backproject_impl(p, r, sv, 1, 0, st)) != KCT_OK) return s;
        kct::sumsq_kernel<<<nb, T, 0, st>>>(sv, nvol, part_ss);
        kct::store_sum_kernel<<<1, T, 0, st>>>(part_ss, nb, &sc->atb2);
    }
    kct::cgls_p_kernel<<<nb, T, 0, st>>>(sv, pv, nvol, part_ss, part_rr, nb, nullptr, &sc->gamma[0], sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CGLS start kernels");

    auto read_residuals = [&](double* out2) -> kct_status {
        cudaError_t e2 = cudaMemcpyAsync(out2, &sc->normal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
        return e2 == cudaSuccess ? KCT_OK : cuda_fail(e2, "CGLS residual read");
    };
    double res[2] = {0.0, 0.0};
    if ((s = read_residuals(res)) != KCT_OK) return s;
    if (h_normal) h_normal[0] = res[0];
    if (h_data) h_data[0] = res[1];
    int k = 0;
    while (k < max_iter && !(res[0] <= tol)) {
        double* g_cur = &sc->gamma[k & 1];
        double* g_next = &sc->gamma[(k + 1) & 1];
        if ((s = project_impl(p, pv, q, 1, 0, st)) != KCT_OK) return s;
        kct::sumsq_kernel<<<nb, T, 0, st>>>(q, nproj, part_qq);
        kct::cgls_xr_kernel<<<nb, T, 0, st>>>(d_x, pv, nvol, r, q, nproj, part_qq, nb, g_cur, part_rr);
        if ((s = backproject_impl(p, r, sv, 1, 0, st)) != KCT_OK) return s;
        kct::sumsq_kernel<<<nb, T, 0, st>>>(sv, nvol, part_ss);
        kct::cgls_p_kernel<<<nb, T, 0, st>>>(sv, pv, nvol, part_ss, part_rr, nb, g_cur, g_next, sc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "CGLS step kernels");
        if ((s = read_residuals(res)) != KCT_OK) return s;
        ++k;
        if (h_normal) h_normal[k] = res[0];
        if (h_data) h_data[k] = res[1];
    }
    if (report) {
        report->iterations = k;
        report->converged = res[0] <= tol ? 1 : 0;
        report->normal_residual = res[0];
        report->data_residual = res[1];
    }
    return KCT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Forward projection without any allocation: scratch in a fixed device array
// ---------------------------------------------------------------------------------------
//
// For callers that may not allocate device memory at all (code running inside another
// library's memory pool or an allocator-free runtime, where every cudaMalloc would break the
// host application's accounting). Layout of the array: per-view parameters, the error word,
// the unscaled sums of every pixel.
namespace {

constexpr size_t kStaticViews = 4096;                     // views per call, at most
constexpr size_t kStaticSums = size_t(8) << 20;           // pixels x views per call, at most
constexpr size_t kStaticViewBytes = kStaticViews * sizeof(View);
constexpr size_t kStaticErrOffset = kStaticViewBytes;
constexpr size_t kStaticSumOffset = kStaticViewBytes + 256;
constexpr size_t kStaticBytes = kStaticSumOffset + kStaticSums * sizeof(float);   // about 32.5 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices];

// Device address of g_static_scratch on the current device, looked up once per device.
cudaError_t static_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = ptr;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

// Up to 32 views' parameters, passed by value as a kernel argument (about 4.4 KB).
constexpr int kStaticViewBatch = 32;
struct StaticViewBatch {
    View v[kStaticViewBatch];
};

// Writes the views of one batch into the array; the parameters travel with the launch.
__global__ void static_views_kernel(StaticViewBatch batch, int nb, View* __restrict__ dst) {
    for (int q = threadIdx.x; q < nb; q += blockDim.x) dst[q] = batch.v[q];
}

}  // namespace

extern "C" kct_status kct_project_static(const kct_volume_desc* vol, const kct_detector_desc* det,
                                         const double* pmats, int32_t nviews, kct_variant variant,
                                         kct_scaling scaling, const float* d_vol, float* d_proj,
                                         int32_t accumulate, void* stream) {
    g_last_error.clear();
    if (!vol || !det || !pmats || !d_vol || !d_proj) return fail(KCT_ERR_INVALID_ARG, "null pointer argument");
    if (vol->nx <= 0 || vol->ny <= 0 || vol->nz <= 0) return fail(KCT_ERR_INVALID_ARG, "volume sizes must be positive");
    if (!(vol->ax > 0.0) || !(vol->ay > 0.0) || !(vol->az > 0.0) || !std::isfinite(vol->ax) ||
        !std::isfinite(vol->ay) || !std::isfinite(vol->az))
        return fail(KCT_ERR_INVALID_ARG, "voxel sizes must be positive and finite");
    if (det->nu <= 0 || det->nv <= 0) return fail(KCT_ERR_INVALID_ARG, "detector sizes must be positive");
    if (nviews <= 0) return fail(KCT_ERR_INVALID_ARG, "nviews must be positive");
    if (variant != KCT_CVP_EXACT && variant != KCT_CVP_RELAXED) return fail(KCT_ERR_INVALID_ARG, "unknown variant");
    if (scaling != KCT_SCALE_COS && scaling != KCT_SCALE_EXACT) return fail(KCT_ERR_INVALID_ARG, "unknown scaling");
    const long long npix = (long long)det->nu * det->nv * nviews;
    if ((size_t)nviews > kStaticViews)
        return fail(KCT_ERR_UNSUPPORTED, "kct_project_static: more than 4096 views");
    if ((size_t)npix > kStaticSums)
        return fail(KCT_ERR_UNSUPPORTED, "kct_project_static: detector pixels x views exceed 8388608");
    if ((long long)vol->nx * vol->ny * vol->nz > (1LL << 31) - 1)
        return fail(KCT_ERR_UNSUPPORTED, "problem too large for 32-bit voxel indexing");

    void* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    e = brick_kernel_attributes();
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    View* d_views = (View*)base;
    int* d_err = (int*)((unsigned char*)base + kStaticErrOffset);
    float* S = (float*)((unsigned char*)base + kStaticSumOffset);
    cudaStream_t st = (cudaStream_t)stream;

    // per-view parameters: every view is validated first, so that a rejected geometry
    // enqueues nothing; then they go to the array in batches of 32, each batch as the
    // by-value argument of one small kernel (no host buffer has to outlive the call)
    StaticViewBatch batch;
    for (int q = 0; q < nviews; ++q) {
        std::string why = setup_view(pmats + 12 * (size_t)q, *vol, batch.v[0]);
        if (!why.empty()) {
            char buf[64];
            std::snprintf(buf, sizeof buf, "view %d: ", q);
            bool unsup = why.compare(0, 12, "unsupported:") == 0;
            return fail(unsup ? KCT_ERR_UNSUPPORTED : KCT_ERR_GEOMETRY, buf + why);
        }
    }
    for (int q0 = 0; q0 < nviews; q0 += kStaticViewBatch) {
        const int nb = (nviews - q0 < kStaticViewBatch) ? nviews - q0 : kStaticViewBatch;
        for (int q = 0; q < nb; ++q) setup_view(pmats + 12 * (size_t)(q0 + q), *vol, batch.v[q]);
        static_views_kernel<<<1, 32, 0, st>>>(batch, nb, d_views + q0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "uploading view parameters");
    }
    Grid G;
    G.nx = vol->nx; G.ny = vol->ny; G.nz = vol->nz;
    G.nu = det->nu; G.nv = det->nv; G.nviews = nviews;
    G.ax = (float)vol->ax; G.ay = (float)vol->ay; G.az = (float)vol->az;
    G.x0 = (float)(0.5 * (1 - vol->nx) * vol->ax);
    G.y0 = (float)(0.5 * (1 - vol->ny) * vol->ay);
    G.z0 = (float)(0.5 * (1 - vol->nz) * vol->az);
    set_grid_doubles(G, *vol);
    // the array keeps the previous call's contents: clear the sums and the error word
    e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, sizeof(float) * (size_t)npix, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const unsigned chunks = (unsigned)((G.nviews + kct::VIEW_CHUNK - 1) / kct::VIEW_CHUNK);
    if (variant == KCT_CVP_RELAXED)
        kct::fwd_kernel<1, -1><<<dim3(bricks(G), segments<1>(G), chunks), kct::NTHREADS, brick_dyn_smem<1>(), st>>>(
            d_views, G, d_vol, S, 0, 0, kct::VIEW_CHUNK, d_err);
    else
        kct::fwd_kernel<0, -1><<<dim3(bricks(G), segments<0>(G), chunks), kct::NTHREADS, brick_dyn_smem<0>(), st>>>(
            d_views, G, d_vol, S, 0, 0, kct::VIEW_CHUNK, d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "forward projection launch");
    dim3 sgrid((unsigned)(((long)G.nu * G.nv + 255) / 256), G.nviews);
    if (scaling == KCT_SCALE_EXACT)
        kct::scale_kernel<1><<<sgrid, 256, 0, st>>>(d_views, G, S, d_proj, accumulate ? 1 : 0);
    else
        kct::scale_kernel<0><<<sgrid, 256, 0, st>>>(d_views, G, S, d_proj, accumulate ? 1 : 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pixel factor launch");
    return KCT_OK;
}

extern "C" kct_status kct_project_static_device_error(int32_t* code, void* stream) {
    g_last_error.clear();
    if (!code) return fail(KCT_ERR_INVALID_ARG, "null output pointer");
    void* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    int* d_err = (int*)((unsigned char*)base + kStaticErrOffset);
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    *code = h;
    return KCT_OK;
}
