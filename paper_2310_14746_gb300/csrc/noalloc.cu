// Allocation-free variant of the FP64 diagnostics reduction.
//
// Some callers cannot allocate device memory at the point where they need the
// diagnostics: code running inside a custom allocator or memory-pool callback,
// an embedding host that hands the library a fixed arena and forbids further
// cudaMalloc calls, or a monitoring hook that must never fail for lack of
// memory. For them this entry point runs the same two reduction kernels as
// hlbm_reduce, but puts the per-block partial sums in a fixed array that lives
// in this file's device memory instead of in memory the library allocates.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (4 MiB + 64 bytes) until the process exits, and every call
// on a device shares it, so two calls whose work overlaps on that GPU (on
// different streams, or from different threads) race on it. The partials are
// fully rewritten by each call before they are read and the final 8 values
// likewise, so nothing in it has to start at zero and it keeps the last
// call's contents.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/hlbm.h"
#include "internal.h"

namespace {

constexpr size_t kMaxPartialBlocks = 65536;  // 8 doubles each: 4 MiB
constexpr size_t kScratchDoubles = kMaxPartialBlocks * 8 + 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct DeviceScratch {
    std::once_flag once;
    cudaError_t status = cudaErrorNotReady;
    double* ptr = nullptr;
};
DeviceScratch g_dev[kMaxDevices];

// Device address of the array on the current device (set up once per device).
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    DeviceScratch& d = g_dev[dev];
    std::call_once(d.once, [&d]() {
        void* p = nullptr;
        d.status = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (d.status == cudaSuccess) d.ptr = static_cast<double*>(p);
    });
    if (d.status != cudaSuccess) return d.status;
    *out = d.ptr;
    return cudaSuccess;
}

// The storage-scale rule of hlbm_set_storage_scale: a power of two in [1, 2^20]
// for FP16 deviations, exactly 1 for the other storage types.
bool scale_ok(int storage, double s) {
    if (!std::isfinite(s)) return false;
    if (storage != HLBM_F16DEV) return s == 1.0;
    int ex = 0;
    return std::frexp(s, &ex) == 0.5 && s >= 1.0 && s <= 1048576.0;
}

}  // namespace

extern "C" int hlbm_reduce_noalloc(int velset, int nx, int ny, int nz, int storage, const int* bc, double tau,
                                   const double* F, double storage_scale, int form, const float* varpi,
                                   const void* f, void* u_prev, hlbm_stats* out, void* cuda_stream) {
    if (!f || !u_prev || !out || !bc || !F) return HLBM_ERR_INVALID_ARG;
    if (velset != HLBM_D2Q9 && velset != HLBM_D3Q19) return HLBM_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (velset == HLBM_D2Q9 && nz != 1)) return HLBM_ERR_INVALID_ARG;
    // the size limits of hlbm_create
    if (ny > 65535 || nz > 65535 || (size_t)nx * ny * nz > ((size_t)1 << 34)) return HLBM_ERR_INVALID_ARG;
    if (storage < HLBM_F64 || storage > HLBM_BF16DEV) return HLBM_ERR_INVALID_ARG;
    if (!(tau > 0.5) || !std::isfinite(tau) || !scale_ok(storage, storage_scale)) return HLBM_ERR_INVALID_ARG;
    if (form != HLBM_HOMOG_SHIFT && form != HLBM_HOMOG_DRAG) return HLBM_ERR_INVALID_ARG;
    if (form == HLBM_HOMOG_DRAG && !varpi) return HLBM_ERR_INVALID_ARG;
    hlbm::LaunchCtx c;
    c.q = velset;
    c.storage = storage;
    c.nx = nx;
    c.ny = ny;
    c.nz = nz;
    for (int a = 0; a < 3; ++a) {
        if (bc[a] != HLBM_PERIODIC && bc[a] != HLBM_HALFWAY_BOUNCE_BACK) return HLBM_ERR_INVALID_ARG;
        if (!std::isfinite(F[a])) return HLBM_ERR_INVALID_ARG;
        c.wall[a] = bc[a] == HLBM_HALFWAY_BOUNCE_BACK;
        c.F[a] = F[a];
    }
    c.tau = tau;
    c.scale = storage_scale;
    c.stream = static_cast<cudaStream_t>(cuda_stream);
    c.drag = form == HLBM_HOMOG_DRAG;
    c.varpi = c.drag ? varpi : nullptr;  // the shift form's moments do not depend on varpi
    if (!hlbm::reduce_grid_fits(c)) return HLBM_ERR_INVALID_ARG;
    if (hlbm::reduce_partials_count(c) > kMaxPartialBlocks) return HLBM_ERR_SCRATCH_LIMIT;

    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e == cudaSuccess) e = hlbm::launch_reduce(c, 0 /* NATURAL layout */, f, u_prev, 1, scratch,
                                                  scratch + kMaxPartialBlocks * 8);
    double v[8];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v, scratch + kMaxPartialBlocks * 8, sizeof(v), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? HLBM_ERR_OOM : HLBM_ERR_CUDA;
    out->mass = v[0];
    out->momentum[0] = v[1];
    out->momentum[1] = v[2];
    out->momentum[2] = v[3];
    out->plane_flux = v[4];
    out->k_app = v[5];
    out->max_du = v[6];
    out->max_u = v[7];
    out->step = 0;
    return HLBM_OK;
}
