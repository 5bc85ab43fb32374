// C ABI of the HBGK library (include/hlbm.h): handles, validation, state
// bookkeeping, CUDA-graph replay of step sequences, checkpoints.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hlbm.h"
#include "internal.h"

using namespace hlbm;

namespace {

thread_local char g_last_cuda[256] = "";

int cuda_fail(cudaError_t e) {
    std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HLBM_ERR_OOM : HLBM_ERR_CUDA;
}

#define HLBM_CUDA(call)                               \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_);  \
    } while (0)

constexpr int kGraphSteps = 8;  // even: a graph returns the state to its starting layout

// The lattice Layout enum values (lattice.cuh), repeated for host code.
constexpr int kNatural = 0, kStreamed = 1, kSwapped = 2;

}  // namespace

struct hlbm_lattice {
    int q = 19, nx = 0, ny = 0, nz = 0, storage = HLBM_F32, pattern = HLBM_TWO_LATTICE;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    double tau = 1.0;
    double F[3] = {0.0, 0.0, 0.0};
    int bc[3] = {HLBM_PERIODIC, HLBM_PERIODIC, HLBM_PERIODIC};
    double scale = 1.0;
    int homog = HLBM_HOMOG_SHIFT;
    size_t cells = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;     // two-lattice: buffer holding the state
    int aa_odd = 0;  // AA: 1 when the state is in the SWAPPED layout
    long long step = 0;
    float* varpi = nullptr;
    float* varpi3 = nullptr;  // diagonal porosity tensor (allocated on first use)
    int aniso = 0;
    unsigned* links = nullptr;  // solid-link masks (resolved obstacles), or null
    void* u_prev = nullptr;
    double* partials = nullptr;
    double* out8 = nullptr;
    double* out8_host = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    int step_variant = HLBM_STEP_AUTO;
    cudaMemPool_t pool = nullptr;  // scratch of the calls that need temporary device memory

    size_t state_bytes() const { return (size_t)q * cells * storage_bytes(storage); }
    size_t arith_bytes() const { return storage == HLBM_F64 ? 8 : 4; }
    int layout() const {
        if (pattern == HLBM_TWO_LATTICE) return kNatural;
        return aa_odd ? kSwapped : kStreamed;
    }
    void* state() const { return buf[pattern == HLBM_TWO_LATTICE ? cur : 0]; }
    LaunchCtx ctx(cudaStream_t s) const {
        LaunchCtx c;
        c.q = q;
        c.storage = storage;
        c.nx = nx;
        c.ny = ny;
        c.nz = nz;
        for (int a = 0; a < 3; ++a) c.wall[a] = bc[a] == HLBM_HALFWAY_BOUNCE_BACK;
        c.tau = tau;
        for (int a = 0; a < 3; ++a) c.F[a] = F[a];
        c.scale = scale;
        c.stream = s;
        c.drag = homog == HLBM_HOMOG_DRAG;
        c.varpi = varpi;
        c.varpi3 = aniso ? varpi3 : nullptr;
        c.links = links;
        c.variant = step_variant;
        return c;
    }
};

namespace {

// All n values in [0, 1] (NaN fails)? The input may be a whole lattice (64 MiB
// at 256^3), so the test runs in blocks without an early exit inside a block:
// the inner loop vectorises, and a bad value still stops the scan at the end
// of its block.
bool host_unit_interval(const float* v, size_t n) {
    constexpr size_t kBlock = 4096;
    for (size_t b = 0; b < n; b += kBlock) {
        const size_t e = b + kBlock < n ? b + kBlock : n;
        int good = 1;
        for (size_t k = b; k < e; ++k) good &= (v[k] >= 0.0f) & (v[k] <= 1.0f);
        if (!good) return false;
    }
    return true;
}

// Make the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Temporary device memory of a call (the adjoint's checkpoints, staging buffers of host
// I/O), stream-ordered on the handle's stream, from a memory pool private to the handle that
// keeps what it has mapped for the next call. With the default pool (release threshold 0) the
// 14.5 GB of checkpoints of a 128^3 x 2000-step gradient were unmapped at every
// synchronisation and mapped again by the next call (0.395 s vs 0.370 s per gradient).
// hlbm_release_scratch hands the memory back; hlbm_destroy destroys the pool.
cudaError_t scratch_alloc(hlbm_t* h, void** p, size_t bytes) {
    if (!h->pool) {
        cudaMemPoolProps pr;
        std::memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = h->device;
        cudaError_t e = cudaMemPoolCreate(&h->pool, &pr);
        if (e != cudaSuccess) {
            h->pool = nullptr;
            return e;
        }
        unsigned long long keep = ~0ull;  // never hand memory back on synchronisation
        e = cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    return cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream);
}

void free_all(hlbm_t* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->varpi);
    cudaFree(h->varpi3);
    cudaFree(h->links);
    cudaFree(h->u_prev);
    cudaFree(h->partials);
    cudaFree(h->out8);
    if (h->out8_host) cudaFreeHost(h->out8_host);
    if (h->pool) cudaMemPoolDestroy(h->pool);  // every scratch block was freed on the stream
}

// One direct time step on `s`, updating the bookkeeping.
int step_once(hlbm_t* h, cudaStream_t s) {
    const LaunchCtx c = h->ctx(s);
    if (h->pattern == HLBM_TWO_LATTICE) {
        HLBM_CUDA(launch_step(c, MODE_TWO_LATTICE, h->buf[h->cur], h->buf[1 - h->cur], h->varpi));
        h->cur = 1 - h->cur;
    } else {
        HLBM_CUDA(launch_step(c, h->aa_odd ? MODE_AA_ODD : MODE_AA_EVEN, h->buf[0], h->buf[0], h->varpi));
        h->aa_odd = 1 - h->aa_odd;
    }
    return HLBM_OK;
}

bool at_graph_origin(const hlbm_t* h) { return h->pattern == HLBM_TWO_LATTICE ? h->cur == 0 : h->aa_odd == 0; }

// Capture kGraphSteps steps starting from the graph origin layout.
int build_graph(hlbm_t* h) {
    if (!h->cap_stream) HLBM_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int cur0 = h->cur, odd0 = h->aa_odd;
    cudaGraph_t graph = nullptr;
    HLBM_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = HLBM_OK;
    for (int k = 0; k < kGraphSteps && rc == HLBM_OK; ++k) rc = step_once(h, h->cap_stream);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    h->cur = cur0;
    h->aa_odd = odd0;
    if (rc != HLBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    h->graph_dirty = false;
    return HLBM_OK;
}

int reset_counters(hlbm_t* h) {
    h->step = 0;
    HLBM_CUDA(cudaMemsetAsync(h->u_prev, 0, 3 * h->cells * h->arith_bytes(), h->stream));
    return HLBM_OK;
}

// Write natural FP64 populations (device pointer; q values if uniform) as the new state.
int write_state(hlbm_t* h, const double* fnat_dev, int uniform) {
    h->cur = 0;
    h->aa_odd = 0;
    const int lay = h->layout();
    HLBM_CUDA(launch_write_state(h->ctx(h->stream), lay, fnat_dev, uniform, h->buf[0]));
    return reset_counters(h);
}

bool is_finite(double v) { return std::isfinite(v); }

// Host-side equilibrium at (rho0, u0) in the documented direction order
// (the same second-order expansion the kernels use, evaluated once).
void host_equilibrium(int q, double rho, const double u[3], double* out) {
    static const int c9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    static const int c19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                   {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                   {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                   {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < q; ++i) {
        const int* c = q == 9 ? c9[i] : c19[i];
        const int c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        const double w = q == 9 ? (c2 == 0 ? 4.0 / 9 : (c2 == 1 ? 1.0 / 9 : 1.0 / 36))
                                : (c2 == 0 ? 1.0 / 3 : (c2 == 1 ? 1.0 / 18 : 1.0 / 36));
        const double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        out[i] = w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

struct CkptHeader {
    char magic[8];
    int q, nx, ny, nz, storage, pattern, cur, aa_odd;
    long long step;
    double tau, F[3], scale;
    int bc[3], pad;
};

}  // namespace

extern "C" {

const char* hlbm_strerror(int status) {
    switch (status) {
        case HLBM_OK: return "ok";
        case HLBM_ERR_INVALID_ARG: return "invalid argument";
        case HLBM_ERR_OOM: return "out of memory";
        case HLBM_ERR_CUDA: return "CUDA error";
        case HLBM_ERR_NOT_CONVERGED: return "not converged";
        case HLBM_ERR_TIMEOUT: return "timeout";
        case HLBM_ERR_BUSY: return "busy";
        case HLBM_ERR_IO: return "I/O error";
        case HLBM_ERR_STATE: return "invalid state for this call";
        case HLBM_ERR_CANCELLED: return "cancelled";
        case HLBM_ERR_SCRATCH_LIMIT: return "lattice too large for the fixed scratch of the allocation-free call";
    }
    return "unknown status";
}

const char* hlbm_last_cuda_error(void) { return g_last_cuda; }

int hlbm_create(hlbm_t** out, int velset, int nx, int ny, int nz, int storage, int pattern, void* cuda_stream) {
    if (!out) return HLBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (velset != HLBM_D2Q9 && velset != HLBM_D3Q19) return HLBM_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return HLBM_ERR_INVALID_ARG;
    if (velset == HLBM_D2Q9 && nz != 1) return HLBM_ERR_INVALID_ARG;
    if (storage < HLBM_F64 || storage > HLBM_BF16DEV) return HLBM_ERR_INVALID_ARG;
    if (pattern != HLBM_TWO_LATTICE && pattern != HLBM_AA) return HLBM_ERR_INVALID_ARG;
    if (ny > 65535 || nz > 65535) return HLBM_ERR_INVALID_ARG;  // launch-grid y and z limits
    const size_t cells = (size_t)nx * ny * nz;
    if (cells > ((size_t)1 << 34)) return HLBM_ERR_INVALID_ARG;

    hlbm_t* h = new (std::nothrow) hlbm_lattice();
    if (!h) return HLBM_ERR_OOM;
    h->q = velset;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->storage = storage;
    h->pattern = pattern;
    h->cells = cells;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->scale = storage == HLBM_F16DEV ? 4096.0 : 1.0;
    cudaError_t e = cudaGetDevice(&h->device);
    const size_t nparts = reduce_partials_count(h->ctx(h->stream));
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[0], h->state_bytes());
    if (e == cudaSuccess && pattern == HLBM_TWO_LATTICE) e = cudaMalloc(&h->buf[1], h->state_bytes());
    if (e == cudaSuccess) e = cudaMalloc(&h->varpi, cells * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->u_prev, 3 * cells * h->arith_bytes());
    if (e == cudaSuccess) e = cudaMalloc(&h->partials, nparts * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->out8, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h->out8_host, 8 * sizeof(double));
    if (e == cudaSuccess) e = launch_fill_f32(h->varpi, cells, 1.0f, h->stream);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e);
        free_all(h);
        delete h;
        return rc;
    }
    int rc = hlbm_init_equilibrium(h, 1.0, 0.0, 0.0, 0.0);
    if (rc == HLBM_OK) {
        cudaError_t s = cudaStreamSynchronize(h->stream);
        if (s != cudaSuccess) rc = cuda_fail(s);
    }
    if (rc != HLBM_OK) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return HLBM_OK;
}

void hlbm_destroy(hlbm_t* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int hlbm_release_scratch(hlbm_t* h) {
    if (!h) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    HLBM_CUDA(cudaStreamSynchronize(h->stream));
    if (h->pool) HLBM_CUDA(cudaMemPoolTrimTo(h->pool, 0));
    return HLBM_OK;
}

int hlbm_set_stream(hlbm_t* h, void* cuda_stream) {
    if (!h) return HLBM_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return HLBM_OK;
}

int hlbm_set_relaxation(hlbm_t* h, double tau) {
    if (!h || !is_finite(tau) || !(tau > 0.5)) return HLBM_ERR_INVALID_ARG;
    h->tau = tau;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_set_force(hlbm_t* h, double Fx, double Fy, double Fz) {
    if (!h || !is_finite(Fx) || !is_finite(Fy) || !is_finite(Fz)) return HLBM_ERR_INVALID_ARG;
    h->F[0] = Fx;
    h->F[1] = Fy;
    h->F[2] = h->q == HLBM_D2Q9 ? 0.0 : Fz;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_set_boundary(hlbm_t* h, int axis, int type) {
    if (!h || axis < 0 || axis > 2) return HLBM_ERR_INVALID_ARG;
    if (type != HLBM_PERIODIC && type != HLBM_HALFWAY_BOUNCE_BACK) return HLBM_ERR_INVALID_ARG;
    if (h->q == HLBM_D2Q9 && axis == 2 && type != HLBM_PERIODIC) return HLBM_ERR_INVALID_ARG;
    if (h->bc[axis] == type) return HLBM_OK;
    if (h->links) return HLBM_ERR_STATE;  // set boundaries before the solid mask
    if (h->pattern == HLBM_AA) {
        // The AA layouts place bounced populations according to the walls:
        // re-lay the post-collision state under the new boundary.
        DeviceGuard g(h->device);
        double* tmp = nullptr;
        HLBM_CUDA(scratch_alloc(h, (void**)&tmp, (size_t)h->q * h->cells * sizeof(double)));
        cudaError_t e = launch_read_state(h->ctx(h->stream), h->layout(), h->state(), tmp);
        h->bc[axis] = type;
        if (e == cudaSuccess) e = launch_write_state(h->ctx(h->stream), h->layout(), tmp, 0, h->buf[0]);
        cudaFreeAsync(tmp, h->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    h->bc[axis] = type;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_set_homogenization(hlbm_t* h, int form) {
    if (!h || (form != HLBM_HOMOG_SHIFT && form != HLBM_HOMOG_DRAG)) return HLBM_ERR_INVALID_ARG;
    if (form == HLBM_HOMOG_DRAG && h->aniso) return HLBM_ERR_STATE;  // the tensor form is a shift form
    h->homog = form;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_set_step_kernel(hlbm_t* h, int variant) {
    if (!h || (variant != HLBM_STEP_AUTO && variant != HLBM_STEP_PER_CELL)) return HLBM_ERR_INVALID_ARG;
    h->step_variant = variant;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_set_storage_scale(hlbm_t* h, double s) {
    if (!h || !is_finite(s)) return HLBM_ERR_INVALID_ARG;
    if (h->storage != HLBM_F16DEV) return s == 1.0 ? HLBM_OK : HLBM_ERR_INVALID_ARG;
    int ex = 0;
    const double m = std::frexp(s, &ex);
    if (m != 0.5 || s < 1.0 || s > 1048576.0) return HLBM_ERR_INVALID_ARG;
    h->scale = s;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_porosity_from_permeability(const float* K, double nu, double tau, float* varpi, size_t n) {
    if ((!K || !varpi) && n) return HLBM_ERR_INVALID_ARG;
    if (!is_finite(nu) || !is_finite(tau) || nu <= 0.0 || tau <= 0.0) return HLBM_ERR_INVALID_ARG;
    for (size_t k = 0; k < n; ++k) {
        const double Kk = K[k];
        double v = Kk > 0.0 ? 1.0 - nu * tau / Kk : 0.0;  // NaN and K <= 0 give 0
        if (!(v >= 0.0)) v = 0.0;
        if (v > 1.0) v = 1.0;
        varpi[k] = (float)v;
    }
    return HLBM_OK;
}

// The handle returns to the scalar porosity field; the captured step graph
// only needs rebuilding when the tensor form was in use (the field's device
// buffer itself does not move).
static void use_scalar_porosity(hlbm_t* h) {
    if (h->aniso) {
        h->aniso = 0;
        h->graph_dirty = true;
    }
}

// Check a device array of n porosity values and copy it into the handle's
// field; the field is unchanged when a value is rejected. Synchronises.
static int porosity_from_device(hlbm_t* h, const float* varpi, size_t n) {
    int* bad = nullptr;
    HLBM_CUDA(scratch_alloc(h, (void**)&bad, sizeof(int)));
    int nbad = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = launch_check_unit_interval(varpi, n, bad, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(bad, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (nbad) return HLBM_ERR_INVALID_ARG;
    HLBM_CUDA(cudaMemcpyAsync(h->varpi, varpi, n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    use_scalar_porosity(h);
    return HLBM_OK;
}

int hlbm_set_porosity(hlbm_t* h, const float* varpi, int on_device) {
    if (!h || !varpi) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const size_t n = h->cells;
    if (on_device) return porosity_from_device(h, varpi, n);
    // A host array goes to a device staging buffer and is checked there (a
    // single host core reads the 64 MiB of a 256^3 field far slower than the
    // copy and a check kernel take); without room for the staging buffer it is
    // checked on the host and copied straight into the field.
    float* stage = nullptr;
    if (scratch_alloc(h, (void**)&stage, n * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();  // the failed allocation leaves no sticky error
        if (!host_unit_interval(varpi, n)) return HLBM_ERR_INVALID_ARG;
        HLBM_CUDA(cudaMemcpyAsync(h->varpi, varpi, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        HLBM_CUDA(cudaStreamSynchronize(h->stream));
        use_scalar_porosity(h);
        return HLBM_OK;
    }
    cudaError_t e = cudaMemcpyAsync(stage, varpi, n * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    const int rc = e == cudaSuccess ? porosity_from_device(h, stage, n) : cuda_fail(e);
    cudaFreeAsync(stage, h->stream);
    if (rc != HLBM_OK) cudaStreamSynchronize(h->stream);  // the host array may be reused at once
    return rc;
}

int hlbm_set_solid_mask(hlbm_t* h, const unsigned char* solid, int on_device) {
    if (!h) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!solid) {  // remove the obstacles
        if (h->links) {
            HLBM_CUDA(cudaStreamSynchronize(h->stream));
            cudaFree(h->links);
            h->links = nullptr;
        }
        h->graph_dirty = true;
        return HLBM_OK;
    }
    // the state's layout (AA) depends on the obstacles: keep the post-collision
    // state across the change, as hlbm_set_boundary does
    double* tmp = nullptr;
    unsigned char* dsolid = nullptr;
    HLBM_CUDA(scratch_alloc(h, (void**)&tmp, (size_t)h->q * h->cells * sizeof(double)));
    cudaError_t e = launch_read_state(h->ctx(h->stream), h->layout(), h->state(), tmp);
    if (e == cudaSuccess && !h->links) e = cudaMalloc(&h->links, h->cells * sizeof(unsigned));
    if (e == cudaSuccess && !on_device) e = scratch_alloc(h, (void**)&dsolid, h->cells);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(dsolid, solid, h->cells, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_build_links(h->ctx(h->stream), on_device ? solid : dsolid, h->links);
    if (e == cudaSuccess) e = launch_write_state(h->ctx(h->stream), h->layout(), tmp, 0, h->state());
    if (dsolid) cudaFreeAsync(dsolid, h->stream);
    cudaFreeAsync(tmp, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_set_porosity_tensor(hlbm_t* h, const float* varpi3, int on_device) {
    if (!h || !varpi3) return HLBM_ERR_INVALID_ARG;
    if (h->homog != HLBM_HOMOG_SHIFT) return HLBM_ERR_STATE;
    DeviceGuard g(h->device);
    const size_t n = 3 * h->cells;
    if (!h->varpi3) HLBM_CUDA(cudaMalloc(&h->varpi3, n * sizeof(float)));
    if (!on_device) {
        if (!host_unit_interval(varpi3, n)) return HLBM_ERR_INVALID_ARG;
        HLBM_CUDA(cudaMemcpyAsync(h->varpi3, varpi3, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        HLBM_CUDA(cudaStreamSynchronize(h->stream));
    } else {
        int* bad = nullptr;
        HLBM_CUDA(scratch_alloc(h, (void**)&bad, sizeof(int)));
        int nbad = 0;
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = launch_check_unit_interval(varpi3, n, bad, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFreeAsync(bad, h->stream);
        if (e != cudaSuccess) return cuda_fail(e);
        if (nbad) return HLBM_ERR_INVALID_ARG;
        HLBM_CUDA(cudaMemcpyAsync(h->varpi3, varpi3, n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    }
    h->aniso = 1;
    h->graph_dirty = true;
    return HLBM_OK;
}

int hlbm_init_equilibrium(hlbm_t* h, double rho0, double ux, double uy, double uz) {
    if (!h || !is_finite(rho0) || !is_finite(ux) || !is_finite(uy) || !is_finite(uz) || !(rho0 > 0.0))
        return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    double u[3] = {ux, uy, h->q == HLBM_D2Q9 ? 0.0 : uz};
    double feq[19];
    host_equilibrium(h->q, rho0, u, feq);
    double* dev = nullptr;
    HLBM_CUDA(scratch_alloc(h, (void**)&dev, sizeof(feq)));
    cudaError_t e = cudaMemcpyAsync(dev, feq, h->q * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    int rc = e == cudaSuccess ? write_state(h, dev, 1) : cuda_fail(e);
    // the pageable source above is consumed before cudaMemcpyAsync returns
    cudaFreeAsync(dev, h->stream);
    return rc;
}

int hlbm_set_populations(hlbm_t* h, const double* f, int on_device) {
    if (!h || !f) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const size_t bytes = (size_t)h->q * h->cells * sizeof(double);
    if (on_device) return write_state(h, f, 0);
    double* dev = nullptr;
    HLBM_CUDA(scratch_alloc(h, (void**)&dev, bytes));
    cudaError_t e = cudaMemcpyAsync(dev, f, bytes, cudaMemcpyHostToDevice, h->stream);
    int rc = e == cudaSuccess ? write_state(h, dev, 0) : cuda_fail(e);
    cudaFreeAsync(dev, h->stream);
    if (rc == HLBM_OK) {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    return rc;
}

int hlbm_get_populations(hlbm_t* h, double* f, int on_device) {
    if (!h || !f) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const LaunchCtx c = h->ctx(h->stream);
    if (on_device) {
        HLBM_CUDA(launch_read_state(c, h->layout(), h->state(), f));
        return HLBM_OK;
    }
    const size_t bytes = (size_t)h->q * h->cells * sizeof(double);
    double* dev = nullptr;
    HLBM_CUDA(scratch_alloc(h, (void**)&dev, bytes));
    cudaError_t e = launch_read_state(c, h->layout(), h->state(), dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, dev, bytes, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(dev, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? HLBM_OK : cuda_fail(e);
}

int hlbm_step(hlbm_t* h, long nsteps) {
    if (!h || nsteps < 0) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    long left = nsteps;
    while (left > 0) {
        if (left >= kGraphSteps && at_graph_origin(h)) {
            if (h->graph_dirty || !h->gexec) {
                int rc = build_graph(h);
                if (rc != HLBM_OK) return rc;
            }
            HLBM_CUDA(cudaGraphLaunch(h->gexec, h->stream));
            left -= kGraphSteps;
            h->step += kGraphSteps;
        } else {
            int rc = step_once(h, h->stream);
            if (rc != HLBM_OK) return rc;
            --left;
            ++h->step;
        }
    }
    return HLBM_OK;
}

int hlbm_get_step(hlbm_t* h, long long* step) {
    if (!h || !step) return HLBM_ERR_INVALID_ARG;
    *step = h->step;
    return HLBM_OK;
}

static int moments_common(hlbm_t* h, void* rho, void* u, int on_device, int f64) {
    if (!h) return HLBM_ERR_INVALID_ARG;
    if (!rho && !u) return HLBM_OK;
    DeviceGuard g(h->device);
    const LaunchCtx c = h->ctx(h->stream);
    if (on_device) {
        HLBM_CUDA(launch_moments(c, h->layout(), h->state(), rho, u, f64));
        return HLBM_OK;
    }
    const size_t es = f64 ? 8 : 4;
    void* drho = nullptr;
    void* du = nullptr;
    cudaError_t e = cudaSuccess;
    if (rho) e = scratch_alloc(h, (void**)&drho, h->cells * es);
    if (e == cudaSuccess && u) e = scratch_alloc(h, (void**)&du, 3 * h->cells * es);
    if (e == cudaSuccess) e = launch_moments(c, h->layout(), h->state(), drho, du, f64);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, drho, h->cells * es, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, 3 * h->cells * es, cudaMemcpyDeviceToHost, h->stream);
    if (drho) cudaFreeAsync(drho, h->stream);
    if (du) cudaFreeAsync(du, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? HLBM_OK : cuda_fail(e);
}

int hlbm_moments(hlbm_t* h, float* rho, float* u, int on_device) { return moments_common(h, rho, u, on_device, 0); }

int hlbm_moments_f64(hlbm_t* h, double* rho, double* u, int on_device) {
    return moments_common(h, rho, u, on_device, 1);
}

int hlbm_reduce(hlbm_t* h, hlbm_stats* out) {
    if (!h || !out) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    HLBM_CUDA(launch_reduce(h->ctx(h->stream), h->layout(), h->state(), h->u_prev, 1, h->partials, h->out8));
    HLBM_CUDA(cudaMemcpyAsync(h->out8_host, h->out8, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(cudaStreamSynchronize(h->stream));
    const double* v = h->out8_host;
    out->mass = v[0];
    out->momentum[0] = v[1];
    out->momentum[1] = v[2];
    out->momentum[2] = v[3];
    out->plane_flux = v[4];
    out->k_app = v[5];
    out->max_du = v[6];
    out->max_u = v[7];
    out->step = h->step;
    return HLBM_OK;
}

int hlbm_reduce_series(hlbm_t* h, long nsamples, int every, double* out, int on_device) {
    if (!h || !out || nsamples < 1 || every < 1) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    const size_t bytes = (size_t)nsamples * 8 * sizeof(double);
    double* dst = out;
    if (!on_device) HLBM_CUDA(scratch_alloc(h, (void**)&dst, bytes));
    int rc = HLBM_OK;
    for (long k = 0; k < nsamples && rc == HLBM_OK; ++k) {
        if (k) rc = hlbm_step(h, every);
        if (rc == HLBM_OK) {
            const cudaError_t e = launch_reduce(h->ctx(h->stream), h->layout(), h->state(), h->u_prev, 0,
                                                h->partials, dst + 8 * k);
            if (e != cudaSuccess) rc = cuda_fail(e);
        }
    }
    if (!on_device) {
        cudaError_t e = cudaSuccess;
        if (rc == HLBM_OK) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
        const cudaError_t ef = cudaFreeAsync(dst, h->stream);
        if (e == cudaSuccess) e = ef;
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (rc == HLBM_OK && e != cudaSuccess) rc = cuda_fail(e);
    }
    return rc;
}

namespace {

// Device allocations of one call, released on every exit path (stream-ordered).
struct Scratch {
    hlbm_t* h;
    std::vector<void*> ptrs;
    explicit Scratch(hlbm_t* hh) : h(hh) {}
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, h->stream);
    }
    cudaError_t alloc(void** p, size_t bytes) {
        cudaError_t e = scratch_alloc(h, p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// Copy the current state into `dst` in the NATURAL layout.
int copy_natural(hlbm_t* h, void* dst, Scratch& sc) {
    if (h->pattern == HLBM_TWO_LATTICE) {
        HLBM_CUDA(cudaMemcpyAsync(dst, h->state(), h->state_bytes(), cudaMemcpyDeviceToDevice, h->stream));
        return HLBM_OK;
    }
    double* tmp = nullptr;
    HLBM_CUDA(sc.alloc((void**)&tmp, (size_t)h->q * h->cells * sizeof(double)));
    HLBM_CUDA(launch_read_state(h->ctx(h->stream), h->layout(), h->state(), tmp));
    HLBM_CUDA(launch_write_state(h->ctx(h->stream), kNatural, tmp, 0, dst));
    return HLBM_OK;
}

// Make a NATURAL-layout buffer the handle's state.
int adopt_natural(hlbm_t* h, const void* src, Scratch& sc) {
    if (h->pattern == HLBM_TWO_LATTICE) {
        HLBM_CUDA(cudaMemcpyAsync(h->buf[0], src, h->state_bytes(), cudaMemcpyDeviceToDevice, h->stream));
        h->cur = 0;
        return HLBM_OK;
    }
    double* tmp = nullptr;
    HLBM_CUDA(sc.alloc((void**)&tmp, (size_t)h->q * h->cells * sizeof(double)));
    HLBM_CUDA(launch_read_state(h->ctx(h->stream), kNatural, src, tmp));
    h->aa_odd = 0;
    HLBM_CUDA(launch_write_state(h->ctx(h->stream), h->layout(), tmp, 0, h->buf[0]));
    return HLBM_OK;
}

}  // namespace

int hlbm_adjoint_flux_grad(hlbm_t* h, long nsteps, int every, int plane_x, double* J, float* grad, int on_device) {
    if (!h || !J || !grad || nsteps < 0 || every < 1 || plane_x < 0 || plane_x >= (h ? h->nx : 0))
        return HLBM_ERR_INVALID_ARG;
    // the adjoint differentiates the isotropic shift form without obstacles
    if (h->homog != HLBM_HOMOG_SHIFT || h->aniso || h->links) return HLBM_ERR_STATE;
    DeviceGuard g(h->device);
    const size_t sb = h->state_bytes();
    const size_t N = h->cells;
    const long nsnap = nsteps > 0 ? (nsteps - 1) / every + 1 : 1;
    const int nseg = every > 2 ? every : 2;  // slot 0/1 double as forward ping-pong buffers
    const LaunchCtx c = h->ctx(h->stream);
    Scratch sc(h);
    char *snaps = nullptr, *seg = nullptr;
    float *lam_a = nullptr, *lam_b = nullptr, *gacc = nullptr;
    double* jdev = nullptr;
    HLBM_CUDA(sc.alloc((void**)&snaps, sb * nsnap));
    HLBM_CUDA(sc.alloc((void**)&seg, sb * nseg));
    HLBM_CUDA(sc.alloc((void**)&lam_a, (size_t)h->q * N * sizeof(float)));
    HLBM_CUDA(sc.alloc((void**)&lam_b, (size_t)h->q * N * sizeof(float)));
    HLBM_CUDA(sc.alloc((void**)&gacc, N * sizeof(float)));
    HLBM_CUDA(sc.alloc((void**)&jdev, sizeof(double)));
    int rc = copy_natural(h, snaps, sc);
    if (rc != HLBM_OK) return rc;

    // forward sweep, keeping f^{k*every}
    void* a = snaps;
    for (long s = 0; s < nsteps; ++s) {
        const bool keep = (s + 1) % every == 0 && (s + 1) / every < nsnap;
        void* b = keep ? (void*)(snaps + sb * ((s + 1) / every)) : (void*)(seg + sb * ((s + 1) & 1));
        HLBM_CUDA(launch_step(c, MODE_TWO_LATTICE, a, b, h->varpi));
        a = b;
    }
    HLBM_CUDA(launch_plane_flux(c, kNatural, a, plane_x, jdev));
    rc = adopt_natural(h, a, sc);
    if (rc != HLBM_OK) return rc;

    // reverse sweep
    HLBM_CUDA(launch_flux_seed(c, lam_a, plane_x));
    HLBM_CUDA(cudaMemsetAsync(gacc, 0, N * sizeof(float), h->stream));
    for (long sg = nsnap - 1; sg >= 0 && nsteps > 0; --sg) {
        const long s0 = sg * every;
        const long s1 = s0 + every < nsteps ? s0 + every : nsteps;
        auto state = [&](long k) -> void* { return k == 0 ? (void*)(snaps + sb * sg) : (void*)(seg + sb * k); };
        for (long k = 0; k + 1 < s1 - s0; ++k) HLBM_CUDA(launch_step(c, MODE_TWO_LATTICE, state(k), state(k + 1), h->varpi));
        for (long s = s1 - 1; s >= s0; --s) {
            HLBM_CUDA(launch_adjoint_step(c, state(s - s0), lam_a, lam_b, h->varpi, gacc));
            float* t = lam_a;
            lam_a = lam_b;
            lam_b = t;
        }
    }
    HLBM_CUDA(cudaMemcpyAsync(grad, gacc, N * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(cudaMemcpyAsync(J, jdev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(cudaStreamSynchronize(h->stream));
    h->step += nsteps;
    return HLBM_OK;
}

int hlbm_save(hlbm_t* h, const char* path) {
    if (!h || !path) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    std::vector<char> st(h->state_bytes());
    std::vector<float> vp(h->cells);
    HLBM_CUDA(cudaMemcpyAsync(st.data(), h->state(), st.size(), cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(cudaMemcpyAsync(vp.data(), h->varpi, vp.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    HLBM_CUDA(cudaStreamSynchronize(h->stream));
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "HLBMCKP1", 8);
    hd.q = h->q;
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.nz = h->nz;
    hd.storage = h->storage;
    hd.pattern = h->pattern;
    hd.cur = 0;
    hd.aa_odd = h->aa_odd;
    hd.step = h->step;
    hd.tau = h->tau;
    for (int a = 0; a < 3; ++a) {
        hd.F[a] = h->F[a];
        hd.bc[a] = h->bc[a];
    }
    hd.scale = h->scale;
    hd.pad = h->homog;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return HLBM_ERR_IO;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(st.data(), 1, st.size(), fp) == st.size() &&
              std::fwrite(vp.data(), sizeof(float), vp.size(), fp) == vp.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? HLBM_OK : HLBM_ERR_IO;
}

int hlbm_load(hlbm_t* h, const char* path) {
    if (!h || !path) return HLBM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return HLBM_ERR_IO;
    CkptHeader hd;
    bool ok = std::fread(&hd, sizeof(hd), 1, fp) == 1 && std::memcmp(hd.magic, "HLBMCKP1", 8) == 0;
    ok = ok && hd.q == h->q && hd.nx == h->nx && hd.ny == h->ny && hd.nz == h->nz && hd.storage == h->storage &&
         hd.pattern == h->pattern;
    std::vector<char> st(ok ? h->state_bytes() : 0);
    std::vector<float> vp(ok ? h->cells : 0);
    ok = ok && std::fread(st.data(), 1, st.size(), fp) == st.size() &&
         std::fread(vp.data(), sizeof(float), vp.size(), fp) == vp.size();
    std::fclose(fp);
    if (!ok) return HLBM_ERR_IO;
    if (!(hd.tau > 0.5)) return HLBM_ERR_IO;
    h->cur = 0;
    h->aa_odd = hd.aa_odd;
    h->step = hd.step;
    h->tau = hd.tau;
    for (int a = 0; a < 3; ++a) {
        h->F[a] = hd.F[a];
        h->bc[a] = hd.bc[a];
    }
    h->scale = hd.scale;
    h->homog = hd.pad == HLBM_HOMOG_DRAG ? HLBM_HOMOG_DRAG : HLBM_HOMOG_SHIFT;
    h->graph_dirty = true;
    HLBM_CUDA(cudaMemcpyAsync(h->buf[0], st.data(), st.size(), cudaMemcpyHostToDevice, h->stream));
    HLBM_CUDA(cudaMemcpyAsync(h->varpi, vp.data(), vp.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    HLBM_CUDA(cudaMemsetAsync(h->u_prev, 0, 3 * h->cells * h->arith_bytes(), h->stream));
    HLBM_CUDA(cudaStreamSynchronize(h->stream));
    return HLBM_OK;
}

}  // extern "C"
