// Continuous-batching solve server: many D3Q19 HBGK lattices of different sizes
// advance together in batched persistent launches.
//
// Each admitted request owns a slot: two population buffers (two-lattice
// streaming), its porosity field, and its residual reference velocity. A
// device slot table lists the small slots of the current round with their tile
// ranges, grouped by kernel class (storage and collision form); one launch
// per class advances every listed slot by one time step, one block per tile
// (a tile never mixes slots). Large slots (kDirectCells) run the single-lattice
// step kernels instead. check_every steps are captured once in a CUDA graph of
// parallel branches (the tile kernels on one, each large slot on one of the
// others) that reads the table from device memory, so admissions, retirements,
// precision changes and the round's set of small slots only rewrite the
// table. After each graph replay a per-slot FP64 reduction (a fixed partition
// per slot, so a slot's result does not depend on its neighbours in the
// batch) gives the residual and the apparent permeability; converged slots
// retire and free their memory, and waiting requests are admitted first-come
// first-served while they fit the memory budget. Each round runs the oldest
// live request and younger ones within a cell budget (choose_run).
//
// Precision ladder. With FP16 or BF16 storage a slot first runs in that
// storage (half the bytes of FP32). Reduced-precision rounding puts a floor
// under the residual that scales with the flow speed (measured for FP16 near
// 6e-4 * max|u|), so a fast flow can never reach an absolute tolerance of
// 1e-6 there. When the residual reaches that floor (or stops improving), the
// slot's state is converted in place to FP32 deviations and the solve
// finishes in FP32 against the requested tolerance.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hlbm.h"
#include "internal.h"
#include "lattice.cuh"
#include "diag.cuh"
#include "k_step_pair.cuh"

namespace hlbm {
namespace srv {

constexpr int kMaxSlots = 1024;
// Kernel classes: 2 * storage + fast for the tile kernel (2..7), and kDirectClass
// for the large slots that run the single-lattice kernels.
constexpr int kDirectClass = 8;
constexpr int kClasses = 9;
// Slots of at least this many cells (64^3 and larger at the serving edges) run the
// single-lattice step kernels, one launch per slot and step inside the round's
// graph, each slot in a branch of the graph (kGraphBranches) so that the
// launches of several slots overlap: the tile kernel's per-block slot lookup (a
// chain of dependent loads before the first population load) costs 10 to 15 % of
// the copy bandwidth (measured: 128^3 FP32 0.90 vs 0.99, 192^3 FP16 0.70 vs 0.83;
// eight 64^3 slots in parallel branches 0.80 vs 0.70 FP16, 0.98 vs 0.89 FP32).
// Smaller slots share the tile kernel, where one launch per class replaces one
// launch per slot.
constexpr size_t kDirectCells = (size_t)1 << 18;
constexpr int kBlock = 256;  // threads per block; a tile is tw x (256 / tw) threads of one slot
// Parallel branches of a round's graph: the tile-kernel classes on one, the large
// slots spread over the others. A slot's steps depend only on its own previous
// step, so the branches are independent, and their kernels (and the partly
// filled last wave of each launch) overlap on the GPU.
constexpr int kGraphBranches = 8;

struct DevSlot {
    void* f[2];
    float* varpi;
    float* u_prev;
    int nx, ny, nz;
    int pair;     // 16-bit storage with an even nx: a thread owns the cells (2 xp, 2 xp + 1)
    int tw_log2;  // tile width in threads along x (cells, or cell pairs when `pair`)
    int tiles_x, tiles_y;
    float rcp_tiles_x, rcp_tiles_y;  // 1/tiles_x, 1/tiles_y for the quotient estimate
    int tile_begin;
    int ntiles;
    int storage;  // HLBM_F32, HLBM_F16DEV or HLBM_BF16DEV
    int fx_only;  // body force along x only
    int direct;   // advanced by the single-lattice step kernels (a large slot), not the tile kernel
    float scale, inv_scale;
    Phys<float> ph;
    double nu, Fx64;
};

struct DevTable {
    int nslots;
    int total_tiles;
    int lo[kClasses], hi[kClasses];  // tile range of each kernel class (kernel_class below)
    int begin[kMaxSlots];   // first tile of each slot (ascending): the slot lookup reads only this
    DevSlot slot[kMaxSlots];
};

__device__ __forceinline__ int find_slot(const DevTable* tab, int t, int ns) {
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&tab->begin[mid]) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Kernel class of a slot: 2 * storage + 1 for the fast form of its storage (the
// force along x, and for 16-bit storage the paired cells: the common serving
// case, compiled on its own for 64 registers), else 2 * storage. The table
// keeps the slots of a class contiguous.
__host__ __device__ inline int kernel_class(const DevSlot& d) {
    if (d.direct) return kDirectClass;
    const bool fast = d.fx_only && (d.storage == HLBM_F32 || d.pair);
    return 2 * d.storage + (fast ? 1 : 0);
}

// Tile geometry of a slot: the tile width is the largest power of two (up to
// 128) that divides the row's thread count, so the serving edges 32..192
// leave no idle lanes; rows whose count has no such divisor of at least 16
// use the next power of two instead.
inline void set_tiles(DevSlot& d) {
    d.pair = d.storage != HLBM_F32 && d.nx % 2 == 0;
    const int w = d.pair ? d.nx / 2 : d.nx;
    int tw = 1;
    while (tw < 128 && w % (2 * tw) == 0) tw *= 2;
    if (tw < 16 && tw < w) {
        tw = 16;
        while (tw < 128 && tw < w) tw *= 2;
    }
    d.tw_log2 = 0;
    while ((1 << d.tw_log2) < tw) ++d.tw_log2;
    const int th = kBlock / tw;
    d.tiles_x = (w + tw - 1) / tw;
    d.tiles_y = (d.ny + th - 1) / th;
    d.rcp_tiles_x = 1.0f / (float)d.tiles_x;
    d.rcp_tiles_y = 1.0f / (float)d.tiles_y;
    d.ntiles = d.tiles_x * d.tiles_y * d.nz;
}

// One cell update of a slot in storage S; launch k of an interval reads f[k&1]
// and writes f[(k+1)&1] (each interval has an even number of steps).
template <class S, bool FX>
__device__ __forceinline__ void advance_cell(const DevSlot& sl, int k, int x, int y, int z) {
    using C = typename S::C;
    using T = typename S::T;
    const Geometry g{sl.nx, sl.ny, sl.nz, 0, 0, 0, (size_t)sl.nx * sl.ny * sl.nz};
    const Phys<C> ph = sl.ph;
    const T* fin = static_cast<const T*>(sl.f[k & 1]);
    T* fout = static_cast<T*>(sl.f[(k + 1) & 1]);
    const Nbr<int> nb(g, x, y, z);
    const int cell = x + g.nx * (y + g.ny * z);
    C d[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) d[i] = S::load_raw(fin, gather_index<19, false>(g, nb, cell, i, NATURAL));
    const C vp = C(__ldg(sl.varpi + cell));
    if (FX) collide<19, C, S::scaled, true>(d, vp, ph, C(sl.scale), C(sl.inv_scale), WriteBack<C>{d});  // fx_only
    else collide<19, C, S::scaled, false>(d, vp, ph, C(sl.scale), C(sl.inv_scale), WriteBack<C>{d});
#pragma unroll
    for (int i = 0; i < 19; ++i) S::store_raw(fout, i * (int)g.N + cell, d[i]);
}

// Update of the cell pair (x0, x0 + 1) of a 16-bit slot (the paired scheme of
// the single-lattice 16-bit kernel: shared y/z neighbour arithmetic, 32-bit
// word loads where the pair's populations share a word, one paired
// conversion per stored word).
template <class S, bool FX>
__device__ __forceinline__ void advance_pair(const DevSlot& sl, int k, int x0, int y, int z) {
    using P = Pair16<S>;
    using T = typename S::T;
    const Geometry g{sl.nx, sl.ny, sl.nz, 0, 0, 0, (size_t)sl.nx * sl.ny * sl.nz};
    const int N = (int)g.N;
    Planes<const T, 19> fin;
    const T* base = static_cast<const T*>(sl.f[k & 1]);
#pragma unroll
    for (int i = 0; i < 19; ++i) fin.p[i] = base + i * N;
    T* fout = static_cast<T*>(sl.f[(k + 1) & 1]);
    const int cell = x0 + g.nx * (y + g.ny * z);
    const Nbr<int> nb(g, x0, y, z);
    const int xm1 = x0 == 0 ? g.nx - 1 : -1;
    const int xp2 = x0 + 2 >= g.nx ? -x0 : 2;
    const float2 vp = __ldg(reinterpret_cast<const float2*>(sl.varpi + cell));
    const Phys<float> ph = sl.ph;
    PackedPairs<S, 19> d;  // the loaded words; lane 0: cell x0, lane 1: cell x0 + 1
    if (FX) pair_gather_words<19, S, LD_WORDS>(fin, cell, nb, xm1, xp2, d.w);
    else pair_gather_words<19, S, LD_HALVES>(fin, cell, nb, xm1, xp2, d.w);
    const auto store = [&](int i, F2 v) {  // one 32-bit word per direction, stored once final
        const float2 f = v.split();
        *reinterpret_cast<unsigned*>(fout + (i * N + cell)) = P::pack(f.x, f.y);
    };
    if (FX) collide<19, F2, S::scaled, true>(d, F2(vp.x, vp.y), ph, sl.scale, sl.inv_scale, store);  // fx_only
    else collide<19, F2, S::scaled, false>(d, F2(vp.x, vp.y), ph, sl.scale, sl.inv_scale, store);
}

// q = n / d and r = n % d for 0 <= n < 2^21, d >= 1 (a slot has fewer tiles): a float-reciprocal
// estimate corrected to the exact quotient (no integer division; checked
// exhaustively on the host for n < 2^21 and d up to 256 plus larger samples).
__device__ __forceinline__ int divmod(int n, int d, float rcp, int& r) {
    int q = __float2int_rz(__int2float_rn(n) * rcp);
    r = n - q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
    return q;
}

// Thread `tid` of tile `lt` of a slot: its x thread index (a cell, or a cell
// pair), y and z; false past the lattice edge.
__device__ __forceinline__ bool tile_cell(const DevSlot& sl, int lt, int tid, int& xt, int& y, int& z) {
    int tx, ty;
    const int rest = divmod(lt, sl.tiles_x, sl.rcp_tiles_x, tx);
    z = divmod(rest, sl.tiles_y, sl.rcp_tiles_y, ty);
    const int tw = 1 << sl.tw_log2;
    xt = tx * tw + (tid & (tw - 1));
    y = ty * (kBlock >> sl.tw_log2) + (tid >> sl.tw_log2);
    return xt < (sl.pair ? sl.nx >> 1 : sl.nx) && y < sl.ny;
}

// One time step of one tile of a live slot stored as S: block b handles tile
// lo[c] + b of the table, c = 2 * S::kind + FAST (the slots of each kernel
// class form one contiguous tile range, so each class has its own kernel and
// register budget); blocks past the range exit at once. The tile's slot
// descriptor is staged in shared memory, so its fields are read where they
// are used instead of held in registers.
template <class S, bool FAST>
__global__ void __launch_bounds__(kBlock, FAST ? 4 : 3)
k_batched_step(const DevTable* __restrict__ tab, int k) {
    __shared__ DevSlot sl;
    constexpr int kWords = (int)(sizeof(DevSlot) / sizeof(int));
    constexpr int cls = 2 * S::kind + (FAST ? 1 : 0);
    constexpr bool k16 = S::kind == HLBM_F16DEV || S::kind == HLBM_BF16DEV;
    const int t = tab->lo[cls] + blockIdx.x;
    if (t >= tab->hi[cls]) return;  // uniform over the block
    if ((int)threadIdx.x < kWords)
        reinterpret_cast<int*>(&sl)[threadIdx.x] =
            reinterpret_cast<const int*>(&tab->slot[find_slot(tab, t, tab->nslots)])[threadIdx.x];
    __syncthreads();
    int x, y, z;
    if (!tile_cell(sl, t - sl.tile_begin, threadIdx.x, x, y, z)) return;
    if constexpr (FAST) {  // force along x; 16-bit slots of this class are paired
        if constexpr (k16) advance_pair<S, true>(sl, k, 2 * x, y, z);
        else advance_cell<S, true>(sl, k, x, y, z);
    } else {
        if constexpr (k16) {
            if (sl.pair) {  // uniform over the block
                advance_pair<S, false>(sl, k, 2 * x, y, z);
                return;
            }
        }
        if (sl.fx_only) advance_cell<S, true>(sl, k, x, y, z);
        else advance_cell<S, false>(sl, k, x, y, z);
    }
}

// Diagnostics of one cell of a slot in storage S, added to the thread's
// accumulator (see k_batched_partials).
template <class S>
__device__ __forceinline__ void cell_stats(const DevSlot& sl, int x, int y, int z, DiagCell<typename S::C>& a) {
    using C = typename S::C;
    using T = typename S::T;
    const Geometry g{sl.nx, sl.ny, sl.nz, 0, 0, 0, (size_t)sl.nx * sl.ny * sl.nz};
    const Phys<C> ph = sl.ph;
    const T* f = static_cast<const T*>(sl.f[0]);
    const Nbr<int> nb(g, x, y, z);
    const int cell = x + g.nx * (y + g.ny * z);
    C d[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) d[i] = S::load(f, gather_index<19, false>(g, nb, cell, i, NATURAL), C(sl.inv_scale));
    C drho, jx, jy, jz;
    moments<19, C>(d, drho, jx, jy, jz);
    C u3[3];
    velocity<C>(jx, jy, jz, C(1) / (C(1) + drho), ph, u3[0], u3[1], u3[2]);
    C up[3];
    const int N = (int)g.N;
#pragma unroll
    for (int c = 0; c < 3; ++c) up[c] = sl.u_prev[c * N + cell];
    a.fluid += 1;
    a.p[0] += drho;  // rho*u = j + F/2: F/2 is added per block from the counts
    a.p[1] += jx;
    a.p[2] += jy;
    a.p[3] += jz;
    if (x == g.nx - 1) {
        a.plane += 1;
        a.p[4] += jx;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.du = nan_max(a.du, fabsf(u3[c] - up[c]));
        a.um = nan_max(a.um, fabsf(u3[c]));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) sl.u_prev[c * N + cell] = u3[c];
}

// Per-tile FP64 partials of the diagnostics (one block per tile of any slot,
// the tiles of the step kernel: one or two cells per thread): sum drho, sum
// rho*u (3), plane flux, 0, max|du|, max|u|; fixed-order fold.
__global__ void __launch_bounds__(kBlock)
k_batched_partials(const DevTable* __restrict__ tab, double* __restrict__ partials) {
    __shared__ DiagShared sh;
    const int t = blockIdx.x;
    const DevSlot& sl = tab->slot[find_slot(tab, t, tab->nslots)];
    int xt, y, z;
    DiagCell<float> a;
    if (tile_cell(sl, t - sl.tile_begin, threadIdx.x, xt, y, z)) {
        const int n = sl.pair ? 2 : 1;
        for (int h = 0; h < n; ++h) {
            const int x = sl.pair ? 2 * xt + h : xt;
            switch (sl.storage) {
                case HLBM_F16DEV: cell_stats<StoreF16>(sl, x, y, z, a); break;
                case HLBM_BF16DEV: cell_stats<StoreBF16>(sl, x, y, z, a); break;
                default: cell_stats<StoreF32>(sl, x, y, z, a); break;
            }
        }
    }
    diag_fold<float>(a, sh, threadIdx.x, kBlock, (double)sl.ph.Fx, (double)sl.ph.Fy, (double)sl.ph.Fz,
                        partials + (size_t)t * 8);
}

// One block per slot folds that slot's tile partials in a fixed order.
__global__ void __launch_bounds__(256)
k_batched_final(const DevTable* __restrict__ tab, const double* __restrict__ partials, double* __restrict__ out) {
    __shared__ double buf[256];
    const DevSlot& sl = tab->slot[blockIdx.x];
    const double* p = partials + (size_t)sl.tile_begin * 8;
    double v[8];
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        v[c] = c == 5 ? 0.0 : fold_column(p, (size_t)sl.ntiles, c, buf);
        __syncthreads();  // buf is reused by the next column
    }
    if (threadIdx.x == 0) {
        const double cells = (double)sl.nx * sl.ny * sl.nz;
        double* o = out + (size_t)blockIdx.x * 8;
        o[0] = cells + v[0];
        o[1] = v[1];
        o[2] = v[2];
        o[3] = v[3];
        o[4] = v[4];
        o[5] = sl.Fx64 != 0.0 ? sl.nu * (v[1] / cells) / sl.Fx64 : 0.0;
        o[6] = v[6];
        o[7] = v[7];
    }
}

// Reduced-precision deviations (times s) -> FP32 deviations, element-wise.
template <class S>
__global__ void k_widen(const typename S::T* __restrict__ in, float* __restrict__ out, size_t n, float inv_s) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = S::load(in, i, inv_s);
}

}  // namespace srv
}  // namespace hlbm

using namespace hlbm;
using namespace hlbm::srv;

namespace {

thread_local char g_srv_err[256] = "";

int srv_cuda_fail(cudaError_t e) {
    std::snprintf(g_srv_err, sizeof(g_srv_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HLBM_ERR_OOM : HLBM_ERR_CUDA;
}

#define SRV_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return srv_cuda_fail(e_); \
    } while (0)

struct Pending {
    uint64_t id;
    hlbm_request req;
    float* field = nullptr;  // pinned host copy of varpi
    double t_submit = 0.0;
    int alloc_failures = 0;  // admissions that failed for lack of device memory
};

// With no live slot nothing will free memory; after this many failed
// admissions in a row the request fails with HLBM_ERR_OOM.
constexpr int kMaxAllocRetries = 8;
// A reduced-precision slot moves to FP32 once its residual is below
// floor_coef * max|u| (or the tolerance), or its relative residual has not
// improved by 10 % for this many checks while within kStallBand times the floor.
constexpr int kStallChecks = 20;
constexpr double kStallBand = 10.0;

struct Live {
    Pending p;
    DevSlot ds;
    size_t bytes = 0;
    long long steps = 0;
    long long steps_low = 0;  // steps run in the reduced-precision storage
    double t_admit = 0.0;
    double best_du = 1e300;  // best relative residual max|du| / max|u| so far
    int stall = 0;
    bool cancel = false;
};

double feq_rest(int i) {
    // lattice weights of D3Q19 in the documented order: rest 1/3, faces 1/18, edges 1/36
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

double scale_of(int storage) { return storage == HLBM_F16DEV ? 4096.0 : 1.0; }

}  // namespace

struct hlbm_server {
    int storage = HLBM_F16DEV;  // storage new slots start in
    int check_every = 100;
    int refine = 1;             // move reduced-precision slots to FP32 at their floor
    double floor_coef = 2e-3;   // reduced-precision residual floor, in units of max|u|
    double backfill = 0.1;      // cells younger requests may add to a round, per cell of the oldest
    std::vector<int> run;       // live slots (indices) that run this round, in table order
    std::vector<uint64_t> table_ids;  // request ids of the slots in the device table, in order
    size_t budget = 0, used = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaStream_t branch[kGraphBranches] = {};  // capture streams of the graph's parallel branches
    cudaEvent_t fork_ev = nullptr, join_ev[kGraphBranches] = {};
    int device = 0;
    std::mutex mu;
    std::deque<Pending> waiting;
    std::vector<Live> live;
    std::deque<hlbm_result> done;
    DevTable* dtab = nullptr;
    DevTable* htab = nullptr;
    bool table_dirty = true;
    cudaGraphExec_t gexec = nullptr;
    int grid[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // blocks of the captured launches per tile-kernel class (>= its tiles)
    // large slots advanced by single-lattice launches in the captured graph: (id, storage) of each
    std::vector<std::pair<uint64_t, int>> graph_direct;
    double* dpartials = nullptr;
    size_t partial_cap = 0;  // tiles
    double* dout = nullptr;
    double* hout = nullptr;
    double* dfeq = nullptr;
    uint64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    int inject_alloc_failures = 0;
    long long lups = 0;  // lattice updates done
    long long rounds = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    static size_t bytes_for(int st, size_t n) { return 2 * 19 * n * storage_bytes(st) + n * sizeof(float) * 4; }
    size_t slot_bytes(const hlbm_request& r) const {
        return bytes_for(storage, (size_t)r.nx * r.ny * r.nz);
    }
    LaunchCtx ctx_for(const Live& l) const {
        LaunchCtx c;
        c.q = 19;
        c.storage = l.ds.storage;
        c.nx = l.ds.nx;
        c.ny = l.ds.ny;
        c.nz = l.ds.nz;
        c.wall[0] = c.wall[1] = c.wall[2] = 0;
        c.tau = l.p.req.tau;
        c.F[0] = l.p.req.F[0];
        c.F[1] = l.p.req.F[1];
        c.F[2] = l.p.req.F[2];
        c.scale = l.ds.scale;
        c.stream = stream;
        return c;
    }
};

namespace {

void free_slot(hlbm_server_t* s, Live& l) {
    cudaFreeAsync(l.ds.f[0], s->stream);
    cudaFreeAsync(l.ds.f[1], s->stream);
    cudaFreeAsync(l.ds.varpi, s->stream);
    cudaFreeAsync(l.ds.u_prev, s->stream);
    s->used -= l.bytes;
}

void finish(hlbm_server_t* s, Live& l, int status, const double* o) {
    hlbm_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = l.p.id;
    r.tag = l.p.req.tag;
    r.status = status;
    r.nx = l.ds.nx;
    r.ny = l.ds.ny;
    r.nz = l.ds.nz;
    r.steps = l.steps;
    r.steps_low = l.steps_low;
    r.final_storage = l.ds.storage;
    if (o) {
        r.mass = o[0];
        r.plane_flux = o[4];
        r.k_app = o[5];
        r.max_du = o[6];
        r.max_u = o[7];
    }
    r.t_submit = l.p.t_submit;
    r.t_admit = l.t_admit;
    r.t_finish = s->now();
    s->done.push_back(r);
}

void finish_pending(hlbm_server_t* s, Pending& p, int status) {
    hlbm_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = p.id;
    r.tag = p.req.tag;
    r.status = status;
    r.nx = p.req.nx;
    r.ny = p.req.ny;
    r.nz = p.req.nz;
    r.final_storage = s->storage;
    r.t_submit = p.t_submit;
    r.t_admit = -1.0;
    r.t_finish = s->now();
    s->done.push_back(r);
    cudaFreeHost(p.field);
    p.field = nullptr;
}

cudaError_t alloc_or_inject(hlbm_server_t* s, void** p, size_t bytes) {
    if (s->inject_alloc_failures > 0) {
        --s->inject_alloc_failures;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s->stream);
}

// Allocate and initialise a slot; returns cudaSuccess or the failing error (nothing leaked).
cudaError_t admit(hlbm_server_t* s, Pending& p, Live& l) {
    const hlbm_request& r = p.req;
    const size_t n = (size_t)r.nx * r.ny * r.nz;
    const size_t fb = 19 * n * storage_bytes(s->storage);
    std::memset(&l.ds, 0, sizeof(l.ds));
    void* ptrs[4] = {nullptr, nullptr, nullptr, nullptr};
    const size_t sizes[4] = {fb, fb, n * sizeof(float), 3 * n * sizeof(float)};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = alloc_or_inject(s, &ptrs[k], sizes[k]);
    if (e != cudaSuccess) {
        for (void* q : ptrs)
            if (q) cudaFreeAsync(q, s->stream);
        return e;
    }
    l.p = p;
    l.ds.f[0] = ptrs[0];
    l.ds.f[1] = ptrs[1];
    l.ds.varpi = static_cast<float*>(ptrs[2]);
    l.ds.u_prev = static_cast<float*>(ptrs[3]);
    l.ds.nx = r.nx;
    l.ds.ny = r.ny;
    l.ds.nz = r.nz;
    l.ds.fx_only = r.F[1] == 0.0 && r.F[2] == 0.0;
    l.ds.direct = n >= kDirectCells ? 1 : 0;
    l.ds.storage = s->storage;
    set_tiles(l.ds);
    l.ds.scale = (float)scale_of(s->storage);
    l.ds.inv_scale = (float)(1.0 / scale_of(s->storage));
    l.ds.ph = make_phys<float, 19>(r.tau, r.F);
    l.ds.nu = (r.tau - 0.5) / 3.0;
    l.ds.Fx64 = r.F[0];
    l.bytes = s->slot_bytes(r);
    l.steps = 0;
    l.t_admit = s->now();
    e = cudaMemcpyAsync(l.ds.varpi, p.field, n * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(l.ds.u_prev, 0, 3 * n * sizeof(float), s->stream);
    if (e == cudaSuccess) e = launch_write_state(s->ctx_for(l), 0 /*NATURAL*/, s->dfeq, 1, l.ds.f[0]);
    if (e != cudaSuccess) {
        for (void* q : ptrs) cudaFreeAsync(q, s->stream);
        return e;
    }
    s->used += l.bytes;
    return cudaSuccess;
}

// Move a reduced-precision slot to FP32 storage (state converted in place).
// Returns cudaErrorMemoryAllocation (nothing changed) when it does not fit.
cudaError_t widen_to_fp32(hlbm_server_t* s, Live& l) {
    const size_t n = (size_t)l.ds.nx * l.ds.ny * l.ds.nz;
    const size_t extra = hlbm_server::bytes_for(HLBM_F32, n) - l.bytes;
    if (s->used + extra > s->budget) return cudaErrorMemoryAllocation;
    void* a = nullptr;
    void* b = nullptr;
    cudaError_t e = alloc_or_inject(s, &a, 19 * n * sizeof(float));
    if (e == cudaSuccess) e = alloc_or_inject(s, &b, 19 * n * sizeof(float));
    if (e != cudaSuccess) {
        if (a) cudaFreeAsync(a, s->stream);
        return e;
    }
    const unsigned grid = (unsigned)std::min<size_t>((19 * n + 255) / 256, 152 * 16);
    if (l.ds.storage == HLBM_F16DEV)
        k_widen<StoreF16><<<grid, 256, 0, s->stream>>>(static_cast<const __half*>(l.ds.f[0]), static_cast<float*>(a),
                                                       19 * n, l.ds.inv_scale);
    else
        k_widen<StoreBF16><<<grid, 256, 0, s->stream>>>(static_cast<const __nv_bfloat16*>(l.ds.f[0]),
                                                        static_cast<float*>(a), 19 * n, l.ds.inv_scale);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(a, s->stream);
        cudaFreeAsync(b, s->stream);
        return e;
    }
    cudaFreeAsync(l.ds.f[0], s->stream);
    cudaFreeAsync(l.ds.f[1], s->stream);
    l.ds.f[0] = a;
    l.ds.f[1] = b;
    l.ds.storage = HLBM_F32;
    set_tiles(l.ds);  // per-cell tiles from now on
    l.ds.scale = 1.0f;
    l.ds.inv_scale = 1.0f;
    s->used += extra;
    l.bytes += extra;
    l.best_du = 1e300;
    l.stall = 0;
    return cudaSuccess;
}

// Capture check_every steps of this round's slots with the current grid sizes:
// the tile-kernel classes (per step: the reduced-precision classes, then the
// FP32 ones) on one branch, each large slot's single-lattice launches on one of
// the other branches (round robin), all forked from and joined into the
// capture stream.
int build_graph(hlbm_server_t* s) {
    if (!s->cap_stream) SRV_CUDA(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
    if (!s->fork_ev) SRV_CUDA(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    for (int b = 0; b < kGraphBranches; ++b) {
        if (!s->branch[b]) SRV_CUDA(cudaStreamCreateWithFlags(&s->branch[b], cudaStreamNonBlocking));
        if (!s->join_ev[b]) SRV_CUDA(cudaEventCreateWithFlags(&s->join_ev[b], cudaEventDisableTiming));
    }
    s->graph_direct.clear();
    std::vector<const Live*> direct;
    for (int idx : s->run) {
        const Live& l = s->live[idx];
        if (l.ds.direct) {
            direct.push_back(&l);
            s->graph_direct.emplace_back(l.p.id, l.ds.storage);
        }
    }
    bool tiles = false;
    for (int c = 0; c < 8; ++c) tiles = tiles || s->grid[c] > 0;
    const int first_direct = tiles ? 1 : 0;  // branch 0 carries the tile kernels when there are any
    const int direct_branches = kGraphBranches - first_direct;
    const int used = std::min<int>(kGraphBranches, first_direct + (int)direct.size());
    cudaGraph_t graph = nullptr;
    SRV_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaEventRecord(s->fork_ev, s->cap_stream);
    for (int b = 0; b < used && le == cudaSuccess; ++b) le = cudaStreamWaitEvent(s->branch[b], s->fork_ev, 0);
    const auto launch = [&](auto kern, int blocks, int k) {
        if (blocks > 0 && le == cudaSuccess) {
            kern<<<blocks, kBlock, 0, s->branch[0]>>>(s->dtab, k);
            le = cudaGetLastError();
        }
    };
    for (int k = 0; k < s->check_every && le == cudaSuccess; ++k) {
        const int* g = s->grid;
        for (size_t d = 0; d < direct.size(); ++d) {  // launch k reads f[k & 1], writes f[(k + 1) & 1]
            if (le != cudaSuccess) break;
            const Live* l = direct[d];
            LaunchCtx c = s->ctx_for(*l);
            c.stream = s->branch[first_direct + (int)(d % direct_branches)];
            le = launch_step(c, MODE_TWO_LATTICE, l->ds.f[k & 1], l->ds.f[(k + 1) & 1], l->ds.varpi);
        }
        launch(k_batched_step<StoreF16, true>, g[2 * HLBM_F16DEV + 1], k);
        launch(k_batched_step<StoreF16, false>, g[2 * HLBM_F16DEV], k);
        launch(k_batched_step<StoreBF16, true>, g[2 * HLBM_BF16DEV + 1], k);
        launch(k_batched_step<StoreBF16, false>, g[2 * HLBM_BF16DEV], k);
        launch(k_batched_step<StoreF32, true>, g[2 * HLBM_F32 + 1], k);
        launch(k_batched_step<StoreF32, false>, g[2 * HLBM_F32], k);
    }
    for (int b = 0; b < used && le == cudaSuccess; ++b) {
        le = cudaEventRecord(s->join_ev[b], s->branch[b]);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(s->cap_stream, s->join_ev[b], 0);
    }
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &graph);
    if (e == cudaSuccess && le != cudaSuccess) {
        cudaGraphDestroy(graph);
        e = le;
    }
    if (e != cudaSuccess) return srv_cuda_fail(e);
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    e = cudaGraphInstantiate(&s->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return srv_cuda_fail(e);
    return HLBM_OK;
}

// Grid for `tiles` tiles: a power of two >= tiles, kept while it stays within 8x;
// no launch for an empty class.
int fit_grid(int cur, int tiles) {
    if (tiles == 0) return 0;
    if (cur >= tiles && cur <= 8 * tiles) return cur;
    int g = 256;
    while (g < tiles) g *= 2;
    return g;
}

// This round's slots. The oldest live request (lowest id) runs every round;
// younger slots are added in age order (skipping those that do not fit, so a
// small request can pass a large one) while the round stays within a cell
// budget of max(kRoundCells, (1 + backfill) * the oldest request's cells).
// The oldest request therefore never runs slower than 1 / (1 + backfill) of
// its speed alone, however long the queue behind it: the batch approaches
// first-come first-served for long solves (which bounds the tail) while short
// requests fill the rest of each round. kRoundCells keeps a small oldest
// request from leaving the GPU idle: about a million cells (some 4000 blocks
// of 256 cells, six waves over 152 SMs) keep every SM streaming, and a larger
// floor would let younger requests slow an oldest request of 128^3 (2.1M
// cells) by far more than the backfill allows. A very large backfill is plain processor
// sharing. Returns true when the set (or its order) differs from the device
// table.
constexpr double kRoundCells = 1.0e6;

bool choose_run(hlbm_server_t* s) {
    std::vector<int> age(s->live.size());
    for (int i = 0; i < (int)age.size(); ++i) age[i] = i;
    std::sort(age.begin(), age.end(), [s](int a, int b) { return s->live[a].p.id < s->live[b].p.id; });
    s->run.clear();
    double cells = 0.0, budget = 0.0;
    for (size_t r = 0; r < age.size(); ++r) {
        const Live& l = s->live[age[r]];
        const double n = (double)l.ds.nx * l.ds.ny * l.ds.nz;
        if (r == 0) {
            budget = std::max(kRoundCells, (1.0 + s->backfill) * n);
        } else if (cells + n > budget) {
            continue;
        }
        s->run.push_back(age[r]);
        cells += n;
    }
    std::stable_sort(s->run.begin(), s->run.end(), [s](int a, int b) {
        const int ca = kernel_class(s->live[a].ds), cb = kernel_class(s->live[b].ds);
        return ca != cb ? ca < cb : s->live[a].p.id < s->live[b].p.id;
    });
    if (s->run.size() != s->table_ids.size()) return true;
    for (size_t k = 0; k < s->run.size(); ++k)
        if (s->live[s->run[k]].p.id != s->table_ids[k]) return true;
    return false;
}

int upload_table(hlbm_server_t* s) {
    // the running slots grouped by kernel class (each class kernel strides over its own
    // range); a slot's arithmetic does not depend on its position in the table
    int tiles = 0;
    s->htab->nslots = (int)s->run.size();
    s->table_ids.clear();
    for (int c = 0; c < kClasses; ++c) s->htab->lo[c] = s->htab->hi[c] = 0;
    for (size_t k = 0; k < s->run.size(); ++k) {
        Live& l = s->live[s->run[k]];
        const int c = kernel_class(l.ds);
        if (k == 0 || kernel_class(s->live[s->run[k - 1]].ds) != c) s->htab->lo[c] = tiles;
        l.ds.tile_begin = tiles;
        s->htab->begin[k] = tiles;
        tiles += l.ds.ntiles;
        s->htab->hi[c] = tiles;
        s->htab->slot[k] = l.ds;
        s->table_ids.push_back(l.p.id);
    }
    s->htab->total_tiles = tiles;
    if ((size_t)tiles > s->partial_cap) {
        if (s->dpartials) cudaFreeAsync(s->dpartials, s->stream);
        s->dpartials = nullptr;
        s->partial_cap = 0;
        size_t cap = std::max<size_t>((size_t)tiles * 2, 4096);
        SRV_CUDA(cudaMallocAsync(&s->dpartials, cap * 8 * sizeof(double), s->stream));
        s->partial_cap = cap;
    }
    const size_t bytes = offsetof(DevTable, slot) + sizeof(DevSlot) * s->run.size();
    SRV_CUDA(cudaMemcpyAsync(s->dtab, s->htab, bytes, cudaMemcpyHostToDevice, s->stream));
    s->table_dirty = false;
    bool rebuild = !s->gexec;
    {  // the large slots are launched one by one: a change in their set needs a new graph
        std::vector<std::pair<uint64_t, int>> direct;
        for (int idx : s->run)
            if (s->live[idx].ds.direct) direct.emplace_back(s->live[idx].p.id, s->live[idx].ds.storage);
        rebuild = rebuild || direct != s->graph_direct;
    }
    for (int c = 0; c < 8; ++c) {
        const int gc = fit_grid(s->grid[c], s->htab->hi[c] - s->htab->lo[c]);
        rebuild = rebuild || gc != s->grid[c];
        s->grid[c] = gc;
    }
    if (rebuild) {
        return build_graph(s);
    }
    return HLBM_OK;
}

}  // namespace

extern "C" {

int hlbm_server_create(hlbm_server_t** out, size_t mem_budget, int storage, int check_every, void* cuda_stream) {
    if (!out) return HLBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (storage != HLBM_F32 && storage != HLBM_F16DEV && storage != HLBM_BF16DEV) return HLBM_ERR_INVALID_ARG;
    if (check_every < 2 || check_every % 2 || check_every > 10000 || mem_budget == 0) return HLBM_ERR_INVALID_ARG;
    hlbm_server_t* s = new (std::nothrow) hlbm_server();
    if (!s) return HLBM_ERR_OOM;
    s->storage = storage;
    s->check_every = check_every;
    s->budget = mem_budget;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->floor_coef = storage == HLBM_BF16DEV ? 1.6e-2 : 2e-3;
    s->t0 = std::chrono::steady_clock::now();
    double feq[19];
    for (int i = 0; i < 19; ++i) feq[i] = feq_rest(i);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->dtab, sizeof(DevTable));
    if (e == cudaSuccess) e = cudaMallocHost(&s->htab, sizeof(DevTable));
    if (e == cudaSuccess) e = cudaMalloc(&s->dout, kMaxSlots * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&s->hout, kMaxSlots * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->dfeq, sizeof(feq));
    if (e == cudaSuccess) e = cudaMemcpy(s->dfeq, feq, sizeof(feq), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::memset(s->htab, 0, sizeof(DevTable));
        e = cudaMemcpy(s->dtab, s->htab, sizeof(DevTable), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        int rc = srv_cuda_fail(e);
        hlbm_server_destroy(s);
        return rc;
    }
    *out = s;
    return HLBM_OK;
}

int hlbm_server_set_refinement(hlbm_server_t* s, int enable, double floor_coef) {
    if (!s || !(floor_coef >= 0.0) || !std::isfinite(floor_coef)) return HLBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->refine = enable ? 1 : 0;
    s->floor_coef = floor_coef;
    return HLBM_OK;
}

int hlbm_server_set_priority(hlbm_server_t* s, double backfill) {
    if (!s || !(backfill >= 0.0) || !std::isfinite(backfill)) return HLBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->backfill = backfill;
    return HLBM_OK;
}

void hlbm_server_destroy(hlbm_server_t* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (Live& l : s->live) {
        free_slot(s, l);
        cudaFreeHost(l.p.field);
    }
    for (Pending& p : s->waiting) cudaFreeHost(p.field);
    if (s->dpartials) cudaFreeAsync(s->dpartials, s->stream);
    cudaStreamSynchronize(s->stream);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    for (int b = 0; b < kGraphBranches; ++b) {
        if (s->branch[b]) cudaStreamDestroy(s->branch[b]);
        if (s->join_ev[b]) cudaEventDestroy(s->join_ev[b]);
    }
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    cudaFree(s->dtab);
    cudaFree(s->dout);
    cudaFree(s->dfeq);
    if (s->htab) cudaFreeHost(s->htab);
    if (s->hout) cudaFreeHost(s->hout);
    delete s;
}

int hlbm_server_submit(hlbm_server_t* s, const hlbm_request* r, uint64_t* id) {
    if (!s || !r || !r->varpi) return HLBM_ERR_INVALID_ARG;
    if (r->nx < 1 || r->ny < 1 || r->nz < 1 || !(r->tau > 0.5) || !std::isfinite(r->tau)) return HLBM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(r->F[a])) return HLBM_ERR_INVALID_ARG;
    if (!(r->tol > 0.0) || r->max_steps < 1) return HLBM_ERR_INVALID_ARG;
    const size_t n = (size_t)r->nx * r->ny * r->nz;
    if (n > ((size_t)1 << 31) / 19) return HLBM_ERR_INVALID_ARG;
    for (size_t k = 0; k < n; ++k)
        if (!(r->varpi[k] >= 0.0f && r->varpi[k] <= 1.0f)) return HLBM_ERR_INVALID_ARG;
    if (s->slot_bytes(*r) > s->budget) return HLBM_ERR_OOM;
    Pending p;
    p.req = *r;
    if (cudaMallocHost(&p.field, n * sizeof(float)) != cudaSuccess) return HLBM_ERR_OOM;
    std::memcpy(p.field, r->varpi, n * sizeof(float));
    p.req.varpi = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    p.id = s->next_id++;
    p.t_submit = s->now();
    s->waiting.push_back(p);
    if (id) *id = p.id;
    return HLBM_OK;
}

int hlbm_server_cancel(hlbm_server_t* s, uint64_t id) {
    if (!s) return HLBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->waiting.begin(); it != s->waiting.end(); ++it)
        if (it->id == id) {
            finish_pending(s, *it, HLBM_ERR_CANCELLED);
            s->waiting.erase(it);
            return HLBM_OK;
        }
    for (Live& l : s->live)
        if (l.p.id == id) {
            l.cancel = true;
            return HLBM_OK;
        }
    return HLBM_ERR_INVALID_ARG;
}

int hlbm_server_inject_alloc_failures(hlbm_server_t* s, int n) {
    if (!s || n < 0) return HLBM_ERR_INVALID_ARG;
    s->inject_alloc_failures = n;
    return HLBM_OK;
}

int hlbm_server_pump(hlbm_server_t* s, int* active, int* waiting) {
    if (!s) return HLBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    // 1. admission, first come first served, while the memory budget allows
    while (!s->waiting.empty() && s->live.size() < (size_t)kMaxSlots) {
        Pending& p = s->waiting.front();
        if (s->used + s->slot_bytes(p.req) > s->budget) break;
        Live l;
        cudaError_t e = admit(s, p, l);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            if (s->live.empty() && ++p.alloc_failures >= kMaxAllocRetries) {
                finish_pending(s, p, HLBM_ERR_OOM);  // nothing will free memory
                s->waiting.pop_front();
                continue;
            }
            break;  // back off: retry at the next round
        }
        if (e != cudaSuccess) return srv_cuda_fail(e);
        s->live.push_back(l);
        s->waiting.pop_front();
        s->table_dirty = true;
    }
    if (!s->live.empty()) {
        // 2. this round's slots, then check_every batched steps of each of them
        if (choose_run(s) || s->table_dirty) {
            int rc = upload_table(s);
            if (rc != HLBM_OK) return rc;
        }
        SRV_CUDA(cudaGraphLaunch(s->gexec, s->stream));
        // 3. per-slot FP64 diagnostics
        const int tiles = s->htab->total_tiles;
        k_batched_partials<<<tiles, kBlock, 0, s->stream>>>(s->dtab, s->dpartials);
        SRV_CUDA(cudaGetLastError());
        const int ns = (int)s->run.size();
        k_batched_final<<<ns, 256, 0, s->stream>>>(s->dtab, s->dpartials, s->dout);
        SRV_CUDA(cudaGetLastError());
        SRV_CUDA(cudaMemcpyAsync(s->hout, s->dout, (size_t)ns * 8 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        SRV_CUDA(cudaStreamSynchronize(s->stream));
        s->rounds++;
        // 4. retire converged / exhausted / cancelled slots; widen slots at their floor
        std::vector<char> gone(s->live.size(), 0);
        auto retire = [&](int i, int status, const double* o) -> int {
            Live& l = s->live[i];
            if (l.p.req.u_out && status != HLBM_ERR_CANCELLED) {
                const size_t n = (size_t)l.ds.nx * l.ds.ny * l.ds.nz;
                void* du = nullptr;
                cudaError_t e = cudaMallocAsync(&du, 3 * n * sizeof(float), s->stream);
                if (e == cudaSuccess) e = launch_moments(s->ctx_for(l), 0, l.ds.f[0], nullptr, du, 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(l.p.req.u_out, du, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
                if (du) cudaFreeAsync(du, s->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
                if (e != cudaSuccess) return srv_cuda_fail(e);
            }
            finish(s, l, status, o);
            free_slot(s, l);
            cudaFreeHost(l.p.field);
            gone[i] = 1;
            s->table_dirty = true;
            return HLBM_OK;
        };
        for (int k = 0; k < ns; ++k) {
            Live& l = s->live[s->run[k]];
            l.steps += s->check_every;
            if (l.ds.storage != HLBM_F32) l.steps_low += s->check_every;
            s->lups += (long long)s->check_every * l.ds.nx * l.ds.ny * l.ds.nz;
            const double* o = s->hout + (size_t)k * 8;
            const bool low = l.ds.storage != HLBM_F32;
            int status = 1;
            if (l.cancel) status = HLBM_ERR_CANCELLED;
            else if (o[6] < l.p.req.tol && !(low && s->refine)) status = HLBM_OK;
            else if (l.steps >= l.p.req.max_steps) status = HLBM_ERR_NOT_CONVERGED;
            if (status == 1 && low && s->refine) {
                // Stall test on the relative residual max|du| / max|u|: during the start-up
                // transient the flow accelerates almost uniformly, so max|du| over an interval
                // stays flat while max|u| grows, and only the ratio shows the progress. A ratio
                // that stops falling counts as a stall only near the rounding floor (within
                // kStallBand of it).
                const double rel = o[7] > 0.0 ? o[6] / o[7] : o[6];
                if (rel < 0.9 * l.best_du) {
                    l.best_du = rel;
                    l.stall = 0;
                } else if (rel < kStallBand * s->floor_coef) {
                    ++l.stall;
                } else {
                    l.stall = 0;
                }
                const bool at_floor = o[6] < std::max(l.p.req.tol, s->floor_coef * o[7]) || l.stall >= kStallChecks;
                if (at_floor) {
                    cudaError_t e = widen_to_fp32(s, l);
                    if (e == cudaErrorMemoryAllocation) cudaGetLastError();  // retry at a later round
                    else if (e != cudaSuccess) return srv_cuda_fail(e);
                    else s->table_dirty = true;
                }
            }
            if (status != 1) {
                int rc = retire(s->run[k], status, o);
                if (rc != HLBM_OK) return rc;
            }
        }
        // a cancelled slot that did not run this round leaves at once
        for (int i = 0; i < (int)s->live.size(); ++i)
            if (!gone[i] && s->live[i].cancel) {
                int rc = retire(i, HLBM_ERR_CANCELLED, nullptr);
                if (rc != HLBM_OK) return rc;
            }
        std::vector<Live> keep;
        keep.reserve(s->live.size());
        for (int i = 0; i < (int)s->live.size(); ++i)
            if (!gone[i]) keep.push_back(s->live[i]);
        s->live.swap(keep);
        s->run.clear();  // indices into the old live list
    }
    if (active) *active = (int)s->live.size();
    if (waiting) *waiting = (int)s->waiting.size();
    return HLBM_OK;
}

int hlbm_server_poll(hlbm_server_t* s, hlbm_result* out, int max, int* n) {
    if (!s || !n || (max > 0 && !out) || max < 0) return HLBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return HLBM_OK;
}

int hlbm_server_info(hlbm_server_t* s, hlbm_server_stats* out) {
    if (!s || !out) return HLBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->active = (int)s->live.size();
    out->waiting = (int)s->waiting.size();
    out->done_unpolled = (int)s->done.size();
    out->mem_used = s->used;
    out->mem_budget = s->budget;
    out->lattice_updates = s->lups;
    out->rounds = s->rounds;
    out->elapsed_s = s->now();
    return HLBM_OK;
}

}  // extern "C"
