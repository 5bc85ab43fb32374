// Observables and state I/O: moments, FP64 diagnostics, population
// conversion, input validation.
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"
#include "diag.cuh"

namespace hlbm {

static dim3 block_for(int nx) {
    int bx = ((nx + 31) / 32) * 32;
    if (bx > 128) bx = 128;
    return dim3(bx, 256 / bx, 1);
}

static Geometry geom(const LaunchCtx& c) {
    return Geometry{c.nx, c.ny, c.nz, c.wall[0], c.wall[1], c.wall[2], (size_t)c.nx * c.ny * c.nz};
}

template <class C, int Q>
static Phys<C> phys(const LaunchCtx& c) {
    return make_phys<C, Q>(c.tau, c.F);
}

// ---------------------------------------------------------------------------
// Moments (Def. moments of the streamed populations, half-force velocity).
// ---------------------------------------------------------------------------
template <int Q, class S, bool WALLS, class Out>
__global__ void __launch_bounds__(256)
k_moments(const typename S::T* f, int lay, Geometry g, Phys<typename S::C> ph, typename S::C inv_s,
          Out* rho, Out* u, const float* varpi, int drag, const unsigned* links) {
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
    const unsigned lm = links ? links[cell] : 0u;
    if (lm & kSolidBit) {  // resolved obstacle: at rest
        if (rho) rho[cell] = Out(1);
        if (u) u[cell] = u[g.N + cell] = u[2 * g.N + cell] = Out(0);
        return;
    }
    const Nbr<long long> nb(g, x, y, z, lm);
    C d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = S::load(f, gather_index<Q, WALLS>(g, nb, cell, i, lay), inv_s);
    C drho, jx, jy, jz;
    moments<Q, C>(d, drho, jx, jy, jz);
    const C r = C(1) + drho;
    if (rho) rho[cell] = Out(r);
    if (u) {
        C ux, uy, uz;
        velocity_form<C>(jx, jy, jz, r, drag ? C(varpi[cell]) : C(1), drag, ph, ux, uy, uz);
        u[cell] = Out(ux);
        u[g.N + cell] = Out(uy);
        u[2 * g.N + cell] = Out(uz);
    }
}

template <int Q, class S, bool WALLS>
static cudaError_t moments_impl(const LaunchCtx& c, int lay, const void* f, void* rho, void* u, int f64) {
    using C = typename S::C;
    const Geometry g = geom(c);
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    const auto* a = static_cast<const typename S::T*>(f);
    if (f64)
        k_moments<Q, S, WALLS, double><<<grd, blk, 0, c.stream>>>(a, lay, g, phys<C, Q>(c), C(1.0 / c.scale),
                                                                  (double*)rho, (double*)u, c.varpi, c.drag, c.links);
    else
        k_moments<Q, S, WALLS, float><<<grd, blk, 0, c.stream>>>(a, lay, g, phys<C, Q>(c), C(1.0 / c.scale),
                                                                 (float*)rho, (float*)u, c.varpi, c.drag, c.links);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 diagnostics. Stage 1: each block folds its cells (256 threads over x
// rows, kReduceZ z planes per thread) into 8 doubles (sum drho, sum rho*u
// (3), plane flux, 0, max|du|, max|u|) in a fixed order (diag.cuh). Stage 2:
// one block per column folds the block rows in a fixed order. The result does
// not depend on scheduling.
//
// The first version (64-bit indices, the layout chosen per direction at run
// time, residual reference loads ordered behind the previous component's
// store, one cell per thread) was latency-bound at 0.87 TB/s; 32-bit indices
// with the two-lattice layout fixed at compile time and all loads issued
// before any store bring the cell work to the copy bandwidth.
// ---------------------------------------------------------------------------
constexpr int kReduceZ = 4;

template <int Q, class S, bool WALLS, bool FAST>
__global__ void __launch_bounds__(256)
k_reduce_partials(const typename S::T* __restrict__ f, int lay, Geometry g, Phys<typename S::C> ph,
                  typename S::C inv_s, typename S::C* __restrict__ u_prev, int update_prev,
                  double* __restrict__ partials, const float* __restrict__ varpi, int drag,
                  const unsigned* __restrict__ links) {
    using C = typename S::C;
    using I = typename std::conditional<FAST, int, long long>::type;  // FAST: 32-bit indices, natural layout
    __shared__ DiagShared sh;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    DiagCell<C> a;
    a.shifted = drag != 0;
    if (x < g.nx && y < g.ny) {
        const I N = (I)g.N;
        const int z0 = blockIdx.z * kReduceZ;
        const int z1 = z0 + kReduceZ < g.nz ? z0 + kReduceZ : g.nz;
        for (int z = z0; z < z1; ++z) {
            const I cell = (I)x + (I)g.nx * ((I)y + (I)g.ny * (I)z);
            const unsigned lm = links ? links[cell] : 0u;
            if (lm & kSolidBit) {
                // resolved obstacle: rho = 1, u = 0 (contributes nothing but its residual reference)
                if (update_prev)
                    for (int k = 0; k < 3; ++k) u_prev[(I)k * N + cell] = C(0);
                continue;
            }
            const Nbr<I> nb(g, x, y, z, lm);
            C d[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i)
                d[i] = S::load(f, gather_index<Q, WALLS>(g, nb, cell, i, FAST ? (int)NATURAL : lay), inv_s);
            C up[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) up[k] = u_prev[(I)k * N + cell];
            C drho, jx, jy, jz;
            moments<Q, C>(d, drho, jx, jy, jz);
            C u3[3];
            const C vp = drag ? C(varpi[cell]) : C(1);
            velocity_form<C>(jx, jy, jz, C(1) + drho, vp, drag, ph, u3[0], u3[1], u3[2]);
            a.fluid += 1;
            a.p[0] += drho;
            C mx = jx, my = jy, mz = jz;
            if (drag) {  // rho*u = (j + F/2) / (1 + lam/2)
                const C hd = C(1) / fma_(C(0.5), (C(1) - vp) * ph.omega, C(1));
                mx = fma_(C(0.5), ph.Fx, jx) * hd;
                my = fma_(C(0.5), ph.Fy, jy) * hd;
                mz = fma_(C(0.5), ph.Fz, jz) * hd;
            }  // else rho*u = j + F/2, the F/2 added per block from the fluid-cell count
            a.p[1] += mx;
            a.p[2] += my;
            a.p[3] += mz;
            if (x == g.nx - 1) {
                a.plane += 1;
                a.p[4] += mx;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a.du = nan_max(a.du, C(fabs(u3[k] - up[k])));
                a.um = nan_max(a.um, C(fabs(u3[k])));
            }
            if (update_prev)
#pragma unroll
                for (int k = 0; k < 3; ++k) u_prev[(I)k * N + cell] = u3[k];
        }
    }
    const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    diag_fold<C>(a, sh, threadIdx.x + blockDim.x * threadIdx.y, blockDim.x * blockDim.y, (double)ph.Fx,
                 (double)ph.Fy, (double)ph.Fz, partials + b * 8);
}

// Block k folds column k of the partials; block 1 also forms k_app.
__global__ void __launch_bounds__(256)
k_reduce_final(const double* partials, size_t nblocks, double cells, double nu, double Fx, double* out8) {
    __shared__ double buf[256];
    const int k = blockIdx.x;
    if (k == 5) {
        return;  // column 5 is k_app, written by block 1
    }
    const double v = fold_column(partials, nblocks, k, buf);
    if (threadIdx.x == 0) {
        if (k == 0) {
            out8[0] = cells + v;  // mass = sum (1 + drho)
        } else {
            out8[k] = v;
            if (k == 1) out8[5] = (Fx != 0.0) ? nu * (v / cells) / Fx : 0.0;
        }
    }
}

size_t reduce_partials_count(const LaunchCtx& c) {
    const dim3 blk = block_for(c.nx);
    return (size_t)((c.nx + blk.x - 1) / blk.x) * ((c.ny + blk.y - 1) / blk.y) * ((c.nz + kReduceZ - 1) / kReduceZ);
}

bool reduce_grid_fits(const LaunchCtx& c) {
    const dim3 blk = block_for(c.nx);
    return (size_t)(c.ny + blk.y - 1) / blk.y <= 65535 && (size_t)(c.nz + kReduceZ - 1) / kReduceZ <= 65535 &&
           (size_t)(c.nx + blk.x - 1) / blk.x <= 0x7fffffff;
}

template <int Q, class S, bool WALLS>
static cudaError_t reduce_impl(const LaunchCtx& c, int lay, const void* f, void* u_prev, int upd,
                               double* partials, double* out8) {
    using C = typename S::C;
    const Geometry g = geom(c);
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, (c.nz + kReduceZ - 1) / kReduceZ);
    const auto* fs = static_cast<const typename S::T*>(f);
    C* up = static_cast<C*>(u_prev);
    if (lay == NATURAL && (size_t)Q * g.N < ((size_t)1 << 31))
        k_reduce_partials<Q, S, WALLS, true><<<grd, blk, 0, c.stream>>>(fs, lay, g, phys<C, Q>(c), C(1.0 / c.scale),
                                                                        up, upd, partials, c.varpi, c.drag, c.links);
    else
        k_reduce_partials<Q, S, WALLS, false><<<grd, blk, 0, c.stream>>>(fs, lay, g, phys<C, Q>(c), C(1.0 / c.scale),
                                                                         up, upd, partials, c.varpi, c.drag, c.links);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<8, 256, 0, c.stream>>>(partials, reduce_partials_count(c), (double)g.N,
                                            (c.tau - 0.5) / 3.0, c.F[0], out8);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State conversion (natural FP64 full populations <-> stored deviations).
// ---------------------------------------------------------------------------
template <int Q, class S, bool WALLS>
__global__ void __launch_bounds__(256)
k_write_state(const double* fnat, int uniform, int lay, Geometry g, typename S::C s, typename S::T* f,
              const unsigned* links) {
    using C = typename S::C;
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
    const unsigned lm = links ? links[cell] : 0u;
    if (lm & kSolidBit) return;  // solid cells hold no state (their slots may belong to neighbours)
    const Nbr<long long> nb(g, x, y, z, lm);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double fi = uniform ? fnat[i] : fnat[(size_t)i * g.N + cell];
        S::store(f, natural_index<Q, WALLS>(g, nb, cell, i, lay), C(fi - L::w(i)), s);
    }
}

template <int Q, class S, bool WALLS>
__global__ void __launch_bounds__(256)
k_read_state(const typename S::T* f, int lay, Geometry g, typename S::C inv_s, double* fnat,
             const unsigned* links) {
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
    const unsigned lm = links ? links[cell] : 0u;
    if (lm & kSolidBit) {  // solid cells read as the rest state
#pragma unroll
        for (int i = 0; i < Q; ++i) fnat[(size_t)i * g.N + cell] = L::w(i);
        return;
    }
    const Nbr<long long> nb(g, x, y, z, lm);
#pragma unroll
    for (int i = 0; i < Q; ++i)
        fnat[(size_t)i * g.N + cell] =
            L::w(i) + (double)S::load(f, natural_index<Q, WALLS>(g, nb, cell, i, lay), inv_s);
}

// The same state as k_write_state with uniform = 1 (every cell holds fnat[i]),
// for kFillZ consecutive z planes per thread: the deviation of each direction
// is formed once per thread (in double, as k_write_state forms it, so the bits
// are the same), and the per-cell work is only the index and the store. GB300's
// FP64 rate is a small fraction of its FP32 rate, and the per-cell double
// subtract and conversion had limited the initial write to about 1.2 TB/s.
constexpr int kFillZ = 8;

template <int Q, class S, bool WALLS>
__global__ void __launch_bounds__(256)
k_fill_state(const double* fnat, int lay, Geometry g, typename S::C s, typename S::T* f, const unsigned* links) {
    using C = typename S::C;
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    C v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = C(fnat[i] - L::w(i));
    const int z0 = blockIdx.z * kFillZ;
    const int z1 = z0 + kFillZ < g.nz ? z0 + kFillZ : g.nz;
    for (int z = z0; z < z1; ++z) {
        const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
        const unsigned lm = links ? links[cell] : 0u;
        if (lm & kSolidBit) continue;
        const Nbr<long long> nb(g, x, y, z, lm);
#pragma unroll
        for (int i = 0; i < Q; ++i) S::store(f, natural_index<Q, WALLS>(g, nb, cell, i, lay), v[i], s);
    }
}

template <int Q, class S, bool WALLS>
static cudaError_t write_impl(const LaunchCtx& c, int lay, const double* fnat, int uniform, void* f) {
    using C = typename S::C;
    const dim3 blk = block_for(c.nx);
    if (uniform) {
        const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, (c.nz + kFillZ - 1) / kFillZ);
        k_fill_state<Q, S, WALLS><<<grd, blk, 0, c.stream>>>(fnat, lay, geom(c), C(c.scale),
                                                             static_cast<typename S::T*>(f), c.links);
        return cudaGetLastError();
    }
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    k_write_state<Q, S, WALLS><<<grd, blk, 0, c.stream>>>(fnat, uniform, lay, geom(c), C(c.scale),
                                                          static_cast<typename S::T*>(f), c.links);
    return cudaGetLastError();
}

template <int Q, class S, bool WALLS>
static cudaError_t read_impl(const LaunchCtx& c, int lay, const void* f, double* fnat) {
    using C = typename S::C;
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    k_read_state<Q, S, WALLS><<<grd, blk, 0, c.stream>>>(static_cast<const typename S::T*>(f), lay, geom(c),
                                                         C(1.0 / c.scale), fnat, c.links);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dispatch on (q, storage, walls)
// ---------------------------------------------------------------------------
template <int Q, class S, class Fn>
static cudaError_t with_walls(const LaunchCtx& c, Fn&& fn) {
    const bool walls = c.wall[0] || c.wall[1] || c.wall[2] || c.links;
    return walls ? fn.template operator()<Q, S, true>() : fn.template operator()<Q, S, false>();
}
template <int Q, class Fn>
static cudaError_t with_storage(const LaunchCtx& c, Fn&& fn) {
    switch (c.storage) {
        case 0: return with_walls<Q, StoreF64>(c, fn);
        case 1: return with_walls<Q, StoreF32>(c, fn);
        case 2: return with_walls<Q, StoreF16>(c, fn);
        case 3: return with_walls<Q, StoreBF16>(c, fn);
    }
    return cudaErrorInvalidValue;
}
template <class Fn>
static cudaError_t dispatch(const LaunchCtx& c, Fn&& fn) {
    if (c.q == 9) return with_storage<9>(c, fn);
    if (c.q == 19) return with_storage<19>(c, fn);
    return cudaErrorInvalidValue;
}

cudaError_t launch_moments(const LaunchCtx& c, int layout, const void* f, void* rho, void* u, int out_f64) {
    return dispatch(c, [&]<int Q, class S, bool W>() { return moments_impl<Q, S, W>(c, layout, f, rho, u, out_f64); });
}

cudaError_t launch_reduce(const LaunchCtx& c, int layout, const void* f, void* u_prev, int update_prev,
                          double* partials, double* out8) {
    return dispatch(c, [&]<int Q, class S, bool W>() {
        return reduce_impl<Q, S, W>(c, layout, f, u_prev, update_prev, partials, out8);
    });
}

cudaError_t launch_write_state(const LaunchCtx& c, int layout, const double* fnat, int uniform, void* f) {
    return dispatch(c, [&]<int Q, class S, bool W>() { return write_impl<Q, S, W>(c, layout, fnat, uniform, f); });
}

cudaError_t launch_read_state(const LaunchCtx& c, int layout, const void* f, double* fnat) {
    return dispatch(c, [&]<int Q, class S, bool W>() { return read_impl<Q, S, W>(c, layout, f, fnat); });
}

// ---------------------------------------------------------------------------
// small utilities
// ---------------------------------------------------------------------------
__global__ void k_check_unit(const float* __restrict__ v, size_t n, int* bad) {
    int local = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float a = v[i];
        if (!(a >= 0.0f && a <= 1.0f)) ++local;  // NaN fails both comparisons
    }
    if (local) atomicAdd(bad, local);
}

__global__ void k_fill_f32(float* v, size_t n, float value) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[i] = value;
}

static unsigned grid_1d(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b == 0) b = 1;
    return (unsigned)b;
}

cudaError_t launch_check_unit_interval(const float* v, size_t n, int* bad, cudaStream_t s) {
    k_check_unit<<<grid_1d(n), 256, 0, s>>>(v, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(float* v, size_t n, float value, cudaStream_t s) {
    k_fill_f32<<<grid_1d(n), 256, 0, s>>>(v, n, value);
    return cudaGetLastError();
}

cudaError_t launch_fill_bytes0(void* p, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(p, 0, bytes, s); }

size_t storage_bytes(int storage) {
    switch (storage) {
        case 0: return 8;
        case 1: return 4;
        case 2: return 2;
        case 3: return 2;
    }
    return 0;
}

}  // namespace hlbm
