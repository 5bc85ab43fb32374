// Observables and state I/O: moments, FP64 diagnostics, population
// conversion, input validation.
#include "internal.h"
#include "lattice.cuh"

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
// FP64 diagnostics. Stage 1: each block reduces its cells into 8 doubles
// (sum drho, sum rho*u (3), plane flux, -, max|du|, max|u|) with a fixed
// shuffle tree. Stage 2: one block folds the block rows in a fixed order.
// The result does not depend on scheduling.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <int Q, class S, bool WALLS>
__global__ void __launch_bounds__(256)
k_reduce_partials(const typename S::T* f, int lay, Geometry g, Phys<typename S::C> ph,
                  typename S::C inv_s, typename S::C* u_prev, int update_prev, double* partials, const float* varpi,
                  int drag, const unsigned* links) {
    using C = typename S::C;
    __shared__ double sh[8][8];  // [warp][quantity]
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
    const unsigned lm = (links && x < g.nx && y < g.ny) ? links[cell] : 0u;
    if (x < g.nx && y < g.ny && (lm & kSolidBit)) {
        // resolved obstacle: rho = 1, u = 0 (contributes nothing but its residual reference)
        if (update_prev)
            for (int k = 0; k < 3; ++k) u_prev[k * g.N + cell] = typename S::C(0);
    } else if (x < g.nx && y < g.ny) {
        const Nbr<long long> nb(g, x, y, z, lm);
        C d[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = S::load(f, gather_index<Q, WALLS>(g, nb, cell, i, lay), inv_s);
        C drho, jx, jy, jz;
        moments<Q, C>(d, drho, jx, jy, jz);
        C u3[3];
        const C vp = drag ? C(varpi[cell]) : C(1);
        velocity_form<C>(jx, jy, jz, C(1) + drho, vp, drag, ph, u3[0], u3[1], u3[2]);
        // rho*u = (j + F/2) (/(1 + lam/2) in the drag form), formed in FP64
        const double hd = drag ? 1.0 / (1.0 + 0.5 * (1.0 - (double)vp) * (double)ph.omega) : 1.0;
        const double mx = ((double)jx + 0.5 * (double)ph.Fx) * hd;
        v[0] = (double)drho;
        v[1] = mx;
        v[2] = ((double)jy + 0.5 * (double)ph.Fy) * hd;
        v[3] = ((double)jz + 0.5 * (double)ph.Fz) * hd;
        v[4] = (x == g.nx - 1) ? mx : 0.0;
        double du = 0.0, um = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const C up = u_prev[k * g.N + cell];
            du = fmax(du, fabs((double)u3[k] - (double)up));
            um = fmax(um, fabs((double)u3[k]));
            if (update_prev) u_prev[k * g.N + cell] = u3[k];
        }
        v[6] = du;
        v[7] = um;
    }
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (k >= 6) ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (t < 8) {
        double a = sh[0][t];
        for (int w = 1; w < (int)(blockDim.x * blockDim.y) / 32; ++w) a = (t >= 6) ? fmax(a, sh[w][t]) : a + sh[w][t];
        const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
        partials[b * 8 + t] = a;
    }
}

__global__ void __launch_bounds__(256)
k_reduce_final(const double* partials, size_t nblocks, double cells, double nu, double Fx, double* out8) {
    __shared__ double sh[8][256];
    const int t = threadIdx.x;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t b = t; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = (k >= 6) ? fmax(v[k], partials[b * 8 + k]) : v[k] + partials[b * 8 + k];
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[k][t] = v[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k][t] = (k >= 6) ? fmax(sh[k][t], sh[k][t + s]) : sh[k][t] + sh[k][t + s];
        __syncthreads();
    }
    if (t == 0) {
        out8[0] = cells + sh[0][0];  // mass = sum (1 + drho)
        out8[1] = sh[1][0];
        out8[2] = sh[2][0];
        out8[3] = sh[3][0];
        out8[4] = sh[4][0];
        out8[5] = (Fx != 0.0) ? nu * (sh[1][0] / cells) / Fx : 0.0;
        out8[6] = sh[6][0];
        out8[7] = sh[7][0];
    }
}

size_t reduce_partials_count(const LaunchCtx& c) {
    const dim3 blk = block_for(c.nx);
    return (size_t)((c.nx + blk.x - 1) / blk.x) * ((c.ny + blk.y - 1) / blk.y) * c.nz;
}

template <int Q, class S, bool WALLS>
static cudaError_t reduce_impl(const LaunchCtx& c, int lay, const void* f, void* u_prev, int upd,
                               double* partials, double* out8) {
    using C = typename S::C;
    const Geometry g = geom(c);
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    k_reduce_partials<Q, S, WALLS><<<grd, blk, 0, c.stream>>>(static_cast<const typename S::T*>(f), lay, g,
                                                              phys<C, Q>(c), C(1.0 / c.scale),
                                                              static_cast<C*>(u_prev), upd, partials, c.varpi,
                                                              c.drag, c.links);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, 256, 0, c.stream>>>(partials, reduce_partials_count(c), (double)g.N,
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

template <int Q, class S, bool WALLS>
static cudaError_t write_impl(const LaunchCtx& c, int lay, const double* fnat, int uniform, void* f) {
    using C = typename S::C;
    const dim3 blk = block_for(c.nx);
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
