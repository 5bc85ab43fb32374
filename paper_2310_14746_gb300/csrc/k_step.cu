// Fused HBGK stream-and-collide kernels (one time step over every cell).
//
// One thread per cell; threads run along x so that each of the q population
// planes is read and written by whole warps over contiguous x (the +-1 x
// shifts of the pull make those loads straddle a sector boundary, which the
// L1/L2 absorb). Per cell: q loads, moments, the homogenized equilibrium at
// varpi*u (Sec. 3.2, eq. porousVeloMaxwellian), Guo forcing, BGK relaxation
// (eq. collisionOperatorQ), q stores. Bytes per cell update: 2*q*sizeof(T)
// for the populations plus 4 for varpi.
#include "internal.h"
#include "lattice.cuh"

namespace hlbm {

// Base pointer of every population plane, passed by value (kernel parameter
// space), so an access is one wide multiply-add of a 32/64-bit cell offset.
template <class T, int Q>
struct Planes {
    T* p[Q];
};

// Plane and cell of g_i(x) (the population the collision at x consumes) for a
// state in layout LAY; see gather_index in lattice.cuh for the three layouts.
template <int Q, bool WALLS, int LAY, class T, class I>
__device__ __forceinline__ T* gather_ptr(const Planes<T, Q>& pl, const Nbr<I>& nb, I cell, int i) {
    if (LAY == STREAMED) return pl.p[i] + cell;
    const bool wall = WALLS && nb.template beyond_wall<Q>(i, -1);
    const I src = cell + nb.template offset<Q>(i, -1);
    if (LAY == NATURAL) return wall ? pl.p[opp<Q>(i)] + cell : pl.p[i] + src;
    return wall ? pl.p[i] + cell : pl.p[opp<Q>(i)] + src;  // SWAPPED
}

// Plane and cell that receive the post-collision f_i(x) in layout LAY.
template <int Q, bool WALLS, int LAY, class T, class I>
__device__ __forceinline__ T* scatter_ptr(const Planes<T, Q>& pl, const Nbr<I>& nb, I cell, int i) {
    if (LAY == NATURAL) return pl.p[i] + cell;
    if (LAY == SWAPPED) return pl.p[opp<Q>(i)] + cell;
    const bool wall = WALLS && nb.template beyond_wall<Q>(i, +1);  // STREAMED
    return wall ? pl.p[opp<Q>(i)] + cell : pl.p[i] + (cell + nb.template offset<Q>(i, +1));
}

template <int Q, class S, bool WALLS, int MODE, class I>
__global__ void __launch_bounds__(256)
k_step(Planes<const typename S::T, Q> fin, Planes<typename S::T, Q> fout, const float* __restrict__ varpi,
       Geometry g, Phys<typename S::C> ph, typename S::C s, typename S::C inv_s, int fx_only) {
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const Nbr<I> nb(g, x, y, z);
    const I cell = (I)x + (I)g.nx * ((I)y + (I)g.ny * (I)z);
    constexpr int lay_in = MODE == MODE_TWO_LATTICE ? NATURAL : (MODE == MODE_AA_EVEN ? STREAMED : SWAPPED);
    constexpr int lay_out = MODE == MODE_TWO_LATTICE ? NATURAL : (MODE == MODE_AA_EVEN ? SWAPPED : STREAMED);

    C d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = S::load_raw(gather_ptr<Q, WALLS, lay_in>(fin, nb, cell, i), 0);

    const C vp = C(__ldg(varpi + cell));
    if (fx_only) collide<Q, C, S::scaled, true>(d, vp, ph, s, inv_s);
    else collide<Q, C, S::scaled, false>(d, vp, ph, s, inv_s);

#pragma unroll
    for (int i = 0; i < Q; ++i) S::store_raw(scatter_ptr<Q, WALLS, lay_out>(fout, nb, cell, i), 0, d[i]);
}

static dim3 block_for(int nx) {
    int bx = ((nx + 31) / 32) * 32;
    if (bx > 128) bx = 128;
    return dim3(bx, 256 / bx, 1);
}

template <int Q, class S, bool WALLS, class I>
static cudaError_t step_impl(const LaunchCtx& c, int mode, const void* fin, void* fout,
                             const float* varpi) {
    using C = typename S::C;
    using T = typename S::T;
    Geometry g{c.nx, c.ny, c.nz, c.wall[0], c.wall[1], c.wall[2], (size_t)c.nx * c.ny * c.nz};
    const Phys<C> ph = make_phys<C, Q>(c.tau, c.F);
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    const C s = C(c.scale), inv_s = C(1.0 / c.scale);
    Planes<const T, Q> a;
    Planes<T, Q> b;
    for (int i = 0; i < Q; ++i) {
        a.p[i] = static_cast<const T*>(fin) + (size_t)i * g.N;
        b.p[i] = static_cast<T*>(fout) + (size_t)i * g.N;
    }
    const int fx = (Q == 9 || c.F[2] == 0.0) && c.F[1] == 0.0;
    switch (mode) {
        case MODE_TWO_LATTICE:
            k_step<Q, S, WALLS, MODE_TWO_LATTICE, I><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, s, inv_s, fx);
            break;
        case MODE_AA_EVEN:
            k_step<Q, S, WALLS, MODE_AA_EVEN, I><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, s, inv_s, fx);
            break;
        case MODE_AA_ODD:
            k_step<Q, S, WALLS, MODE_AA_ODD, I><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, s, inv_s, fx);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int Q, class S>
static cudaError_t step_w(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    const bool walls = c.wall[0] || c.wall[1] || c.wall[2];
    // 32-bit element indices while every index of the [q][cells] array fits
    const bool small = (size_t)Q * c.nx * c.ny * c.nz < ((size_t)1 << 31);
    if (small)
        return walls ? step_impl<Q, S, true, int>(c, mode, fin, fout, varpi)
                     : step_impl<Q, S, false, int>(c, mode, fin, fout, varpi);
    return walls ? step_impl<Q, S, true, long long>(c, mode, fin, fout, varpi)
                 : step_impl<Q, S, false, long long>(c, mode, fin, fout, varpi);
}

template <int Q>
static cudaError_t step_s(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    switch (c.storage) {
        case 0: return step_w<Q, StoreF64>(c, mode, fin, fout, varpi);
        case 1: return step_w<Q, StoreF32>(c, mode, fin, fout, varpi);
        case 2: return step_w<Q, StoreF16>(c, mode, fin, fout, varpi);
        case 3: return step_w<Q, StoreBF16>(c, mode, fin, fout, varpi);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    if (c.q == 9) return step_s<9>(c, mode, fin, fout, varpi);
    if (c.q == 19) return step_s<19>(c, mode, fin, fout, varpi);
    return cudaErrorInvalidValue;
}

}  // namespace hlbm
