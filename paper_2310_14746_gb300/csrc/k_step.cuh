// Templates of the fused HBGK stream-and-collide kernels (one time step over
// every cell); instantiated once per storage policy in k_step_<policy>.cu.
#pragma once
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

// Collision forms of the step: FORM_AUTO picks at run time (used for the
// 64-bit index kernels, which only very large lattices need); the others are
// compiled separately so each kernel carries only its own code and registers.
enum StepForm { FORM_AUTO = 0, FORM_SHIFT_FX = 1, FORM_SHIFT = 2, FORM_DRAG = 3, FORM_ANISO = 4 };

template <int Q, class S, bool WALLS, int MODE, class I, int FORM>
__global__ void __launch_bounds__(256)
k_step(Planes<const typename S::T, Q> fin, Planes<typename S::T, Q> fout, const float* __restrict__ varpi,
       Geometry g, Phys<typename S::C> ph, typename S::C s, typename S::C inv_s, int fx_only, int drag,
       const float* __restrict__ varpi3, const unsigned* __restrict__ links) {
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const I cell = (I)x + (I)g.nx * ((I)y + (I)g.ny * (I)z);
    unsigned lm = 0;
    if (WALLS && links) {
        lm = __ldg(links + cell);
        if (lm & kSolidBit) return;  // solid cells are not updated
    }
    const Nbr<I> nb(g, x, y, z, lm);
    constexpr int lay_in = MODE == MODE_TWO_LATTICE ? NATURAL : (MODE == MODE_AA_EVEN ? STREAMED : SWAPPED);
    constexpr int lay_out = MODE == MODE_TWO_LATTICE ? NATURAL : (MODE == MODE_AA_EVEN ? SWAPPED : STREAMED);

    C d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = S::load_raw(gather_ptr<Q, WALLS, lay_in>(fin, nb, cell, i), 0);

    const bool aniso = FORM == FORM_ANISO || (FORM == FORM_AUTO && varpi3);
    if (aniso) {  // diagonal porosity tensor [3][cells]
        collide_aniso<Q, C, S::scaled>(d, C(__ldg(varpi3 + cell)), C(__ldg(varpi3 + (I)g.N + cell)),
                                       C(__ldg(varpi3 + 2 * (I)g.N + cell)), ph, s, inv_s, WriteBack<C>{d});
    } else {
        const C vp = C(__ldg(varpi + cell));
        if (FORM == FORM_DRAG || (FORM == FORM_AUTO && drag))
            collide_drag<Q, C, S::scaled>(d, vp, ph, s, inv_s, WriteBack<C>{d});
        else if (FORM == FORM_SHIFT_FX || (FORM == FORM_AUTO && fx_only))
            collide<Q, C, S::scaled, true>(d, vp, ph, s, inv_s, WriteBack<C>{d});
        else collide<Q, C, S::scaled, false>(d, vp, ph, s, inv_s, WriteBack<C>{d});
    }

#pragma unroll
    for (int i = 0; i < Q; ++i) S::store_raw(scatter_ptr<Q, WALLS, lay_out>(fout, nb, cell, i), 0, d[i]);
}

inline dim3 step_block_for(int nx) {
    int bx = ((nx + 31) / 32) * 32;
    if (bx > 128) bx = 128;
    return dim3(bx, 256 / bx, 1);
}

template <int Q, class S, bool WALLS, class I, int FORM>
cudaError_t step_impl(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    using C = typename S::C;
    using T = typename S::T;
    Geometry g{c.nx, c.ny, c.nz, c.wall[0], c.wall[1], c.wall[2], (size_t)c.nx * c.ny * c.nz};
    const Phys<C> ph = make_phys<C, Q>(c.tau, c.F);
    const dim3 blk = step_block_for(c.nx);
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
            k_step<Q, S, WALLS, MODE_TWO_LATTICE, I, FORM><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, s, inv_s, fx,
                                                                                    c.drag, c.varpi3, c.links);
            break;
        case MODE_AA_EVEN:
            k_step<Q, S, WALLS, MODE_AA_EVEN, I, FORM><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, s, inv_s, fx,
                                                                                c.drag, c.varpi3, c.links);
            break;
        case MODE_AA_ODD:
            k_step<Q, S, WALLS, MODE_AA_ODD, I, FORM><<<grd, blk, 0, c.stream>>>(a, b, varpi, g, ph, s, inv_s, fx,
                                                                               c.drag, c.varpi3, c.links);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The form a launch needs for the handle's settings.
inline int step_form(const LaunchCtx& c, int q) {
    if (c.varpi3) return FORM_ANISO;
    if (c.drag) return FORM_DRAG;
    return ((q == 9 || c.F[2] == 0.0) && c.F[1] == 0.0) ? FORM_SHIFT_FX : FORM_SHIFT;
}

template <int Q, class S, bool WALLS>
cudaError_t step_forms(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    // 32-bit element indices while every index of the [q][cells] array fits
    const bool small = (size_t)Q * c.nx * c.ny * c.nz < ((size_t)1 << 31);
    if (!small) return step_impl<Q, S, WALLS, long long, FORM_AUTO>(c, mode, fin, fout, varpi);
    switch (step_form(c, Q)) {
        case FORM_SHIFT_FX: return step_impl<Q, S, WALLS, int, FORM_SHIFT_FX>(c, mode, fin, fout, varpi);
        case FORM_SHIFT: return step_impl<Q, S, WALLS, int, FORM_SHIFT>(c, mode, fin, fout, varpi);
        case FORM_DRAG: return step_impl<Q, S, WALLS, int, FORM_DRAG>(c, mode, fin, fout, varpi);
        default: return step_impl<Q, S, WALLS, int, FORM_ANISO>(c, mode, fin, fout, varpi);
    }
}

// All step kernels of storage policy S (one translation unit per policy).
template <class S>
cudaError_t step_for_storage(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    const bool walls = c.wall[0] || c.wall[1] || c.wall[2] || c.links;  // obstacles use the wall path
    if (c.q == 9)
        return walls ? step_forms<9, S, true>(c, mode, fin, fout, varpi) : step_forms<9, S, false>(c, mode, fin, fout, varpi);
    if (c.q == 19)
        return walls ? step_forms<19, S, true>(c, mode, fin, fout, varpi)
                     : step_forms<19, S, false>(c, mode, fin, fout, varpi);
    return cudaErrorInvalidValue;
}

}  // namespace hlbm
