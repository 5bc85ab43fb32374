// Lattice constants, storage policies and the per-cell HBGK collision.
//
// Velocity sets D2Q9 / D3Q19 (c_s^2 = 1/3) in the direction order of the
// public header. Weights are derived from |c|^2 and opposites from c at
// compile time, so every table lookup inside an unrolled direction loop
// folds to an immediate.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstddef>
#include <cstdint>

namespace hlbm {

template <int Q>
struct Lat;

template <>
struct Lat<9> {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (cx(i) * cx(i) + cy(i) * cy(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <>
struct Lat<19> {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    // 1..6 faces (+x,-x,+y,-y,+z,-z), 7..18 edges in opposite pairs
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
               : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                     : 0;
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)   ? 1
               : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                                     : 0;
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)   ? 1
               : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                      : 0;
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0
                      : (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i) == 1 ? 1.0 / 18.0
                                                                            : 1.0 / 36.0);
    }
};

// Opposite direction: the j with c_j = -c_i.
template <int Q>
__host__ __device__ constexpr int opp(int i) {
    using L = Lat<Q>;
    int r = 0;
    for (int j = 0; j < Q; ++j)
        if (L::cx(j) == -L::cx(i) && L::cy(j) == -L::cy(i) && L::cz(j) == -L::cz(i)) r = j;
    return r;
}

// ---------------------------------------------------------------------------
// Storage policies: populations live as deviations d_i = (f_i - w_i) * s.
// T = element type in HBM, C = arithmetic type.
// ---------------------------------------------------------------------------
struct StoreF64 {
    using T = double;
    using C = double;
    static constexpr int kind = 0;
    __device__ __forceinline__ static C load(const T* p, size_t i, C) { return __ldg(p + i); }
    __device__ __forceinline__ static void store(T* p, size_t i, C v, C) { p[i] = v; }
};
struct StoreF32 {
    using T = float;
    using C = float;
    static constexpr int kind = 1;
    __device__ __forceinline__ static C load(const T* p, size_t i, C) { return __ldg(p + i); }
    __device__ __forceinline__ static void store(T* p, size_t i, C v, C) { p[i] = v; }
};
struct StoreF16 {
    using T = __half;
    using C = float;
    static constexpr int kind = 2;
    __device__ __forceinline__ static C load(const T* p, size_t i, C inv_s) {
        return __half2float(__ldg(p + i)) * inv_s;
    }
    __device__ __forceinline__ static void store(T* p, size_t i, C v, C s) {
        p[i] = __float2half_rn(v * s);
    }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    using C = float;
    static constexpr int kind = 3;
    __device__ __forceinline__ static C load(const T* p, size_t i, C inv_s) {
        return __bfloat162float(__ldg(p + i)) * inv_s;
    }
    __device__ __forceinline__ static void store(T* p, size_t i, C v, C s) {
        p[i] = __float2bfloat16_rn(v * s);
    }
};

// ---------------------------------------------------------------------------
// Where the state lives between steps.
//   NATURAL  (two-lattice): slot (x, i) holds the post-collision f_i(x).
//   STREAMED (AA, even count): slot (x, i) holds g_i(x) = f_i(x - c_i), i.e.
//            the populations the next collision at x consumes.
//   SWAPPED  (AA, odd count): slot (x, opp(i)) holds the post-collision f_i(x).
// ---------------------------------------------------------------------------
enum Layout { NATURAL = 0, STREAMED = 1, SWAPPED = 2 };

struct Geometry {
    int nx, ny, nz;
    int wall_x, wall_y, wall_z;  // 1 = half-way bounce-back at both ends
    size_t N;                    // cells
};

// Neighbour bookkeeping of one cell: coordinates of x - 1 / x + 1 (periodic
// wrap) along each axis, and whether the step crosses a wall.
struct Nbr {
    int x, y, z, xm, xp, ym, yp, zm, zp;
    bool lo_x, hi_x, lo_y, hi_y, lo_z, hi_z;  // at the low / high end of a wall axis

    __device__ __forceinline__ Nbr(const Geometry& g, int x_, int y_, int z_) {
        x = x_;
        y = y_;
        z = z_;
        xm = x == 0 ? g.nx - 1 : x - 1;
        xp = x == g.nx - 1 ? 0 : x + 1;
        ym = y == 0 ? g.ny - 1 : y - 1;
        yp = y == g.ny - 1 ? 0 : y + 1;
        zm = z == 0 ? g.nz - 1 : z - 1;
        zp = z == g.nz - 1 ? 0 : z + 1;
        lo_x = g.wall_x && x == 0;
        hi_x = g.wall_x && x == g.nx - 1;
        lo_y = g.wall_y && y == 0;
        hi_y = g.wall_y && y == g.ny - 1;
        lo_z = g.wall_z && z == 0;
        hi_z = g.wall_z && z == g.nz - 1;
    }

    // Cell index of x + s*c_i (s = -1 pull source, +1 push target) with wrap.
    template <int Q>
    __device__ __forceinline__ size_t cell_at(const Geometry& g, int i, int s) const {
        using L = Lat<Q>;
        const int dx = s * L::cx(i), dy = s * L::cy(i), dz = s * L::cz(i);
        const int sx = dx > 0 ? xp : (dx < 0 ? xm : x);
        const int sy = dy > 0 ? yp : (dy < 0 ? ym : y);
        const int sz = dz > 0 ? zp : (dz < 0 ? zm : z);
        return (size_t)sx + (size_t)g.nx * ((size_t)sy + (size_t)g.ny * (size_t)sz);
    }

    // Does x + s*c_i lie beyond a wall?
    template <int Q>
    __device__ __forceinline__ bool beyond_wall(int i, int s) const {
        using L = Lat<Q>;
        const int dx = s * L::cx(i), dy = s * L::cy(i), dz = s * L::cz(i);
        return (dx < 0 && lo_x) || (dx > 0 && hi_x) || (dy < 0 && lo_y) || (dy > 0 && hi_y) ||
               (dz < 0 && lo_z) || (dz > 0 && hi_z);
    }
};

// Flat index (into the [q][cells] array) holding g_i(x), the population the
// collision at x consumes, for a state in layout `lay`.
template <int Q, bool WALLS>
__device__ __forceinline__ size_t gather_index(const Geometry& g, const Nbr& nb, size_t cell,
                                               int i, int lay) {
    const size_t N = g.N;
    if (lay == STREAMED) return (size_t)i * N + cell;
    const bool wall = WALLS && nb.beyond_wall<Q>(i, -1);
    if (lay == NATURAL)
        return wall ? (size_t)opp<Q>(i) * N + cell : (size_t)i * N + nb.cell_at<Q>(g, i, -1);
    // SWAPPED: f_i(x - c_i) sits in slot opp(i) of cell x - c_i; across a
    // wall the bounce-back f_opp(i)(x) sits in slot i of x.
    return wall ? (size_t)i * N + cell : (size_t)opp<Q>(i) * N + nb.cell_at<Q>(g, i, -1);
}

// Flat index of the post-collision f_i(x) for a state in layout `lay`.
template <int Q, bool WALLS>
__device__ __forceinline__ size_t natural_index(const Geometry& g, const Nbr& nb, size_t cell,
                                                int i, int lay) {
    const size_t N = g.N;
    if (lay == NATURAL) return (size_t)i * N + cell;
    if (lay == SWAPPED) return (size_t)opp<Q>(i) * N + cell;
    // STREAMED: f_i(x) travelled to x + c_i (slot i), or bounced back into
    // slot opp(i) of x when x + c_i lies beyond a wall.
    const bool wall = WALLS && nb.beyond_wall<Q>(i, +1);
    return wall ? (size_t)opp<Q>(i) * N + cell : (size_t)i * N + nb.cell_at<Q>(g, i, +1);
}

// ---------------------------------------------------------------------------
// Per-cell physics in arithmetic type C.
// ---------------------------------------------------------------------------
template <class C>
struct Phys {
    C omega;       // 1/tau
    C guo;         // 1 - 1/(2 tau)
    C Fx, Fy, Fz;  // body force
};

// Moments of deviations d_i = g_i - w_i: drho = sum d, j = sum c d (the
// weights carry no momentum), rho = 1 + drho, rho*u = j + F/2.
template <int Q, class C>
__device__ __forceinline__ void moments(const C* d, const Phys<C>& ph, C& drho, C& mx, C& my,
                                        C& mz) {
    using L = Lat<Q>;
    C s = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s += d[i];
        if (L::cx(i) > 0) jx += d[i];
        if (L::cx(i) < 0) jx -= d[i];
        if (L::cy(i) > 0) jy += d[i];
        if (L::cy(i) < 0) jy -= d[i];
        if (L::cz(i) > 0) jz += d[i];
        if (L::cz(i) < 0) jz -= d[i];
    }
    drho = s;
    mx = jx + C(0.5) * ph.Fx;
    my = jy + C(0.5) * ph.Fy;
    mz = jz + C(0.5) * ph.Fz;
}

// HBGK collision of one cell, in place on the deviations d (Sec. 3.2:
// relaxation toward the Maxwellian at varpi*u; Guo's source built with u).
template <int Q, class C>
__device__ __forceinline__ void collide(C* d, C varpi, const Phys<C>& ph) {
    using L = Lat<Q>;
    C drho, mx, my, mz;
    moments<Q, C>(d, ph, drho, mx, my, mz);
    const C rho = C(1) + drho;
    const C inv_rho = C(1) / rho;
    const C ux = mx * inv_rho, uy = my * inv_rho, uz = mz * inv_rho;
    const C vx = varpi * ux, vy = varpi * uy, vz = varpi * uz;
    const C vv15 = C(1.5) * (vx * vx + vy * vy + vz * vz);
    const C uF3 = C(3) * (ux * ph.Fx + uy * ph.Fy + uz * ph.Fz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const C cx = C(L::cx(i)), cy = C(L::cy(i)), cz = C(L::cz(i));
        const C w = C(L::w(i));
        const C cv = cx * vx + cy * vy + cz * vz;
        const C cu = cx * ux + cy * uy + cz * uz;
        const C cF = cx * ph.Fx + cy * ph.Fy + cz * ph.Fz;
        // deviation of the equilibrium from w_i
        const C eq = w * (drho + rho * (C(3) * cv + C(4.5) * cv * cv - vv15));
        const C src = ph.guo * w * (C(3) * cF - uF3 + C(9) * cu * cF);
        d[i] = d[i] + ph.omega * (eq - d[i]) + src;
    }
}

}  // namespace hlbm
