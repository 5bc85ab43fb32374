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
#include <cmath>
#include <cstdint>
#include <type_traits>

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
// `scaled` policies keep deviations times a power-of-two scale s; the step
// kernel then works in scaled units throughout (load_raw / store_raw), which
// is exact because multiplying by a power of two commutes with rounding.
struct StoreF64 {
    using T = double;
    using C = double;
    static constexpr int kind = 0;
    static constexpr bool scaled = false;
    template <class I>
    __device__ __forceinline__ static C load_raw(const T* p, I i) { return __ldg(p + i); }
    template <class I>
    __device__ __forceinline__ static void store_raw(T* p, I i, C v) { p[i] = v; }
    template <class I>
    __device__ __forceinline__ static C load(const T* p, I i, C) { return __ldg(p + i); }
    template <class I>
    __device__ __forceinline__ static void store(T* p, I i, C v, C) { p[i] = v; }
};
struct StoreF32 {
    using T = float;
    using C = float;
    static constexpr int kind = 1;
    static constexpr bool scaled = false;
    template <class I>
    __device__ __forceinline__ static C load_raw(const T* p, I i) { return __ldg(p + i); }
    template <class I>
    __device__ __forceinline__ static void store_raw(T* p, I i, C v) { p[i] = v; }
    template <class I>
    __device__ __forceinline__ static C load(const T* p, I i, C) { return __ldg(p + i); }
    template <class I>
    __device__ __forceinline__ static void store(T* p, I i, C v, C) { p[i] = v; }
};
struct StoreF16 {
    using T = __half;
    using C = float;
    static constexpr int kind = 2;
    static constexpr bool scaled = true;
    template <class I>
    __device__ __forceinline__ static C load_raw(const T* p, I i) { return __half2float(__ldg(p + i)); }
    template <class I>
    __device__ __forceinline__ static void store_raw(T* p, I i, C v) { p[i] = __float2half_rn(v); }
    template <class I>
    __device__ __forceinline__ static C load(const T* p, I i, C inv_s) {
        return __half2float(__ldg(p + i)) * inv_s;
    }
    template <class I>
    __device__ __forceinline__ static void store(T* p, I i, C v, C s) {
        p[i] = __float2half_rn(v * s);
    }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    using C = float;
    static constexpr int kind = 3;
    static constexpr bool scaled = false;
    template <class I>
    __device__ __forceinline__ static C load_raw(const T* p, I i) { return __bfloat162float(__ldg(p + i)); }
    template <class I>
    __device__ __forceinline__ static void store_raw(T* p, I i, C v) { p[i] = __float2bfloat16_rn(v); }
    template <class I>
    __device__ __forceinline__ static C load(const T* p, I i, C inv_s) {
        return __bfloat162float(__ldg(p + i)) * inv_s;
    }
    template <class I>
    __device__ __forceinline__ static void store(T* p, I i, C v, C s) {
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

// Neighbour bookkeeping of one cell: element offsets from the cell to its
// periodic neighbours at -1 / +1 along each axis (wrap folded in), and
// whether the cell sits at the low / high end of a wall axis. I is the index
// type: int when q*cells < 2^31 (cheaper address arithmetic), else long long.
// Resolved obstacles: links[cell] bit i says that the pull source x - c_i is a
// solid cell (bounce-back on that link), bit 31 that the cell itself is solid.
constexpr unsigned kSolidBit = 1u << 31;

template <class I = long long>
struct Nbr {
    I oxm, oxp, oym, oyp, ozm, ozp;
    bool lo_x, hi_x, lo_y, hi_y, lo_z, hi_z;
    unsigned lm = 0;  // solid-link mask of the cell (0 without obstacles)

    __device__ __forceinline__ Nbr(const Geometry& g, int x, int y, int z, unsigned links = 0) : lm(links) {
        const I sy = (I)g.nx, sz = (I)g.nx * (I)g.ny;
        oxm = x == 0 ? (I)(g.nx - 1) : (I)-1;
        oxp = x == g.nx - 1 ? (I)(1 - g.nx) : (I)1;
        oym = y == 0 ? (I)(g.ny - 1) * sy : -sy;
        oyp = y == g.ny - 1 ? (I)(1 - g.ny) * sy : sy;
        ozm = z == 0 ? (I)(g.nz - 1) * sz : -sz;
        ozp = z == g.nz - 1 ? (I)(1 - g.nz) * sz : sz;
        lo_x = g.wall_x && x == 0;
        hi_x = g.wall_x && x == g.nx - 1;
        lo_y = g.wall_y && y == 0;
        hi_y = g.wall_y && y == g.ny - 1;
        lo_z = g.wall_z && z == 0;
        hi_z = g.wall_z && z == g.nz - 1;
    }

    // Offset from the cell to x + s*c_i (s = -1 pull source, +1 push target).
    template <int Q>
    __device__ __forceinline__ I offset(int i, int s) const {
        using L = Lat<Q>;
        const int dx = s * L::cx(i), dy = s * L::cy(i), dz = s * L::cz(i);
        I o = 0;
        if (dx > 0) o += oxp;
        if (dx < 0) o += oxm;
        if (dy > 0) o += oyp;
        if (dy < 0) o += oym;
        if (dz > 0) o += ozp;
        if (dz < 0) o += ozm;
        return o;
    }

    // Does x + s*c_i lie beyond a wall or in a solid cell? (x + c_i is the pull
    // source of the opposite direction.)
    template <int Q>
    __device__ __forceinline__ bool beyond_wall(int i, int s) const {
        using L = Lat<Q>;
        const int dx = s * L::cx(i), dy = s * L::cy(i), dz = s * L::cz(i);
        const int link = s < 0 ? i : opp<Q>(i);
        return (dx < 0 && lo_x) || (dx > 0 && hi_x) || (dy < 0 && lo_y) || (dy > 0 && hi_y) ||
               (dz < 0 && lo_z) || (dz > 0 && hi_z) || ((lm >> link) & 1u);
    }
};

// Flat index (into the [q][cells] array) holding g_i(x), the population the
// collision at x consumes, for a state in layout `lay`.
template <int Q, bool WALLS, class I>
__device__ __forceinline__ I gather_index(const Geometry& g, const Nbr<I>& nb, I cell, int i, int lay) {
    const I N = (I)g.N;
    if (lay == STREAMED) return (I)i * N + cell;
    const bool wall = WALLS && nb.template beyond_wall<Q>(i, -1);
    if (lay == NATURAL)
        return wall ? (I)opp<Q>(i) * N + cell : (I)i * N + cell + nb.template offset<Q>(i, -1);
    // SWAPPED: f_i(x - c_i) sits in slot opp(i) of cell x - c_i; across a
    // wall the bounce-back f_opp(i)(x) sits in slot i of x.
    return wall ? (I)i * N + cell : (I)opp<Q>(i) * N + cell + nb.template offset<Q>(i, -1);
}

// Flat index of the post-collision f_i(x) for a state in layout `lay`.
template <int Q, bool WALLS, class I>
__device__ __forceinline__ I natural_index(const Geometry& g, const Nbr<I>& nb, I cell, int i, int lay) {
    const I N = (I)g.N;
    if (lay == NATURAL) return (I)i * N + cell;
    if (lay == SWAPPED) return (I)opp<Q>(i) * N + cell;
    // STREAMED: f_i(x) travelled to x + c_i (slot i), or bounced back into
    // slot opp(i) of x when x + c_i lies beyond a wall.
    const bool wall = WALLS && nb.template beyond_wall<Q>(i, +1);
    return wall ? (I)opp<Q>(i) * N + cell : (I)i * N + cell + nb.template offset<Q>(i, +1);
}

// ---------------------------------------------------------------------------
// Per-cell physics in arithmetic type C.
//
// Rounding. In FP32 two habits bias the momentum budget systematically
// (measured at ~1e-5 relative velocity error after 1000 steps of a forced
// sphere-pack flow): (a) adding a constant (F/2, a force term) to a value
// gives the same rounding error for every value of a binade, so it does not
// average out; (b) per-direction constants such as w_i*omega*3, each rounded
// on its own, make the equilibrium's first moment differ from the omega in
// (1 - omega) by a fixed factor. So: the force never enters j; the linear
// (odd) part of each pair is one fma with a varying product; and its
// coefficients are derived from the rounded omega and guo so that
// sum_i c_ix^2 k_i = omega and sum_i c_ix^2 g_i = guo hold exactly.
// ---------------------------------------------------------------------------
template <class C>
struct Phys {
    C omega;       // 1/tau, rounded to C
    C guo;         // 1 - omega/2 (exact in C)
    C k1, k2;      // odd equilibrium coefficients of |c|^2 = 1 and 2 directions (~3 w omega)
    C g1, g2;      // odd force coefficients (~3 w guo)
    C Fx, Fy, Fz;  // body force
};

// Coefficients k1 (|c|^2 = 1, na directions along an axis) and k2 (|c|^2 = 2,
// nb of them touch an axis) with na*k1 + nb*k2 == target exactly (checked in
// double for float; FP64 keeps the plain rounding, its bias is at 1e-16).
template <class C>
__host__ inline void split_exact(C target, double w1x3, double w2x3, int na, int nb, C& k1, C& k2) {
    const C base = C((double)target * w2x3);
    if (sizeof(C) == 4) {
        // try base, base+1ulp, base-1ulp, base+2ulp, ... until the split is exact
        for (int k = 0; k < 64; ++k) {
            const int off = (k + 1) / 2 * ((k & 1) ? 1 : -1);
            float t2 = (float)base;
            for (int s = 0; s < (off < 0 ? -off : off); ++s) t2 = nextafterf(t2, off > 0 ? 1e30f : -1e30f);
            const float t1 = (float)(((double)target - nb * (double)t2) / na);
            if ((double)na * (double)t1 + (double)nb * (double)t2 == (double)target) {
                k1 = C(t1);
                k2 = C(t2);
                return;
            }
        }
    }
    k2 = base;
    k1 = C(((double)target - nb * (double)base) / na);
}

template <class C, int Q>
__host__ inline Phys<C> make_phys(double tau, const double F[3]) {
    Phys<C> p;
    p.omega = C(1.0 / tau);
    p.guo = C(1) - p.omega / C(2);
    // x-momentum: D3Q19 has 2 faces and 8 edges with c_x != 0 (w = 1/18, 1/36);
    // D2Q9 has 2 faces and 4 diagonals (w = 1/9, 1/36).
    const double w1x3 = Q == 19 ? 3.0 / 18.0 : 3.0 / 9.0, w2x3 = 3.0 / 36.0;
    const int nb = Q == 19 ? 8 : 4;
    split_exact<C>(p.omega, w1x3, w2x3, 2, nb, p.k1, p.k2);
    split_exact<C>(p.guo, w1x3, w2x3, 2, nb, p.g1, p.g2);
    p.Fx = C(F[0]);
    p.Fy = C(F[1]);
    p.Fz = Q == 9 ? C(0) : C(F[2]);
    return p;
}

// ---------------------------------------------------------------------------
// Lane arithmetic of the collision. Every operation of the collision below is
// written out and rounded on its own (a product is never contracted into a
// following add, nothing is reassociated), so the collision is the same
// sequence of IEEE operations whether a thread updates one cell (lane type
// float or double) or two neighbouring cells at once (F2: the paired FP32
// instructions add/sub/mul/fma .rn.f32x2 of sm_100-class GPUs, one issue slot
// for both lanes, each lane rounded exactly as the scalar instruction). Every
// step kernel therefore produces the same bits for a cell, and the paired
// 16-bit kernels issue about half the floating-point instructions.
// ---------------------------------------------------------------------------
// All helpers are PTX instructions with an explicit rounding modifier. Measured
// on GB300 (4M random operand triples): each paired instruction rounds every lane
// exactly as the scalar instruction does, and a scalar multiply followed by a
// scalar add is never fused; but a paired multiply whose result only feeds a
// paired add or subtract is contracted into a paired fma by the code generator
// (about 20 % of random x + a*b then differ from the separately rounded value).
// The collision below is therefore written so that no product is added or
// subtracted after rounding.
__device__ __forceinline__ float add_(float a, float b) {
    float d;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float sub_(float a, float b) {
    float d;
    asm("sub.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float mul_(float a, float b) {
    float d;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float fma_(float a, float b, float c) {
    float d;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float rcp_(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double add_(double a, double b) {
    double d;
    asm("add.rn.f64 %0, %1, %2;" : "=d"(d) : "d"(a), "d"(b));
    return d;
}
__device__ __forceinline__ double sub_(double a, double b) {
    double d;
    asm("sub.rn.f64 %0, %1, %2;" : "=d"(d) : "d"(a), "d"(b));
    return d;
}
__device__ __forceinline__ double mul_(double a, double b) {
    double d;
    asm("mul.rn.f64 %0, %1, %2;" : "=d"(d) : "d"(a), "d"(b));
    return d;
}
__device__ __forceinline__ double fma_(double a, double b, double c) {
    double d;
    asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(b), "d"(c));
    return d;
}
__device__ __forceinline__ double rcp_(double a) { return __drcp_rn(a); }

// Two FP32 lanes in one 64-bit register pair (lane 0 = the lower cell of a pair).
struct F2 {
    unsigned long long v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ explicit F2(float a) { asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(a)); }
    __device__ __forceinline__ F2(float lo, float hi) { asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi)); }
    __device__ __forceinline__ float2 split() const {
        float2 r;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
        return r;
    }
};
__device__ __forceinline__ F2 add_(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 sub_(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 mul_(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ F2 rcp_(F2 a) {
    const float2 x = a.split();
    return F2(__frcp_rn(x.x), __frcp_rn(x.y));
}

// Scalar type of a lane type; V(k) broadcasts a scalar to every lane.
template <class V>
struct Lane {
    using S = V;
};
template <>
struct Lane<F2> {
    using S = float;
};

// sum_a c_a x_a for a direction with components in {-1, 0, 1} and at least one
// +1: the +1 terms in axis order, then the -1 terms subtracted (no products).
template <int CX, int CY, int CZ, class V>
__device__ __forceinline__ V cdot(V x, V y, V z) {
    static_assert(CX == 1 || CY == 1 || CZ == 1, "cdot needs a +1 component");
    V r = CX == 1 ? x : (CY == 1 ? y : z);
    if (CY == 1 && CX == 1) r = add_(r, y);
    if (CZ == 1 && (CX == 1 || CY == 1)) r = add_(r, z);
    if (CX == -1) r = sub_(r, x);
    if (CY == -1) r = sub_(r, y);
    if (CZ == -1) r = sub_(r, z);
    return r;
}
template <int Q, int I, class V>
__device__ __forceinline__ V cdot_i(V x, V y, V z) {
    using L = Lat<Q>;
    return cdot<L::cx(I), L::cy(I), L::cz(I), V>(x, y, z);
}
// The same for uniform scalars with a general sign pattern (force components).
template <int Q, int I, class S>
__device__ __forceinline__ S cdot_s(S x, S y, S z) {
    using L = Lat<Q>;
    S r = S(0);
    if (L::cx(I) > 0) r = add_(r, x);
    if (L::cx(I) < 0) r = sub_(r, x);
    if (L::cy(I) > 0) r = add_(r, y);
    if (L::cy(I) < 0) r = sub_(r, y);
    if (L::cz(I) > 0) r = add_(r, z);
    if (L::cz(I) < 0) r = sub_(r, z);
    return r;
}

// Moments of the deviations for the collision: drho = sum d (index order) and
// j = sum c d (per axis: from the first +1 direction, then in index order).
template <int Q, int A, class V, class Pop>
__device__ __forceinline__ V axis_sum(const Pop& d) {
    using L = Lat<Q>;
    constexpr int first = A == 0 ? 1 : (Q == 9 ? 2 : (A == 1 ? 3 : 5));  // first direction with c_A = +1
    V r = d[first];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (i == first) continue;
        const int c = A == 0 ? L::cx(i) : (A == 1 ? L::cy(i) : L::cz(i));
        if (c > 0) r = add_(r, d[i]);
        if (c < 0) r = sub_(r, d[i]);
    }
    return r;
}
template <int Q, class V, class Pop>
__device__ __forceinline__ void moments_x(const Pop& d, V& drho, V& jx, V& jy, V& jz) {
    V s = d[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) s = add_(s, d[i]);
    drho = s;
    jx = axis_sum<Q, 0, V>(d);
    jy = axis_sum<Q, 1, V>(d);
    jz = Q == 9 ? V(typename Lane<V>::S(0)) : axis_sum<Q, 2, V>(d);
}

// Zeroth and first moments of deviations d_i = g_i - w_i (Def. moments): drho =
// sum d, j = sum c d (the weights carry no momentum); rho = 1 + drho and the
// half-force momentum is rho*u = j + F/2 (added by the caller in the precision it needs).
template <int Q, class C>
__device__ __forceinline__ void moments(const C* d, C& drho, C& jx, C& jy, C& jz) {
    using L = Lat<Q>;
    C s = 0, ax = 0, ay = 0, az = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s += d[i];
        if (L::cx(i) > 0) ax += d[i];
        if (L::cx(i) < 0) ax -= d[i];
        if (L::cy(i) > 0) ay += d[i];
        if (L::cy(i) < 0) ay -= d[i];
        if (L::cz(i) > 0) az += d[i];
        if (L::cz(i) < 0) az -= d[i];
    }
    drho = s;
    jx = ax;
    jy = ay;
    jz = az;
}

// Half-force velocity u = (j + F/2)/rho, with F/2 folded in by an fma.
template <class C>
__device__ __forceinline__ void velocity(C jx, C jy, C jz, C inv_rho, const Phys<C>& ph, C& ux, C& uy, C& uz) {
    const C h = C(0.5) * inv_rho;
    ux = fma_(ph.Fx, h, jx * inv_rho);
    uy = fma_(ph.Fy, h, jy * inv_rho);
    uz = fma_(ph.Fz, h, jz * inv_rho);
}

// The collision reads its input populations through `d` (d[i], i < q: an
// array, or an object that unpacks stored words on each use) and hands every
// final post-collision value to a sink, out(i, value), as soon as it is known,
// so a kernel can store it at once instead of keeping all q values live.
// WriteBack makes the collision in place on an array.
template <class V>
struct WriteBack {
    V* d;
    __device__ __forceinline__ void operator()(int i, V v) const { d[i] = v; }
};

// One opposite pair (I, opp(I)) of the collision: d_I = keep d_I + even + odd,
// d_opp = keep d_opp + even - odd.
template <int Q, int I, class V, class Pop, class Sink>
__device__ __forceinline__ void relax_pair(const Pop& d, V keep, V even, V odd, Sink& out) {
    constexpr int J = opp<Q>(I);
    const V a = add_(fma_(keep, V(d[I]), even), odd);
    const V b = sub_(fma_(keep, V(d[J]), even), odd);
    out(I, a);
    out(J, b);
}

// As relax_pair for an odd part that is a single product k (c.j): it enters
// through an fma (k and -k), never as a product added afterwards.
template <int Q, int I, class V, class Pop, class Sink>
__device__ __forceinline__ void relax_pair_prod(const Pop& d, V keep, V even, V k, V nk, V cj, Sink& out) {
    constexpr int J = opp<Q>(I);
    const V a = fma_(k, cj, fma_(keep, V(d[I]), even));
    const V b = fma_(nk, cj, fma_(keep, V(d[J]), even));
    out(I, a);
    out(J, b);
}

// sum_a c_a w_a x_a over the nonzero components of direction I as an fma chain
// (c_a w_a is w_a or -w_a, an exact negation of an input), so no product is
// added after it has been rounded.
template <int Q, int I, class V>
__device__ __forceinline__ V cdot_w(V wx, V wy, V wz, V nwx, V nwy, V nwz, V x, V y, V z) {
    using L = Lat<Q>;
    constexpr int cx = L::cx(I), cy = L::cy(I), cz = L::cz(I);
    V r;
    bool have = false;
    if (cx != 0) {
        r = mul_(cx > 0 ? wx : nwx, x);
        have = true;
    }
    if (cy != 0) {
        r = have ? fma_(cy > 0 ? wy : nwy, y, r) : mul_(cy > 0 ? wy : nwy, y);
        have = true;
    }
    if (cz != 0) r = have ? fma_(cz > 0 ? wz : nwz, z, r) : mul_(cz > 0 ? wz : nwz, z);
    return r;
}

// Compile-time loop over the pairs of a velocity set (each pair from its lower
// index, which has a +1 component in both orderings).
template <int Q, int I = 1, class F>
__device__ __forceinline__ void for_pairs(F&& f) {
    if constexpr (I < Q) {
        if constexpr (opp<Q>(I) > I) f(std::integral_constant<int, I>{});
        for_pairs<Q, I + 1>(f);
    }
}

// HBGK collision of one cell (or of two, V = F2), in place on the deviations d
// (Sec. 3.2: relaxation toward the Maxwellian at varpi*u; Guo's source built
// with u). Opposite directions share the even part of the equilibrium and of
// the source and differ in the sign of the odd part, so each pair costs one
// evaluation:
//   M_i - w_i = w_i [drho + rho (4.5 (c.v)^2 - 1.5 v.v)]  +-  3 w_i rho (c.v)
//   S_i       = guo w_i [9 (c.u)(c.F) - 3 u.F]            +-  3 w_i guo (c.F)
// and with rho (c.v) = varpi (c.j + c.F/2) the odd part of omega*M_i + S_i is
//   k_i varpi (c.j) + (k_i varpi / 2 + g_i) (c.F).
// c.u is formed as (c.j)/rho + (c.F)/(2 rho) and c.v as varpi (c.u). The code
// generator may contract a paired multiply into a following paired add (it does
// on GB300) but not a scalar one, so no product here is added or subtracted
// after rounding: products only feed multiplies and fmas. That keeps the paired
// and the scalar evaluations bit-identical.
template <int Q, class V, bool SCALED, bool FX_ONLY, class Pop, class Sink>
__device__ __forceinline__ void collide(const Pop& d, V varpi, const Phys<typename Lane<V>::S>& ph,
                                        typename Lane<V>::S s, typename Lane<V>::S inv_s, Sink out) {
    // FX_ONLY: the caller guarantees F = (Fx, 0, 0); the terms with c.F = 0 drop out.
    // With SCALED the d are s * (f - w) on entry and exit; every term below
    // that adds into d carries the factor s (a power of two: exact).
    using L = Lat<Q>;
    using S = typename Lane<V>::S;
    V drho_s, jxs, jys, jzs;  // sums in the units of d
    moments_x<Q, V>(d, drho_s, jxs, jys, jzs);
    const V rho = SCALED ? fma_(drho_s, V(inv_s), V(S(1))) : add_(V(S(1)), drho_s);
    const V inv_rho = rcp_(rho);
    const V im = SCALED ? mul_(inv_rho, V(inv_s)) : inv_rho;  // 1/rho in the units of d (exact scaling)
    const V h = mul_(V(S(0.5)), inv_rho);
    const V ux = fma_(V(ph.Fx), h, mul_(jxs, im));
    const V uy = FX_ONLY ? mul_(jys, im) : fma_(V(ph.Fy), h, mul_(jys, im));
    const V uz = FX_ONLY ? mul_(jzs, im) : fma_(V(ph.Fz), h, mul_(jzs, im));
    const V rho_s = SCALED ? mul_(rho, V(s)) : rho;
    const V uu = fma_(uz, uz, fma_(uy, uy, mul_(ux, ux)));
    const V vv = mul_(mul_(varpi, varpi), uu);
    const V A = fma_(mul_(rho_s, V(S(-1.5))), vv, drho_s);
    // -3 u.F
    const V nuF3 = FX_ONLY ? mul_(ux, V(mul_(S(-3), ph.Fx)))
                           : mul_(V(S(-3)), fma_(uz, V(ph.Fz), fma_(uy, V(ph.Fy), mul_(ux, V(ph.Fx)))));
    const V r45 = mul_(V(S(4.5)), rho_s);
    const V keep = V(sub_(S(1), ph.omega));
    const S guo_s = SCALED ? mul_(ph.guo, s) : ph.guo;
    {  // rest population
        const S w = S(L::w(0));
        out(0, fma_(keep, V(d[0]), fma_(V(mul_(ph.omega, w)), A, mul_(V(mul_(guo_s, w)), nuF3))));
    }
    const V kv1 = mul_(V(ph.k1), varpi), kv2 = mul_(V(ph.k2), varpi);
    const S g1 = SCALED ? mul_(ph.g1, s) : ph.g1, g2 = SCALED ? mul_(ph.g2, s) : ph.g2;
    const V kvs1 = SCALED ? mul_(kv1, V(s)) : kv1, kvs2 = SCALED ? mul_(kv2, V(s)) : kv2;
    for_pairs<Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int c2 = L::cx(I) * L::cx(I) + L::cy(I) * L::cy(I) + L::cz(I) * L::cz(I);
        const S w = S(L::w(I));
        const V ow = V(mul_(ph.omega, w)), gw = V(mul_(guo_s, w));
        const V cj = cdot_i<Q, I>(jxs, jys, jzs);  // c.j in the units of d
        const V kv = c2 == 1 ? kv1 : kv2;
        if (FX_ONLY && L::cx(I) == 0) {  // c.F = 0: the odd part is the product kv (c.j)
            const V cu = mul_(cj, im);
            const V cv = mul_(varpi, cu);
            const V even = fma_(ow, fma_(r45, mul_(cv, cv), A), mul_(gw, nuF3));
            const V nkv = mul_(V(c2 == 1 ? -ph.k1 : -ph.k2), varpi);
            relax_pair_prod<Q, I>(d, keep, even, kv, nkv, cj, out);
        } else {
            const S cF = FX_ONLY ? (L::cx(I) > 0 ? ph.Fx : -ph.Fx) : cdot_s<Q, I>(ph.Fx, ph.Fy, ph.Fz);
            const V cu = fma_(V(cF), h, mul_(cj, im));
            const V cv = mul_(varpi, cu);
            const V kvs = c2 == 1 ? kvs1 : kvs2;
            const S g = c2 == 1 ? g1 : g2;
            const V even = fma_(ow, fma_(r45, mul_(cv, cv), A), mul_(gw, fma_(mul_(V(S(9)), cu), V(cF), nuF3)));
            const V odd = fma_(kv, cj, fma_(kvs, V(mul_(S(0.5), cF)), V(mul_(g, cF))));
            relax_pair<Q, I>(d, keep, even, odd, out);
        }
    });
}

// Explicit-drag form of the homogenization (Sec. 3.3, eq. momentumHLBM): the
// equilibrium stays at u and the drag -lam rho u, lam = nu/K = (1 - varpi)/tau,
// joins the body force, G = F - lam rho u, in Guo's scheme; u is the half-force
// velocity of the total force, u = (j + F/2) / (rho (1 + lam/2)). With
// h = 1/(1 + lam/2), rho (c.u) = h (c.j + c.F/2) and c.G = c.F - lam rho (c.u),
// so the odd part of omega*M_i + S_i is kk (c.j) + (kk/2 + g)(c.F) with
// kk = (k - g lam) h: the same fma shape as the shift form (and the same rule:
// no product is added after rounding).
template <int Q, class V, bool SCALED, class Pop, class Sink>
__device__ __forceinline__ void collide_drag(const Pop& d, V varpi, const Phys<typename Lane<V>::S>& ph,
                                             typename Lane<V>::S s, typename Lane<V>::S inv_s, Sink out) {
    using L = Lat<Q>;
    using S = typename Lane<V>::S;
    V drho_s, jxs, jys, jzs;
    moments_x<Q, V>(d, drho_s, jxs, jys, jzs);
    const V rho = SCALED ? fma_(drho_s, V(inv_s), V(S(1))) : add_(V(S(1)), drho_s);
    const V lam = mul_(sub_(V(S(1)), varpi), V(ph.omega));
    const V nlam = mul_(sub_(varpi, V(S(1))), V(ph.omega));  // -lam, exactly
    const V h = rcp_(fma_(V(S(0.5)), lam, V(S(1))));
    const V hr = mul_(h, rcp_(rho));
    const V hm = SCALED ? mul_(hr, V(inv_s)) : hr;  // in the units of d (exact scaling)
    const V hh = mul_(V(S(0.5)), hr);
    const V ux = fma_(V(ph.Fx), hh, mul_(jxs, hm));
    const V uy = fma_(V(ph.Fy), hh, mul_(jys, hm));
    const V uz = fma_(V(ph.Fz), hh, mul_(jzs, hm));
    const V nlr = mul_(nlam, rho);  // -lam rho
    const V Gx = fma_(nlr, ux, V(ph.Fx)), Gy = fma_(nlr, uy, V(ph.Fy)), Gz = fma_(nlr, uz, V(ph.Fz));
    const V rho_s = SCALED ? mul_(rho, V(s)) : rho;
    const V uu = fma_(uz, uz, fma_(uy, uy, mul_(ux, ux)));
    const V A = fma_(mul_(rho_s, V(S(-1.5))), uu, drho_s);
    const V nuG3 = mul_(V(S(-3)), fma_(uz, Gz, fma_(uy, Gy, mul_(ux, Gx))));
    const V r45 = mul_(V(S(4.5)), rho_s);
    const V keep = V(sub_(S(1), ph.omega));
    const S guo_s = SCALED ? mul_(ph.guo, s) : ph.guo;
    {
        const S w = S(L::w(0));
        out(0, fma_(keep, V(d[0]), fma_(V(mul_(ph.omega, w)), A, mul_(V(mul_(guo_s, w)), nuG3))));
    }
    const V kk1 = mul_(fma_(V(-ph.g1), lam, V(ph.k1)), h), kk2 = mul_(fma_(V(-ph.g2), lam, V(ph.k2)), h);
    const S g1 = SCALED ? mul_(ph.g1, s) : ph.g1, g2 = SCALED ? mul_(ph.g2, s) : ph.g2;
    const V kks1 = SCALED ? mul_(kk1, V(s)) : kk1, kks2 = SCALED ? mul_(kk2, V(s)) : kk2;
    for_pairs<Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int c2 = L::cx(I) * L::cx(I) + L::cy(I) * L::cy(I) + L::cz(I) * L::cz(I);
        const S w = S(L::w(I));
        const V ow = V(mul_(ph.omega, w)), gw = V(mul_(guo_s, w));
        const V cu = cdot_i<Q, I>(ux, uy, uz);
        const V cG = cdot_i<Q, I>(Gx, Gy, Gz);
        const V cj = cdot_i<Q, I>(jxs, jys, jzs);
        const S cF = cdot_s<Q, I>(ph.Fx, ph.Fy, ph.Fz);
        const V kk = c2 == 1 ? kk1 : kk2;
        const V kks = c2 == 1 ? kks1 : kks2;
        const S g = c2 == 1 ? g1 : g2;
        const V even = fma_(ow, fma_(r45, mul_(cu, cu), A), mul_(gw, fma_(mul_(V(S(9)), cu), cG, nuG3)));
        const V odd = fma_(kk, cj, fma_(kks, V(mul_(S(0.5), cF)), V(mul_(g, cF))));
        relax_pair<Q, I>(d, keep, even, odd, out);
    });
}

// Anisotropic (diagonal-tensor) porosity control: the Maxwellian at
// v = (vx ux, vy uy, vz uz), a per-axis drag nu/K_a. As collide(), with the
// odd part k (c.(varpi o j)) + (k/2 c.(varpi o F) + g c.F); the weighted dot
// products are fma chains.
template <int Q, class V, bool SCALED, class Pop, class Sink>
__device__ __forceinline__ void collide_aniso(const Pop& d, V wx, V wy, V wz, const Phys<typename Lane<V>::S>& ph,
                                              typename Lane<V>::S s, typename Lane<V>::S inv_s, Sink out) {
    using L = Lat<Q>;
    using S = typename Lane<V>::S;
    V drho_s, jxs, jys, jzs;
    moments_x<Q, V>(d, drho_s, jxs, jys, jzs);
    const V rho = SCALED ? fma_(drho_s, V(inv_s), V(S(1))) : add_(V(S(1)), drho_s);
    const V inv_rho = rcp_(rho);
    const V im = SCALED ? mul_(inv_rho, V(inv_s)) : inv_rho;
    const V h = mul_(V(S(0.5)), inv_rho);
    const V ux = fma_(V(ph.Fx), h, mul_(jxs, im));
    const V uy = fma_(V(ph.Fy), h, mul_(jys, im));
    const V uz = fma_(V(ph.Fz), h, mul_(jzs, im));
    const V nwx = sub_(V(S(0)), wx), nwy = sub_(V(S(0)), wy), nwz = sub_(V(S(0)), wz);
    const V rho_s = SCALED ? mul_(rho, V(s)) : rho;
    const V vx = mul_(wx, ux), vy = mul_(wy, uy), vz = mul_(wz, uz);
    const V vv = fma_(vz, vz, fma_(vy, vy, mul_(vx, vx)));
    const V A = fma_(mul_(rho_s, V(S(-1.5))), vv, drho_s);
    const V nuF3 = mul_(V(S(-3)), fma_(uz, V(ph.Fz), fma_(uy, V(ph.Fy), mul_(ux, V(ph.Fx)))));
    const V r45 = mul_(V(S(4.5)), rho_s);
    const V keep = V(sub_(S(1), ph.omega));
    const S guo_s = SCALED ? mul_(ph.guo, s) : ph.guo;
    {
        const S w = S(L::w(0));
        out(0, fma_(keep, V(d[0]), fma_(V(mul_(ph.omega, w)), A, mul_(V(mul_(guo_s, w)), nuF3))));
    }
    const V hFx = V(mul_(S(0.5), ph.Fx)), hFy = V(mul_(S(0.5), ph.Fy)), hFz = V(mul_(S(0.5), ph.Fz));
    const S g1 = SCALED ? mul_(ph.g1, s) : ph.g1, g2 = SCALED ? mul_(ph.g2, s) : ph.g2;
    const S ks1 = SCALED ? mul_(ph.k1, s) : ph.k1, ks2 = SCALED ? mul_(ph.k2, s) : ph.k2;
    for_pairs<Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int c2 = L::cx(I) * L::cx(I) + L::cy(I) * L::cy(I) + L::cz(I) * L::cz(I);
        const S w = S(L::w(I));
        const V ow = V(mul_(ph.omega, w)), gw = V(mul_(guo_s, w));
        const V cv = cdot_w<Q, I>(wx, wy, wz, nwx, nwy, nwz, ux, uy, uz);
        const V cu = cdot_i<Q, I>(ux, uy, uz);
        const S cF = cdot_s<Q, I>(ph.Fx, ph.Fy, ph.Fz);
        const V cpj = cdot_w<Q, I>(wx, wy, wz, nwx, nwy, nwz, jxs, jys, jzs);  // c.(varpi o j), units of d
        const V cpF = cdot_w<Q, I>(wx, wy, wz, nwx, nwy, nwz, hFx, hFy, hFz);  // c.(varpi o F)/2
        const S k = c2 == 1 ? ph.k1 : ph.k2;
        const S ks = c2 == 1 ? ks1 : ks2;
        const S g = c2 == 1 ? g1 : g2;
        const V even = fma_(ow, fma_(r45, mul_(cv, cv), A), mul_(gw, fma_(mul_(V(S(9)), cu), V(cF), nuF3)));
        const V odd = fma_(V(k), cpj, fma_(V(ks), cpF, V(mul_(g, cF))));
        relax_pair<Q, I>(d, keep, even, odd, out);
    });
}

// Velocity seen by the collision of either form: u = (j + F/2)/rho for the
// shift form, divided by (1 + lam/2) for the drag form.
template <class C>
__device__ __forceinline__ void velocity_form(C jx, C jy, C jz, C rho, C varpi, int drag, const Phys<C>& ph, C& ux,
                                              C& uy, C& uz) {
    C inv = C(1) / rho;
    if (drag) inv = inv / fma_(C(0.5), (C(1) - varpi) * ph.omega, C(1));
    velocity<C>(jx, jy, jz, inv, ph, ux, uy, uz);
}

}  // namespace hlbm
