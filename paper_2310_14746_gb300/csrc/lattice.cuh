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

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

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

// HBGK collision of one cell, in place on the deviations d (Sec. 3.2:
// relaxation toward the Maxwellian at varpi*u; Guo's source built with u).
// Opposite directions share the even part of the equilibrium and of the
// source and differ in the sign of the odd part, so each pair costs one
// evaluation:
//   M_i - w_i = w_i [drho + rho (4.5 (c.v)^2 - 1.5 v.v)]  +-  3 w_i rho (c.v)
//   S_i       = guo w_i [9 (c.u)(c.F) - 3 u.F]            +-  3 w_i guo (c.F)
// and with rho (c.v) = varpi (c.j + c.F/2) the odd part of omega*M_i + S_i is
//   k_i varpi (c.j) + (k_i varpi / 2 + g_i) (c.F).
template <int Q, class C, bool SCALED = false, bool FX_ONLY = false>
__device__ __forceinline__ void collide(C* d, C varpi, const Phys<C>& ph, C s = C(1), C inv_s = C(1)) {
    // FX_ONLY: the caller guarantees F = (Fx, 0, 0); the terms with c.F = 0 drop out.
    // With SCALED the d are s * (f - w) on entry and exit; every term below
    // that adds into d carries the factor s (a power of two: exact).
    using L = Lat<Q>;
    C drho_s, jxs, jys, jzs;  // sums in the units of d
    moments<Q, C>(d, drho_s, jxs, jys, jzs);
    const C drho = SCALED ? drho_s * inv_s : drho_s;
    const C jx = SCALED ? jxs * inv_s : jxs, jy = SCALED ? jys * inv_s : jys, jz = SCALED ? jzs * inv_s : jzs;
    const C rho = C(1) + drho;
    const C inv_rho = C(1) / rho;
    C ux, uy, uz;
    velocity<C>(jx, jy, jz, inv_rho, ph, ux, uy, uz);
    if (FX_ONLY) {
        uy = jy * inv_rho;
        uz = jz * inv_rho;
    }
    const C vx = varpi * ux, vy = varpi * uy, vz = varpi * uz;
    const C rho_s = SCALED ? rho * s : rho;
    const C A = fma_(-rho_s, C(1.5) * (vx * vx + vy * vy + vz * vz), drho_s);
    const C uF3 = FX_ONLY ? C(3) * (ux * ph.Fx) : C(3) * (ux * ph.Fx + uy * ph.Fy + uz * ph.Fz);
    const C r45 = C(4.5) * rho_s;
    const C keep = C(1) - ph.omega;
    const C guo_s = SCALED ? ph.guo * s : ph.guo;
    {  // rest population
        const C w = C(L::w(0));
        d[0] = fma_(keep, d[0], fma_(ph.omega * w, A, -(guo_s * w) * uF3));
    }
    const C kv1 = ph.k1 * varpi, kv2 = ph.k2 * varpi;
    const C g1 = SCALED ? ph.g1 * s : ph.g1, g2 = SCALED ? ph.g2 * s : ph.g2;
    const C kvs1 = SCALED ? kv1 * s : kv1, kvs2 = SCALED ? kv2 * s : kv2;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int j = opp<Q>(i);
        if (j < i) continue;  // each pair once, from its lower index
        const int c2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
        const C cx = C(L::cx(i)), cy = C(L::cy(i)), cz = C(L::cz(i));
        const C w = C(L::w(i));
        const C cv = cx * vx + cy * vy + cz * vz;
        const C cu = cx * ux + cy * uy + cz * uz;
        // c.j in the units of d (scaled j when SCALED)
        const C cj = cx * jxs + cy * jys + cz * jzs;
        const C kv = c2 == 1 ? kv1 : kv2;
        const C kvs = c2 == 1 ? kvs1 : kvs2;
        const C g = c2 == 1 ? g1 : g2;
        C even, odd;
        if (FX_ONLY && L::cx(i) == 0) {  // c.F = 0
            even = fma_(ph.omega * w, fma_(r45, cv * cv, A), -(guo_s * w) * uF3);
            odd = kv * cj;
        } else {
            const C cF = FX_ONLY ? cx * ph.Fx : cx * ph.Fx + cy * ph.Fy + cz * ph.Fz;
            even = fma_(ph.omega * w, fma_(r45, cv * cv, A), (guo_s * w) * fma_(C(9) * cu, cF, -uF3));
            odd = fma_(kv, cj, fma_(kvs, C(0.5) * cF, g * cF));
        }
        d[i] = fma_(keep, d[i], even) + odd;
        d[j] = fma_(keep, d[j], even) - odd;
    }
}

// Explicit-drag form of the homogenization (Sec. 3.3, eq. momentumHLBM): the
// equilibrium stays at u and the drag -lam rho u, lam = nu/K = (1 - varpi)/tau,
// joins the body force, G = F - lam rho u, in Guo's scheme; u is the half-force
// velocity of the total force, u = (j + F/2) / (rho (1 + lam/2)). With
// h = 1/(1 + lam/2), rho (c.u) = h (c.j + c.F/2) and c.G = c.F - lam rho (c.u),
// so the odd part of omega*M_i + S_i is kk (c.j) + (kk/2 + g)(c.F) with
// kk = (k - g lam) h: the same fma shape as the shift form.
template <int Q, class C, bool SCALED = false>
__device__ __forceinline__ void collide_drag(C* d, C varpi, const Phys<C>& ph, C s = C(1), C inv_s = C(1)) {
    using L = Lat<Q>;
    C drho_s, jxs, jys, jzs;
    moments<Q, C>(d, drho_s, jxs, jys, jzs);
    const C drho = SCALED ? drho_s * inv_s : drho_s;
    const C jx = SCALED ? jxs * inv_s : jxs, jy = SCALED ? jys * inv_s : jys, jz = SCALED ? jzs * inv_s : jzs;
    const C rho = C(1) + drho;
    const C lam = (C(1) - varpi) * ph.omega;
    const C h = C(1) / fma_(C(0.5), lam, C(1));
    C ux, uy, uz;
    velocity<C>(jx, jy, jz, h / rho, ph, ux, uy, uz);
    const C lr = -lam * rho;
    const C Gx = fma_(lr, ux, ph.Fx), Gy = fma_(lr, uy, ph.Fy), Gz = fma_(lr, uz, ph.Fz);
    const C rho_s = SCALED ? rho * s : rho;
    const C A = fma_(-rho_s, C(1.5) * (ux * ux + uy * uy + uz * uz), drho_s);
    const C uG3 = C(3) * (ux * Gx + uy * Gy + uz * Gz);
    const C r45 = C(4.5) * rho_s;
    const C keep = C(1) - ph.omega;
    const C guo_s = SCALED ? ph.guo * s : ph.guo;
    {
        const C w = C(L::w(0));
        d[0] = fma_(keep, d[0], fma_(ph.omega * w, A, -(guo_s * w) * uG3));
    }
    const C kk1 = fma_(-ph.g1, lam, ph.k1) * h, kk2 = fma_(-ph.g2, lam, ph.k2) * h;
    const C g1 = SCALED ? ph.g1 * s : ph.g1, g2 = SCALED ? ph.g2 * s : ph.g2;
    const C kks1 = SCALED ? kk1 * s : kk1, kks2 = SCALED ? kk2 * s : kk2;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int j = opp<Q>(i);
        if (j < i) continue;
        const int c2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
        const C cx = C(L::cx(i)), cy = C(L::cy(i)), cz = C(L::cz(i));
        const C w = C(L::w(i));
        const C cu = cx * ux + cy * uy + cz * uz;
        const C cG = cx * Gx + cy * Gy + cz * Gz;
        const C cF = cx * ph.Fx + cy * ph.Fy + cz * ph.Fz;
        const C cj = cx * jxs + cy * jys + cz * jzs;
        const C kk = c2 == 1 ? kk1 : kk2;
        const C kks = c2 == 1 ? kks1 : kks2;
        const C g = c2 == 1 ? g1 : g2;
        const C even = fma_(ph.omega * w, fma_(r45, cu * cu, A), (guo_s * w) * fma_(C(9) * cu, cG, -uG3));
        const C odd = fma_(kk, cj, fma_(kks, C(0.5) * cF, g * cF));
        d[i] = fma_(keep, d[i], even) + odd;
        d[j] = fma_(keep, d[j], even) - odd;
    }
}

// Anisotropic (diagonal-tensor) porosity control: the Maxwellian at
// v = (vx ux, vy uy, vz uz), a per-axis drag nu/K_a. As collide(), with the
// odd part k (c.(varpi o j)) + (k/2 c.(varpi o F) + g c.F).
template <int Q, class C, bool SCALED = false>
__device__ __forceinline__ void collide_aniso(C* d, C wx, C wy, C wz, const Phys<C>& ph, C s = C(1), C inv_s = C(1)) {
    using L = Lat<Q>;
    C drho_s, jxs, jys, jzs;
    moments<Q, C>(d, drho_s, jxs, jys, jzs);
    const C drho = SCALED ? drho_s * inv_s : drho_s;
    const C jx = SCALED ? jxs * inv_s : jxs, jy = SCALED ? jys * inv_s : jys, jz = SCALED ? jzs * inv_s : jzs;
    const C rho = C(1) + drho;
    const C inv_rho = C(1) / rho;
    C ux, uy, uz;
    velocity<C>(jx, jy, jz, inv_rho, ph, ux, uy, uz);
    const C vx = wx * ux, vy = wy * uy, vz = wz * uz;
    const C rho_s = SCALED ? rho * s : rho;
    const C A = fma_(-rho_s, C(1.5) * (vx * vx + vy * vy + vz * vz), drho_s);
    const C uF3 = C(3) * (ux * ph.Fx + uy * ph.Fy + uz * ph.Fz);
    const C r45 = C(4.5) * rho_s;
    const C keep = C(1) - ph.omega;
    const C guo_s = SCALED ? ph.guo * s : ph.guo;
    {
        const C w = C(L::w(0));
        d[0] = fma_(keep, d[0], fma_(ph.omega * w, A, -(guo_s * w) * uF3));
    }
    const C pjx = wx * jxs, pjy = wy * jys, pjz = wz * jzs;             // varpi o j (units of d)
    const C hFx = C(0.5) * wx * ph.Fx, hFy = C(0.5) * wy * ph.Fy, hFz = C(0.5) * wz * ph.Fz;
    const C g1 = SCALED ? ph.g1 * s : ph.g1, g2 = SCALED ? ph.g2 * s : ph.g2;
    const C ks1 = SCALED ? ph.k1 * s : ph.k1, ks2 = SCALED ? ph.k2 * s : ph.k2;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int j = opp<Q>(i);
        if (j < i) continue;
        const int c2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
        const C cx = C(L::cx(i)), cy = C(L::cy(i)), cz = C(L::cz(i));
        const C w = C(L::w(i));
        const C cv = cx * vx + cy * vy + cz * vz;
        const C cu = cx * ux + cy * uy + cz * uz;
        const C cF = cx * ph.Fx + cy * ph.Fy + cz * ph.Fz;
        const C cpj = cx * pjx + cy * pjy + cz * pjz;
        const C cpF = cx * hFx + cy * hFy + cz * hFz;
        const C k = c2 == 1 ? ph.k1 : ph.k2;
        const C ks = c2 == 1 ? ks1 : ks2;
        const C g = c2 == 1 ? g1 : g2;
        const C even = fma_(ph.omega * w, fma_(r45, cv * cv, A), (guo_s * w) * fma_(C(9) * cu, cF, -uF3));
        const C odd = fma_(k, cpj, fma_(ks, cpF, g * cF));
        d[i] = fma_(keep, d[i], even) + odd;
        d[j] = fma_(keep, d[j], even) - odd;
    }
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
