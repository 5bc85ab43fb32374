// Discrete adjoint of the HBGK step, for the gradient of the outflow flux
// J = sum_{y,z} rho*u_x over a plane x = plane_x of the final state with
// respect to the per-cell porosity control varpi (eq. "d definition").
//
// Forward step: f^{n+1} = C(S f^n; varpi) with S the pull streaming and C the
// per-cell HBGK collision. Reverse step, with lam = dJ/df^{n+1}:
//   mu(x)    = (dC/dg)^T lam(x)   at g = (S f^n)(x)
//   grad(x) += (dC/dvarpi(x))^T lam(x)
//   dJ/df^n  = S^T mu,  (S^T mu)_k(y) = mu_k(y + c_k), or mu_opp(k)(y) when
//              y + c_k lies beyond a wall.
// (dC/dg)^T lam = (1 - 1/tau) lam + a_rho + c . a_j is the diagonal plus a
// rank-4 correction through the moments (rho, j); the kernel evaluates it
// per cell and pushes mu to its transposed-streaming destinations. Bytes per
// cell update: q loads of the forward state, q loads and q stores of the
// adjoint (FP32), varpi, and the gradient read-modify-write.
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

// I: index type (int while every index of the [q][cells] arrays fits). Four
// blocks of 256 per SM (64 registers, no spills): the kernel moves 240 B per
// cell and needs resident warps to keep that many loads in flight (five blocks
// would spill).
template <int Q, class S, bool WALLS, class I>
__global__ void __launch_bounds__(256, 4)
k_adjoint_step(const typename S::T* __restrict__ fn, const float* __restrict__ lam_in, float* __restrict__ lam_out,
               const float* __restrict__ varpi, float* __restrict__ grad, Geometry g, Phys<typename S::C> ph,
               typename S::C inv_s) {
    using C = typename S::C;
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const Nbr<I> nb(g, x, y, z);
    const I cell = (I)x + (I)g.nx * ((I)y + (I)g.ny * (I)z);
    const I N = (I)g.N;

    // forward quantities at g = S f^n
    C d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = S::load(fn, gather_index<Q, WALLS>(g, nb, cell, i, NATURAL), inv_s);
    C drho, jx, jy, jz;
    moments<Q, C>(d, drho, jx, jy, jz);
    const C rho = C(1) + drho;
    const C inv_rho = C(1) / rho;
    C ux, uy, uz;
    velocity<C>(jx, jy, jz, inv_rho, ph, ux, uy, uz);
    const C vp = C(__ldg(varpi + cell));
    const C vx = vp * ux, vy = vp * uy, vz = vp * uz;
    const C vv = vx * vx + vy * vy + vz * vz;

    // Every sum over directions below is linear in lw_i = lam_i w_i with a
    // polynomial of degree <= 2 in c_i, so it is a contraction of the moments
    //   S0 = sum lw_i,  S1 = sum lw_i c_i,  S2 = sum lw_i c_i c_i^T
    // with v = varpi u, F and u (P_i = 1 + 3 c.v + 4.5 (c.v)^2 - 1.5 v.v,
    // dP_i/dv = 3 c + 9 (c.v) c - 3 v):
    //   b_u    = sum lam_i d(M_i/tau + S_i)/du
    //          = rho varpi omega (3 S1 + 9 S2 v - 3 v S0) + guo (9 S2 F - 3 F S0)
    //   b_rho  = sum lam_i w_i P_i / tau = omega (S0 + 3 S1.v + 4.5 v.S2 v - 1.5 v.v S0)
    //   dvarpi = sum lam_i w_i rho (dP_i/dv . u) / tau = rho omega (3 S1.u + 9 v.S2 u - 3 v.u S0)
    // The moments take only adds of +-lw (c_i has components in {-1, 0, 1},
    // known at compile time per direction), so the per-cell cost stays close
    // to the loads and stores.
    C lam[Q];
    C S0 = 0, S1x = 0, S1y = 0, S1z = 0, Sxx = 0, Syy = 0, Szz = 0, Sxy = 0, Sxz = 0, Syz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        lam[i] = __ldg(lam_in + (I)i * N + cell);
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const C lw = lam[i] * C(L::w(i));
        S0 += lw;
        if (cx) {
            S1x += cx > 0 ? lw : -lw;
            Sxx += lw;
        }
        if (cy) {
            S1y += cy > 0 ? lw : -lw;
            Syy += lw;
        }
        if (cz) {
            S1z += cz > 0 ? lw : -lw;
            Szz += lw;
        }
        if (cx && cy) Sxy += cx * cy > 0 ? lw : -lw;
        if (cx && cz) Sxz += cx * cz > 0 ? lw : -lw;
        if (cy && cz) Syz += cy * cz > 0 ? lw : -lw;
    }
    const C omega = ph.omega;
    // S2 v, S2 F, S2 u
    const C S2vx = Sxx * vx + Sxy * vy + Sxz * vz, S2vy = Sxy * vx + Syy * vy + Syz * vz,
            S2vz = Sxz * vx + Syz * vy + Szz * vz;
    const C S2Fx = Sxx * ph.Fx + Sxy * ph.Fy + Sxz * ph.Fz, S2Fy = Sxy * ph.Fx + Syy * ph.Fy + Syz * ph.Fz,
            S2Fz = Sxz * ph.Fx + Syz * ph.Fy + Szz * ph.Fz;
    const C ra = rho * vp * omega;
    const C bux = ra * (C(3) * S1x + C(9) * S2vx - C(3) * vx * S0) + ph.guo * (C(9) * S2Fx - C(3) * ph.Fx * S0);
    const C buy = ra * (C(3) * S1y + C(9) * S2vy - C(3) * vy * S0) + ph.guo * (C(9) * S2Fy - C(3) * ph.Fy * S0);
    const C buz = ra * (C(3) * S1z + C(9) * S2vz - C(3) * vz * S0) + ph.guo * (C(9) * S2Fz - C(3) * ph.Fz * S0);
    const C S1v = S1x * vx + S1y * vy + S1z * vz;
    const C vS2v = vx * S2vx + vy * S2vy + vz * S2vz;
    const C brho = omega * (S0 + C(3) * S1v + C(4.5) * vS2v - C(1.5) * vv * S0);
    const C S1u = S1x * ux + S1y * uy + S1z * uz;
    const C vS2u = ux * S2vx + uy * S2vy + uz * S2vz;  // S2 is symmetric: u.S2 v = v.S2 u
    const C vu = vx * ux + vy * uy + vz * uz;
    const C dvp = rho * omega * (C(3) * S1u + C(9) * vS2u - C(3) * vu * S0);
    // u = (j + F/2)/rho: du/dj = I/rho, du/drho = -u/rho
    const C a_rho = brho - (bux * ux + buy * uy + buz * uz) * inv_rho;
    const C ajx = bux * inv_rho, ajy = buy * inv_rho, ajz = buz * inv_rho;
    grad[cell] += float(dvp);

    const C keep = C(1) - omega;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        C mu = fma_(keep, lam[k], a_rho);
        if (L::cx(k)) mu += L::cx(k) > 0 ? ajx : -ajx;
        if (L::cy(k)) mu += L::cy(k) > 0 ? ajy : -ajy;
        if (L::cz(k)) mu += L::cz(k) > 0 ? ajz : -ajz;
        // (S^T mu)_k(y) = mu_k(y + c_k): mu_k(x) goes to y = x - c_k, or, when x - c_k
        // lies beyond a wall, to slot opp(k) of x itself.
        const bool wall = WALLS && nb.template beyond_wall<Q>(k, -1);
        const I dst = wall ? (I)opp<Q>(k) * N + cell : (I)k * N + cell + nb.template offset<Q>(k, -1);
        lam_out[dst] = float(mu);
    }
}

// Seed dJ/df^N = S^T e, e_k(x) = c_kx on the plane x = plane_x (rho*u_x of the
// streamed populations is sum_k c_kx g_k + F_x/2).
template <int Q, bool WALLS>
__global__ void __launch_bounds__(256) k_flux_seed(float* lam, Geometry g, int plane_x) {
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const Nbr<long long> nb(g, x, y, z);
    const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        // (S^T e)_k(y) = e_k(y + c_k), or e_opp(k)(y) across a wall
        float v;
        if (WALLS && nb.template beyond_wall<Q>(k, +1)) {
            v = (x == plane_x) ? float(L::cx(opp<Q>(k))) : 0.0f;
        } else {
            const int dx = L::cx(k);
            const int xs = dx > 0 ? (x == g.nx - 1 ? 0 : x + 1) : (dx < 0 ? (x == 0 ? g.nx - 1 : x - 1) : x);
            v = (xs == plane_x) ? float(dx) : 0.0f;
        }
        lam[(size_t)k * g.N + cell] = v;
    }
}

// J = sum over the plane x = plane_x of rho*u_x = (j_x + F_x/2), FP64, one block,
// fixed order.
template <int Q, class S, bool WALLS>
__global__ void __launch_bounds__(256)
k_plane_flux(const typename S::T* f, int lay, Geometry g, Phys<typename S::C> ph, typename S::C inv_s,
             int plane_x, double* out) {
    using C = typename S::C;
    __shared__ double sh[256];
    double acc = 0.0;
    const int rows = g.ny * g.nz;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int y = r % g.ny, z = r / g.ny;
        const Nbr<long long> nb(g, plane_x, y, z);
        const long long cell = (long long)plane_x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
        C d[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = S::load(f, gather_index<Q, WALLS>(g, nb, cell, i, lay), inv_s);
        C drho, jx, jy, jz;
        moments<Q, C>(d, drho, jx, jy, jz);
        acc += (double)jx + 0.5 * (double)ph.Fx;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <int Q, class S, bool WALLS>
static cudaError_t adjoint_impl(const LaunchCtx& c, const void* fn, const float* lam_in, float* lam_out,
                                const float* varpi, float* grad) {
    using C = typename S::C;
    const Geometry g = geom(c);
    const Phys<C> ph = make_phys<C, Q>(c.tau, c.F);
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    const auto* f = static_cast<const typename S::T*>(fn);
    if ((size_t)Q * g.N < ((size_t)1 << 31))
        k_adjoint_step<Q, S, WALLS, int><<<grd, blk, 0, c.stream>>>(f, lam_in, lam_out, varpi, grad, g, ph,
                                                                    C(1.0 / c.scale));
    else
        k_adjoint_step<Q, S, WALLS, long long><<<grd, blk, 0, c.stream>>>(f, lam_in, lam_out, varpi, grad, g, ph,
                                                                          C(1.0 / c.scale));
    return cudaGetLastError();
}

template <int Q, class S, class Fn>
static cudaError_t with_walls(const LaunchCtx& c, Fn&& fn) {
    const bool walls = c.wall[0] || c.wall[1] || c.wall[2];
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

cudaError_t launch_adjoint_step(const LaunchCtx& c, const void* fn, const float* lam_in, float* lam_out,
                                const float* varpi, float* grad) {
    return dispatch(c, [&]<int Q, class S, bool W>() { return adjoint_impl<Q, S, W>(c, fn, lam_in, lam_out, varpi, grad); });
}

cudaError_t launch_flux_seed(const LaunchCtx& c, float* lam, int plane_x) {
    const Geometry g = geom(c);
    const dim3 blk = block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    const bool walls = c.wall[0] || c.wall[1] || c.wall[2];
    if (c.q == 9) {
        if (walls) k_flux_seed<9, true><<<grd, blk, 0, c.stream>>>(lam, g, plane_x);
        else k_flux_seed<9, false><<<grd, blk, 0, c.stream>>>(lam, g, plane_x);
    } else {
        if (walls) k_flux_seed<19, true><<<grd, blk, 0, c.stream>>>(lam, g, plane_x);
        else k_flux_seed<19, false><<<grd, blk, 0, c.stream>>>(lam, g, plane_x);
    }
    return cudaGetLastError();
}

cudaError_t launch_plane_flux(const LaunchCtx& c, int layout, const void* f, int plane_x, double* out) {
    return dispatch(c, [&]<int Q, class S, bool W>() {
        using C = typename S::C;
        const Phys<C> ph = make_phys<C, Q>(c.tau, c.F);
        k_plane_flux<Q, S, W><<<1, 256, 0, c.stream>>>(static_cast<const typename S::T*>(f), layout, geom(c), ph,
                                                       C(1.0 / c.scale), plane_x, out);
        return cudaGetLastError();
    });
}

}  // namespace hlbm
