/*
 * FP64 CPU oracle for the homogenized lattice BGK (HBGK) time step.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference the CUDA
 * path is checked against. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product never does. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes (Simonis et al., arXiv:2310.14746, Part I):
 *   - the homogenized Maxwellian M_eq = f_eq(n, varpi*u, T), i.e. the BGK
 *     equilibrium evaluated at the porosity-scaled velocity varpi*u
 *     (Sec. 3.2, eq. porousVeloMaxwellian, with varpi = 1 - nu*tau/K from
 *     eq. "d definition");
 *   - the BGK relaxation Q(f) = -(f - M_eq)/tau (Sec. 3.1, eq.
 *     collisionOperatorQ) of the HBGKBE (Sec. 3.2, eq. HBGKBE);
 *   - moments rho = sum f, rho*u = sum c f (Sec. 3.1, Def. moments).
 * Part I stops at the continuous kinetic model; its lattice discretization is
 * deferred to Part II. The discrete pieces here are the textbook ones and are
 * readings, not quotations: DdQq velocity sets with c_s^2 = 1/3 (the
 * covariance 1/(3 eps^2) of Sec. 3.3 in lattice units), the second-order
 * Hermite truncation of the Maxwellian, Guo's forcing for the F.grad_v f term
 * of eq. BGKBE, pull streaming with periodic wrap, and half-way bounce-back
 * for the no-slip condition u = 0 on the boundary of eq. targetEBTL.
 *
 * Conventions (the same ones the public header documents):
 *   populations f[q][z][y][x], x fastest; cell index = x + nx*(y + ny*z);
 *   the stored state is the post-collision population; a step pulls
 *   g_i(x) = f_i(x - c_i) (or f_opp(i)(x) across a wall) and collides g.
 *   Velocity ordering, D2Q9:  0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1)
 *                             5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 *   D3Q19: 0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0) 5 (0,0,1)
 *          6 (0,0,-1) 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
 *          11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1)
 *          16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *
 * Everything is plain loops in double precision. OpenMP (if enabled) only
 * splits the cell loop of a step; each cell's arithmetic is identical
 * whatever the thread count, and every reduction runs serially in cell order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 19

typedef struct {
    int q;
    int c[OR_MAXQ][3];
    double w[OR_MAXQ];
    int opp[OR_MAXQ];
} or_velset;

/* Standard D2Q9 and D3Q19 sets (lattice weights 4/9,1/9,1/36 and
 * 1/3,1/18,1/36), in the ordering stated above. */
static int or_get_velset(int q, or_velset* vs)
{
    static const int c9[9][3] = {
        {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
        {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    static const int c19[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    int i, j, d;
    if (q != 9 && q != 19) return -1;
    vs->q = q;
    for (i = 0; i < q; ++i) {
        int s2 = 0;
        for (d = 0; d < 3; ++d) {
            vs->c[i][d] = (q == 9) ? c9[i][d] : c19[i][d];
            s2 += vs->c[i][d] * vs->c[i][d];
        }
        if (q == 9)
            vs->w[i] = (s2 == 0) ? 4.0 / 9.0 : (s2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else
            vs->w[i] = (s2 == 0) ? 1.0 / 3.0 : (s2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    /* opposite direction: the one with c_j = -c_i (searched, not tabulated) */
    for (i = 0; i < q; ++i) {
        vs->opp[i] = -1;
        for (j = 0; j < q; ++j)
            if (vs->c[j][0] == -vs->c[i][0] && vs->c[j][1] == -vs->c[i][1] &&
                vs->c[j][2] == -vs->c[i][2])
                vs->opp[i] = j;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-cell pieces                                                            */
/* ------------------------------------------------------------------------ */

/* Homogenized Maxwellian on the lattice: the second-order expansion of
 * f_eq(n, v, T) with covariance c_s^2 = 1/3, evaluated at v = varpi*u
 * (Sec. 3.2, eq. porousVeloMaxwellian). Its zeroth moment is rho and its
 * first moment rho*v (eqs. hbgk statistic equilibrium 1-2). */
static void or_equilibrium(const or_velset* vs, double rho, const double v[3], double* feq)
{
    int i;
    double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    for (i = 0; i < vs->q; ++i) {
        double cv = vs->c[i][0] * v[0] + vs->c[i][1] * v[1] + vs->c[i][2] * v[2];
        feq[i] = vs->w[i] * rho * (1.0 + 3.0 * cv + 4.5 * cv * cv - 1.5 * vv);
    }
}

/* Zeroth and first moments (Def. moments) of the streamed populations g,
 * with Guo's half-force shift: u = (sum c g + F/2) / rho. */
static void or_moments_cell(const or_velset* vs, const double* g, const double F[3],
                            double* rho_out, double u[3])
{
    int i, d;
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (i = 0; i < vs->q; ++i) {
        rho += g[i];
        for (d = 0; d < 3; ++d) j[d] += vs->c[i][d] * g[i];
    }
    for (d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * F[d]) / rho;
    *rho_out = rho;
}

/* One HBGK collision of a cell's streamed populations g (Sec. 3.2):
 *   out_i = g_i - (g_i - M_eq_i)/tau + S_i,
 * M_eq at (rho, varpi*u), and Guo's source built with u:
 *   S_i = (1 - 1/(2 tau)) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)]. */
static void or_collide_cell(const or_velset* vs, const double* g, double varpi, double tau,
                            const double F[3], double* out)
{
    int i;
    double rho, u[3], v[3], feq[OR_MAXQ];
    or_moments_cell(vs, g, F, &rho, u);
    v[0] = varpi * u[0];
    v[1] = varpi * u[1];
    v[2] = varpi * u[2];
    or_equilibrium(vs, rho, v, feq);
    for (i = 0; i < vs->q; ++i) {
        const int* c = vs->c[i];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        double cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2];
        double cmuF = (c[0] - u[0]) * F[0] + (c[1] - u[1]) * F[1] + (c[2] - u[2]) * F[2];
        double S = (1.0 - 0.5 / tau) * vs->w[i] * (3.0 * cmuF + 9.0 * cu * cF);
        out[i] = g[i] - (g[i] - feq[i]) / tau + S;
    }
}

/* The explicit-drag form of the homogenization (Sec. 3.3, eq. momentumHLBM:
 * the equilibrium shift acts as the drag -nu K^{-1} rho u, and with
 * varpi = 1 - nu tau/K, nu/K = (1 - varpi)/tau =: lam). The equilibrium stays
 * at the velocity u and the drag joins the body force, G = F - lam rho u, in
 * Guo's scheme; u is the half-force velocity of the total force, which is
 * implicit in u: rho u = j + G/2 = j + F/2 - lam rho u / 2, so
 * u = (j + F/2) / (rho (1 + lam/2)). */
static void or_collide_cell_drag(const or_velset* vs, const double* g, double varpi, double tau,
                                 const double F[3], double* out)
{
    int i, d;
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3], G[3], feq[OR_MAXQ];
    const double lam = (1.0 - varpi) / tau;
    for (i = 0; i < vs->q; ++i) {
        rho += g[i];
        for (d = 0; d < 3; ++d) j[d] += vs->c[i][d] * g[i];
    }
    for (d = 0; d < 3; ++d) {
        u[d] = (j[d] + 0.5 * F[d]) / (rho * (1.0 + 0.5 * lam));
        G[d] = F[d] - lam * rho * u[d];
    }
    or_equilibrium(vs, rho, u, feq);
    for (i = 0; i < vs->q; ++i) {
        const int* c = vs->c[i];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        double cG = c[0] * G[0] + c[1] * G[1] + c[2] * G[2];
        double cmuG = (c[0] - u[0]) * G[0] + (c[1] - u[1]) * G[1] + (c[2] - u[2]) * G[2];
        double S = (1.0 - 0.5 / tau) * vs->w[i] * (3.0 * cmuG + 9.0 * cu * cG);
        out[i] = g[i] - (g[i] - feq[i]) / tau + S;
    }
}

/* Anisotropic (diagonal-tensor) porosity control, beyond the isotropy assumption
 * of Sec. 2.5 (Assumption thmAssump, item 3) and listed as future work in the
 * outlook: the Maxwellian is evaluated at v = (varpi_x u_x, varpi_y u_y,
 * varpi_z u_z), i.e. a drag -nu K_a^{-1} rho u_a per axis with
 * varpi_a = 1 - nu tau / K_a. Otherwise as or_collide_cell. */
static void or_collide_cell_aniso(const or_velset* vs, const double* g, const double varpi[3], double tau,
                                  const double F[3], double* out)
{
    int i;
    double rho, u[3], v[3], feq[OR_MAXQ];
    or_moments_cell(vs, g, F, &rho, u);
    v[0] = varpi[0] * u[0];
    v[1] = varpi[1] * u[1];
    v[2] = varpi[2] * u[2];
    or_equilibrium(vs, rho, v, feq);
    for (i = 0; i < vs->q; ++i) {
        const int* c = vs->c[i];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        double cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2];
        double cmuF = (c[0] - u[0]) * F[0] + (c[1] - u[1]) * F[1] + (c[2] - u[2]) * F[2];
        double S = (1.0 - 0.5 / tau) * vs->w[i] * (3.0 * cmuF + 9.0 * cu * cF);
        out[i] = g[i] - (g[i] - feq[i]) / tau + S;
    }
}

/* Velocity of the streamed populations g as the collision of `mode` sees it
 * (0: equilibrium shift, half-force velocity of F; 1: explicit drag, half-force
 * velocity of F + drag). */
static void or_velocity_mode(const or_velset* vs, const double* g, double varpi, double tau,
                             const double F[3], int mode, double* rho_out, double u[3])
{
    int d;
    or_moments_cell(vs, g, F, rho_out, u);
    if (mode == 1) {
        const double lam = (1.0 - varpi) / tau;
        for (d = 0; d < 3; ++d) u[d] /= (1.0 + 0.5 * lam);
    }
}

/* ------------------------------------------------------------------------ */
/* Streaming                                                                  */
/* ------------------------------------------------------------------------ */

/* Source of the population arriving at (x,y,z) in direction i: the cell
 * (x,y,z) - c_i with periodic wrap, or, when that cell lies beyond a wall
 * (bc[axis] = 1), the same cell's opposite population (half-way bounce-back).
 * Returns the flat index into f[q][cells]. */
static int64_t or_pull_source(const or_velset* vs, const int n[3], const int bc[3], int i,
                              int x, int y, int z)
{
    int p[3] = {x, y, z}, s[3], d, wall = 0;
    int64_t cells = (int64_t)n[0] * n[1] * n[2];
    for (d = 0; d < 3; ++d) {
        s[d] = p[d] - vs->c[i][d];
        if (s[d] < 0 || s[d] >= n[d]) {
            if (bc[d]) wall = 1;
            else s[d] = (s[d] + n[d]) % n[d];
        }
    }
    if (wall)
        return (int64_t)vs->opp[i] * cells + x + (int64_t)n[0] * (y + (int64_t)n[1] * z);
    return (int64_t)i * cells + s[0] + (int64_t)n[0] * (s[1] + (int64_t)n[1] * s[2]);
}

static void or_gather(const or_velset* vs, const int n[3], const int bc[3], const double* f,
                      int x, int y, int z, double* g)
{
    int i;
    for (i = 0; i < vs->q; ++i) g[i] = f[or_pull_source(vs, n, bc, i, x, y, z)];
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                      */
/* ------------------------------------------------------------------------ */

/* Thread control for the step loop (no effect without OpenMP). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_velset(int q, int* c_out /* q x 3 */, double* w_out, int* opp_out)
{
    or_velset vs;
    int i, d;
    if (or_get_velset(q, &vs)) return -1;
    for (i = 0; i < q; ++i) {
        for (d = 0; d < 3; ++d) c_out[3 * i + d] = vs.c[i][d];
        w_out[i] = vs.w[i];
        opp_out[i] = vs.opp[i];
    }
    return 0;
}

/* Equilibrium populations at density rho and velocity v (already scaled). */
int oracle_equilibrium(int q, double rho, const double* v, double* feq)
{
    or_velset vs;
    if (or_get_velset(q, &vs)) return -1;
    or_equilibrium(&vs, rho, v, feq);
    return 0;
}

/* Collision of one cell's streamed populations. */
int oracle_collide(int q, const double* g, double varpi, double tau, const double* F,
                   double* out)
{
    or_velset vs;
    if (or_get_velset(q, &vs)) return -1;
    or_collide_cell(&vs, g, varpi, tau, F, out);
    return 0;
}

/* Pull streaming only: g = S f. */
int oracle_stream(int q, int nx, int ny, int nz, const int* bc, const double* f, double* g)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, x, y, z, i;
    int64_t cells = (int64_t)nx * ny * nz;
    if (or_get_velset(q, &vs)) return -1;
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x)
                for (i = 0; i < q; ++i)
                    g[(int64_t)i * cells + x + (int64_t)nx * (y + (int64_t)ny * z)] =
                        f[or_pull_source(&vs, n, bc, i, x, y, z)];
    return 0;
}

/* One cell's collision in the chosen homogenization form (0: shift, 1: drag). */
int oracle_collide_mode(int q, const double* g, double varpi, double tau, const double* F, int mode,
                        double* out)
{
    or_velset vs;
    if (or_get_velset(q, &vs) || mode < 0 || mode > 1) return -1;
    if (mode == 1) or_collide_cell_drag(&vs, g, varpi, tau, F, out);
    else or_collide_cell(&vs, g, varpi, tau, F, out);
    return 0;
}

/* As oracle_run with the homogenization form `mode` (0: shift, 1: drag). */
int oracle_run_mode(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
                    const double* varpi, double* f, double* tmp, long nsteps, int mode)
{
    or_velset vs;
    int n[3] = {nx, ny, nz};
    int64_t cells = (int64_t)nx * ny * nz;
    long s;
    double *src = f, *dst = tmp;
    if (or_get_velset(q, &vs) || mode < 0 || mode > 1) return -1;
    if (!(tau > 0.5)) return -1;
    for (s = 0; s < nsteps; ++s) {
        int z;
#pragma omp parallel for schedule(static)
        for (z = 0; z < nz; ++z) {
            int x, y, i;
            double g[OR_MAXQ], out[OR_MAXQ];
            for (y = 0; y < ny; ++y)
                for (x = 0; x < nx; ++x) {
                    int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                    or_gather(&vs, n, bc, src, x, y, z, g);
                    if (mode == 1) or_collide_cell_drag(&vs, g, varpi[cell], tau, F, out);
                    else or_collide_cell(&vs, g, varpi[cell], tau, F, out);
                    for (i = 0; i < q; ++i) dst[(int64_t)i * cells + cell] = out[i];
                }
        }
        {
            double* t = src;
            src = dst;
            dst = t;
        }
    }
    if (src != f) memcpy(f, src, sizeof(double) * (size_t)(cells * q));
    return 0;
}

/* nsteps of the anisotropic form; varpi3 is [3][cells] (x, y, z components). */
int oracle_run_aniso(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
                     const double* varpi3, double* f, double* tmp, long nsteps)
{
    or_velset vs;
    int n[3] = {nx, ny, nz};
    int64_t cells = (int64_t)nx * ny * nz;
    long s;
    double *src = f, *dst = tmp;
    if (or_get_velset(q, &vs) || !(tau > 0.5)) return -1;
    for (s = 0; s < nsteps; ++s) {
        int z;
#pragma omp parallel for schedule(static)
        for (z = 0; z < nz; ++z) {
            int x, y, i;
            double g[OR_MAXQ], out[OR_MAXQ], vp[3];
            for (y = 0; y < ny; ++y)
                for (x = 0; x < nx; ++x) {
                    int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                    vp[0] = varpi3[cell];
                    vp[1] = varpi3[cells + cell];
                    vp[2] = varpi3[2 * cells + cell];
                    or_gather(&vs, n, bc, src, x, y, z, g);
                    or_collide_cell_aniso(&vs, g, vp, tau, F, out);
                    for (i = 0; i < q; ++i) dst[(int64_t)i * cells + cell] = out[i];
                }
        }
        {
            double* t = src;
            src = dst;
            dst = t;
        }
    }
    if (src != f) memcpy(f, src, sizeof(double) * (size_t)(cells * q));
    return 0;
}

/* Resolved obstacles: solid[cell] != 0 marks a solid cell. A fluid cell whose
 * pull source is solid takes the bounce-back population of its own opposite
 * direction (half-way bounce-back on the solid surface, no slip); solid cells
 * are not updated (their populations are left as they are and never read).
 * Used with varpi = 1 in the fluid for the resolved pore-scale problem whose
 * permeability the homogenized field approximates (Thm. thmStatNSECase4,
 * unit-cell problem for A). */
int oracle_run_masked(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
                      const double* varpi, const unsigned char* solid, double* f, double* tmp, long nsteps)
{
    or_velset vs;
    int n[3] = {nx, ny, nz};
    int64_t cells = (int64_t)nx * ny * nz;
    long s;
    double *src = f, *dst = tmp;
    if (or_get_velset(q, &vs) || !(tau > 0.5)) return -1;
    for (s = 0; s < nsteps; ++s) {
        int z;
#pragma omp parallel for schedule(static)
        for (z = 0; z < nz; ++z) {
            int x, y, i, d;
            double g[OR_MAXQ], out[OR_MAXQ];
            for (y = 0; y < ny; ++y)
                for (x = 0; x < nx; ++x) {
                    int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                    if (solid[cell]) {
                        for (i = 0; i < q; ++i) dst[(int64_t)i * cells + cell] = src[(int64_t)i * cells + cell];
                        continue;
                    }
                    for (i = 0; i < q; ++i) {
                        int p[3] = {x, y, z}, sp[3], wall = 0;
                        for (d = 0; d < 3; ++d) {
                            sp[d] = p[d] - vs.c[i][d];
                            if (sp[d] < 0 || sp[d] >= n[d]) {
                                if (bc[d]) wall = 1;
                                else sp[d] = (sp[d] + n[d]) % n[d];
                            }
                        }
                        if (!wall && solid[sp[0] + (int64_t)nx * (sp[1] + (int64_t)ny * sp[2])]) wall = 1;
                        g[i] = wall ? src[(int64_t)vs.opp[i] * cells + cell]
                                    : src[(int64_t)i * cells + sp[0] + (int64_t)nx * (sp[1] + (int64_t)ny * sp[2])];
                    }
                    or_collide_cell(&vs, g, varpi[cell], tau, F, out);
                    for (i = 0; i < q; ++i) dst[(int64_t)i * cells + cell] = out[i];
                }
        }
        {
            double* t = src;
            src = dst;
            dst = t;
        }
    }
    if (src != f) memcpy(f, src, sizeof(double) * (size_t)(cells * q));
    return 0;
}

/* Moments with resolved obstacles: solid cells report rho = 1, u = 0; fluid
 * cells the moments of their streamed populations (bounce-back at solid
 * sources). */
int oracle_moments_masked(int q, int nx, int ny, int nz, const int* bc, const double* F,
                          const unsigned char* solid, const double* f, double* rho, double* u)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, x, y, z, i, d;
    int64_t cells = (int64_t)nx * ny * nz;
    if (or_get_velset(q, &vs)) return -1;
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x) {
                double g[OR_MAXQ], r, uu[3];
                int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                if (solid[cell]) {
                    rho[cell] = 1.0;
                    u[cell] = u[cells + cell] = u[2 * cells + cell] = 0.0;
                    continue;
                }
                for (i = 0; i < q; ++i) {
                    int p[3] = {x, y, z}, sp[3], wall = 0;
                    for (d = 0; d < 3; ++d) {
                        sp[d] = p[d] - vs.c[i][d];
                        if (sp[d] < 0 || sp[d] >= n[d]) {
                            if (bc[d]) wall = 1;
                            else sp[d] = (sp[d] + n[d]) % n[d];
                        }
                    }
                    if (!wall && solid[sp[0] + (int64_t)nx * (sp[1] + (int64_t)ny * sp[2])]) wall = 1;
                    g[i] = wall ? f[(int64_t)vs.opp[i] * cells + cell]
                                : f[(int64_t)i * cells + sp[0] + (int64_t)nx * (sp[1] + (int64_t)ny * sp[2])];
                }
                or_moments_cell(&vs, g, F, &r, uu);
                rho[cell] = r;
                u[cell] = uu[0];
                u[cells + cell] = uu[1];
                u[2 * cells + cell] = uu[2];
            }
    return 0;
}

/* One cell's anisotropic collision (varpi3 = 3 values). */
int oracle_collide_aniso(int q, const double* g, const double* varpi3, double tau, const double* F, double* out)
{
    or_velset vs;
    if (or_get_velset(q, &vs)) return -1;
    or_collide_cell_aniso(&vs, g, varpi3, tau, F, out);
    return 0;
}

/* Density and velocity of a state as the collision of `mode` sees them. */
int oracle_moments_mode(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
                        const double* varpi, const double* f, int mode, double* rho, double* u)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, x, y, z;
    int64_t cells = (int64_t)nx * ny * nz;
    if (or_get_velset(q, &vs) || mode < 0 || mode > 1) return -1;
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x) {
                double g[OR_MAXQ], r, uu[3];
                int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                or_gather(&vs, n, bc, f, x, y, z, g);
                or_velocity_mode(&vs, g, varpi[cell], tau, F, mode, &r, uu);
                rho[cell] = r;
                u[cell] = uu[0];
                u[cells + cell] = uu[1];
                u[2 * cells + cell] = uu[2];
            }
    return 0;
}

/* nsteps full time steps: stream (pull) then collide, ping-ponging between
 * f (in/out) and the caller's scratch buffer tmp (same size). On return f
 * holds the post-collision state after nsteps. */
int oracle_run(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
               const double* varpi, double* f, double* tmp, long nsteps)
{
    or_velset vs;
    int n[3] = {nx, ny, nz};
    int64_t cells = (int64_t)nx * ny * nz;
    long s;
    double *src = f, *dst = tmp;
    if (or_get_velset(q, &vs)) return -1;
    if (!(tau > 0.5)) return -1;
    for (s = 0; s < nsteps; ++s) {
        int z;
#pragma omp parallel for schedule(static)
        for (z = 0; z < nz; ++z) {
            int x, y, i;
            double g[OR_MAXQ], out[OR_MAXQ];
            for (y = 0; y < ny; ++y)
                for (x = 0; x < nx; ++x) {
                    int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                    or_gather(&vs, n, bc, src, x, y, z, g);
                    or_collide_cell(&vs, g, varpi[cell], tau, F, out);
                    for (i = 0; i < q; ++i) dst[(int64_t)i * cells + cell] = out[i];
                }
        }
        {
            double* t = src;
            src = dst;
            dst = t;
        }
    }
    if (src != f) memcpy(f, src, sizeof(double) * (size_t)(cells * q));
    return 0;
}

/* Macroscopic fields of a state: density and (half-force) velocity of the
 * streamed populations, i.e. what the next collision sees. u is [3][cells]. */
int oracle_moments(int q, int nx, int ny, int nz, const int* bc, const double* F,
                   const double* f, double* rho, double* u)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, x, y, z;
    int64_t cells = (int64_t)nx * ny * nz;
    if (or_get_velset(q, &vs)) return -1;
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x) {
                double g[OR_MAXQ], r, uu[3];
                int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                or_gather(&vs, n, bc, f, x, y, z, g);
                or_moments_cell(&vs, g, F, &r, uu);
                rho[cell] = r;
                u[cell] = uu[0];
                u[cells + cell] = uu[1];
                u[2 * cells + cell] = uu[2];
            }
    return 0;
}

/* Global FP64 diagnostics of a state, summed serially in cell order.
 * out[0] = sum rho, out[1..3] = sum rho*u, out[4] = plane flux
 * sum_{y,z} rho*u_x at x = nx-1, out[5] = apparent permeability
 * nu * mean(rho*u_x) / F_x with nu = (tau - 1/2)/3 (Darcy's law, Thm.
 * thmStatNSECase4: u = A (F - grad p)/nu, mean over all cells),
 * out[6] = max |u - u_prev| over cells and components (0 if u_prev is NULL),
 * out[7] = max |u|. */
int oracle_stats(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
                 const double* f, const double* u_prev, double* out)
{
    int64_t cells = (int64_t)nx * ny * nz, c;
    double *rho = (double*)malloc(sizeof(double) * (size_t)cells);
    double *u = (double*)malloc(sizeof(double) * (size_t)(3 * cells));
    int k, rc;
    if (!rho || !u) {
        free(rho);
        free(u);
        return -2;
    }
    rc = oracle_moments(q, nx, ny, nz, bc, F, f, rho, u);
    if (rc) {
        free(rho);
        free(u);
        return rc;
    }
    for (k = 0; k < 8; ++k) out[k] = 0.0;
    for (c = 0; c < cells; ++c) {
        int64_t x = c % nx;
        out[0] += rho[c];
        for (k = 0; k < 3; ++k) out[1 + k] += rho[c] * u[k * cells + c];
        if (x == nx - 1) out[4] += rho[c] * u[c];
        for (k = 0; k < 3; ++k) {
            double a = fabs(u[k * cells + c]);
            if (a > out[7]) out[7] = a;
            if (u_prev) {
                double d = fabs(u[k * cells + c] - u_prev[k * cells + c]);
                if (d > out[6]) out[6] = d;
            }
        }
    }
    out[5] = (F[0] != 0.0) ? ((tau - 0.5) / 3.0) * (out[1] / (double)cells) / F[0] : 0.0;
    free(rho);
    free(u);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint (reverse mode) of the step, for the gradient of the       */
/* outflow flux J = sum_{y,z} rho*u_x at x = nx-1 of the final state with     */
/* respect to the per-cell porosity control varpi.                            */
/*                                                                            */
/* Forward: f^{n+1} = C(S f^n; varpi), S the pull streaming, C the per-cell   */
/* collision. Reverse: with lam = dJ/df^{n+1},                                */
/*   mu(x)   = (dC/dg)^T lam(x)     (per cell, at g = S f^n)                  */
/*   grad(x) += (dC/dvarpi)^T lam(x)                                          */
/*   dJ/df^n = S^T mu                                                         */
/* The Jacobian products are written out from the collision formula by the   */
/* chain rule through the moments (rho, j) and u = (j + F/2)/rho.             */
/* ------------------------------------------------------------------------ */

/* Vector-Jacobian product of one cell's collision. lam: adjoint of the
 * collision output; g: the streamed input. mu = (dC/dg)^T lam;
 * returns (dC/dvarpi)^T lam. */
static double or_collide_vjp(const or_velset* vs, const double* g, double varpi, double tau,
                             const double F[3], const double* lam, double* mu)
{
    int i, d;
    double rho, u[3], v[3], vv;
    double b_rho = 0.0, b_u[3] = {0.0, 0.0, 0.0}, dvarpi = 0.0, a_rho, a_j[3], bu_dot_u;
    const double beta = 1.0 - 0.5 / tau;
    or_moments_cell(vs, g, F, &rho, u);
    for (d = 0; d < 3; ++d) v[d] = varpi * u[d];
    vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    for (i = 0; i < vs->q; ++i) {
        const int* c = vs->c[i];
        double cv = c[0] * v[0] + c[1] * v[1] + c[2] * v[2];
        double cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2];
        double P = 1.0 + 3.0 * cv + 4.5 * cv * cv - 1.5 * vv;
        double dP_dv[3], dfeq_du[3], dS_du[3];
        for (d = 0; d < 3; ++d) {
            dP_dv[d] = 3.0 * c[d] + 9.0 * cv * c[d] - 3.0 * v[d];
            /* M_eq_i = w_i rho P(varpi u): d/du = w_i rho varpi dP/dv */
            dfeq_du[d] = vs->w[i] * rho * varpi * dP_dv[d];
            /* S_i = beta w_i [3 (c - u).F + 9 (c.u)(c.F)]: d/du */
            dS_du[d] = beta * vs->w[i] * (-3.0 * F[d] + 9.0 * cF * c[d]);
            b_u[d] += lam[i] * (dfeq_du[d] / tau + dS_du[d]);
        }
        b_rho += lam[i] * vs->w[i] * P / tau; /* d(M_eq/tau)/drho at fixed u */
        /* d(M_eq_i/tau)/dvarpi = w_i rho (dP/dv . u) / tau */
        dvarpi += lam[i] * vs->w[i] * rho *
                  (dP_dv[0] * u[0] + dP_dv[1] * u[1] + dP_dv[2] * u[2]) / tau;
    }
    /* u = (j + F/2)/rho: du/dj = I/rho, du/drho = -u/rho */
    bu_dot_u = b_u[0] * u[0] + b_u[1] * u[1] + b_u[2] * u[2];
    a_rho = b_rho - bu_dot_u / rho;
    for (d = 0; d < 3; ++d) a_j[d] = b_u[d] / rho;
    /* rho = sum g, j = sum c g; plus the (1 - 1/tau) g_i diagonal */
    for (i = 0; i < vs->q; ++i) {
        const int* c = vs->c[i];
        mu[i] = (1.0 - 1.0 / tau) * lam[i] + a_rho + c[0] * a_j[0] + c[1] * a_j[1] +
                c[2] * a_j[2];
    }
    return dvarpi;
}

/* Transposed pull streaming: (S^T mu)_i(x) = mu_i(x + c_i) with periodic
 * wrap, or mu_opp(i)(x) when x + c_i lies beyond a wall. */
static void or_stream_transpose(const or_velset* vs, const int n[3], const int bc[3],
                                const double* mu, double* out)
{
    int64_t cells = (int64_t)n[0] * n[1] * n[2];
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < n[2]; ++z) {
        int x, y, i, d;
        for (y = 0; y < n[1]; ++y)
            for (x = 0; x < n[0]; ++x)
                for (i = 0; i < vs->q; ++i) {
                    int p[3] = {x, y, z}, s[3], wall = 0;
                    int64_t cell = x + (int64_t)n[0] * (y + (int64_t)n[1] * z);
                    for (d = 0; d < 3; ++d) {
                        s[d] = p[d] + vs->c[i][d];
                        if (s[d] < 0 || s[d] >= n[d]) {
                            if (bc[d]) wall = 1;
                            else s[d] = (s[d] + n[d]) % n[d];
                        }
                    }
                    if (wall)
                        out[(int64_t)i * cells + cell] = mu[(int64_t)vs->opp[i] * cells + cell];
                    else
                        out[(int64_t)i * cells + cell] =
                            mu[(int64_t)i * cells + s[0] + (int64_t)n[0] * (s[1] + (int64_t)n[1] * s[2])];
                }
    }
}

/* One reverse step: given the forward state f^n (post-collision, before the
 * step) and lam_in = dJ/df^{n+1}, write lam_out = dJ/df^n and add
 * (dC/dvarpi)^T lam_in into grad. */
int oracle_adjoint_step(int q, int nx, int ny, int nz, const int* bc, double tau,
                        const double* F, const double* varpi, const double* f_n,
                        const double* lam_in, double* lam_out, double* grad)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, x, y, z, i;
    int64_t cells = (int64_t)nx * ny * nz;
    double* mu;
    if (or_get_velset(q, &vs)) return -1;
    mu = (double*)malloc(sizeof(double) * (size_t)(q * cells));
    if (!mu) return -2;
#pragma omp parallel for private(x, y, i) schedule(static)
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (x = 0; x < nx; ++x) {
                double g[OR_MAXQ], lam[OR_MAXQ], m[OR_MAXQ];
                int64_t cell = x + (int64_t)nx * (y + (int64_t)ny * z);
                or_gather(&vs, n, bc, f_n, x, y, z, g);
                for (i = 0; i < q; ++i) lam[i] = lam_in[(int64_t)i * cells + cell];
                grad[cell] += or_collide_vjp(&vs, g, varpi[cell], tau, F, lam, m);
                for (i = 0; i < q; ++i) mu[(int64_t)i * cells + cell] = m[i];
            }
    or_stream_transpose(&vs, n, bc, mu, lam_out);
    free(mu);
    return 0;
}

/* Seed of the reverse sweep: dJ/df^N for J = sum_{y,z} rho*u_x at x = nx-1
 * of the streamed final state. rho*u_x = sum_i c_ix g_i + F_x/2, so
 * dJ/dg_i(x) = c_ix on the plane, and dJ/df^N = S^T of that. */
int oracle_flux_seed(int q, int nx, int ny, int nz, const int* bc, double* lam)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, x, y, z, i;
    int64_t cells = (int64_t)nx * ny * nz;
    double* e;
    if (or_get_velset(q, &vs)) return -1;
    e = (double*)calloc((size_t)(q * cells), sizeof(double));
    if (!e) return -2;
    x = nx - 1;
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y)
            for (i = 0; i < q; ++i)
                e[(int64_t)i * cells + x + (int64_t)nx * (y + (int64_t)ny * z)] = vs.c[i][0];
    or_stream_transpose(&vs, n, bc, e, lam);
    free(e);
    return 0;
}

/* Outflow flux J of a state: sum over the plane x = nx-1 of rho*u_x of the
 * streamed populations. */
int oracle_flux(int q, int nx, int ny, int nz, const int* bc, const double* F, const double* f,
                double* J)
{
    or_velset vs;
    int n[3] = {nx, ny, nz}, y, z;
    if (or_get_velset(q, &vs)) return -1;
    *J = 0.0;
    for (z = 0; z < nz; ++z)
        for (y = 0; y < ny; ++y) {
            double g[OR_MAXQ], r, uu[3];
            or_gather(&vs, n, bc, f, nx - 1, y, z, g);
            or_moments_cell(&vs, g, F, &r, uu);
            *J += r * uu[0];
        }
    return 0;
}

/* Gradient dJ/dvarpi after nsteps from the initial state f0, by reverse
 * sweep with recomputation: states are kept every `every` steps and each
 * segment is recomputed forward before its reverse steps. grad must hold
 * cells values and is overwritten. J receives the forward objective. */
int oracle_flux_grad(int q, int nx, int ny, int nz, const int* bc, double tau, const double* F,
                     const double* varpi, const double* f0, long nsteps, int every, double* J,
                     double* grad)
{
    int64_t cells = (int64_t)nx * ny * nz, sz = (int64_t)q * cells;
    long nsnap, s, k, seg;
    double *snaps, *seg_states, *tmp, *lam_a, *lam_b;
    int rc = 0;
    if (every < 1 || nsteps < 0) return -1;
    nsnap = nsteps / every + 1;
    snaps = (double*)malloc(sizeof(double) * (size_t)(sz * nsnap));
    seg_states = (double*)malloc(sizeof(double) * (size_t)(sz * (every + 1)));
    tmp = (double*)malloc(sizeof(double) * (size_t)sz);
    lam_a = (double*)malloc(sizeof(double) * (size_t)sz);
    lam_b = (double*)malloc(sizeof(double) * (size_t)sz);
    if (!snaps || !seg_states || !tmp || !lam_a || !lam_b) {
        rc = -2;
        goto done;
    }
    /* forward sweep, keeping f^{k*every} */
    memcpy(snaps, f0, sizeof(double) * (size_t)sz);
    memcpy(tmp, f0, sizeof(double) * (size_t)sz);
    for (s = 0; s < nsteps; ++s) {
        if ((rc = oracle_run(q, nx, ny, nz, bc, tau, F, varpi, tmp, lam_a, 1))) goto done;
        if ((s + 1) % every == 0 && (s + 1) / every < nsnap)
            memcpy(snaps + sz * ((s + 1) / every), tmp, sizeof(double) * (size_t)sz);
    }
    if ((rc = oracle_flux(q, nx, ny, nz, bc, F, tmp, J))) goto done;
    if ((rc = oracle_flux_seed(q, nx, ny, nz, bc, lam_a))) goto done;
    for (k = 0; k < cells; ++k) grad[k] = 0.0;
    /* reverse sweep over segments [seg*every, min((seg+1)*every, nsteps)) */
    for (seg = (nsteps - 1) / every; seg >= 0 && nsteps > 0; --seg) {
        long s0 = seg * every, s1 = (seg + 1) * every < nsteps ? (seg + 1) * every : nsteps;
        memcpy(seg_states, snaps + sz * seg, sizeof(double) * (size_t)sz);
        for (s = s0; s < s1 - 1; ++s) {
            memcpy(seg_states + sz * (s - s0 + 1), seg_states + sz * (s - s0),
                   sizeof(double) * (size_t)sz);
            if ((rc = oracle_run(q, nx, ny, nz, bc, tau, F, varpi, seg_states + sz * (s - s0 + 1),
                                 tmp, 1)))
                goto done;
        }
        for (s = s1 - 1; s >= s0; --s) {
            if ((rc = oracle_adjoint_step(q, nx, ny, nz, bc, tau, F, varpi,
                                          seg_states + sz * (s - s0), lam_a, lam_b, grad)))
                goto done;
            memcpy(lam_a, lam_b, sizeof(double) * (size_t)sz);
        }
    }
done:
    free(snaps);
    free(seg_states);
    free(tmp);
    free(lam_a);
    free(lam_b);
    return rc;
}

/* Porosity control from a permeability (eq. "d definition"):
 * varpi = 1 - nu*tau/K, clamped to [0, 1]; K <= 0 gives 0 (solid),
 * K = +inf gives 1 (free fluid). */
int oracle_porosity_from_permeability(const double* K, double nu, double tau, double* varpi,
                                      int64_t n)
{
    int64_t k;
    for (k = 0; k < n; ++k) {
        double v;
        if (!(K[k] > 0.0)) v = 0.0;
        else v = 1.0 - nu * tau / K[k];
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        varpi[k] = v;
    }
    return 0;
}
