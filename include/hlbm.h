/*
 * hlbm.h - C ABI of the GB300 homogenized lattice BGK (HBGK) library.
 *
 * The library advances the lattice Boltzmann discretization of the
 * homogenized BGK Boltzmann equation (HBGKBE) of Simonis et al.,
 * arXiv:2310.14746, Part I: BGK relaxation (Sec. 3.1, eq. collisionOperatorQ)
 * toward the homogenized Maxwellian evaluated at the porosity-scaled velocity
 * varpi*u (Sec. 3.2, eqs. porousVeloMaxwellian and "d definition",
 * varpi = 1 - nu*tau/K), with a body force F (the F.grad_v f term of eq.
 * BGKBE) and the data of the target problem eq. targetEBTL (viscosity,
 * force, permeability via varpi, no-slip walls). The lattice pieces follow
 * the textbook scheme, since the paper defers its discretization:
 *   - velocity sets D2Q9 / D3Q19, lattice units dx = dt = 1, c_s^2 = 1/3,
 *     nu = (tau - 1/2)/3;
 *   - one time step = pull streaming g_i(x) = f_i(x - c_i) (periodic wrap, or
 *     half-way bounce-back g_i(x) = f_opp(i)(x) across a wall), then
 *       rho = sum g, u = (sum c g + F/2)/rho, v = varpi*u,
 *       M_i = w_i rho (1 + 3 c_i.v + 4.5 (c_i.v)^2 - 1.5 v.v),
 *       S_i = (1 - 1/(2 tau)) w_i (3 (c_i - u).F + 9 (c_i.u)(c_i.F)),
 *       f_i <- g_i - (g_i - M_i)/tau + S_i;
 *   - the state between steps is the post-collision population f.
 *
 * Layouts. Every cell array is x-fastest: cell = x + nx*(y + ny*z).
 * Population arrays are [q][z][y][x]. Velocity arrays are [3][z][y][x]
 * (component-major). Direction order:
 *   D2Q9 : 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1)
 *          7 (-1,-1) 8 (1,-1)
 *   D3Q19: 0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0) 5 (0,0,1)
 *          6 (0,0,-1) 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
 *          11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1)
 *          16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 * D2Q9 lattices have nz = 1.
 *
 * Storage. Populations are held on the device as deviations from the lattice
 * weights, (f_i - w_i) * s, in FP64, FP32, FP16 (s = 2^12 by default) or
 * BF16 (s = 1); arithmetic is FP32 for the reduced-precision and FP32
 * policies and FP64 for the FP64 policy. Conversions round to nearest.
 *
 * Conventions shared by every call:
 *   - the return value is a status: HLBM_OK (0) or a negative HLBM_ERR_*;
 *     hlbm_strerror() names it. No exception crosses the ABI.
 *   - a handle owns all device memory it allocates; inputs are copied, the
 *     caller keeps ownership of every buffer it passes.
 *   - device work is enqueued on the handle's CUDA stream and is asynchronous
 *     unless the call says it synchronises.
 *   - `on_device` = 1 means the pointer is device memory, 0 host memory.
 *   - a handle is used by one host thread at a time.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HLBM_OK 0
#define HLBM_ERR_INVALID_ARG (-1) /* an argument is out of range or NULL     */
#define HLBM_ERR_OOM (-2)         /* a device or host allocation failed      */
#define HLBM_ERR_CUDA (-3)        /* a CUDA runtime call or launch failed    */
#define HLBM_ERR_NOT_CONVERGED (-4)
#define HLBM_ERR_TIMEOUT (-5)
#define HLBM_ERR_BUSY (-6)
#define HLBM_ERR_IO (-7)          /* file open/read/write failed or bad file */
#define HLBM_ERR_STATE (-8)       /* the call needs a setting not yet made   */
#define HLBM_ERR_CANCELLED (-9)   /* a server request was cancelled          */
#define HLBM_ERR_SCRATCH_LIMIT (-10) /* lattice too large for the fixed scratch
                                        of hlbm_reduce_noalloc                */

/* ---- enumerations ------------------------------------------------------ */
#define HLBM_D2Q9 9
#define HLBM_D3Q19 19

#define HLBM_F64 0
#define HLBM_F32 1
#define HLBM_F16DEV 2
#define HLBM_BF16DEV 3

#define HLBM_TWO_LATTICE 0 /* pull from buffer A into buffer B, swap        */
#define HLBM_AA 1          /* in place, alternating local / neighbour steps */

#define HLBM_PERIODIC 0
#define HLBM_HALFWAY_BOUNCE_BACK 1 /* walls half a cell outside both ends  */

#define HLBM_HOMOG_SHIFT 0 /* equilibrium at varpi*u (eq. porousVeloMaxwellian) */
#define HLBM_HOMOG_DRAG 1  /* equilibrium at u, drag -lam rho u in the force  */

typedef struct hlbm_lattice hlbm_t;

/* FP64 diagnostics of the current state (see hlbm_reduce). */
typedef struct {
    double mass;        /* sum over cells of rho                            */
    double momentum[3]; /* sum over cells of rho*u                          */
    double plane_flux;  /* sum over the plane x = nx-1 of rho*u_x           */
    double k_app;       /* nu * mean(rho*u_x) / F_x (0 if F_x == 0)         */
    double max_du;      /* max over cells, components of |u - u_prev|       */
    double max_u;       /* max over cells, components of |u|                */
    long long step;     /* time steps taken since the last initialisation   */
} hlbm_stats;

/* ---- lattice lifetime -------------------------------------------------- */

/* Create a lattice of nx*ny*nz cells with velocity set `velset`
 * (HLBM_D2Q9 needs nz == 1), storage policy `storage` and streaming
 * pattern `pattern`; work goes on `cuda_stream` (a cudaStream_t; NULL is the
 * legacy default stream) of the current device. Defaults: tau = 1, F = 0,
 * all axes periodic, varpi = 1 everywhere, populations at rest (f = w).
 * Limits: ny and nz at most 65535 (launch-grid dimensions), at most 2^34
 * cells; HLBM_ERR_INVALID_ARG beyond them. On error *out is NULL. Cites: the lattice and its data are the problem
 * statement of eq. targetEBTL and of the HBGKBE (Sec. 3.2). */
int hlbm_create(hlbm_t** out, int velset, int nx, int ny, int nz, int storage, int pattern,
                void* cuda_stream);

/* Free the handle and its device memory (after draining its stream). NULL is a no-op. */
void hlbm_destroy(hlbm_t* h);

/* Temporary device memory of the calls that need it (the checkpoints of
 * hlbm_adjoint_flux_grad, staging buffers of host-array I/O) comes, ordered on
 * the handle's stream, from a memory pool private to the handle, which keeps
 * the memory it has mapped for the next call instead of handing it back at
 * each synchronisation (re-mapping the 14.5 GB of checkpoints of a 128^3 x
 * 2000-step gradient took about 7 % of the call). This call waits for the
 * handle's stream and returns the pool's unused memory to the device; the
 * next call that needs scratch maps it again. Not a paper operation (memory
 * management of this library). */
int hlbm_release_scratch(hlbm_t* h);

/* Replace the stream later work is enqueued on. */
int hlbm_set_stream(hlbm_t* h, void* cuda_stream);

/* ---- problem data ------------------------------------------------------ */

/* BGK relaxation time tau (eq. collisionOperatorQ); viscosity nu = (tau - 1/2)/3.
 * Rejects tau <= 1/2 and non-finite values. */
int hlbm_set_relaxation(hlbm_t* h, double tau);

/* Per-cell porosity control varpi (eq. "d definition"), nx*ny*nz FP32 values,
 * x-fastest; copied. Every value must lie in [0, 1] (NaN rejected), checked
 * by a kernel before the values replace the field: a host array is first
 * copied to a temporary device buffer (or, when that buffer cannot be
 * allocated, checked on the host and copied straight into the field). On
 * HLBM_ERR_INVALID_ARG the field is unchanged. Synchronises; the caller's
 * array may be reused when the call returns. varpi = 1 is plain BGK,
 * varpi = 0 a solid cell. */
int hlbm_set_porosity(hlbm_t* h, const float* varpi, int on_device);

/* Resolved obstacles: nx*ny*nz bytes, nonzero = solid cell (copied; host or
 * device). A fluid cell whose pull source is solid takes the bounce-back
 * population of its opposite direction (no slip half-way on the solid
 * surface); solid cells are not updated and report rho = 1, u = 0 (and rest
 * populations from hlbm_get_populations). With varpi = 1 in the fluid this is
 * the pore-scale problem whose permeability the homogenized field stands in
 * for (Thm. thmStatNSECase4). NULL removes the obstacles. Set the domain
 * boundaries first (hlbm_set_boundary returns HLBM_ERR_STATE while a mask is
 * set); the post-collision state of the fluid cells is kept across the call.
 * Not supported by hlbm_adjoint_flux_grad (HLBM_ERR_STATE). Synchronises. */
int hlbm_set_solid_mask(hlbm_t* h, const unsigned char* solid, int on_device);

/* Anisotropic porosity control: a diagonal tensor per cell, 3*nx*ny*nz FP32
 * values [3][z][y][x] (varpi_x, varpi_y, varpi_z), each in [0, 1]; copied and
 * validated like hlbm_set_porosity. The Maxwellian is then evaluated at
 * (varpi_x u_x, varpi_y u_y, varpi_z u_z): a drag nu/K_a per axis with
 * varpi_a = 1 - nu tau / K_a, beyond the isotropy assumption of Sec. 2.5
 * (Assumption thmAssump, item 3). A later hlbm_set_porosity returns to the
 * isotropic field. Shift form only (HLBM_ERR_STATE with the drag form);
 * hlbm_adjoint_flux_grad needs the isotropic field. Costs 8 more bytes per
 * cell update. */
int hlbm_set_porosity_tensor(hlbm_t* h, const float* varpi3, int on_device);

/* varpi = 1 - nu*tau/K for n host values (eq. "d definition"), clamped to
 * [0, 1]; K <= 0 or NaN gives 0, K = +inf gives 1. Pure host function. */
int hlbm_porosity_from_permeability(const float* K, double nu, double tau, float* varpi,
                                    size_t n);

/* Constant body force (lattice units) F of eq. targetEBTL; D2Q9 ignores Fz. */
int hlbm_set_force(hlbm_t* h, double Fx, double Fy, double Fz);

/* Boundary type of axis 0 (x), 1 (y) or 2 (z): HLBM_PERIODIC or
 * HLBM_HALFWAY_BOUNCE_BACK (no-slip u = 0 on the boundary, eq. targetEBTL). */
int hlbm_set_boundary(hlbm_t* h, int axis, int type);

/* Form of the homogenization term. HLBM_HOMOG_SHIFT (default) evaluates the
 * Maxwellian at varpi*u (Sec. 3.2, eq. porousVeloMaxwellian). HLBM_HOMOG_DRAG
 * uses the equivalent drag of Sec. 3.3 (eq. momentumHLBM: the shift acts as
 * -nu K^{-1} rho u): the equilibrium stays at u and the force becomes
 * G = F - lam rho u with lam = nu/K = (1 - varpi)/tau, u being the half-force
 * velocity of the total force, u = (j + F/2) / (rho (1 + lam/2)); hlbm_moments
 * and hlbm_reduce then report that u. Both forms give Darcy's u = F K / nu at
 * uniform porosity. hlbm_adjoint_flux_grad supports the shift form only
 * (HLBM_ERR_STATE otherwise). */
int hlbm_set_homogenization(hlbm_t* h, int form);

/* Which of the equivalent step kernels runs (no counterpart in the paper: an
 * implementation choice, exposed for testing and measurement).
 * HLBM_STEP_AUTO (default) picks the fastest kernel that applies: for FP16
 * and BF16 storage on periodic lattices with an even nx, a kernel that
 * updates two neighbouring cells per thread with 32-bit words (two-lattice
 * streaming in every homogenization form; in-place AA streaming in the
 * equilibrium-shift form with a scalar varpi field). HLBM_STEP_PER_CELL forces
 * the one-cell-per-thread kernel. Both give bit-identical states. */
#define HLBM_STEP_AUTO 0
#define HLBM_STEP_PER_CELL 1
int hlbm_set_step_kernel(hlbm_t* h, int variant);

/* Storage scale s of the FP16 deviation policy (a power of two in
 * [1, 2^20]); other policies accept only 1. Applies to later writes of
 * the state: call before hlbm_init_equilibrium / hlbm_set_populations. */
int hlbm_set_storage_scale(hlbm_t* h, double s);

/* Set every cell to the equilibrium of (rho0, u0) (unscaled by varpi) and
 * reset the step counter and the residual reference velocity (to 0). */
int hlbm_init_equilibrium(hlbm_t* h, double rho0, double ux, double uy, double uz);

/* Set the post-collision state from q*cells FP64 full populations f
 * ([q][z][y][x]); resets the step counter and the residual reference. */
int hlbm_set_populations(hlbm_t* h, const double* f, int on_device);

/* Read the post-collision state as q*cells FP64 full populations.
 * A host destination synchronises. */
int hlbm_get_populations(hlbm_t* h, double* f, int on_device);

/* ---- time stepping ----------------------------------------------------- */

/* Advance nsteps >= 0 time steps (stream + collide, see above). Asynchronous.
 * Runs of at least 8 steps replay a captured CUDA graph of the step
 * sequence; shorter runs launch directly. */
int hlbm_step(hlbm_t* h, long nsteps);

/* Steps taken since the last initialisation. */
int hlbm_get_step(hlbm_t* h, long long* step);

/* ---- observables ------------------------------------------------------- */

/* Density rho (cells values) and velocity u ([3][cells]) of the current
 * state: the moments of Def. moments of the streamed populations, with the
 * half-force velocity u = (sum c g + F/2)/rho. Either pointer may be NULL.
 * FP32 outputs. A host destination synchronises. */
int hlbm_moments(hlbm_t* h, float* rho, float* u, int on_device);

/* As hlbm_moments with FP64 outputs (for FP64-storage parity checks). */
int hlbm_moments_f64(hlbm_t* h, double* rho, double* u, int on_device);

/* FP64 diagnostics of the current state (struct hlbm_stats): totals in a
 * fixed-order (deterministic) reduction tree, the apparent permeability of
 * Darcy's law (Thm. thmStatNSECase4, u = A(F - grad p)/nu, mean over all
 * cells), and the residual max|u - u_prev| against the velocity seen by the
 * previous hlbm_reduce call (or 0 after initialisation), which this call then
 * replaces. Synchronises. */
int hlbm_reduce(hlbm_t* h, hlbm_stats* out);

/* Time series of the FP64 diagnostics without a host synchronisation per
 * sample: records the diagnostics of the current state, then nsamples - 1
 * times advances `every` time steps and records them again, so record k
 * describes the state k*every steps after the call began. out receives
 * nsamples records of 8 doubles in the order mass, momentum[3], plane_flux,
 * k_app, max_du, max_u (the fields of hlbm_stats); max_du compares with the
 * residual reference of the last hlbm_reduce call, which this call leaves
 * unchanged. Used for the relaxation history of the Darcy law with memory
 * (Sec. 2, the mean momentum of a cell relaxing with no force). A device
 * `out` (8*nsamples doubles) keeps the call asynchronous; a host `out`
 * synchronises once at the end (the call then allocates a device staging
 * buffer for the records). */
int hlbm_reduce_series(hlbm_t* h, long nsamples, int every, double* out, int on_device);

/* ---- differentiation ---------------------------------------------------- */

/* Gradient of the outflow mass flux through the plane x = plane_x,
 *   J = sum_{y,z} rho*u_x  (the moments of Def. moments, half-force velocity),
 * evaluated nsteps time steps after the current state, with respect to the
 * per-cell porosity control varpi (eq. "d definition"), by a hand-written
 * discrete adjoint of the step: the forward run keeps the state every
 * ckpt_every steps, and each segment is recomputed before its reverse steps
 * (memory: about (nsteps/ckpt_every + ckpt_every + 2) lattice states, plus
 * two FP32 adjoint fields, allocated for the call and freed after it).
 * Writes J (one host double) and grad_varpi (cells FP32 values, x-fastest,
 * host or device per on_device). The lattice state afterwards is the forward
 * state after nsteps steps, and the step counter advances by nsteps.
 * Synchronises. Rejects nsteps < 0, ckpt_every < 1, plane_x outside [0, nx). */
int hlbm_adjoint_flux_grad(hlbm_t* h, long nsteps, int ckpt_every, int plane_x, double* J,
                           float* grad_varpi, int on_device);

/* ---- checkpoint -------------------------------------------------------- */

/* Write the state, step counter and parameters to a file / read them back
 * into a handle of the same shape, velocity set and storage. Both
 * synchronise. Resuming gives the same bits as an uninterrupted run. */
int hlbm_save(hlbm_t* h, const char* path);
int hlbm_load(hlbm_t* h, const char* path);

/* ---- serving: continuous batching of many solves ------------------------ */
/*
 * A server advances many independent D3Q19 HBGK solves (fully periodic
 * lattices of any size) together. Requests wait in a first-come first-served
 * queue and are admitted as slots while their device memory fits the budget;
 * each pump round advances every live slot by check_every time steps in
 * batched persistent launches (one CUDA graph replay), then reads a per-slot
 * FP64 residual max|u - u_prev| over that interval and retires the slots
 * whose residual fell below their tolerance (or that reached max_steps),
 * freeing their memory for waiting requests. A slot's arithmetic, including
 * its reduction, does not depend on the other slots in the batch, so a
 * result is bit-identical alone and in a mix. Server calls may come from
 * several host threads (an internal mutex serialises them).
 */
typedef struct hlbm_server hlbm_server_t;

typedef struct {
    int nx, ny, nz;      /* lattice edge lengths (periodic on every axis)      */
    double tau;          /* relaxation time (> 1/2)                            */
    double F[3];         /* body force                                         */
    const float* varpi;  /* host, nx*ny*nz values in [0, 1]; copied at submit  */
    double tol;          /* converged when max|u - u_prev| over one interval < tol */
    long long max_steps; /* give up (HLBM_ERR_NOT_CONVERGED) after this many    */
    float* u_out;        /* optional host buffer of 3*cells floats that receives
                            the final velocity ([3][z][y][x]) at retirement;
                            must stay valid until the result is polled; or NULL */
    uint64_t tag;        /* caller's label, returned in the result             */
} hlbm_request;

typedef struct {
    uint64_t id, tag;
    int status;          /* HLBM_OK (converged), HLBM_ERR_NOT_CONVERGED,
                            HLBM_ERR_CANCELLED or HLBM_ERR_OOM                 */
    int nx, ny, nz;
    long long steps;     /* time steps run                                     */
    double k_app;        /* nu * mean(rho u_x) / F_x at the end                */
    double max_du;       /* last residual                                      */
    double max_u, mass, plane_flux;
    double t_submit, t_admit, t_finish; /* seconds since server creation (host
                                           steady clock); t_admit < 0 if never admitted */
    long long steps_low; /* of `steps`, those run in the reduced-precision storage */
    int final_storage;   /* storage the solve ended in (HLBM_F32 after refinement) */
} hlbm_result;

typedef struct {
    int active, waiting, done_unpolled;
    size_t mem_used, mem_budget;
    long long lattice_updates; /* cell updates performed by all rounds        */
    long long rounds;
    double elapsed_s;
} hlbm_server_stats;

/* Create a server whose slots start in `storage` (HLBM_F32, HLBM_F16DEV or
 * HLBM_BF16DEV) within mem_budget bytes of device memory, checking every
 * check_every (even, 2..10000) steps, on `cuda_stream`. With a reduced-
 * precision storage, refinement is on by default: a slot whose residual
 * reaches the storage's rounding floor (floor_coef * max|u|; 2e-3 for FP16,
 * 1.6e-2 for BF16), or stops improving for 20 checks within 10 times that
 * floor, is converted in place to FP32 storage (when the budget allows) and
 * must then meet its tolerance in FP32. Scheduling: every round the oldest
 * live request advances check_every steps, and younger ones join it in age
 * order within a cell budget (hlbm_server_set_priority). Slots of at least
 * 2^18 cells (64^3) run the single-lattice step kernels inside the round's
 * graph, in parallel branches of it; smaller ones share a batched kernel; both
 * give the same bits. */
int hlbm_server_create(hlbm_server_t** out, size_t mem_budget, int storage, int check_every,
                       void* cuda_stream);
/* Turn refinement on or off and set its floor coefficient (>= 0). With it off,
 * a reduced-precision slot converges only if its own rounding noise stays
 * below the tolerance. */
int hlbm_server_set_refinement(hlbm_server_t* s, int enable, double floor_coef);
/* Age priority of the batch (no counterpart in the paper: a serving policy).
 * Each round runs the oldest live request and, in age order, the younger
 * ones that fit a budget of max(1M, (1 + backfill) * the oldest request's
 * cells) cells; a younger request that does not fit is skipped for that
 * round, so smaller ones behind it can still run. backfill >= 0 (default
 * 0.1) bounds how much the oldest request is slowed by the batch, whatever
 * the queue length; a very large value is plain processor sharing. Results
 * do not depend on it, only when they arrive. */
int hlbm_server_set_priority(hlbm_server_t* s, double backfill);
/* Queue a request (validated and copied); *id receives its identifier.
 * HLBM_ERR_OOM if it could never fit the budget. */
int hlbm_server_submit(hlbm_server_t* s, const hlbm_request* r, uint64_t* id);
/* One scheduling round: admit, run check_every steps of this round's slots
 * (see hlbm_server_set_priority), check them, retire. Synchronises. *active / *waiting (may be NULL) receive the
 * counts after the round. A round with no live slot launches nothing. */
int hlbm_server_pump(hlbm_server_t* s, int* active, int* waiting);
/* Move up to max finished results into out; *n receives how many. */
int hlbm_server_poll(hlbm_server_t* s, hlbm_result* out, int max, int* n);
/* Cancel a waiting (immediately) or live (at the next round) request. */
int hlbm_server_cancel(hlbm_server_t* s, uint64_t id);
/* Counters of the server. */
int hlbm_server_info(hlbm_server_t* s, hlbm_server_stats* out);
/* Fault injection for tests: the next n slot allocations fail as if the
 * device were out of memory (admission then backs off). */
int hlbm_server_inject_alloc_failures(hlbm_server_t* s, int n);
/* Free the server, its slots and its queued requests (results not polled are lost). */
void hlbm_server_destroy(hlbm_server_t* s);

/* ---- allocation-free diagnostics --------------------------------------- */

/* The diagnostics of hlbm_reduce for callers that must not allocate device
 * memory: for example code running inside an allocator or memory-pool
 * callback, a host application that gives the library a fixed arena and
 * forbids further cudaMalloc calls, or a monitoring hook that must not fail
 * for lack of memory. (The paper has no counterpart; this is a systems
 * interface.) The caller passes everything: f, the post-collision state in
 * the two-lattice (NATURAL) layout, q*nx*ny*nz device values of the storage
 * type holding (f_i - w_i) * storage_scale, [q][z][y][x]; u_prev, a device
 * buffer of 3*nx*ny*nz values in the arithmetic type (double for HLBM_F64,
 * float otherwise) holding the previous velocity, which the call compares
 * against (max_du) and then overwrites with the current velocity; the lattice
 * description (velset, sizes, storage, bc[3] boundary types, tau, F[3],
 * storage_scale with the rule of hlbm_set_storage_scale); the homogenization
 * `form` (HLBM_HOMOG_SHIFT or HLBM_HOMOG_DRAG, as hlbm_set_homogenization)
 * with `varpi`, nx*ny*nz device FP32 porosity values that the drag form needs
 * for its velocity (required with HLBM_HOMOG_DRAG, ignored and may be NULL
 * with HLBM_HOMOG_SHIFT); and the host struct `out` (its step field is set to
 * 0). Lattices with resolved obstacles (hlbm_set_solid_mask) are not
 * supported: the call has no solid-cell input and counts every cell as fluid.
 * Sizes follow hlbm_create's limits, and the reduction grid must fit the
 * launch limits; otherwise HLBM_ERR_INVALID_ARG.
 * The call uses no memory the library allocates: its scratch is a fixed 4 MiB
 * array in the library's device memory, which every GPU that loads the
 * library keeps until the process exits. A lattice whose reduction needs more
 * than 65536 partial blocks (blocks of 256 threads over x-rows of up to 128
 * cells and four z planes; 384^3 is the largest cube that fits) returns
 * HLBM_ERR_SCRATCH_LIMIT. The first call on a device looks up the array's
 * device address (once per device); make that first call before any stream
 * capture. Every call on a device shares the array: calls whose work
 * overlaps on the same GPU race on it, so serialise them. Synchronises
 * `cuda_stream`. */
int hlbm_reduce_noalloc(int velset, int nx, int ny, int nz, int storage, const int* bc, double tau,
                        const double* F, double storage_scale, int form, const float* varpi, const void* f,
                        void* u_prev, hlbm_stats* out, void* cuda_stream);

/* ---- misc -------------------------------------------------------------- */

/* Static description of a status code. */
const char* hlbm_strerror(int status);

/* Last CUDA error string recorded by the library on this thread ("" if none). */
const char* hlbm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HLBM_H */
