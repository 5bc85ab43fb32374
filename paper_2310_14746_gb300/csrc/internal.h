// Internal interface between the C ABI (api.cu) and the kernel translation
// units. Not installed; callers use include/hlbm.h.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace hlbm {

enum StepMode { MODE_TWO_LATTICE = 0, MODE_AA_EVEN = 1, MODE_AA_ODD = 2 };

// Everything a launch needs to know about a lattice, in plain types.
struct LaunchCtx {
    int q;          // 9 or 19
    int storage;    // HLBM_F64 / F32 / F16DEV / BF16DEV
    int nx, ny, nz;
    int wall[3];    // 1 = half-way bounce-back on that axis
    double tau;
    double F[3];
    double scale;   // storage scale s (deviations are stored times s)
    cudaStream_t stream;
    int drag = 0;                  // homogenization form: 0 equilibrium shift, 1 explicit drag
    const float* varpi = nullptr;  // porosity control (observables need it in the drag form)
    const float* varpi3 = nullptr; // diagonal porosity tensor [3][cells], or null (isotropic)
    const unsigned* links = nullptr; // solid-link masks (resolved obstacles), or null
    int variant = 0;                 // 0: fastest applicable step kernel; 1: per-cell kernel only
};

// Solid-link masks from a solid flag per cell (uint8, nonzero = solid): bit i of
// links[cell] is set when the pull source x - c_i is solid (periodic wrap; a
// source beyond a domain wall is left to the wall logic), bit 31 when the
// cell itself is solid.
cudaError_t launch_build_links(const LaunchCtx& c, const unsigned char* solid, unsigned* links);

// One time step: read `fin` in the layout implied by `mode`, write `fout`
// (== fin for the AA modes).
cudaError_t launch_step(const LaunchCtx& c, int mode, const void* fin, void* fout,
                        const float* varpi);

// Moments of a state stored in `layout` (Layout enum of lattice.cuh). rho
// and/or u may be null. out_f64 selects double outputs, else float.
cudaError_t launch_moments(const LaunchCtx& c, int layout, const void* f, void* rho, void* u,
                           int out_f64);

// Per-block FP64 partials of the diagnostics, then a fixed-order final
// reduction (one block per quantity) into out8[8] (device). u_prev (arithmetic type of the
// storage: double for F64, float otherwise; 3*cells) is compared against and,
// if update_prev, overwritten. `partials` is caller-provided scratch of at
// least reduce_partials_count(c) * 8 doubles.
size_t reduce_partials_count(const LaunchCtx& c);
// Whether the partials kernel's grid for this lattice is within the launch limits.
bool reduce_grid_fits(const LaunchCtx& c);
cudaError_t launch_reduce(const LaunchCtx& c, int layout, const void* f, void* u_prev,
                          int update_prev, double* partials, double* out8);

// Write the natural post-collision populations fnat (FP64 full values) into
// the state buffer in `layout`. fnat is [q][cells] when uniform == 0, or q
// values applied to every cell when uniform == 1.
cudaError_t launch_write_state(const LaunchCtx& c, int layout, const double* fnat, int uniform,
                               void* f);
// Read the state as natural FP64 full populations [q][cells].
cudaError_t launch_read_state(const LaunchCtx& c, int layout, const void* f, double* fnat);

// Count values outside [0, 1] (or NaN) into *bad (device int, accumulated).
cudaError_t launch_check_unit_interval(const float* v, size_t n, int* bad, cudaStream_t s);
cudaError_t launch_fill_f32(float* v, size_t n, float value, cudaStream_t s);
cudaError_t launch_fill_bytes0(void* p, size_t bytes, cudaStream_t s);

size_t storage_bytes(int storage);

// Reverse step of the outflow-flux adjoint: fn is the forward state before the
// step (NATURAL layout), lam_in = dJ/df^{n+1} and lam_out = dJ/df^n ([q][cells]
// FP32, distinct buffers); grad (FP32 cells) accumulates dJ/dvarpi.
cudaError_t launch_adjoint_step(const LaunchCtx& c, const void* fn, const float* lam_in, float* lam_out,
                                const float* varpi, float* grad);
// dJ/df of the final state for J = sum over the plane x = plane_x of rho*u_x.
cudaError_t launch_flux_seed(const LaunchCtx& c, float* lam, int plane_x);
// J of a state in `layout` into out (one double, device).
cudaError_t launch_plane_flux(const LaunchCtx& c, int layout, const void* f, int plane_x, double* out);

}  // namespace hlbm
