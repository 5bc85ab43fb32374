// Solid-link masks and the storage dispatch of the step kernels.
#include "k_step.cuh"

namespace hlbm {

cudaError_t step_f64(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi);
cudaError_t step_f32(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi);
cudaError_t step_f16(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi);
cudaError_t step_bf16(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi);

template <int Q>
__global__ void k_build_links(const unsigned char* __restrict__ solid, unsigned* __restrict__ links, Geometry g) {
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long cell = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
    if (solid[cell]) {
        links[cell] = kSolidBit;
        return;
    }
    const Nbr<long long> nb(g, x, y, z);
    unsigned m = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const bool wall = nb.template beyond_wall<Q>(i, -1);  // domain walls only (lm = 0 here)
        if (!wall && solid[cell + nb.template offset<Q>(i, -1)]) m |= 1u << i;
    }
    links[cell] = m;
}

cudaError_t launch_build_links(const LaunchCtx& c, const unsigned char* solid, unsigned* links) {
    Geometry g{c.nx, c.ny, c.nz, c.wall[0], c.wall[1], c.wall[2], (size_t)c.nx * c.ny * c.nz};
    const dim3 blk = step_block_for(c.nx);
    const dim3 grd((c.nx + blk.x - 1) / blk.x, (c.ny + blk.y - 1) / blk.y, c.nz);
    if (c.q == 9) k_build_links<9><<<grd, blk, 0, c.stream>>>(solid, links, g);
    else k_build_links<19><<<grd, blk, 0, c.stream>>>(solid, links, g);
    return cudaGetLastError();
}

cudaError_t launch_step(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    switch (c.storage) {
        case 0: return step_f64(c, mode, fin, fout, varpi);
        case 1: return step_f32(c, mode, fin, fout, varpi);
        case 2: return step_f16(c, mode, fin, fout, varpi);
        case 3: return step_bf16(c, mode, fin, fout, varpi);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hlbm
