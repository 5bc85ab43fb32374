// Step kernels for the StoreF64 storage policy.
#include "k_step.cuh"

namespace hlbm {

cudaError_t step_f64(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    return step_for_storage<StoreF64>(c, mode, fin, fout, varpi);
}

}  // namespace hlbm
