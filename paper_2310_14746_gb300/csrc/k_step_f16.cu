// Step kernels for the StoreF16 storage policy.
#include "k_step_pair.cuh"

namespace hlbm {

cudaError_t step_f16(const LaunchCtx& c, int mode, const void* fin, void* fout, const float* varpi) {
    return step_for_storage16<StoreF16>(c, mode, fin, fout, varpi);
}

}  // namespace hlbm
