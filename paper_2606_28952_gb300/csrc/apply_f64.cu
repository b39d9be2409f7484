// apply_f64.cu -- double instantiations of the gather kernels of apply_kernels.cuh
// (split from apply.cu so the two precisions compile in parallel).
#include "apply_kernels.cuh"

namespace ps {
void launch_apply_f64(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out,
                      double *partials, void *split_buf, cudaStream_t st) {
    launch_apply_prec<double>(cfg, p, v, in, out, partials, split_buf, st);
}
}  // namespace ps
