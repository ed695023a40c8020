// BF16 tensor-core LUT build (tcgen05): not yet built in this revision.
#include "../fa_internal.h"

namespace fa {

void launch_lut_tc(const DeviceIndex &ix, const float *q, int64_t nq, int prec, void *lut,
                   float *lut_scale, cudaStream_t st) {
    (void)ix, (void)q, (void)nq, (void)prec, (void)lut, (void)lut_scale, (void)st;
    throw Error{FA_ERR_ARG, "the BF16 tensor-core LUT is not available in this build"};
}

}  // namespace fa
