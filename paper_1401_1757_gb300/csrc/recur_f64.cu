// FP64 variants of the recurrence kernel (plain double arithmetic).
#include "recur_kernel.cuh"

namespace rsv {
// The tunable fast variants come first; then the one with trajectory /
// per-step-mean outputs and those that pay within the step or take varying
// cash flows.
static const Variant kF64[] = {
    RSV_VARIANT(F_F64, 2, 2, 128, 1, false, "f64 P2xM2 nt128"),
    RSV_VARIANT(F_F64, 4, 1, 128, 1, false, "f64 P4xM1 nt128"),
    RSV_VARIANT(F_F64, 2, 1, 128, 1, false, "f64 P2xM1 nt128"),
    RSV_VARIANT(F_F64, 2, 1, 128, 1, true, "f64 P2xM1 nt128 side-outputs"),
    RSV_VARIANT_PAY(F_F64, 2, 1, 128, 1, false, PAY_START, "f64 P2xM1 nt128 pay-start"),
    RSV_VARIANT_PAY(F_F64, 2, 1, 128, 1, false, PAY_FRACTION, "f64 P2xM1 nt128 pay-fraction"),
    RSV_VARIANT_PAY(F_F64, 2, 1, 128, 1, false, PAY_END_GENERAL, "f64 P2xM1 nt128 pay-end-general"),
};
const Variant* variants_f64(int* n) {
    *n = (int)(sizeof(kF64) / sizeof(kF64[0]));
    return kF64;
}
}  // namespace rsv
