// Compensated (double-float) FP32 variants of the recurrence kernel.
#include "recur_kernel.cuh"

namespace rsv {
// (form, policies per thread P, scenarios per thread M, threads per CTA, minimum
// resident CTAs per SM (caps registers), side outputs)
static const Variant kComp[] = {
    // the tuned best on the 100,000-policy mix first: the default before tuning
    RSV_VARIANT(F_COMP, 8, 1, 128, 4, false, "comp P8xM1 nt128 min4"),
    RSV_VARIANT(F_COMP, 8, 1, 256, 2, false, "comp P8xM1 nt256 min2"),
    RSV_VARIANT(F_COMP, 8, 1, 64, 8, false, "comp P8xM1 nt64 min8"),
    RSV_VARIANT(F_COMP, 12, 1, 128, 3, false, "comp P12xM1 nt128 min3"),
    RSV_VARIANT(F_COMP, 4, 1, 128, 4, false, "comp P4xM1 nt128 min4"),
    RSV_VARIANT(F_COMP, 4, 1, 256, 2, false, "comp P4xM1 nt256 min2"),
    RSV_VARIANT(F_COMP, 2, 2, 256, 3, false, "comp P2xM2 nt256 min3"),
    RSV_VARIANT(F_COMP, 2, 1, 256, 1, true, "comp P2xM1 nt256 side-outputs"),
    RSV_VARIANT_PAY(F_COMP, 4, 1, 128, 4, false, PAY_START, "comp P4xM1 nt128 pay-start"),
    RSV_VARIANT_PAY(F_COMP, 4, 1, 128, 4, false, PAY_FRACTION, "comp P4xM1 nt128 pay-fraction"),
    RSV_VARIANT_PAY(F_COMP, 4, 1, 128, 4, false, PAY_END_GENERAL, "comp P4xM1 nt128 pay-end-general"),
};
const Variant* variants_comp(int* n) {
    *n = (int)(sizeof(kComp) / sizeof(kComp[0]));
    return kComp;
}
}  // namespace rsv
