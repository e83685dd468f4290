// Compensated (double-float) FP32 variants of the recurrence kernel.
#include "recur_kernel.cuh"

namespace rsv {
static const Variant kComp[] = {
    RSV_VARIANT(F_COMP, 2, 1, 256, false, "comp P2xM1 nt256"),
    RSV_VARIANT(F_COMP, 4, 1, 256, false, "comp P4xM1 nt256"),
    RSV_VARIANT(F_COMP, 2, 2, 256, false, "comp P2xM2 nt256"),
    RSV_VARIANT(F_COMP, 4, 2, 128, false, "comp P4xM2 nt128"),
    RSV_VARIANT(F_COMP, 1, 2, 256, false, "comp P1xM2 nt256"),
    RSV_VARIANT(F_COMP, 2, 1, 256, true, "comp P2xM1 nt256 side-outputs"),
};
const Variant* variants_comp(int* n) {
    *n = (int)(sizeof(kComp) / sizeof(kComp[0]));
    return kComp;
}
}  // namespace rsv
