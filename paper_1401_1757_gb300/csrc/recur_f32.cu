// Plain FP32 variants of the recurrence kernel.
#include "recur_kernel.cuh"

namespace rsv {
static const Variant kF32[] = {
    RSV_VARIANT(F_F32, 8, 4, 128, 1, false, "f32 P8xM4 nt128"),
    RSV_VARIANT(F_F32, 4, 4, 256, 1, false, "f32 P4xM4 nt256"),
    RSV_VARIANT(F_F32, 4, 4, 256, 2, false, "f32 P4xM4 nt256 min2"),
    RSV_VARIANT(F_F32, 8, 2, 256, 1, false, "f32 P8xM2 nt256"),
    RSV_VARIANT(F_F32, 4, 2, 256, 3, false, "f32 P4xM2 nt256 min3"),
    RSV_VARIANT(F_F32, 2, 4, 256, 3, false, "f32 P2xM4 nt256 min3"),
    RSV_VARIANT(F_F32, 4, 2, 256, 1, true, "f32 P4xM2 nt256 side-outputs"),
    RSV_VARIANT_PAY(F_F32, 2, 2, 256, 2, false, PAY_START, "f32 P2xM2 nt256 pay-start"),
    RSV_VARIANT_PAY(F_F32, 2, 2, 256, 2, false, PAY_FRACTION, "f32 P2xM2 nt256 pay-fraction"),
    RSV_VARIANT_PAY(F_F32, 2, 2, 256, 2, false, PAY_END_GENERAL, "f32 P2xM2 nt256 pay-end-general"),
};
const Variant* variants_f32(int* n) {
    *n = (int)(sizeof(kF32) / sizeof(kF32[0]));
    return kF32;
}
}  // namespace rsv
