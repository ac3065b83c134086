// Instantiations of the fused lens kernel for the augmented (widely linear)
// spin-2 estimator: a 2K x 2K real system per target.
#include "lens.cuh"

namespace flints {

cudaError_t launch_lens_spin2a(int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                               cudaStream_t st) {
    const int sms = device_sm_count();
    const bool mixed = precision == FLINTS_MIXED;
    constexpr int A = SPIN2_AUG;
    switch (K) {
        case 16:
            return mixed ? launch_one<16, A, 1>(a, R_rings, cfg, sms, st) : launch_one<16, A, 0>(a, R_rings, cfg, sms, st);
        case 24:
            return mixed ? launch_one<24, A, 1>(a, R_rings, cfg, sms, st) : launch_one<24, A, 0>(a, R_rings, cfg, sms, st);
        case 32:
            return mixed ? launch_one<32, A, 1>(a, R_rings, cfg, sms, st) : launch_one<32, A, 0>(a, R_rings, cfg, sms, st);
        case 48:
            return mixed ? launch_one<48, A, 1>(a, R_rings, cfg, sms, st) : launch_one<48, A, 0>(a, R_rings, cfg, sms, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace flints
