// Instantiations of the fused lens kernel for spin-1 fields (e.g. deflections).
#include "lens.cuh"

namespace flints {

cudaError_t launch_lens_spin1(int K, int precision, const LensArgs &a, int R_rings, const LaunchCfg &cfg,
                              cudaStream_t st) {
    const int sms = device_sm_count();
    const bool mixed = precision == FLINTS_MIXED;
    switch (K) {
        case 16:
            return mixed ? launch_one<16, 1, 1>(a, R_rings, cfg, sms, st) : launch_one<16, 1, 0>(a, R_rings, cfg, sms, st);
        case 24:
            return mixed ? launch_one<24, 1, 1>(a, R_rings, cfg, sms, st) : launch_one<24, 1, 0>(a, R_rings, cfg, sms, st);
        case 32:
            return mixed ? launch_one<32, 1, 1>(a, R_rings, cfg, sms, st) : launch_one<32, 1, 0>(a, R_rings, cfg, sms, st);
        case 48:
            return mixed ? launch_one<48, 1, 1>(a, R_rings, cfg, sms, st) : launch_one<48, 1, 0>(a, R_rings, cfg, sms, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace flints
