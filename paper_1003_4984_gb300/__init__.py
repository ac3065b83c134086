"""GB300-native lensing remap by kriging interpolation on the sphere (FLINTS).

The compute path is the CUDA library ``_lib/libflints.so`` (sm_103a), reached
through the C ABI declared in ``include/flints.h``; ``api`` marshals
arguments for it.  Build with ``paper_1003_4984_gb300.build.build()``.
"""
from .api import (Batch, LaunchCfg, FLINTS_FP64, FLINTS_FORCE_FALLBACK, FLINTS_MIXED, FLINTS_NO_VARIANCE, FLINTS_ROTATE_TO_TARGET, FLINTS_SPIN2_AUGMENTED, ST_FALLBACK, ST_FAILED, ST_INPUT, ST_NUGGET, ST_POLE,
                  ST_WINDOW, FlintsError, PaperPlan, Plan, Synth, header_functions, lens_batch, lens_host, load_library,
                  measure_fma_peak)

__all__ = ["Plan", "PaperPlan", "Synth", "Batch", "LaunchCfg", "FlintsError", "lens_batch", "lens_host", "load_library", "header_functions", "measure_fma_peak", "FLINTS_FP64",
           "FLINTS_MIXED", "FLINTS_NO_VARIANCE", "FLINTS_FORCE_FALLBACK", "FLINTS_ROTATE_TO_TARGET", "FLINTS_SPIN2_AUGMENTED", "ST_NUGGET", "ST_FALLBACK", "ST_WINDOW", "ST_FAILED", "ST_POLE", "ST_INPUT"]
