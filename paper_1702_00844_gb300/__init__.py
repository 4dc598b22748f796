"""GB300-native (sm_103a) radio-astronomy correlator: the X-step of an FX
correlator (van Nieuwpoort & Romein, Section 2) as a C-ABI library with
hand-written CUDA kernels and a thin torch/ctypes binding."""
from .build import build as build_library  # noqa: F401
from .corr import (CorrError, GainCalibrationLoss, Plan, Subarray, lib,  # noqa: F401
                   n_baselines, input_shape, layout_shape, reorder, torch_dtype, FLAG_GAINS,
                   FLAG_NO_AUTOTUNE, FLAG_HOST_IO, LAYOUTS)
