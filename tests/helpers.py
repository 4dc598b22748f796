"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

# Tolerances (relative, per channel, Frobenius norm): FP32 inputs accumulate
# in FP32 over T samples (error ~ sqrt(T) * 2^-24 relative to the norm of the
# products); FP16 inputs are compared against the oracle fed the same FP16
# values, so only the FP32 accumulation differs as well.
TOL_FP32 = 1e-5
TOL_FP16 = 1e-5


def tol_fp16(T: int) -> float:
    """FP16 inputs on the tensor path: every accumulator element receives T/8
    MMA additions (four K=16 steps per block of 32 samples, for Re and for
    Im), each rounding the FP32 running sum by at most one ulp (2^-23 of a
    running sum that the autocorrelations bound by the final norm), so the
    relative Frobenius error is at most (T/8) * 2^-23 = T * 2^-26; never
    tighter than TOL_FP16."""
    return max(TOL_FP16, T * 2.0 ** -26)
# Element-wise bound on the correlation-coefficient error
#   |dV_ab| <= TOL_COEF * sqrt(V_aa V_bb) * (number of terms)^0 ... (see below)
TOL_COEF = 2e-5


def rel_frobenius_per_unit(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    g = got.reshape(got.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    num = np.linalg.norm(g - r, axis=1)
    den = np.linalg.norm(r, axis=1)
    den = np.where(den == 0, 1.0, den)
    return num / den


def coef_error(got: np.ndarray, ref: np.ndarray, S: int) -> float:
    """max |V - V_ref|_ab / sqrt(V_ref_aa V_ref_bb) over units, baselines and
    pol pairs (the error in the normalised correlation coefficient)."""
    units = ref.shape[0]
    auto_idx = np.array([s * (s + 1) // 2 + s for s in range(S)])
    auto = np.stack([ref[:, auto_idx, 0, 0].real, ref[:, auto_idx, 1, 1].real], axis=-1)  # (U,S,2)
    s2 = np.concatenate([np.full(j + 1, j) for j in range(S)])
    s1 = np.concatenate([np.arange(j + 1) for j in range(S)])
    na = np.sqrt(np.maximum(auto[:, s1, :], 1e-300))  # (U,B,2)
    nb = np.sqrt(np.maximum(auto[:, s2, :], 1e-300))
    norm = na[:, :, :, None] * nb[:, :, None, :]
    return float((np.abs(got - ref) / norm).max()) if units else 0.0


def to_numpy_vis(t, dtype: str) -> np.ndarray:
    """Device visibilities -> complex128 (units, B, 2, 2)."""
    a = t.detach().cpu()
    if dtype == "ci8":
        a = a.numpy().astype(np.int64)
        v = a[..., 0] + 1j * a[..., 1]
    else:
        v = a.numpy().astype(np.complex128)
    return v.reshape((-1,) + v.shape[-3:])


def to_numpy_int(t) -> np.ndarray:
    """Device int32 visibilities -> int64 pairs (units, B, 2, 2, 2)."""
    a = t.detach().cpu().numpy().astype(np.int64)
    return a.reshape((-1,) + a.shape[-4:])
