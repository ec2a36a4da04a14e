"""Shared helpers of the GPU parity tests."""
import numpy as np

# Parity bar of the FP64 path: 1e-10 relative on every mass fraction above 1e-10
# and on T; mass fractions at or below 1e-10 are compared absolutely at
# 1e-10 * 1e-10 = 1e-20, the Newton absolute tolerance of the mass fractions.
RTOL = 1e-10
Y_FLOOR = 1e-10


def parity_error(gpu, ref, y_floor=Y_FLOOR):
    """max over entries of |gpu - ref| / max(|ref|, floor) (floor only for Y)."""
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    scale = np.abs(ref).copy()
    scale[..., :-1] = np.maximum(scale[..., :-1], y_floor)
    return float(np.max(np.abs(gpu - ref) / scale)) if gpu.size else 0.0


def assert_parity(gpu, ref, rtol=RTOL, y_floor=Y_FLOOR, what=""):
    err = parity_error(gpu, ref, y_floor)
    assert err <= rtol, f"{what} parity error {err:.3e} > {rtol:.1e}"
    return err
