"""Shared checks of the GPU parity tests."""

import numpy as np


def assert_argmax(got: int, ref, tol: float) -> None:
    """The GPU's grid maximum must be the oracle's exact flat index (ties -> lowest index).  The
    one exception is an FP32 near-tie: when the oracle's two best candidates lie within tol of
    each other, FP32 rounding may order them the other way; the gap is printed (pytest -s) and
    the GPU's pick must then be within tol of the maximum."""
    flat = np.asarray(ref).ravel()
    best = int(np.argmax(flat))
    if got == best:
        return
    gap = float(flat[best] - np.partition(flat, -2)[-2])
    print(f"argmax near-tie: gpu index {got}, oracle index {best}, oracle top-2 gap {gap:.3e}, tol {tol:.3e}")
    assert gap <= tol, f"argmax {got} != oracle {best} with top-2 gap {gap:.3e} > {tol:.3e}"
    assert 0 <= got < flat.size and float(flat[best] - flat[got]) <= tol
