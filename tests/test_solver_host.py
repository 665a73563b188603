"""Host FP64 pieces of the GPU solver loop (Algorithms 1 and 2), on the CPU.

nonneg_quadratic_min solves the LASSO of step 3 on the Gram system; box_bfgs drives the
sliding descent (step 4 / 2b) and the local ascent of the certificate (step 1).  Pins:
scipy's NNLS and the KKT conditions, the closed-form minimiser of a separable quadratic on a
box, and convergence on an objective whose values carry FP32 rounding (as the device loss
does) where a plain Armijo search stops early.
"""

import numpy as np
import pytest

from paper_2009_05473_gb300.solver import box_bfgs, nonneg_quadratic_min


def test_nonneg_quadratic_min_matches_nnls_and_kkt():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    A = rng.normal(size=(40, 12))
    b = rng.normal(size=40)
    G, q = A.T @ A, A.T @ b
    w = nonneg_quadratic_min(G, q)
    w_ref, _ = scipy_opt.nnls(A, b)
    np.testing.assert_allclose(w, w_ref, atol=1e-9)
    grad = G @ w - q
    assert (w >= 0).all()
    assert np.all(grad[w == 0] >= -1e-9)            # no descent into the free set
    np.testing.assert_allclose(grad[w > 0], 0.0, atol=1e-9)


def test_box_bfgs_separable_quadratic_closed_form():
    rng = np.random.default_rng(4)
    c = rng.normal(size=8) * 3
    a = rng.uniform(0.5, 4.0, size=8)
    lo, hi = -np.ones(8), np.ones(8)

    def fg(x):
        return float(0.5 * np.sum(a * (x - c) ** 2)), a * (x - c)

    x, _, _ = box_bfgs(fg, np.zeros(8), lo, hi, gtol=1e-10)
    np.testing.assert_allclose(x, np.clip(c, lo, hi), atol=1e-8)


def _rounded_quadratic(n, seed):
    """Ill-conditioned quadratic whose values carry the error of an FP32 sum over many
    terms: a deterministic, x-dependent perturbation of 2e-7 relative (not monotone along
    a search line), with the exact FP64 gradient."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    H = Q @ np.diag(np.logspace(0, 3, n)) @ Q.T
    xs = rng.uniform(-0.5, 0.5, size=n)
    f0 = 2.0
    mix = rng.normal(size=n) * 1e7

    def fg(x):
        d = x - xs
        f = f0 + 0.5 * d @ H @ d
        return float(f * (1.0 + 2e-7 * np.sin(mix @ x))), H @ d

    return fg, xs


def test_box_bfgs_converges_through_fp32_loss_rounding():
    n = 10
    fg, xs = _rounded_quadratic(n, 5)
    lo, hi = -np.ones(n), np.ones(n)
    x, _, _ = box_bfgs(fg, np.zeros(n), lo, hi, gtol=1e-7, max_iter=400)
    assert np.abs(fg(x)[1]).max() <= 1e-7
    np.testing.assert_allclose(x, xs, atol=1e-8)
    # the Armijo test alone cannot resolve the last decreases of an FP32 objective
    x_a, _, _ = box_bfgs(fg, np.zeros(n), lo, hi, gtol=1e-7, max_iter=400, f_rel_noise=0.0)
    assert np.abs(fg(x_a)[1]).max() > 1e-7
