"""Seeded input generators shared by the oracle and the GPU path (no arithmetic of the
method lives there): the non-separable PSF stand-in."""

import numpy as np

import sfw_inputs


def test_tilted_psf_reduces_to_axis_aligned_gaussian():
    R = (4, 5, 6)
    a = sfw_inputs.tilted_gaussian_psf((1.2, 1.7, 2.5), R, (0.0, 0.0))
    b = sfw_inputs.gaussian_psf((1.2, 1.7, 2.5), R)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)


def test_tilted_psf_moments_and_symmetry():
    sig, ang = (1.0, 1.5, 2.0), (0.5, 0.3)
    R = (12, 14, 16)   # wide enough for the second moments of a sampled Gaussian
    h = sfw_inputs.tilted_gaussian_psf(sig, R, ang)
    assert abs(h.sum() - 1.0) < 1e-12
    np.testing.assert_allclose(h, h[::-1, ::-1, ::-1], rtol=1e-12, atol=1e-18)
    x = np.stack(np.meshgrid(*[np.arange(-r, r + 1, dtype=np.float64) for r in R], indexing="ij"), -1)
    cov = np.einsum("abci,abcj,abc->ij", x, x, h)
    a, b = ang
    r0 = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
    r1 = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    q = r1 @ r0
    np.testing.assert_allclose(cov, q @ np.diag(np.square(sig)) @ q.T, atol=2e-3)
    # not separable: the mode-0 unfolding has rank > 1
    sv = np.linalg.svd(h.reshape(h.shape[0], -1), compute_uv=False)
    assert sv[1] > 0.05 * sv[0]
