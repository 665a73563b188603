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


def test_workload_recipes():
    """Each named workload has the shape, PSF support, atom count, kernel grid and noise
    level its name and the input recipe give; atoms lie inside the margin, at least the
    minimum separation apart, with parameters in their drawing ranges; PSFs sum to 1."""
    import numpy as np
    expect = {"vol32_iso9_n3_k3": ((32, 32, 32), (9, 9, 9), 3, 3, 0.01),
              "vol64_aniso_n10_k15": ((64, 64, 64), (15, 15, 31), 10, 15, 0.02),
              "vol64_tilted_n10_k15": ((64, 64, 64), (15, 15, 31), 10, 15, 0.02),
              "vol128_aniso_n30_k32": ((128, 128, 128), (15, 15, 31), 30, 32, 0.02),
              "vol256x256x64_n100": ((256, 256, 64), (15, 15, 31), 100, 15, 0.02)}
    for name, make in sfw_inputs.WORKLOADS.items():
        v = make(seed=0)
        n, psf_shape, N, K, noise = expect[name]
        assert v.n == n and v.psf.shape == psf_shape and v.N == N and len(v.grid_kernels()) == K
        assert v.noise_frac == noise and v.noise.shape == n
        assert abs(v.psf.sum() - 1.0) < 1e-12
        assert np.all(v.m >= sfw_inputs.MARGIN) and np.all(v.m <= np.array(n) - 1 - sfw_inputs.MARGIN)
        dist = np.linalg.norm(v.m[:, None, :] - v.m[None, :, :], axis=2) + np.eye(N) * 1e9
        assert dist.min() >= 4.0
        assert np.all((v.sigma >= 1.0) & (v.sigma <= 3.0)) and np.all((v.d >= 1.5) & (v.d <= 2.5))
        w_lo, w_hi = (0.2, 2.0) if name == "vol256x256x64_n100" else (0.5, 1.5)
        assert np.all((v.w >= w_lo) & (v.w <= w_hi))
        # the same seed gives the same volume; another seed another one
        assert np.array_equal(make(seed=0).m, v.m) and not np.array_equal(make(seed=1).m, v.m)


def test_uneven_batch_recipe():
    import numpy as np
    vols = sfw_inputs.batch_uneven(64)
    assert len(vols) == 64
    assert {v.n for v in vols} <= set(sfw_inputs.BATCH_SHAPES) and len({v.n for v in vols}) == 4
    assert all(5 <= v.N <= 40 for v in vols)
    assert all(1.2 <= v.psf_sigma[0] == v.psf_sigma[1] <= 2.0 and 2.5 <= v.psf_sigma[2] <= 3.5 for v in vols)
    assert all(len(v.grid_kernels()) == 15 for v in vols)
    assert np.array_equal(sfw_inputs.batch_volume(7).m, vols[7].m)
