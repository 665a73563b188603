"""Pins of the FP64 oracle against facts other than itself (CPU only).

Each test names the equation or section of the paper whose definition it
checks, and pins it with a closed form, an invariant, a library routine or
brute force, so that a dropped term, a wrong sign/index or a transposed
operand in the oracle fails at least one of them.
"""

import math

import numpy as np
import pytest
import scipy.optimize
import scipy.signal

import sfw_inputs


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- Eq. 2: the atom

def test_render_d2_is_separable_gaussian(oracle_mod):
    """d = 2: exp(-|x|^2/(2 sigma^2)) = product of three 1-D Gaussians (textbook identity)."""
    n, R = (9, 10, 11), (2, 1, 3)
    m = np.array([[4.3, 5.1, 4.7]])
    sig, d, w = np.array([1.7]), np.array([2.0]), np.array([1.3])
    f = oracle_mod.render(n, R, m, sig, d, w)
    axes = [np.exp(-(np.arange(n[a] + 2 * R[a]) - R[a] - m[0, a]) ** 2 / (2 * sig[0] ** 2))
            for a in range(3)]
    ref = w[0] * axes[0][:, None, None] * axes[1][None, :, None] * axes[2][None, None, :]
    np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d", [1.25, 1.5, 2.5, 3.0])
def test_render_level_sets(oracle_mod, d):
    """At rho = sigma every atom takes w e^{-1/2}; at rho = sigma 2^{1/d} it takes w e^{-1}."""
    n, R = (8, 8, 8), (1, 1, 1)
    m = np.array([[3.0, 4.0, 2.6]])       # E voxel (4,5,4) sits at grid (3,4,3): rho = 0.4
    rho = 0.4
    f1 = oracle_mod.render(n, R, m, np.array([rho]), np.array([d]), np.array([2.0]))
    f2 = oracle_mod.render(n, R, m, np.array([rho / 2 ** (1 / d)]), np.array([d]), np.array([2.0]))
    assert f1[4, 5, 4] == pytest.approx(2.0 * math.exp(-0.5), rel=1e-14)
    assert f2[4, 5, 4] == pytest.approx(2.0 * math.exp(-1.0), rel=1e-14)
    # the atom peaks at w when a voxel sits on m, whatever sigma and d
    f3 = oracle_mod.render(n, R, np.array([[3.0, 4.0, 3.0]]), np.array([1.1]), np.array([d]),
                           np.array([0.7]))
    assert f3[4, 5, 4] == pytest.approx(0.7, rel=1e-15)
    assert f3.max() == pytest.approx(0.7, rel=1e-15)


def test_render_is_linear_in_atoms(oracle_mod):
    """The measure mu is a weighted sum of Diracs: rendering two atoms = sum of each (Eq. 3)."""
    n, R = (7, 6, 5), (1, 2, 1)
    rng = _rng(1)
    m, s, d, w = sfw_inputs.random_atoms(rng, n, 2, margin=1)
    both = oracle_mod.render(n, R, m, s, d, w)
    one = oracle_mod.render(n, R, m[:1], s[:1], d[:1], w[:1])
    two = oracle_mod.render(n, R, m[1:], s[1:], d[1:], w[1:])
    np.testing.assert_allclose(both, one + two, rtol=1e-14, atol=1e-16)


# ---------------------------------------------------------------- Eq. 3: blur on the grid

def test_forward_conv_matches_scipy_valid_convolution(oracle_mod):
    """Brute-force blur == scipy.signal.convolve(f, H, 'valid') for a random, asymmetric H."""
    n, R = (6, 7, 8), (2, 1, 3)
    rng = _rng(2)
    f = rng.standard_normal(tuple(a + 2 * r for a, r in zip(n, R)))
    H = rng.random(tuple(2 * r + 1 for r in R))
    y = oracle_mod.forward_conv(n, R, H, f)
    ref = scipy.signal.convolve(f, H, mode="valid", method="direct")
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_backproject_matches_scipy_full_correlation(oracle_mod):
    """Back-projection == full convolution of r with the flipped H (the transpose of 'valid')."""
    n, R = (6, 5, 7), (1, 2, 2)
    rng = _rng(3)
    r = rng.standard_normal(n)
    H = rng.random(tuple(2 * q + 1 for q in R))
    b = oracle_mod.backproject(n, R, H, r)
    ref = scipy.signal.convolve(r, H[::-1, ::-1, ::-1], mode="full", method="direct")
    np.testing.assert_allclose(b, ref, rtol=1e-12, atol=1e-12)


def test_adjoint_identity_fp64(oracle_mod):
    """<Phi f, r> = <f, Phi^T r> for random f on E and r on the grid (Eq. 5's transpose)."""
    n, R = (9, 8, 10), (2, 3, 1)
    rng = _rng(4)
    f = rng.standard_normal(tuple(a + 2 * q for a, q in zip(n, R)))
    r = rng.standard_normal(n)
    H = rng.random(tuple(2 * q + 1 for q in R))
    lhs = float(np.sum(oracle_mod.forward_conv(n, R, H, f) * r))
    rhs = float(np.sum(f * oracle_mod.backproject(n, R, H, r)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_forward_closed_form_variances_add(oracle_mod):
    """d = 2 atom through a Gaussian PSF: a Gaussian of variance sigma^2 + sigma_H^2 per axis,
    amplitude w prod sqrt(sigma^2/(sigma^2+sigma_H^2)) (the sampled sums approach the integrals
    to ~exp(-2 pi^2 sigma_eff^2); the PSF is truncated at 7 sigma_H)."""
    sh = (2.0, 2.0, 2.5)
    R = (14, 14, 18)
    n = (20, 20, 22)
    H = sfw_inputs.gaussian_psf(sh, R)
    m = np.array([[9.6, 10.2, 10.9]])
    sig = 2.2
    y = oracle_mod.forward(n, R, H, m, np.array([sig]), np.array([2.0]), np.array([1.4]))
    grid = np.indices(n).astype(np.float64)
    v = np.array([sig ** 2 + s ** 2 for s in sh])
    amp = 1.4 * np.prod(np.sqrt(sig ** 2 / v))
    ref = amp * np.exp(-sum((grid[a] - m[0, a]) ** 2 / (2 * v[a]) for a in range(3)))
    np.testing.assert_allclose(y, ref, rtol=1e-8, atol=1e-12 * amp)


def test_fft_variants_equal_direct_sums(oracle_mod):
    """The Fourier-domain blur/back-projection (library FFT) equal the direct sums."""
    n, R = (10, 9, 12), (2, 3, 4)
    rng = _rng(5)
    H = rng.random(tuple(2 * q + 1 for q in R))
    f = rng.standard_normal(tuple(a + 2 * q for a, q in zip(n, R)))
    r = rng.standard_normal(n)
    np.testing.assert_allclose(oracle_mod.forward_fft(n, R, H, f), oracle_mod.forward_conv(n, R, H, f),
                               rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(oracle_mod.backproject_fft(n, R, H, r), oracle_mod.backproject(n, R, H, r),
                               rtol=1e-10, atol=1e-11)


# ---------------------------------------------------------------- Eq. 4 and its gradient

def _small_problem(seed=6, N=2, n=(12, 11, 13), R=(2, 2, 3)):
    rng = _rng(seed)
    H = sfw_inputs.gaussian_psf((1.2, 1.0, 1.6), R)
    m, s, d, w = sfw_inputs.random_atoms(rng, n, N, margin=3)
    y = rng.standard_normal(n) * 0.3 + 0.2
    return n, R, H, y, m, s, d, w


def test_gradient_matches_central_differences(oracle_mod):
    """Analytic dC/d(m, sigma, d, w) (Section 2) == FP64 central differences of Eq. 4."""
    n, R, H, y, m, s, d, w = _small_problem()
    lam = 0.37
    C, g, _ = oracle_mod.loss_and_grad(n, R, H, y, m, s, d, w, lam)
    x0 = oracle_mod.pack_params(np.concatenate([m, s[:, None], d[:, None]], 1), w)
    h = 1e-5
    fd = np.zeros_like(x0)
    for i in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        xp[i] += h
        xm[i] -= h
        tp, wp = oracle_mod.unpack_params(xp)
        tm, wm = oracle_mod.unpack_params(xm)
        cp = oracle_mod.criterion(n, R, H, y, tp[:, :3], tp[:, 3], tp[:, 4], wp, lam)
        cm = oracle_mod.criterion(n, R, H, y, tm[:, :3], tm[:, 3], tm[:, 4], wm, lam)
        fd[i] = (cp - cm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7 * np.max(np.abs(fd)))


def test_gradient_w_equals_lambda_times_one_minus_eta(oracle_mod):
    """From Eqs. 4-5: dC/dw_n = lambda (1 - eta(theta_n)); ties the gradient to the certificate."""
    n, R, H, y, m, s, d, w = _small_problem(seed=7, N=3)
    lam = 0.21
    _, g, r = oracle_mod.loss_and_grad(n, R, H, y, m, s, d, w, lam)
    b = oracle_mod.backproject(n, R, H, r)
    eta = oracle_mod.eta_points(n, R, b, lam, np.concatenate([m, s[:, None], d[:, None]], 1))
    N = w.size
    np.testing.assert_allclose(g[5 * N:], lam * (1.0 - eta), rtol=1e-11, atol=1e-13)


def test_criterion_at_zero_measure(oracle_mod):
    """mu = 0: C = |y|^2 / 2 (Eq. 4 with an empty sum)."""
    n, R = (5, 6, 7), (1, 1, 1)
    y = _rng(8).standard_normal(n)
    H = sfw_inputs.gaussian_psf((1.0, 1.0, 1.0), R)
    C = oracle_mod.criterion(n, R, H, y, np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros(0), 0.5)
    assert C == pytest.approx(0.5 * float(np.sum(y * y)), rel=1e-15)


def test_eta_gradient_matches_central_differences(oracle_mod):
    """d eta / d theta used by the step-1 ascent == central differences of eta (Eq. 5)."""
    n, R, H, y, m, s, d, w = _small_problem(seed=9, N=1)
    b = oracle_mod.backproject(n, R, H, y)
    th = np.array([5.3, 4.6, 6.2, 1.7, 1.8])
    e, g = oracle_mod.eta_points(n, R, b, 0.4, th[None], with_grad=True)
    h = 1e-5
    for i in range(5):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle_mod.eta_points(n, R, b, 0.4, tp[None])[0] - oracle_mod.eta_points(n, R, b, 0.4, tm[None])[0]) / (2 * h)
        assert g[0, i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- Eq. 5: the certificate

def test_certificate_closed_form_gaussian_overlap(oracle_mod):
    """mu = 0, y = Phi G(theta*, w*), d = 2 and a Gaussian PSF: <Phi g_theta, Phi g*> is the
    integral of two Gaussians of variances v = sigma^2 + sigma_H^2 (far from the faces)."""
    sh = (1.5, 1.5, 1.5)
    R = (11, 11, 11)
    n = (34, 34, 34)
    H = sfw_inputs.gaussian_psf(sh, R)
    ms = np.array([[16.4, 17.1, 16.8]])
    ss, ws = 2.0, 1.3
    y = oracle_mod.forward(n, R, H, ms, np.array([ss]), np.array([2.0]), np.array([ws]))
    b = oracle_mod.backproject(n, R, H, y)
    lam = 0.5
    thetas = np.array([[16.0, 17.0, 17.0, 1.5, 2.0], [15.0, 18.0, 16.0, 2.5, 2.0],
                       [17.4, 16.1, 17.8, 1.2, 2.0]])
    eta = oracle_mod.eta_points(n, R, b, lam, thetas)
    for th, e in zip(thetas, eta):
        val = ws / lam
        for a in range(3):
            v1 = th[3] ** 2 + sh[a] ** 2
            v2 = ss ** 2 + sh[a] ** 2
            val *= (th[3] / math.sqrt(v1)) * (ss / math.sqrt(v2)) * math.sqrt(2 * math.pi * v1 * v2 / (v1 + v2)) \
                * math.exp(-(th[a] - ms[0, a]) ** 2 / (2 * (v1 + v2)))
        assert e == pytest.approx(val, rel=1e-7)


def test_eta_grid_fft_equals_direct_definition(oracle_mod):
    """Grid certificate through the library FFT == the direct definition, faces included."""
    n, R = (8, 9, 7), (2, 1, 3)
    rng = _rng(10)
    H = rng.random(tuple(2 * q + 1 for q in R))
    H /= H.sum()
    r = rng.standard_normal(n)
    kernels = [(1.0, 2.0), (2.3, 1.5), (1.6, 2.7)]
    e1 = oracle_mod.eta_grid(n, R, H, r, 0.3, kernels)
    e2 = oracle_mod.eta_grid_fft(n, R, H, r, 0.3, kernels)
    np.testing.assert_allclose(e2, e1, rtol=1e-10, atol=1e-10 * np.abs(e1).max())


def test_eta_of_unit_atom_is_its_own_energy(oracle_mod):
    """r = Phi G(theta, 1): eta(theta) = |Phi G(theta,1)|^2 / lambda (Cauchy-Schwarz maximum)."""
    n, R = (10, 10, 10), (2, 2, 2)
    H = sfw_inputs.gaussian_psf((1.1, 1.1, 1.4), R)
    th = np.array([4.6, 5.2, 4.9, 1.4, 1.7])
    a = oracle_mod.forward(n, R, H, th[None, :3], th[3:4], th[4:5], np.ones(1))
    b = oracle_mod.backproject(n, R, H, a)
    e = oracle_mod.eta_points(n, R, b, 2.0, th[None])[0]
    assert e == pytest.approx(float(np.sum(a * a)) / 2.0, rel=1e-12)


def test_grid_thetas_flat_order(oracle_mod):
    """Grid candidates (Algorithm 1 step 1) in flat order k*V + lin(m): row i is the voxel
    numpy's unravel_index gives for i mod V and kernel i div V."""
    n = (3, 4, 5)
    kernels = [(1.0, 2.0), (2.5, 1.5), (1.7, 2.9)]
    G = oracle_mod.grid_thetas(n, kernels)
    V = int(np.prod(n))
    assert G.shape == (len(kernels) * V, 5)
    for i in (0, 1, 4, 5, 19, 20, V - 1, V, V + 37, 2 * V + 58, 3 * V - 1):
        k, v = divmod(i, V)
        m = np.unravel_index(v, n)
        np.testing.assert_array_equal(G[i], [m[0], m[1], m[2], kernels[k][0], kernels[k][1]])


@pytest.mark.parametrize("fft", [False, True])
def test_lambda_rule_unit_atom_on_the_grid(oracle_mod, fft):
    """lambda = frac * max over the grid of Phi^T y (the reading of Section 3's lambda).  For
    y = Phi G(theta*, 1), theta* on the grid, one kernel: by Cauchy-Schwarz the maximum is at
    theta* and equals |y|^2, so the rule gives frac |y|^2, and the grid argmax is theta*."""
    n, R = (10, 11, 12), (2, 2, 3)
    H = sfw_inputs.gaussian_psf((1.1, 1.2, 1.6), R)
    kernels = [(1.2, 2.0)]
    m = np.array([[5.0, 5.0, 6.0]])
    y = oracle_mod.forward(n, R, H, m, np.array([1.2]), np.array([2.0]), np.ones(1))
    e = float(np.sum(y * y))
    assert oracle_mod.lambda_rule(n, R, H, y, kernels, frac=0.05, fft=fft) == pytest.approx(0.05 * e, rel=1e-9)
    assert oracle_mod.lambda_rule(n, R, H, y, kernels, frac=1.0, fft=fft) == pytest.approx(e, rel=1e-9)
    eta = (oracle_mod.eta_grid_fft if fft else oracle_mod.eta_grid)(n, R, H, y, 1.0, kernels)
    i, val = oracle_mod.grid_argmax(eta)
    assert i == int(np.ravel_multi_index((5, 5, 6), n))
    assert val == pytest.approx(e, rel=1e-9)


# ---------------------------------------------------------------- argmax (step 1 seed)

@pytest.mark.parametrize("shape", [(3, 8, 8, 8), (15, 12, 12, 12)])
def test_argmax_brute_force_with_ties(oracle_mod, shape):
    """Linear-scan argmax == numpy.argmax (first occurrence) with injected ties."""
    rng = _rng(11)
    v = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    flat = v.ravel()
    top = flat.max() + 1.0
    picks = rng.choice(flat.size, 5, replace=False)
    flat[picks] = top
    assert oracle_mod.argmax(v) == int(np.argmax(v)) == int(np.min(picks))
    flat[picks[0]] = np.nan
    assert oracle_mod.argmax(v) == -1


# ---------------------------------------------------------------- step 3: non-negative LASSO

def test_nnls_gram_matches_scipy_nnls_and_kkt(oracle_mod):
    rng = _rng(12)
    for trial in range(20):
        k = int(rng.integers(1, 9))
        M = rng.standard_normal((30, k))
        v = rng.standard_normal(30)
        A = M.T @ M
        q = M.T @ v
        w = oracle_mod.nnls_gram(A, q)
        w_ref, _ = scipy.optimize.nnls(M, v)
        np.testing.assert_allclose(w, w_ref, rtol=1e-8, atol=1e-10)
        grad = A @ w - q
        assert np.all(w >= 0)
        assert np.all(grad >= -1e-9)
        assert abs(float(w @ grad)) < 1e-9


def test_lasso_single_atom_closed_form(oracle_mod):
    """N = 1: w = max(0, (<a, y> - lambda) / |a|^2)."""
    n, R = (9, 9, 9), (2, 2, 2)
    H = sfw_inputs.gaussian_psf((1.0, 1.0, 1.5), R)
    th = np.array([[4.2, 4.1, 3.9, 1.3, 2.2]])
    rng = _rng(13)
    y = rng.standard_normal(n) + 2 * oracle_mod.forward(n, R, H, th[:, :3], th[:, 3], th[:, 4], np.ones(1))
    a = oracle_mod.forward(n, R, H, th[:, :3], th[:, 3], th[:, 4], np.ones(1)).ravel()
    for lam in (0.1, 1.0, 1e3):
        w = oracle_mod.lasso_weights(n, R, H, y, th, lam)
        assert w[0] == pytest.approx(max(0.0, (a @ y.ravel() - lam) / (a @ a)), rel=1e-10, abs=1e-14)


# ---------------------------------------------------------------- BFGS (steps 1 and 4)

def test_projected_bfgs_box_quadratic(oracle_mod):
    rng = _rng(14)
    M = rng.standard_normal((6, 6))
    A = M @ M.T + 0.5 * np.eye(6)
    c = rng.standard_normal(6) * 3
    lo, hi = -0.2 * np.ones(6), 0.3 * np.ones(6)
    x, f, _ = oracle_mod.projected_bfgs(lambda x: (0.5 * x @ A @ x - c @ x, A @ x - c), np.zeros(6),
                                        lo, hi, gtol=1e-10, max_iter=500)
    ref = scipy.optimize.minimize(lambda x: 0.5 * x @ A @ x - c @ x, np.zeros(6), jac=lambda x: A @ x - c,
                                  bounds=list(zip(lo, hi)), method="L-BFGS-B",
                                  options={"ftol": 1e-15, "gtol": 1e-12}).x
    np.testing.assert_allclose(x, ref, atol=1e-6)


def test_projected_bfgs_rosenbrock(oracle_mod):
    def fun(x):
        f = (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2
        g = np.array([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2), 200 * (x[1] - x[0] ** 2)])
        return f, g
    x, f, _ = oracle_mod.projected_bfgs(fun, np.array([-1.2, 1.0]), np.array([-5.0, -5.0]),
                                        np.array([5.0, 5.0]), gtol=1e-9, max_iter=500)
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-5)


# ---------------------------------------------------------------- Algorithms 1 and 2

def _noise_free_single_atom():
    n, R = (16, 16, 16), (3, 3, 3)
    H = sfw_inputs.gaussian_psf((1.2, 1.2, 1.2), R)
    th = np.array([[7.3, 8.4, 7.8, 1.6, 2.0]])
    return n, R, H, th


def test_sfw_single_atom_noise_free(oracle_mod):
    """Noise-free, one atom: SFW adds one atom, then stops with max eta <= 1 + tau and, at the
    recovered atom, eta = 1 and grad eta = 0 (the optimality conditions of the BLASSO)."""
    n, R, H, th = _noise_free_single_atom()
    y = oracle_mod.forward(n, R, H, th[:, :3], th[:, 3], th[:, 4], np.array([1.0]))
    kernels = [(1.0, 2.0), (2.0, 2.0), (3.0, 2.0)]
    lam = oracle_mod.lambda_rule(n, R, H, y, kernels, frac=0.01)
    out = oracle_mod.sfw(n, R, H, y, lam, kernels)
    assert out["w"].size == 1
    assert len(out["history"]) == 2          # one atom added, then the stopping test
    assert out["history"][-1]["eta_max"] <= 1 + oracle_mod.TAU
    est = out["thetas"]
    r = y - oracle_mod.forward(n, R, H, est[:, :3], est[:, 3], est[:, 4], out["w"])
    b = oracle_mod.backproject(n, R, H, r)
    e, g = oracle_mod.eta_points(n, R, b, lam, est, with_grad=True)
    assert e[0] == pytest.approx(1.0, abs=1e-5)
    lo, hi = oracle_mod.domain_bounds(n)
    # KKT on the box D: the projected ascent direction vanishes
    pg = est[0] - np.clip(est[0] + g[0], lo, hi)
    assert np.max(np.abs(pg)) < 1e-3
    np.testing.assert_allclose(est[0, :3], th[0, :3], atol=0.02)


def test_bsfw_reaches_sfw_criterion(oracle_mod):
    """Section 3: BSFW reaches almost the same criterion as SFW (here: two separated atoms)."""
    n, R = (18, 18, 18), (3, 3, 3)
    H = sfw_inputs.gaussian_psf((1.2, 1.2, 1.6), R)
    th = np.array([[5.2, 6.1, 6.3, 1.4, 2.0], [12.4, 11.3, 11.8, 1.9, 1.7]])
    w = np.array([1.0, 0.8])
    y = oracle_mod.forward(n, R, H, th[:, :3], th[:, 3], th[:, 4], w)
    y = y + 0.01 * y.max() * _rng(15).standard_normal(n)
    kernels = [(s, dd) for s in (1.0, 2.0, 3.0) for dd in (1.5, 2.0, 2.5)]
    lam = oracle_mod.lambda_rule(n, R, H, y, kernels)
    a = oracle_mod.sfw(n, R, H, y, lam, kernels)
    b = oracle_mod.bsfw(n, R, H, y, lam, kernels)
    assert a["w"].size == 2
    assert b["w"].size >= 2
    assert b["C"] == pytest.approx(a["C"], rel=2e-3)
