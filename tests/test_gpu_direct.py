"""GPU parity of the plain FP32 route (SFW_ROUTE_DIRECT: direct sums, no transform) against the
FP64 oracle, and of the route choice (SFW_ROUTE_AUTO + sfw_autotune).

Same tolerances as the transform route: 1e-5 of the largest magnitude for the forward operator,
every grid certificate value and the loss; the grid argmax as the exact flat index k V + lin(m)
(unless the oracle's two best candidates are closer than the tolerance, which is printed);
gradient 1e-4 overall."""

import numpy as np
import pytest

import sfw_inputs
from parity_util import assert_argmax

pytestmark = pytest.mark.gpu

RTOL = 1e-5

CASES = [
    ((13, 17, 22), (2, 3, 4), (1.1, 1.3, 1.8), 3),
    ((9, 20, 11), (1, 4, 2), (0.9, 1.7, 1.2), 4),
    ((24, 24, 24), (3, 3, 6), (1.5, 1.5, 3.0), 5),
]


def _rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def sfw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_05473_gb300 as m
    m.build_library()
    return m


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _case(oracle_mod, n, R, psf_sigma, N, seed=0, asym=True):
    vol = sfw_inputs.make_volume("t", n, R, psf_sigma, N, seed=seed, grid_sigmas=(1.0, 2.0, 3.0),
                                 grid_ds=(1.5, 2.0, 2.5), min_sep=2.0)
    if asym:
        rng = np.random.default_rng(seed + 100)
        psf = vol.psf * (1.0 + 0.3 * rng.random(vol.psf.shape))
        vol.psf = psf / psf.sum()
    return vol, oracle_mod.observe(vol, fft=False)


@pytest.mark.parametrize("case", CASES)
def test_direct_forward_matches_oracle(sfw, oracle_mod, case):
    n, R, ps, N = case
    vol, _ = _case(oracle_mod, n, R, ps, N)
    plan = sfw.Plan(n, R, vol.psf, route="direct")
    assert plan.info["route_blur"] == "direct"
    atoms = sfw.AtomSet.from_numpy(vol.m, vol.sigma, vol.d, vol.w)
    y = plan.forward(atoms).cpu().numpy()
    ref = oracle_mod.forward(n, R, vol.psf, vol.m, vol.sigma, vol.d, vol.w)
    assert _rel_inf(y, ref) <= RTOL
    plan.close()


@pytest.mark.parametrize("case", CASES)
def test_direct_certificate_matches_definition(sfw, oracle_mod, torch_mod, case):
    """eta_k(m) by direct sums == Eq. 5 at every voxel (faces included) and kernel; the grid
    argmax, the per-voxel max and argk; and the same values as the transform route."""
    n, R, ps, N = case
    vol, y = _case(oracle_mod, n, R, ps, N)
    kernels = vol.grid_kernels()
    lam = oracle_mod.lambda_rule(n, R, vol.psf, y, kernels, fft=False)
    r = y - oracle_mod.forward(n, R, vol.psf, vol.m[:1], vol.sigma[:1], vol.d[:1], vol.w[:1])
    r32 = r.astype(np.float32)
    plan = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="direct")
    assert plan.info["route_cert"] == "direct" and plan.info["table_bytes"] == 0
    rt = torch_mod.tensor(r32, device="cuda")
    out = plan.certificate(rt, lam, want_eta=True)
    eta = out["eta"].cpu().numpy()
    ref = oracle_mod.eta_grid(n, R, vol.psf, r32.astype(np.float64), lam, kernels)
    assert _rel_inf(eta, ref) <= RTOL
    assert int(out["best_idx"].item()) == int(np.argmax(eta))
    assert_argmax(int(out["best_idx"].item()), ref, RTOL * np.abs(ref).max())
    np.testing.assert_array_equal(out["max"].cpu().numpy(), eta.max(axis=0))
    np.testing.assert_array_equal(out["argk"].cpu().numpy(), eta.argmax(axis=0))
    fft = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="fft")
    eta_f = fft.certificate(rt, lam, want_eta=True)["eta"].cpu().numpy()
    assert _rel_inf(eta, eta_f) <= 2 * RTOL
    plan.close()
    fft.close()


@pytest.mark.parametrize("case", CASES)
def test_direct_slide_loss_grad_matches_oracle(sfw, oracle_mod, torch_mod, case):
    n, R, ps, N = case
    vol, y = _case(oracle_mod, n, R, ps, N)
    lam = 0.37
    rng = np.random.default_rng(7)
    m = vol.m + rng.normal(0, 0.3, vol.m.shape)
    s = vol.sigma * 1.1
    d = np.clip(vol.d + 0.1, 1.3, 2.9)
    w = vol.w * 0.9
    plan = sfw.Plan(n, R, vol.psf, route="direct")
    atoms = sfw.AtomSet.from_numpy(m, s, d, w)
    m32, s32, d32, w32 = (np.asarray(a, np.float32).astype(np.float64) for a in (m, s, d, w))
    y32 = y.astype(np.float32).astype(np.float64)
    C, g, r = oracle_mod.loss_and_grad(n, R, vol.psf, y32, m32, s32, d32, w32, lam)
    loss, grad, res = plan.slide_loss_grad(torch_mod.tensor(y32, dtype=torch_mod.float32, device="cuda"),
                                           atoms, lam, want_residual=True)
    assert abs(loss.item() - C) <= RTOL * abs(C)
    assert _rel_inf(res.cpu().numpy(), r) <= RTOL * 10
    assert _rel_inf(grad.cpu().numpy(), g) <= 1e-4
    plan.close()


def test_direct_eta_points_and_step(sfw, oracle_mod, torch_mod):
    """Off-grid eta on the direct back-projection, and sfw_step on a DIRECT plan equal to its two
    separate calls (loss, gradient, residual, grid argmax)."""
    n, R, ps, N = CASES[0]
    vol, y = _case(oracle_mod, n, R, ps, N)
    plan = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="direct")
    th = np.concatenate([vol.m + 0.37, (vol.sigma * 0.9)[:, None], (vol.d * 1.05)[:, None]], 1)
    y32 = y.astype(np.float32).astype(np.float64)
    th32 = th.astype(np.float32).astype(np.float64)
    b = oracle_mod.backproject(n, R, vol.psf, y32)
    e_ref, g_ref = oracle_mod.eta_points(n, R, b, 0.5, th32, with_grad=True)
    yt = torch_mod.tensor(y32, dtype=torch_mod.float32, device="cuda")
    e, g = plan.eta_points(yt, 0.5, th)
    assert _rel_inf(e.cpu().numpy(), e_ref) <= RTOL
    assert _rel_inf(g.cpu().numpy(), g_ref) <= 1e-4
    atoms = sfw.AtomSet.from_numpy(vol.m + 0.2, vol.sigma, vol.d, vol.w * 0.8)
    aux = torch_mod.cuda.Stream()
    st = plan.step(yt, atoms, 0.3, aux_stream=aux)
    loss, grad, res = plan.slide_loss_grad(yt, atoms, 0.3, want_residual=True)
    cert = plan.certificate(res, 0.3, want_max=False)
    torch_mod.cuda.synchronize()
    assert st["loss"].item() == loss.item()
    assert torch_mod.equal(st["grad"], grad) and torch_mod.equal(st["residual"], res)
    assert st["best_idx"].item() == cert["best_idx"].item()
    assert st["best_val"].item() == cert["best_val"].item()
    plan.close()


def test_auto_route_autotune_and_cache(sfw, oracle_mod, torch_mod, tmp_path):
    """An AUTO plan builds both routes; sfw_autotune picks one per operation, writes the choice
    to the cache and a second plan of the same geometry reads it back; results stay those of
    the oracle whichever route runs."""
    n, R, ps, N = CASES[2]
    vol, y = _case(oracle_mod, n, R, ps, N, asym=False)
    cache = str(tmp_path / "routes.txt")
    plan = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="auto")
    assert plan.info["route_blur"] == "fft" and plan.info["route_cert"] == "fft"
    assert plan.info["table_bytes"] > 0
    routes = plan.autotune(cache)
    assert routes["blur"] in ("fft", "direct") and routes["cert"] in ("fft", "direct")
    text = open(cache).read()
    assert text.count("|") == 1
    again = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="auto")
    assert again.autotune(cache) == routes
    assert open(cache).read() == text     # read back, not timed again
    kernels = vol.grid_kernels()
    lam = oracle_mod.lambda_rule(n, R, vol.psf, y, kernels, fft=False)
    y32 = y.astype(np.float32)
    out = plan.certificate(torch_mod.tensor(y32, device="cuda"), lam, want_eta=True)
    ref = oracle_mod.eta_grid(n, R, vol.psf, y32.astype(np.float64), lam, kernels)
    assert _rel_inf(out["eta"].cpu().numpy(), ref) <= RTOL
    fixed = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="fft")
    fr = fixed.autotune(cache)
    assert (fr["blur"], fr["cert"], fr["tensor_cores"]) == ("fft", "fft", False)   # nothing to choose
    for p in (plan, again, fixed):
        p.close()


def test_direct_plan_rejected_by_batches(sfw, oracle_mod, torch_mod):
    n, R, ps, N = CASES[1]
    vol, y = _case(oracle_mod, n, R, ps, N)
    plan = sfw.Plan(n, R, vol.psf, vol.grid_sigmas, vol.grid_ds, route="direct")
    yt = torch_mod.tensor(y, dtype=torch_mod.float32, device="cuda")
    atoms = sfw.AtomSet.from_numpy(vol.m, vol.sigma, vol.d, vol.w)
    with pytest.raises(sfw.SfwError) as e:
        sfw.Batch([plan], [yt], [atoms], [0.5])
    assert e.value.status == 7
    plan.close()
