"""Batches of uneven volumes through grouped persistent launches (sfw_batch).

Each volume's loss, gradient, residual and grid argmax from one batch step must equal the
single-volume calls on the same inputs (same kernels, same descriptors: bit-identical), and a
volume of the batch is checked against the FP64 oracle (1e-5 loss, 1e-4 gradient, argmax).
The batch step is also replayed from a captured CUDA graph.
"""

import numpy as np
import pytest

import sfw_inputs
from parity_util import assert_argmax

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_05473_gb300 as m
    m.build_library()
    return m


def _make(sfw, oracle_mod, shapes):
    import torch
    vols, plans, ys, atoms, lams = [], [], [], [], []
    for i, n in enumerate(shapes):
        rng = np.random.default_rng(500 + i)
        lat, ax = rng.uniform(1.2, 2.0), rng.uniform(2.5, 3.5)
        vol = sfw_inputs.make_volume(f"b{i}", n, sfw_inputs.ANISO_R, (lat, lat, ax), int(rng.integers(5, 12)),
                                     seed=600 + i, grid_sigmas=np.linspace(1, 3, 5), grid_ds=(1.5, 2.0, 2.5))
        y = np.asarray(oracle_mod.observe(vol, fft=True), np.float32)
        plan = sfw.Plan(vol.n, vol.R, vol.psf, vol.grid_sigmas, vol.grid_ds)
        est = sfw.AtomSet.from_numpy(vol.m + 0.3, vol.sigma * 1.05, np.clip(vol.d + 0.05, 1.3, 2.9), vol.w * 0.9)
        vols.append(vol); plans.append(plan); ys.append(torch.tensor(y, device="cuda")); atoms.append(est)
        lams.append(0.05 * float(np.abs(y).max()))
    return vols, plans, ys, atoms, lams


def test_batch_equals_single_calls_and_graph_replay(sfw, oracle_mod, tmp_path):
    import json
    import torch
    shapes = [(48, 48, 48), (64, 64, 64), (96, 96, 64), (48, 48, 48), (64, 64, 64)]
    vols, plans, ys, atoms, lams = _make(sfw, oracle_mod, shapes)
    batch = sfw.Batch(plans, ys, atoms, lams)
    # the autotuner only moves work between CTAs: results stay bit-identical
    cache = str(tmp_path / "tune.json")
    batch.autotune(cache)
    rec = json.load(open(cache))
    # persistent launches get a grid; the fixed-shape ones (zeroing, finalisers) keep 0
    assert len(rec["grids"]) == batch.launches_per_step
    assert all(g >= 0 for g in rec["grids"]) and sum(g >= 1 for g in rec["grids"]) >= batch.launches_per_step // 2
    batch.autotune(cache)   # read back from the cache
    batch.step()
    torch.cuda.synchronize()
    print(f"\n[batch] {len(plans)} volumes, {batch.launches_per_step} grouped launches per step")
    assert batch.launches_per_step < 21 * len(plans)
    for v in range(len(plans)):
        loss, grad, r = plans[v].slide_loss_grad(ys[v], atoms[v], lams[v], want_residual=True)
        c = plans[v].certificate(r, lams[v], want_max=False)
        assert batch.loss[v].item() == loss.item()
        assert torch.equal(batch.grad[v], grad)
        assert torch.equal(batch.residual[v], r)
        assert batch.best_idx[v].item() == c["best_idx"].item()
        # a batch records the per-axis certificate passes; a single call on a 64- or
        # 128-point certificate grid runs the slab kernels, whose register transforms
        # round differently from the shared-memory ones (a few FP32 ulp)
        if plans[v].info["P_cert"][1] in (64, 128) and plans[v].info["P_cert"][2] in (64, 128):
            assert abs(batch.best_val[v].item() - c["best_val"].item()) <= 4e-7 * abs(c["best_val"].item())
        else:
            assert batch.best_val[v].item() == c["best_val"].item()
    # one volume against the FP64 oracle
    v = 1
    vol = vols[v]
    a = atoms[v]
    m, s, d, w = (x.double().cpu().numpy() for x in (a.m, a.sigma, a.d, a.w))
    y = ys[v].double().cpu().numpy()
    C, g, _ = oracle_mod.loss_and_grad(vol.n, vol.R, vol.psf, y, m, s, d, w, lams[v], fft=True)
    assert abs(batch.loss[v].item() - C) <= 1e-5 * abs(C)
    gg = batch.grad[v].cpu().numpy()
    assert np.max(np.abs(gg - g)) <= 1e-4 * np.max(np.abs(g))
    eta = oracle_mod.eta_grid_fft(vol.n, vol.R, vol.psf, batch.residual[v].double().cpu().numpy(), lams[v],
                                  vol.grid_kernels())
    assert batch.best_idx[v].item() == int(np.argmax(eta))
    # graph capture of the batch step reproduces the eager step
    ref_loss = batch.loss.clone()
    ref_idx = batch.best_idx.clone()
    graph = torch.cuda.CUDAGraph()
    s_cap = torch.cuda.Stream()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(graph, stream=s_cap):
            batch.step()
    batch.loss.zero_()
    batch.best_idx.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(batch.loss, ref_loss)
    assert torch.equal(batch.best_idx, ref_idx)


def test_batch_with_128_volume_and_bf16_plan(sfw, oracle_mod):
    """The largest member of the uneven batch (128^3) and a bf16-table plan in one batch: every
    volume equals its single calls (loss, gradient, residual bit-identical; grid argmax), and
    the 128^3 volume matches the FP64 oracle (loss 1e-5, gradient 1e-4, grid argmax)."""
    import torch
    shapes = [(128, 128, 128), (64, 64, 64), (48, 48, 48)]
    vols, plans, ys, atoms, lams = _make(sfw, oracle_mod, shapes)
    vb = vols[1]
    plans[1].close()
    plans[1] = sfw.Plan(vb.n, vb.R, vb.psf, vb.grid_sigmas, vb.grid_ds, precision="bf16")
    batch = sfw.Batch(plans, ys, atoms, lams)
    batch.step()
    torch.cuda.synchronize()
    for v in range(len(plans)):
        loss, grad, r = plans[v].slide_loss_grad(ys[v], atoms[v], lams[v], want_residual=True)
        c = plans[v].certificate(r, lams[v], want_max=False)
        assert batch.loss[v].item() == loss.item()
        assert torch.equal(batch.grad[v], grad)
        assert torch.equal(batch.residual[v], r)
        if plans[v].info["tensor_cores"]:
            # a batch records the FFT passes on the bf16 table; a single call on a bf16 plan
            # runs the axis-0 stage on the tensor cores: both carry bf16 rounding
            assert abs(batch.best_val[v].item() - c["best_val"].item()) <= 1e-2 * abs(c["best_val"].item())
        else:
            assert batch.best_idx[v].item() == c["best_idx"].item()
    v = 0
    vol = vols[v]
    a = atoms[v]
    m, s, d, w = (x.double().cpu().numpy() for x in (a.m, a.sigma, a.d, a.w))
    y = ys[v].double().cpu().numpy()
    C, g, _ = oracle_mod.loss_and_grad(vol.n, vol.R, vol.psf, y, m, s, d, w, lams[v], fft=True)
    assert abs(batch.loss[v].item() - C) <= 1e-5 * abs(C)
    gg = batch.grad[v].cpu().numpy()
    assert np.max(np.abs(gg - g)) <= 1e-4 * np.max(np.abs(g))
    eta = oracle_mod.eta_grid_fft(vol.n, vol.R, vol.psf, batch.residual[v].double().cpu().numpy(), lams[v],
                                  vol.grid_kernels())
    assert_argmax(int(batch.best_idx[v].item()), eta, 1e-5 * np.max(np.abs(eta)))
    batch.close()
    for p in plans:
        p.close()
