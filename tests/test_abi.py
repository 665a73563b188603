"""The C-ABI library builds, loads and exports every entry point of include/sfw.h (CPU only:
no compute call is made without a GPU)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sfw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2009_05473_gb300.build import build
    return build()


def test_header_declares_the_hot_path():
    names = _declared()
    for n in ("sfw_forward", "sfw_certificate_grid", "sfw_argmax", "sfw_slide_loss_grad",
              "sfw_plan_create", "sfw_plan_destroy", "sfw_eta_points"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    import ctypes
    lib = ctypes.CDLL(built)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built):
    from paper_2009_05473_gb300 import _abi
    assert sorted(_abi.EXPORTS) == _declared()
    L = _abi.lib()
    assert _abi.sfw_version().startswith("sfw-gb300")
    assert _abi.sfw_launch_count() == 0


def test_build_targets_sm_103a_only():
    from paper_2009_05473_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_argument_checks_need_no_gpu(built):
    """Argument errors are reported before any CUDA call."""
    import ctypes
    from paper_2009_05473_gb300 import _abi
    with pytest.raises(_abi.SfwError) as e:
        _abi.sfw_plan_create(_abi.PlanDesc())          # n = 0: outside [4, 1024]
    assert e.value.status == 2
    with pytest.raises(_abi.SfwError) as e:
        _abi.sfw_argmax(0, 10, 1, 0, 0, 0)             # NULL pointers
    assert e.value.status == 1
    with pytest.raises(_abi.SfwError):
        _abi.sfw_slide_loss_grad(0, 0, _abi.Atoms(), 1.0, 0, 0, 0, 0)
    with pytest.raises(_abi.SfwError) as e:
        _abi.sfw_step_topk(0, 0, _abi.Atoms(), 1.0, 0, 0, 0, 64, 0, 0, 0, 0, 0, 0, 0)   # NULL plan
    assert e.value.status == 1
    # an unknown route is refused before any device work
    import numpy as np
    psf = np.full((3, 3, 3), 1.0 / 27, np.float32)
    d = _abi.PlanDesc()
    d.n[:] = [8, 8, 8]
    d.R[:] = [1, 1, 1]
    d.psf = psf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    d.route = 9
    with pytest.raises(_abi.SfwError) as e:
        _abi.sfw_plan_create(d)
    assert e.value.status == 1 and "route" in str(e.value)
    with pytest.raises(_abi.SfwError) as e:
        _abi.sfw_autotune(0, None, 0)                  # NULL plan
    assert e.value.status == 1
    assert _abi.sfw_launch_count() == 0


def _desc(np, ctypes, _abi, keep, **over):
    """A valid 8^3 plan description (3 x 2 certificate kernels), with fields replaced."""
    psf = np.full((3, 3, 3), 1.0 / 27, np.float32)
    sig = np.array(over.pop("sigmas", [1.0, 2.0, 3.0]), np.float32)
    ds = np.array(over.pop("ds", [1.5, 2.0]), np.float32)
    keep += [psf, sig, ds]
    d = _abi.PlanDesc()
    d.n[:] = over.pop("n", [8, 8, 8])
    d.R[:] = over.pop("R", [1, 1, 1])
    fp = ctypes.POINTER(ctypes.c_float)
    d.psf = psf.ctypes.data_as(fp)
    d.n_sigma, d.n_d = over.pop("n_sigma", sig.size), over.pop("n_d", ds.size)
    d.sigmas, d.ds = sig.ctypes.data_as(fp), ds.ctypes.data_as(fp)
    if over.pop("null_sigmas", False):
        d.sigmas = fp()
    for k, v in over.items():
        setattr(d, k, fp() if v is None else v)
    return d


@pytest.mark.parametrize("over,status,what", [
    (dict(n=[3, 8, 8]), 2, "n[0]"),
    (dict(n=[8, 8, 1025]), 2, "n[2]"),
    (dict(R=[1, -1, 1]), 2, "R[1]"),
    (dict(R=[65, 1, 1]), 2, "R[0]"),
    (dict(psf=None), 1, "psf"),
    (dict(n_sigma=-1), 1, "negative grid"),
    (dict(null_sigmas=True), 1, "grid arrays"),
    (dict(sigmas=[1.0] * 16, ds=[1.5] * 17), 2, "K=272"),
    (dict(sigmas=[0.2, 1.0, 2.0]), 1, "grid sigma"),
    (dict(ds=[1.5, 4.5]), 1, "grid d"),
    (dict(precision=2), 1, "precision"),
    (dict(eps=0.1), 1, "eps"),
    (dict(eps=-1e-3), 1, "eps"),
    (dict(n=[1024, 1024, 1024], sigmas=[1.0, 2.0, 3.0, 4.0], ds=[1.5]), 2, "2^32"),
])
def test_plan_description_errors(built, over, status, what):
    """Every range of the plan description that include/sfw.h documents is refused with the
    documented status before any CUDA call (no GPU needed)."""
    import ctypes
    import numpy as np
    from paper_2009_05473_gb300 import _abi
    keep = []
    d = _desc(np, ctypes, _abi, keep, **over)
    with pytest.raises(_abi.SfwError) as e:
        _abi.sfw_plan_create(d)
    assert e.value.status == status, str(e.value)
    assert what in str(e.value), str(e.value)
    assert _abi.sfw_launch_count() == 0


def test_batch_argument_errors(built):
    """sfw_batch_create refuses a count outside 1..1024 and a NULL plan before any CUDA call."""
    from paper_2009_05473_gb300 import _abi
    for plans, what in (([], "count"), ([None] * 1025, "count"), ([None], "plan 0 is NULL")):
        vols = [_abi.BatchVolume() for _ in plans]
        with pytest.raises(_abi.SfwError) as e:
            _abi.sfw_batch_create(plans, vols, [1.0] * len(plans))
        assert e.value.status == 1 and what in str(e.value), str(e.value)
    assert _abi.sfw_launch_count() == 0


def test_no_cpu_fallback():
    """Without a GPU the product path refuses to run (there is no CPU path), and without the
    built library the binding raises instead of computing anything."""
    import numpy as np
    import torch
    import paper_2009_05473_gb300 as sfw
    from paper_2009_05473_gb300 import _abi
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError, match="no CPU path"):
            sfw.Plan((8, 8, 8), (1, 1, 1), np.full((3, 3, 3), 1.0 / 27, np.float32))
    saved_path, saved_lib = _abi.LIB_PATH, _abi._lib
    try:
        _abi.LIB_PATH, _abi._lib = os.path.join(ROOT, "no_such_dir", "libsfw.so"), None
        with pytest.raises(RuntimeError, match="libsfw.so not found"):
            _abi.lib()
    finally:
        _abi.LIB_PATH, _abi._lib = saved_path, saved_lib
