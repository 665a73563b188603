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
