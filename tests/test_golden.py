"""The FP64 oracle against its frozen record on one small seeded case
(tests/golden/tiny_13x11x9.json, written by tests/golden/make_golden.py from the oracle
alone).  A change of the oracle's arithmetic shows here first; its commit then has to name
the passage of the paper that justifies it."""

import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_matches_golden_record(oracle_mod):
    rec = json.load(open(os.path.join(HERE, "golden", "tiny_13x11x9.json")))
    assert set(rec["citations"]) == set(rec["values"])
    got = _maker().values()
    want = rec["values"]
    assert got["eta_argmax"] == want["eta_argmax"]
    for key in ("forward_sum", "criterion", "eta_max"):
        assert abs(got[key] - want[key]) <= 1e-10 * max(1.0, abs(want[key])), key
    for key in ("forward_sample", "gradient", "eta_sample"):
        a, b = np.asarray(got[key]), np.asarray(want[key])
        assert a.shape == b.shape, key
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(b))), key
