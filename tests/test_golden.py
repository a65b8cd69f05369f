"""The stored oracle digests of the 256 x 256 x 128 benchmark box.

tests/golden/make_medium_box_digest.py writes them with the oracle alone.
These checks need no GPU: the sampled cells are the script's seeded draw, the
two solutions (exactly 641 iterations of Algorithm 1, and converged to tol
1e-12) agree with each other far below the parity bar, and the digests are
internally consistent (the level sums add up to the same total).
"""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def _script():
    spec = importlib.util.spec_from_file_location("make_medium_box_digest",
                                                  os.path.join(HERE, "make_medium_box_digest.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_digest_cells_are_the_seeded_sample():
    m = _script()
    cells = m.sample_cells(256 * 256 * 128)
    for name in ("medium_box_fixed641.json", "medium_box_tol1e-12.json"):
        d = _load(name)
        assert d["cells"] == [int(c) for c in cells]
        assert len(d["x"]) == m.SAMPLES and len(d["level_sums"]) == 128


def test_fixed_count_and_tight_solutions_agree():
    a, b = _load("medium_box_fixed641.json"), _load("medium_box_tol1e-12.json")
    assert a["iterations"] == 641 and not a["converged"] and a["relres_recursive"] < 1e-8
    assert b["converged"] and b["relres_recursive"] < 1e-12 and b["iterations"] > 641
    xa, xb = np.array(a["x"]), np.array(b["x"])
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xb) < 1e-10
    assert abs(a["norm2"] - b["norm2"]) < 1e-12 * b["norm2"]
    assert np.allclose(a["level_sums"], b["level_sums"], rtol=1e-12, atol=0)
