"""Host-side helpers of bench.py (no GPU): the C_eff deviation from stored
dense-oracle columns and the workload naming shared by both arms."""
import importlib.util
import json
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_ceff_error_vs_dense(tmp_path):
    b = _bench()
    path = tmp_path / "g.json"
    json.dump({"columns": {"0": {"sigma_bar_re": [1.4, 0.6, 0.6, 0, 0, 0]},
                           "3": {"sigma_bar_re": [0, 0, 0, 0.4, 0, 0]}}}, open(path, "w"))
    C = np.zeros((6, 6))
    C[:, 0] = [1.54, 0.6, 0.6, 0, 0, 0]
    C[:, 3] = [0, 0, 0, 0.4, 0, 0]
    err = b.ceff_error_vs_dense(C, str(path))
    assert abs(err["0"] - 0.1) < 1e-12 and err["3"] == 0.0
    assert b.ceff_error_vs_dense(C, str(tmp_path / "missing.json")) is None


def test_stored_dense_column_is_readable():
    b = _bench()
    err = b.ceff_error_vs_dense(np.zeros((6, 6)))
    assert err is not None and abs(err["0"] - 1.0) < 1e-12
