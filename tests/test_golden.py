"""The oracle still reproduces the values frozen in tests/golden/oracle_values.json
(written by tests/golden/make_golden.py from the oracle alone): a change to the
oracle's arithmetic must regenerate them deliberately."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_frozen_values():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, "golden", "oracle_values.json")) as fh:
        stored = json.load(fh)
    now = mg.values()

    def cmp(a, b, path):
        if isinstance(a, dict):
            assert set(a) == set(b), path
            for k in a:
                cmp(a[k], b[k], path + "/" + k)
        elif isinstance(a, list):
            x = np.array(a, float)
            y = np.array(b, float)
            assert x.shape == y.shape, path
            assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(y).max()), path
        else:
            assert a == b, path

    cmp(now, stored, "")
