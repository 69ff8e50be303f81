"""Pins for the oracle's Philox4x32-10 and Box-Muller normals (CPU only)."""

import json
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_known_answer_vectors():
    for c in json.load(open(GOLDEN))["cases"]:
        ctr = [np.array([int(x, 16)]) for x in c["ctr"]]
        key = [int(x, 16) for x in c["key"]]
        out = philox.philox4x32_10(*ctr, *key)
        assert ["%08x" % int(o[0]) for o in out] == c["out"]


def test_test_matrix_is_standard_normal():
    O = philox.gaussian_test_matrix(200000, 3, seed=12345)
    assert abs(O.mean()) < 0.01 and abs(O.std() - 1.0) < 0.01
    assert abs((O ** 4).mean() - 3.0) < 0.05          # Gaussian kurtosis
    # distinct columns and seeds give (nearly) uncorrelated draws
    assert abs(np.corrcoef(O[:, 0], O[:, 1])[0, 1]) < 0.01
    O2 = philox.gaussian_test_matrix(200000, 1, seed=12346)
    assert abs(np.corrcoef(O[:, 0], O2[:, 0])[0, 1]) < 0.01
