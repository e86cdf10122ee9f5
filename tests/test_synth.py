"""The seeded input generators: shapes, determinism, and the signal models."""
import json
import os

import numpy as np
import pytest

from paper_2401_12890_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_dictionary_shapes_and_formula():
    for name, w in synth.WORKLOADS.items():
        K = synth.dictionary_for(name)
        assert K.shape == (w.P, w.Q)
        assert np.all(np.isfinite(K))
    K = synth.dictionary_for("dr2d_tiny")
    # p = (b index, TE index) with TE fastest; q = (D index, T2 index) with T2 fastest
    b, te = 600.0 * 2, 60.0 + 35.0 * 3
    D, T2 = np.geomspace(1e-4, 3e-3, 15)[4], np.geomspace(10, 300, 15)[7]
    assert K[2 * 5 + 3, 4 * 15 + 7] == pytest.approx(np.exp(-b * D) * np.exp(-te / T2))
    Kmrf = synth.dictionary_for("mrf2d")
    np.testing.assert_allclose(np.linalg.norm(Kmrf, axis=0), 1.0, rtol=1e-12)


def test_problem_is_deterministic_and_nonnegative_truth():
    K1, M1, (S1, A1) = synth.make_problem("dr2d_tiny")
    K2, M2, (S2, A2) = synth.make_problem("dr2d_tiny")
    assert np.array_equal(M1, M2) and M1.dtype == np.float32
    assert M1.shape == (30, 1024)
    assert np.all(S1 >= 0) and np.all(A1 >= 0)
    np.testing.assert_allclose(S1.sum(axis=0), 1.0)
    # a different seed gives different noise and maps
    _, M3, _ = synth.make_problem("dr2d_tiny", seed=7)
    assert not np.array_equal(M1, M3)
    # noise level: SNR 100 against the strongest image's peak
    clean = K1 @ (S1 @ A1)
    sigma = np.abs(clean[0]).max() / 100.0
    resid = M1.astype(np.float64) - clean
    assert resid.std() == pytest.approx(sigma, rel=0.05)


def test_third_peak_absent_in_part_of_the_image():
    _, _, (S, A) = synth.make_problem("dr2d_tiny")
    assert 0.1 < np.mean(A[2] == 0) < 0.9


def test_grid_override_and_voxel_order():
    _, M, (S, A) = synth.make_problem("dr2d_tiny", dims=(7, 3))
    assert M.shape == (30, 21) and A.shape == (3, 21)


def test_workload_beta_matches_golden_record():
    g = json.load(open(os.path.join(HERE, "golden", "workloads.json")))
    for name, w in list(synth.WORKLOADS.items()) + [("mrf_b1", synth.B1_WORKLOAD)]:
        assert w.beta == pytest.approx(g[name]["beta"], rel=1e-12)
        assert w.P == g[name]["P"] and w.Q == g[name]["Q"]
    assert g["mrf_b1"]["levels"] == synth.B1_LEVELS
