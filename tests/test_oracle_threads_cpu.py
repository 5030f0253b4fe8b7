"""The oracle's OpenMP build (used only to time the oracle on every host
core) gives results identical to the plain build: its parallel loops are
per-pixel values, exact integer sums and min / max, none of which depends on
the order pixels are visited, and the FP64 scatter sums stay serial."""
import numpy as np
import pytest

import oracle
from synth import make_workload


def _all_outputs(w):
    f = oracle.fit(w.cube, w.labels, w.K)
    y = oracle.project(w.cube, f["V"], f["mu"], w.k)
    rt = oracle.range_training(y, w.labels)
    rg = oracle.range_global(y)
    n, s = oracle.class_sums(w.cube, w.labels, w.K)
    return [f["lam"], f["V"], f["Sw"], f["mu"], y, rt, rg, oracle.to_u8(y, rt), oracle.to_u16(y, rg), n, s]


def test_threaded_build_is_identical_to_plain_build():
    w = make_workload(4321, 16, 301, 257, 4, (2000, 1500, 1200, 900), 3, separation=(1.0, 4.0))
    bad = w.labels.copy()
    bad[100, 100] = 9
    try:
        assert oracle.use_threads(1) == 1
        plain = _all_outputs(w)
        with pytest.raises(oracle.OracleError):
            oracle.class_sums(w.cube, bad, w.K)
        try:
            threads = oracle.use_threads(4)
        except Exception as exc:  # noqa: BLE001 - a compiler without OpenMP
            pytest.skip(f"no OpenMP build: {exc}")
        assert threads == 4
        par = _all_outputs(w)
        with pytest.raises(oracle.OracleError):
            oracle.class_sums(w.cube, bad, w.K)
    finally:
        oracle.use_threads(1)
    for a, b in zip(plain, par):
        np.testing.assert_array_equal(a, b)
