"""Stored closed-form spectra (tests/golden/box_spectra.json, written by
tests/golden/make_golden.py from oracle/spectra.py) stay reproducible, and the
workload intervals hold the eigenvalue counts the measurements are read against."""
import json
import os

import numpy as np

from oracle import spectra

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "box_spectra.json")


def test_golden_spectra_reproduce():
    data = json.load(open(GOLDEN))
    for name, d in data.items():
        cells = tuple(d["cells"])
        h = tuple(1.0 / c for c in cells)
        lam = spectra.eigenvalues_in(cells, h, *d["interval"])
        vals, mult = spectra.distinct(lam)
        assert lam.size == d["count"], name
        np.testing.assert_allclose(vals, d["distinct"], rtol=1e-15)
        np.testing.assert_array_equal(mult, d["multiplicity"])


def test_workload_interval_counts():
    data = json.load(open(GOLDEN))
    assert (data["square64"]["count"], len(data["square64"]["distinct"])) == (38, 20)
    assert (data["cube128"]["count"], len(data["cube128"]["distinct"])) == (424, 83)


def test_workload_spectra_agree_with_the_oracle():
    # bench.py counts and checks eigenvalues with fe_inputs.spectra, the tests with the
    # oracle's closed form: the two copies must agree
    from fe_inputs import spectra as wl_spectra
    for cells, h, iv in [((64, 64), (1 / 64, 1 / 64), (20.0, 30.0)), ((23, 19, 17), (1 / 23, 0.9 / 19, 0.8 / 17), (6.0, 10.0)),
                         ((128, 128, 128), (1 / 128,) * 3, (40.0, 45.0))]:
        a = spectra.eigenvalues_in(cells, h, *iv)
        b = wl_spectra.omega2_in(cells, h, *iv)
        np.testing.assert_allclose(b, a, rtol=1e-14)
        va, ma = spectra.distinct(a)
        vb, mb = wl_spectra.cluster(b)
        np.testing.assert_allclose(vb, va, rtol=1e-14)
        np.testing.assert_array_equal(mb, ma)
