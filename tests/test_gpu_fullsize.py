"""Parity at the measured size: the 128^3 Kuhn cube (2,048,383 dofs, 30.3M
entries), interval [40, 45], L = 600, Krylov dimension 60, in the launch
configuration the benchmark times (SELL-32, CUDA graph, default grid).

The oracle cannot produce single outputs of a 600-step filter one by one, so
the full-length filter is checked through a property that holds at any size
(Lemma 2.3: an eigenvector is scaled by beta~(omega)), element-wise parity is
checked on a full-size trajectory of 60 steps, and the solver's accepted
pairs are checked against the exact spectrum.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2402_08515_gb300 as K
from fe_inputs import WORKLOADS, start_vectors
from oracle import spectra
from tests.tolerances import EIG_REL, elementwise_bound, filter_error, filter_tol

pytestmark = pytest.mark.gpu

WL = WORKLOADS["cube128_fp64"]


@pytest.fixture(scope="module")
def cube():
    p = WL.build()
    v0 = start_vectors(p.n, 1, WL.seed)[0]
    with K.Context(p) as c:
        w_gpu, _ = K.kes_estimate_omega_max(c.handle, WL.power_iters, v0)
    return p, v0, w_gpu


def test_power_iteration_full_size(cube):
    p, v0, w_gpu = cube
    w_ref = O.power_iteration(p.to_scipy(), p.m, v0, WL.power_iters)
    assert w_gpu == pytest.approx(w_ref, rel=1e-10)
    assert w_gpu <= math.sqrt(spectra.box_spectrum(p.cells, p.h).max()) * (1 + 1e-12)


def _modes(p):
    n = p.cells[0]
    out = []
    for k in [(1, 1, 1), (2, 1, 1), (3, 2, 1), (5, 4, 3), (7, 6, 5), (40, 60, 90), (127, 127, 127)]:
        lam = sum(4 * n * n * math.sin(ki * math.pi / (2 * n)) ** 2 for ki in k)
        out.append((k, lam))
    # the one mode with omega closest to the middle of the interval
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_filter_scales_exact_eigenvectors_full_length(cube, precision):
    p, _, w_gpu = cube
    tau = WL.cfl * 2 / w_gpu
    L = WL.L
    alpha = O.alpha_table(WL.omega_min, WL.omega_max, tau, L)
    modes = _modes(p)
    # add modes inside the interval
    lam_in = spectra.eigenvalues_in(p.cells, p.h, WL.omega_min, WL.omega_max)
    with K.Context(p, precision=precision) as c:
        K.kes_set_filter(c.handle, WL.omega_min, WL.omega_max, tau, L)
        worst = 0.0
        for k, lam in modes + [((3, 7, 11), None)]:
            v = spectra.box_eigenvector(p.cells, k)
            if lam is None:
                lam = sum(4 * 128 * 128 * math.sin(ki * math.pi / 256) ** 2 for ki in k)
            beta = O.beta_tilde(np.array([math.sqrt(lam)]), alpha, tau)[0]
            out = np.zeros((1, 1, p.n))
            K.kes_filter_apply(c.handle, v[None, :], out, 1)
            err = filter_error(out[0], beta * v, v[None, :], p.m, alpha)
            worst = max(worst, err)
            assert err <= filter_tol(L, precision), (k, beta, err)
    print(f"{precision}: worst Lemma 2.3 error {worst:.3e} (tol {filter_tol(L, precision):.3e}); "
          f"{lam_in.size} eigenvalues in the interval")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_filter_elementwise_parity_full_size(cube, precision):
    p, v0, w_gpu = cube
    tau = WL.cfl * 2 / w_gpu
    L = 60
    alpha = O.alpha_table(WL.omega_min, WL.omega_max, tau, L)
    ref = O.filter_apply(p.to_scipy(), p.m, v0, tau, alpha)
    with K.Context(p, precision=precision) as c:
        K.kes_set_filter(c.handle, WL.omega_min, WL.omega_max, tau, L)
        out = np.zeros((1, 1, p.n))
        K.kes_filter_apply(c.handle, v0[None, :], out, 1)
    tol = filter_tol(L, precision)
    err = filter_error(out[0], ref, v0[None, :], p.m, alpha)
    print(f"{precision}: full-size L={L} error {err:.3e} (tol {tol:.3e})")
    assert err <= tol
    np.testing.assert_array_less(np.abs(out[0, 0] - ref), elementwise_bound(tol, v0, p.m, alpha))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_krylov_solve_full_size_matches_exact_spectrum(cube, precision):
    p, v0, w_gpu = cube
    tau = WL.cfl * 2 / w_gpu
    tol = 1e-8 if precision == "fp64" else 1e-5
    with K.Context(p, precision=precision) as c:
        K.kes_set_filter(c.handle, WL.omega_min, WL.omega_max, tau, WL.L)
        so = K.kes_solve_opts_default()
        so.kmax, so.tol = WL.kmax, tol
        res = K.kes_krylov_solve(c.handle, v0, so)
    exact, _ = spectra.distinct(spectra.eigenvalues_in(p.cells, p.h, WL.omega_min, WL.omega_max))
    everything = spectra.box_spectrum(p.cells, p.h)
    print(f"{precision}: {res['n_pairs']} accepted of {exact.size} distinct, k={res['k_used']}, "
          f"{res['solve_ms']:.0f} ms")
    assert res["k_used"] == WL.kmax and res["time_steps"] == (WL.kmax - 1) * WL.L
    assert np.all(res["rel_res"] <= tol)
    for th in res["omega2"]:
        assert np.min(np.abs(exact - th) / th) <= EIG_REL[precision]
    # Every Ritz pair in the interval, converged or not, obeys the residual bound of a
    # symmetric definite pencil: some eigenvalue lies within ||(S - theta M) x||_{M^-1}
    # of theta (||x||_M = 1); with M = h^3 I that radius is rel_res * theta.
    inside = ~np.isnan(res["ritz_rel_res"])
    assert inside.any()
    for th, rel in zip(res["ritz_omega2"][inside], res["ritz_rel_res"][inside]):
        gap = np.min(np.abs(everything - th))
        assert gap <= rel * th * (1 + 1e-6) + 1e-12 * th, (th, rel, gap)
