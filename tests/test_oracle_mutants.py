"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching) and
check that the pins of tests/test_oracle_pins.py catch every one of them.

A pin that keeps passing on a broken oracle would prove nothing; these tests
show that each slip listed below breaks at least one pin.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.kes_oracle as K
from tests import test_oracle_pins as pins


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(K, name, fn)
    monkeypatch.setattr(oracle, name, fn)


def _leapfrog(S, m, r, tau, alpha, *, start_prev=None, sign=-1.0, shift=1,
              use_mass=True, first_term=True, last_term=True):
    """filter_apply with one configurable slip."""
    L = len(alpha) - 1
    y_prev = np.array(r if start_prev is None else start_prev(r), dtype=np.float64)
    y = np.array(r, dtype=np.float64)
    acc = alpha[0] * y if first_term else np.zeros_like(y)
    for l in range(L):
        sy = S @ y
        if use_mass:
            sy = sy / m
        y_next = sign * tau * tau * sy + 2.0 * y - y_prev
        if last_term or l < L - 1:
            acc = acc + alpha[min(l + shift, L)] * y_next
        y_prev, y = y, y_next
    return acc


MUTANTS_FILTER = {
    "zero_previous_state": dict(start_prev=np.zeros_like),
    "wrong_sign_of_stiffness_term": dict(sign=+1.0),
    "weights_shifted_by_one_step": dict(shift=0),
    "mass_inverse_dropped": dict(use_mass=False),
    # the first or the last weighted term left out of the sum (eq. disc_filtercoeff runs
    # over n = 0..L): the slips a regrouped accumulation could make at either end
    "first_term_dropped": dict(first_term=False),
    "last_term_dropped": dict(last_term=False),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS_FILTER))
def test_filter_mutants_are_caught(monkeypatch, mutant):
    kw = MUTANTS_FILTER[mutant]
    _patch(monkeypatch, "filter_apply", lambda S, m, r, tau, a: _leapfrog(S, m, r, tau, a, **kw))
    caught = 0
    for kind in ["random", "box"]:
        try:
            pins.test_filter_maps_eigenvectors_by_beta_tilde(kind)
        except AssertionError:
            caught += 1
    assert caught >= 1


def test_weight_factor_mutant_is_caught(monkeypatch):
    orig = K.weight

    def halved(t, wmin, wmax, T):
        return 0.5 * orig(t, wmin, wmax, T)
    _patch(monkeypatch, "weight", halved)
    with pytest.raises(AssertionError):
        pins.test_beta_tilde_tends_to_indicator()


def test_weight_sum_difference_mutant_is_caught(monkeypatch):
    def swapped(t, wmin, wmax, T):   # sum and difference frequencies swapped
        t = np.asarray(t, dtype=np.float64)
        out = np.zeros_like(t)
        out[t == 0] = 2 * (wmax - wmin) / math.pi
        i = (t > 0) & (t <= T)
        ti = t[i]
        out[i] = 4 / (math.pi * ti) * np.sin(0.5 * ti * (wmax + wmin)) * np.cos(0.5 * ti * (wmax - wmin))
        return out
    _patch(monkeypatch, "weight", swapped)
    with pytest.raises(AssertionError):
        pins.test_weight_equals_sine_difference_form()


def test_alpha_without_tau_is_caught(monkeypatch):
    def no_tau(wmin, wmax, tau, L):
        return K.weight(np.arange(L + 1) * tau, wmin, wmax, L * tau)
    _patch(monkeypatch, "alpha_table", no_tau)
    with pytest.raises(AssertionError):
        pins.test_alpha_table_indexing()


def test_recurrence_mutant_is_caught(monkeypatch):
    def q_bad(omega, tau, L):       # q_{-1} = 0 instead of 1
        omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
        q = np.empty((L + 1, omega.size))
        qp, qc = np.zeros_like(omega), np.ones_like(omega)
        q[0] = qc
        for l in range(L):
            qn = (2 - tau * tau * omega * omega) * qc - qp
            q[l + 1] = qn
            qp, qc = qc, qn
        return q
    _patch(monkeypatch, "q_values", q_bad)
    with pytest.raises(AssertionError):
        pins.test_q_is_chebyshev_third_kind()


def test_euclidean_gram_schmidt_is_caught(monkeypatch):
    def cgs2_l2(B, w, m):
        w = np.array(w, dtype=np.float64)
        nb = np.linalg.norm(w)
        for _ in range(2):
            if B.shape[0]:
                w = w - (B @ w) @ B
        na = np.linalg.norm(w)
        return w / na, nb, na
    _patch(monkeypatch, "orthonormalize_cgs2", cgs2_l2)
    with pytest.raises(AssertionError):
        pins.test_cgs2_gives_m_orthonormal_basis()


def test_residual_without_mass_is_caught(monkeypatch):
    def res_bad(S, m, B, theta, Y):
        X = Y.T @ B
        a = np.array([np.linalg.norm(S @ x - th * x) for th, x in zip(theta, X)])
        return X, a, a / np.maximum(theta, 1e-300)
    _patch(monkeypatch, "ritz_residuals", res_bad)
    with pytest.raises(AssertionError):
        pins.test_krylov_finds_every_distinct_eigenvalue_in_interval()


def test_gaussian_normalisation_mutant_is_caught(monkeypatch):
    orig = K.gaussian_weight

    def half(t, c, sigma):
        return 0.5 * orig(t, c, sigma)
    monkeypatch.setattr(K, "gaussian_weight", half)
    monkeypatch.setattr(oracle, "gaussian_weight", half)
    with pytest.raises(AssertionError):
        pins.test_gaussian_weight_matches_numerical_inverse_transform()


def test_every_interval_searching_the_first_is_caught(monkeypatch):
    orig = K.block_krylov_solve
    lo0, hi0 = pins.MULTI_BANDS[0]

    def first_only(S, m, R0, omega_min, omega_max, *a, **kw):
        return orig(S, m, R0, lo0, hi0, *a, **kw)
    _patch(monkeypatch, "block_krylov_solve", first_only)
    with pytest.raises(AssertionError):
        pins.test_multi_interval_solver_finds_every_eigenvalue_of_each_interval()


def test_labels_not_following_the_merge_order_are_caught(monkeypatch):
    orig = K.multi_interval_krylov_solve

    def stale_labels(*a, **kw):
        r = orig(*a, **kw)
        r.interval = np.sort(r.interval)        # labels in interval order, not the merged order
        return r
    _patch(monkeypatch, "multi_interval_krylov_solve", stale_labels)
    with pytest.raises(AssertionError):
        pins.test_multi_interval_solver_finds_every_eigenvalue_of_each_interval()


def test_triangle_sinc_not_squared_is_caught(monkeypatch):
    def unsquared(t, c, h):
        t = np.asarray(t, dtype=np.float64)
        x = 0.5 * t * h
        sinc = np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))
        return 2.0 * h / math.pi * np.cos(c * t) * sinc
    monkeypatch.setattr(K, "triangle_weight", unsquared)
    monkeypatch.setattr(oracle, "triangle_weight", unsquared)
    with pytest.raises(AssertionError):
        pins.test_triangle_weight_matches_numerical_inverse_transform()


def test_leapfrog4_wrong_correction_in_filter_is_caught(monkeypatch):
    def halved_correction(S, m, r, tau, alpha):    # tau^4 / 24 instead of tau^4 / 12
        L = len(alpha) - 1
        y_prev, y = np.array(r, dtype=np.float64), np.array(r, dtype=np.float64)
        acc = alpha[0] * y
        for l in range(L):
            Ky = (S @ y) / m
            y_next = 2.0 * y - y_prev - tau * tau * Ky + tau ** 4 / 24.0 * ((S @ Ky) / m)
            acc = acc + alpha[l + 1] * y_next
            y_prev, y = y, y_next
        return acc
    _patch(monkeypatch, "filter_apply_leapfrog4", halved_correction)
    with pytest.raises(AssertionError):
        pins.test_leapfrog4_filter_maps_eigenvectors_by_its_beta_tilde("box")


def test_leapfrog4_wrong_recurrence_is_caught(monkeypatch):
    def q_bad(omega, tau, L):                       # x^2 / 6 instead of x^2 / 12
        omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
        x = tau * tau * omega * omega
        q = np.empty((L + 1, omega.size))
        qp, qc = np.ones_like(omega), np.ones_like(omega)
        q[0] = qc
        for l in range(L):
            qn = (2 - x + x * x / 6) * qc - qp
            q[l + 1] = qn
            qp, qc = qc, qn
        return q
    _patch(monkeypatch, "q_values_leapfrog4", q_bad)
    with pytest.raises(AssertionError):
        pins.test_leapfrog4_recurrence_is_third_kind_chebyshev_of_its_phase()


def test_subspace_iteration_without_filter_is_caught(monkeypatch):
    def no_filter(S, m, r, tau, alpha):
        return np.array(r, dtype=np.float64)
    _patch(monkeypatch, "filter_apply", no_filter)
    with pytest.raises(AssertionError):
        pins.test_subspace_iteration_finds_the_dominant_eigenvalues_of_the_filter()


def test_refinement_buffer_farthest_instead_of_nearest_is_caught(monkeypatch):
    def farthest(theta, omega_min, omega_max, extra=0):
        omega = np.sqrt(np.maximum(np.asarray(theta, dtype=np.float64), 0.0))
        inside = (omega >= omega_min) & (omega <= omega_max)
        out = np.flatnonzero(~inside)
        dist = np.where(omega[out] < omega_min, omega_min - omega[out], omega[out] - omega_max)
        keep = out[np.argsort(-dist, kind="stable")[:max(extra, 0)]]
        return np.sort(np.concatenate([np.flatnonzero(inside), keep]))
    _patch(monkeypatch, "refine_selection", farthest)
    with pytest.raises(AssertionError):
        pins.test_refine_selection_keeps_the_interval_and_the_nearest_outside()


def test_refinement_dropping_the_buffer_is_caught(monkeypatch):
    real = K.refine_selection
    _patch(monkeypatch, "refine_selection", lambda theta, lo, hi, extra=0: real(theta, lo, hi, 0))
    with pytest.raises(AssertionError):
        pins.test_refine_selection_keeps_the_interval_and_the_nearest_outside()
