"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped factor,
a wrong sign or start value, a shifted index, the wrong inner product) breaks
at least one of them; tests/test_oracle_mutants.py plants such slips and
checks that they are caught.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from oracle import spectra
from fe_inputs import box_grid, square_grid, start_vectors, flared_tube


def random_pencil(n, seed, density=0.2):
    """A random sparse symmetric PSD S (graph Laplacian with random positive
    weights plus a positive shift on a few nodes) and positive lumped masses."""
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=seed, format="csr")
    A = abs(A + A.T)
    A.setdiag(0)
    A.eliminate_zeros()
    Lap = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    shift = np.zeros(n)
    shift[rng.choice(n, size=max(1, n // 5), replace=False)] = rng.uniform(0.5, 2, max(1, n // 5))
    S = (Lap + sp.diags(shift)).tocsr()
    m = rng.uniform(0.5, 2.0, n)
    return S, m


def dense_pencil(S, m):
    w2, V = sla.eigh(S.toarray(), np.diag(m))    # V^T M V = I
    return np.maximum(w2, 0.0), V


# ---------------------------------------------------------------- eq. weightf

def test_weight_at_zero_is_the_limit_of_the_formula():
    for wmin, wmax in [(20.0, 30.0), (0.0, 3.0), (40.0, 45.0), (12.2, 12.5)]:
        a0 = O.weight(np.array([0.0]), wmin, wmax, 1.0)[0]
        assert a0 == pytest.approx(2.0 * (wmax - wmin) / math.pi, rel=1e-15)
        t = np.array([1e-7])
        assert O.weight(t, wmin, wmax, 1.0)[0] == pytest.approx(a0, rel=1e-9)


def test_weight_equals_sine_difference_form():
    # 2 sin(a) cos(b) = sin(a+b) + sin(a-b) turns eq. weightf into
    # 2/(pi t) (sin(t wmax) - sin(t wmin)): a different expression of the same function
    wmin, wmax, T = 1.6, 2.3, 30.0
    t = np.linspace(1e-3, T, 5001)
    ref = 2.0 / (math.pi * t) * (np.sin(t * wmax) - np.sin(t * wmin))
    np.testing.assert_allclose(O.weight(t, wmin, wmax, T), ref, rtol=0, atol=1e-13)


def test_weight_support_is_closed_interval():
    wmin, wmax, T = 2.0, 4.0, 5.0
    vals = O.weight(np.array([T, T * (1 + 1e-12), 2 * T]), wmin, wmax, T)
    assert vals[0] != 0.0
    assert vals[1] == 0.0 and vals[2] == 0.0


def test_shorter_filter_is_a_truncated_table():
    # alpha(t) of eq. (weightf) does not depend on T: the weights of L' < L steps are the
    # first L' + 1 of the L-step table (what a shorter refinement filter runs)
    full = O.alpha_table(20.0, 30.0, 0.01, 600)
    np.testing.assert_array_equal(O.alpha_table(20.0, 30.0, 0.01, 150), full[:151])


def test_alpha_table_indexing():
    wmin, wmax, tau, L = 20.0, 30.0, 0.0099, 300
    a = O.alpha_table(wmin, wmax, tau, L)
    assert a.shape == (L + 1,)
    assert a[0] == pytest.approx(tau * 2 * (wmax - wmin) / math.pi, rel=1e-15)
    t = L * tau
    last = tau * 2.0 / (math.pi * t) * (math.sin(t * wmax) - math.sin(t * wmin))
    assert a[L] == pytest.approx(last, rel=1e-10, abs=1e-15)
    t = 7 * tau
    a7 = tau * 2.0 / (math.pi * t) * (math.sin(t * wmax) - math.sin(t * wmin))
    assert a[7] == pytest.approx(a7, rel=1e-12)


# ---------------------------------------------------------------- eq. scalartimestep

def test_q_is_chebyshev_third_kind():
    # q_l = cos((l + 1/2) theta) / cos(theta / 2), cos(theta) = 1 - tau^2 w^2 / 2
    tau, L = 0.01, 400
    w = np.linspace(0.5, 1.99 / tau, 97)
    q = O.q_values(w, tau, L)
    theta = np.arccos(1.0 - 0.5 * tau * tau * w * w)
    l = np.arange(L + 1)[:, None]
    ref = np.cos((l + 0.5) * theta) / np.cos(0.5 * theta)
    np.testing.assert_allclose(q, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_q_special_cases():
    tau, L = 0.5, 200                    # tau^2 w^2 = 4 exactly at w = 4
    q0 = O.q_values([0.0], tau, L)[:, 0]
    np.testing.assert_array_equal(q0, np.ones(L + 1))
    qe = O.q_values([2.0 / tau], tau, L)[:, 0]
    l = np.arange(L + 1)
    np.testing.assert_allclose(qe, (-1.0) ** l * (2 * l + 1), rtol=1e-12)


def test_q_bounded_inside_cfl_and_growing_outside():
    tau, L = 0.1, 500
    inside = O.q_values([0.95 * 2 / tau], tau, L)[:, 0]
    theta = math.acos(1 - 0.5 * (0.95 * 2) ** 2)
    assert np.abs(inside).max() <= 1 / math.cos(theta / 2) + 1e-9
    outside = O.q_values([1.05 * 2 / tau], tau, L)[:, 0]
    assert abs(outside[-1]) > 1e20


# ---------------------------------------------------------------- Lemma 2.2 limit

def test_beta_tilde_tends_to_indicator():
    # Lemma 2.2 with eq. weightf: beta -> chi_[wmin, wmax] (1/2 at the ends)
    # as tau -> 0 and T -> infinity
    wmin, wmax = 2.0, 4.0
    tau, L = 0.002, 200000               # T = 400
    a = O.alpha_table(wmin, wmax, tau, L)
    w = np.array([0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 6.0, 10.0])
    b = O.beta_tilde(w, a, tau)
    expect = np.array([0, 0, 0, 0.5, 1, 1, 1, 0.5, 0, 0, 0])
    # the ends sit on the transition (width ~ pi/T) and move with the
    # O(tau^2 w^2) phase error of the leapfrog, hence the looser bound there
    atol = np.where(expect == 0.5, 2e-2, 6e-3)
    assert np.all(np.abs(b - expect) <= atol), b


def test_beta_tilde_is_rectangle_rule_of_beta():
    # for tau -> 0 with T fixed, beta~ tends to the integral of eq. filterfunc
    wmin, wmax, T = 2.0, 4.0, 6.0
    w = np.array([1.0, 3.0, 5.0])
    ts = np.linspace(0, T, 2_000_001)
    f = O.weight(ts, wmin, wmax, T)[:, None] * np.cos(ts[:, None] * w[None, :])
    integral = np.trapezoid(f, ts, axis=0)
    L = 60000
    tau = T / L
    b = O.beta_tilde(w, O.alpha_table(wmin, wmax, tau, L), tau)
    # rectangle rule = trapezoid + tau/2 (f(0) + f(T)), plus O(tau^2) from q_l ~ cos
    np.testing.assert_allclose(b, integral, atol=2e-3)


# ---------------------------------------------------------------- Lemma 2.3

@pytest.mark.parametrize("kind", ["square", "box", "random", "tube"])
def test_filter_maps_eigenvectors_by_beta_tilde(kind):
    if kind == "square":
        p = square_grid(7); S, m = p.to_scipy(), p.m
    elif kind == "box":
        p = box_grid((5, 4, 6), extent=(1.0, 0.7, 1.3)); S, m = p.to_scipy(), p.m
    elif kind == "tube":
        p = flared_tube(0.125, length=1.0, r0=0.2, growth=0.8); S, m = p.to_scipy(), p.m
    else:
        S, m = random_pencil(40, seed=3)
    w2, V = dense_pencil(S, m)
    w = np.sqrt(w2)
    tau = 0.95 * 2 / w.max()
    L = 60
    alpha = O.alpha_table(0.3 * w.max(), 0.45 * w.max(), tau, L)
    bt = O.beta_tilde(w, alpha, tau)
    scale = np.abs(alpha).sum() * 2
    for j in range(len(w)):
        c = O.filter_apply(S, m, V[:, j], tau, alpha)
        err = np.abs(c - bt[j] * V[:, j]).max() / np.abs(V[:, j]).max()
        assert err < 1e-12 * scale, (j, err)


def test_filter_is_polynomial_in_minv_s():
    # eq. polyFilter: C = beta~(M^-1 S) = V diag(beta~) V^T M for M-orthonormal V
    S, m = random_pencil(30, seed=11)
    w2, V = dense_pencil(S, m)
    w = np.sqrt(w2)
    tau = 0.9 * 2 / w.max()
    alpha = O.alpha_table(0.2 * w.max(), 0.5 * w.max(), tau, 45)
    r = start_vectors(30, 1, 5)[0]
    ref = V @ (O.beta_tilde(w, alpha, tau) * (V.T @ (m * r)))
    got = O.filter_apply(S, m, r, tau, alpha)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_filter_is_m_self_adjoint():
    S, m = random_pencil(50, seed=7)
    w2, _ = dense_pencil(S, m)
    tau = 0.9 * 2 / math.sqrt(w2.max())
    alpha = O.alpha_table(1.0, 2.0, tau, 80)
    x, y = start_vectors(50, 2, 9)
    cx = O.filter_apply(S, m, x, tau, alpha)
    cy = O.filter_apply(S, m, y, tau, alpha)
    lhs, rhs = O.m_inner(cx, y, m), O.m_inner(x, cy, m)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1)


def test_filter_multi_equals_separate_runs():
    p = square_grid(9)
    S, m = p.to_scipy(), p.m
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    L = 40
    alphas = np.stack([O.alpha_table(a, b, tau, L) for a, b in [(5, 9), (9, 14), (14, 20)]])
    R = start_vectors(p.n, 2, 4)
    out = O.filter_apply_multi(S, m, R, tau, alphas)
    for f in range(3):
        for j in range(2):
            np.testing.assert_allclose(out[f, j], O.filter_apply(S, m, R[j], tau, alphas[f]),
                                       rtol=0, atol=1e-15)


# ---------------------------------------------------------------- closed-form spectra

@pytest.mark.parametrize("cells,extent", [((8, 8), None), ((6, 9), (1.0, 2.0)),
                                          ((4, 4, 4), None), ((5, 6, 7), (1.0, 1.3, 0.8))])
def test_tensor_grid_spectrum_matches_dense(cells, extent):
    p = box_grid(cells, extent)
    w2, _ = dense_pencil(p.to_scipy(), p.m)
    ref = spectra.box_spectrum(p.cells, p.h)
    np.testing.assert_allclose(np.sort(w2), ref, rtol=1e-13)


def test_tensor_grid_eigenvector_closed_form():
    p = box_grid((7, 5, 6))
    S = p.to_scipy()
    lam = 4 * 49 * math.sin(2 * math.pi / 14) ** 2 + 4 * 25 * math.sin(3 * math.pi / 10) ** 2 \
        + 4 * 36 * math.sin(1 * math.pi / 12) ** 2
    v = spectra.box_eigenvector(p.cells, (2, 3, 1))
    r = S @ v - lam * p.m * v
    assert np.abs(r).max() < 1e-13 * lam * np.abs(p.m * v).max()


# ---------------------------------------------------------------- power iteration

def test_power_iteration_reaches_largest_frequency():
    S, m = random_pencil(60, seed=2)
    w2, _ = dense_pencil(S, m)
    got = O.power_iteration(S, m, start_vectors(60, 1, 0)[0], 2000)
    assert got == pytest.approx(math.sqrt(w2.max()), rel=1e-6)


def test_power_iteration_underestimates_within_cfl_margin():
    p = square_grid(64)
    wmax = math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    got = O.power_iteration(p.to_scipy(), p.m, start_vectors(p.n, 1, 0)[0], 300)
    assert got <= wmax * (1 + 1e-12)
    assert got >= wmax / 1.05          # tau = 0.9 * 2 / got stays below 2 / wmax


# ---------------------------------------------------------------- Gram-Schmidt

def test_cgs2_gives_m_orthonormal_basis():
    p = square_grid(12)
    m = p.m
    X = start_vectors(p.n, 25, 1)
    X[5] = X[2] + 1e-6 * start_vectors(p.n, 1, 99)[0]   # nearly dependent column
    B = np.zeros((0, p.n))
    for x in X:
        b, nb, na = O.orthonormalize_cgs2(B, x, m)
        assert b is not None
        B = np.vstack([B, b])
    G = B @ (m[:, None] * B.T)
    np.testing.assert_allclose(G, np.eye(len(B)), atol=1e-14)


def test_cgs2_reports_breakdown_for_dependent_vector():
    p = square_grid(10)
    X = start_vectors(p.n, 3, 1)
    B = np.zeros((0, p.n))
    for x in X:
        B = np.vstack([B, O.orthonormalize_cgs2(B, x, p.m)[0]])
    b, nb, na = O.orthonormalize_cgs2(B, 2.0 * B[0] - 3.0 * B[2], p.m)
    assert b is None and na < O.BREAKDOWN_RATIO * nb


# ---------------------------------------------------------------- full solver

def test_krylov_finds_every_distinct_eigenvalue_in_interval():
    p = square_grid(32)
    S = p.to_scipy()
    exact, mult = spectra.distinct(spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0))
    wmax = math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    tau = 0.9 * 2 / wmax
    res = O.krylov_solve(S, p.m, start_vectors(p.n, 1, 0)[0], 20.0, 30.0, tau, 300, 60, 1e-8)
    assert len(res.omega2) == len(exact)
    np.testing.assert_allclose(res.omega2, exact, rtol=1e-10)
    assert np.all(res.rel_res <= 1e-8)
    # residual recomputed from the returned vectors
    for th, x in zip(res.omega2, res.vectors):
        assert np.linalg.norm(S @ x - th * p.m * x) <= 1e-8 * th * np.linalg.norm(p.m * x)
        assert O.m_norm(x, p.m) == pytest.approx(1.0, rel=1e-12)
    assert res.time_steps == 59 * 300


def test_krylov_breakdown_on_eigenvector_start():
    p = square_grid(16)
    v = spectra.box_eigenvector(p.cells, (3, 2))
    lam = 4 * 256 * (math.sin(3 * math.pi / 32) ** 2 + math.sin(2 * math.pi / 32) ** 2)
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    res = O.krylov_solve(p.to_scipy(), p.m, v, 0.8 * math.sqrt(lam), 1.2 * math.sqrt(lam),
                         tau, 100, 10, 1e-8)
    assert res.breakdown and res.k_used == 1
    assert res.omega2[0] == pytest.approx(lam, rel=1e-13)


# ---------------------------------------------------------------- block version (Sec. 4)

def test_block_solver_with_one_vector_is_the_krylov_solver():
    p = square_grid(24)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    r = start_vectors(p.n, 1, 4)
    a = O.krylov_solve(S, p.m, r[0], 15.0, 25.0, tau, 200, 40, 1e-8)
    b = O.block_krylov_solve(S, p.m, r, 15.0, 25.0, tau, 200, 40, 1e-8)
    np.testing.assert_array_equal(a.omega2, b.omega2)
    np.testing.assert_array_equal(a.basis, b.basis)


def test_block_solver_resolves_multiple_eigenvalues():
    # the square has double eigenvalues (k1, k2) ~ (k2, k1); one start vector sees one
    # vector per eigenspace (Lemma 2.2), a block of two sees both copies
    p = square_grid(32)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    exact = spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0)
    res = O.block_krylov_solve(S, p.m, start_vectors(p.n, 2, 3), 20.0, 30.0, tau, 300, 100, 1e-8)
    assert len(res.omega2) == len(exact) == 36
    np.testing.assert_allclose(np.sort(res.omega2), exact, rtol=1e-10)
    G = res.vectors @ (p.m[:, None] * res.vectors.T)     # accepted vectors M-orthonormal
    np.testing.assert_allclose(G, np.eye(len(exact)), atol=1e-8)


# ---------------------------------------------------------------- several intervals (Sec. 4)

# listed high band first, so that the merge into ascending order permutes the labels
MULTI_BANDS = [(36.0, 39.0), (20.0, 25.0)]


def test_multi_interval_solver_finds_every_eigenvalue_of_each_interval():
    # two intervals, two start vectors each (double eigenvalues of the square need a
    # block of two): every eigenvalue of each interval, found by that interval
    p = square_grid(32)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    res = O.multi_interval_krylov_solve(S, p.m, start_vectors(p.n, 4, 3), MULTI_BANDS, tau, 300, 120, 1e-8)
    for f, (lo, hi) in enumerate(MULTI_BANDS):
        exact = spectra.eigenvalues_in(p.cells, p.h, lo, hi)
        got = res.omega2[res.interval == f]
        assert len(got) == len(exact)
        np.testing.assert_allclose(got, exact, rtol=1e-10)
        assert np.all((np.sqrt(got) >= lo) & (np.sqrt(got) <= hi))
    assert np.all(np.diff(res.omega2) >= 0)
    for th, x in zip(res.omega2, res.vectors):
        assert np.linalg.norm(S @ x - th * p.m * x) <= 1e-8 * th * np.linalg.norm(p.m * x)


def test_multi_interval_with_one_interval_is_the_block_solver():
    p = square_grid(20)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    R = start_vectors(p.n, 2, 1)
    a = O.block_krylov_solve(S, p.m, R, 15.0, 25.0, tau, 150, 40, 1e-8)
    b = O.multi_interval_krylov_solve(S, p.m, R, [(15.0, 25.0)], tau, 150, 40, 1e-8)
    np.testing.assert_array_equal(a.omega2, b.omega2)
    assert np.all(b.interval == 0) and b.k_used == a.k_used


# ---------------------------------------------------------------- FP64 refinement

def test_refinement_keeps_exact_eigenvectors():
    p = square_grid(20)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    modes = [(2, 3), (3, 2), (4, 1)]
    X = np.stack([spectra.box_eigenvector(p.cells, k) for k in modes])
    lam = sorted(4 * 400 * (math.sin(a * math.pi / 40) ** 2 + math.sin(b * math.pi / 40) ** 2) for a, b in modes)
    th, rel, Xa, thi, reli = O.refine_subspace(S, p.m, X, 0.9 * math.sqrt(lam[0]), 1.1 * math.sqrt(lam[-1]),
                                               tau, 150, 1e-10)
    np.testing.assert_allclose(np.sort(th), lam, rtol=1e-12)
    assert np.all(rel < 1e-12)


def test_refinement_damps_noise_by_the_filter_contrast():
    p = square_grid(24)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    k = (3, 5)
    v = spectra.box_eigenvector(p.cells, k)
    lam = 4 * 576 * (math.sin(3 * math.pi / 48) ** 2 + math.sin(5 * math.pi / 48) ** 2)
    noisy = v + 1e-5 * np.abs(v).max() * start_vectors(p.n, 1, 8)[0]
    rq = (noisy @ (S @ noisy)) / (noisy @ (p.m * noisy))
    rel0 = np.linalg.norm(S @ noisy - rq * p.m * noisy) / (rq * np.linalg.norm(p.m * noisy))
    # neighbours at omega = 17.57 and 18.64: a narrow interval and a long filter isolate
    # omega = 18.05 (its twin (5, 3) is the same eigenvalue, so its noise is harmless)
    th, rel, Xa, thi, reli = O.refine_subspace(S, p.m, noisy[None, :], 17.8, 18.3, tau, 2000, 1e-8)
    # the largest |beta~| outside the interval is ~0.08 against ~0.95 inside
    assert len(thi) == 1 and thi[0] == pytest.approx(lam, rel=1e-12)
    assert reli[0] < 1e-3 * rel0


# ---------------------------------------------------------------- other weights (Sec. 4)

def test_gaussian_weight_gives_gaussian_band():
    # the inverse cosine transform of a Gaussian band, sampled by the rectangle rule,
    # reproduces the band (Lemma 2.2 with a Gaussian peak instead of the indicator)
    c, sigma = 3.0, 0.5
    tau, L = 0.001, 20000                      # sigma * T = 10: truncation negligible
    a = O.alpha_table_gaussian(c, sigma, tau, L)
    w = np.array([1.0, 2.0, 2.5, 3.0, 3.4, 4.0, 5.0])
    ref = np.exp(-(w - c) ** 2 / (2 * sigma ** 2)) + np.exp(-(w + c) ** 2 / (2 * sigma ** 2))
    # the rectangle rule (full weight at t = 0) and the leapfrog phase error are O(tau):
    # about 1e-3 at this tau, halving with tau
    np.testing.assert_allclose(O.beta_tilde(w, a, tau), ref, atol=1.5e-3)


def test_gaussian_weight_matches_numerical_inverse_transform():
    c, sigma = 2.0, 0.7
    s = np.linspace(0, 12, 120001)
    band = np.exp(-(s - c) ** 2 / (2 * sigma ** 2)) + np.exp(-(s + c) ** 2 / (2 * sigma ** 2))
    for t in [0.0, 0.3, 1.1, 2.5]:
        num = 2 / math.pi * np.trapezoid(band * np.cos(t * s), s)
        assert O.gaussian_weight(np.array([t]), c, sigma)[0] == pytest.approx(num, abs=1e-8)


def test_triangle_weight_matches_numerical_inverse_transform():
    c, h = 3.0, 1.2
    s = np.linspace(0, 12, 240001)
    band = np.maximum(0, 1 - np.abs(s - c) / h) + np.maximum(0, 1 - np.abs(s + c) / h)
    for t in [0.0, 0.4, 1.7, 3.3, 9.0]:
        num = 2 / math.pi * np.trapezoid(band * np.cos(t * s), s)
        assert O.triangle_weight(np.array([t]), c, h)[0] == pytest.approx(num, abs=1e-8)


def test_triangle_weight_gives_triangle_band():
    c, h = 3.0, 1.0
    tau, L = 0.001, 40000
    a = O.alpha_table_triangle(c, h, tau, L)
    # smooth points of the hat: rectangle rule and leapfrog phase error, O(tau)
    w = np.array([1.0, 2.2, 2.5, 3.5, 3.9, 5.0])
    ref = np.maximum(0, 1 - np.abs(w - c) / h)
    np.testing.assert_allclose(O.beta_tilde(w, a, tau), ref, atol=2e-3)
    # the peak is a kink: the transform decays like 1/t^2, and the tail cut at T = L tau
    # is bounded there by int_T^inf |alpha| dt <= 8 / (pi h T)
    T = L * tau
    assert abs(O.beta_tilde(np.array([c]), a, tau)[0] - 1.0) <= 8 / (math.pi * h * T) + 2e-3


# ---------------------------------------------------------------- fourth-order stepper (Remark 2.4)

def test_leapfrog4_recurrence_is_third_kind_chebyshev_of_its_phase():
    # with 2 cos(theta) = 2 - x + x^2/12 the recurrence is the leapfrog's with that
    # theta: q_l = cos((l + 1/2) theta) / cos(theta / 2)
    tau, L = 0.05, 60
    omega = np.array([0.5, 3.0, 20.0, 40.0, 60.0, 69.0])
    x = (tau * omega) ** 2
    theta = np.arccos(1 - x / 2 + x * x / 24)
    l = np.arange(L + 1)[:, None]
    ref = np.cos((l + 0.5) * theta) / np.cos(theta / 2)
    np.testing.assert_allclose(O.q_values_leapfrog4(omega, tau, L), ref, atol=1e-9)


def test_leapfrog4_phase_error_is_fourth_order():
    # theta - omega tau = O((omega tau)^5) for the modified-equation scheme, O(^3) for
    # the plain leapfrog: halving omega tau divides the errors by ~32 and ~8
    def theta4(z):
        return np.arccos(1 - z * z / 2 + z ** 4 / 24)

    def theta2(z):
        return np.arccos(1 - z * z / 2)
    z = np.array([0.4, 0.2, 0.1])
    e4 = np.abs(theta4(z) - z)
    e2 = np.abs(theta2(z) - z)
    np.testing.assert_allclose(e4[:-1] / e4[1:], 32.0, rtol=0.05)
    np.testing.assert_allclose(e2[:-1] / e2[1:], 8.0, rtol=0.05)
    # and the oracle's q follows its phase: q_l(omega) for a tiny tau tracks cos(l omega tau)
    tau, L, om = 1e-3, 2000, np.array([7.0])
    q = O.q_values_leapfrog4(om, tau, L)[:, 0]
    assert np.max(np.abs(q - np.cos((np.arange(L + 1) + 0.5) * om * tau) / np.cos(om * tau / 2))) < 1e-9


def test_leapfrog4_stable_to_2_sqrt3():
    tau, L = 0.01, 200                         # just past the bound q grows ~1.6x a step
    w_ok = np.array([0.99 * 2 * math.sqrt(3) / tau])
    w_bad = np.array([1.01 * 2 * math.sqrt(3) / tau])
    assert np.max(np.abs(O.q_values_leapfrog4(w_ok, tau, L))) < 50
    assert np.max(np.abs(O.q_values_leapfrog4(w_bad, tau, L))) > 1e6


@pytest.mark.parametrize("kind", ["random", "box"])
def test_leapfrog4_filter_maps_eigenvectors_by_its_beta_tilde(kind):
    if kind == "random":
        S, m = random_pencil(40, 5)
        w2, V = dense_pencil(S, m)
        vecs, omegas = V.T[::7], np.sqrt(w2[::7])
    else:
        p = box_grid((6, 5, 4))
        S, m = p.to_scipy(), p.m
        w2, V = dense_pencil(S, m)
        vecs, omegas = V.T[::11], np.sqrt(w2[::11])
    tau = 0.9 * 2 * math.sqrt(3) / math.sqrt(w2.max())
    alpha = O.alpha_table(0.3 * omegas.max(), 0.6 * omegas.max(), tau, 40)
    beta = O.beta_tilde_leapfrog4(omegas, alpha, tau)
    for v, b in zip(vecs, beta):
        out = O.filter_apply_leapfrog4(S, m, v, tau, alpha)
        np.testing.assert_allclose(out, b * v, atol=1e-10 * np.abs(v).max() * np.abs(alpha).sum())


# ---------------------------------------------------------------- fixed-dimension iteration (Sec. 4)

def test_subspace_iteration_from_exact_eigenvectors_is_exact():
    p = square_grid(20)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    modes = [(2, 3), (3, 2), (4, 1), (1, 4), (6, 6)]       # (6, 6) lies outside the interval
    X = np.stack([spectra.box_eigenvector(p.cells, k) for k in modes])
    lam = [4 * 400 * (math.sin(a * math.pi / 40) ** 2 + math.sin(b * math.pi / 40) ** 2) for a, b in modes]
    th, rel, Xa, tha, rela = O.subspace_iteration(S, p.m, X, 10.0, 15.0, tau, 150, 1e-10, 1)
    np.testing.assert_allclose(np.sort(tha), np.sort(lam), rtol=1e-12)
    inside = sorted(x for x in lam if 10.0 <= math.sqrt(x) <= 15.0)
    np.testing.assert_allclose(np.sort(th), inside, rtol=1e-12)


def test_subspace_iteration_finds_the_dominant_eigenvalues_of_the_filter():
    # from p random vectors the iteration converges to the p eigenvectors with the largest
    # |beta~|: every eigenvalue of the interval whose |beta~| is at least twice the
    # (p+1)-th largest of the whole spectrum is found, and nothing else is accepted
    p = square_grid(24)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    lo, hi, L, dim = 15.0, 22.0, 200, 36
    lam = spectra.box_spectrum(p.cells, p.h)
    beta = np.abs(O.beta_tilde(np.sqrt(lam), O.alpha_table(lo, hi, tau, L), tau))
    cut = np.sort(beta)[::-1][dim]
    w = np.sqrt(lam)
    must = np.sort(lam[(w >= lo) & (w <= hi) & (beta >= 2 * cut)])
    th, rel, X, tha, rela = O.subspace_iteration(S, p.m, start_vectors(p.n, dim, 5), lo, hi, tau, L, 1e-8, 14)
    exact = spectra.eigenvalues_in(p.cells, p.h, lo, hi)
    assert len(must) >= 15 and len(th) >= len(must)
    for t in th:
        assert np.min(np.abs(exact - t)) <= 1e-10 * t
    for t in must:
        assert np.min(np.abs(th - t)) <= 1e-10 * t


def test_refine_selection_keeps_the_interval_and_the_nearest_outside():
    # omega = 1, 2, 3, 4, 5, 6 for the interval [2.5, 4.2]: inside 3 and 4; outside, by
    # distance to the interval, 2 (0.5), 5 (0.8), 1 (1.5), 6 (1.8)
    theta = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0]) ** 2
    assert list(O.refine_selection(theta, 2.5, 4.2)) == [2, 3]
    assert list(O.refine_selection(theta, 2.5, 4.2, 1)) == [1, 2, 3]
    assert list(O.refine_selection(theta, 2.5, 4.2, 3)) == [0, 1, 2, 3, 4]
    assert list(O.refine_selection(theta, 2.5, 4.2, 10)) == [0, 1, 2, 3, 4, 5]
    # equal distances (omega = 0.5 and 4 to [1.5, 3]) go to the lower index
    assert list(O.refine_selection(np.array([0.25, 4.0, 16.0]), 1.5, 3.0, 1)) == [0, 1]
    # negative rounding noise counts as omega = 0
    assert list(O.refine_selection(np.array([-1e-12, 4.0]), 1.0, 3.0, 1)) == [0, 1]


def test_refinement_buffer_lets_rayleigh_ritz_remove_outside_noise():
    # an eigenvector of the interval polluted along an eigenvector just outside it: a
    # short filter only damps that component by its contrast, while with the outside
    # direction in the refined subspace (the buffer) Rayleigh-Ritz removes it
    p = square_grid(24)
    S = p.to_scipy()
    tau = 0.9 * 2 / math.sqrt(spectra.box_spectrum(p.cells, p.h).max())
    v = spectra.box_eigenvector(p.cells, (3, 5))          # omega = 18.05
    u = spectra.box_eigenvector(p.cells, (1, 6))          # omega = 18.64, outside [17.8, 18.3]
    lam_u = 4 * 576 * (math.sin(1 * math.pi / 48) ** 2 + math.sin(6 * math.pi / 48) ** 2)
    assert 18.3 < math.sqrt(lam_u) < 18.7
    noisy = v + 1e-4 * (np.abs(v).max() / np.abs(u).max()) * u
    lo, hi, L = 17.8, 18.3, 300
    _, _, _, th0, rel0 = O.refine_subspace(S, p.m, noisy[None, :], lo, hi, tau, L, 1e-8)
    _, _, _, th1, rel1 = O.refine_subspace(S, p.m, np.stack([noisy, u + 1e-3 * v]), lo, hi, tau, L, 1e-8)
    assert len(th0) == 1 and len(th1) == 1
    assert rel1[0] < 1e-11 and rel0[0] > 1e3 * rel1[0]
