"""Block (SpMM) filter, multi-mesh batches and the block Krylov solver (Sec. 4,
block version) of the CUDA path against the FP64 oracle and the exact spectra."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2402_08515_gb300 as K
from fe_inputs import box_grid, flared_tube, square_grid, start_vectors
from oracle import spectra
from tests.tolerances import EIG_REL, filter_error, filter_tol, filter_tol_leapfrog4

pytestmark = pytest.mark.gpu


def _tau(p):
    return 0.9 * 2 / O.power_iteration(p.to_scipy(), p.m, start_vectors(p.n, 1, 0)[0], 300)


@pytest.fixture(scope="module")
def meshes():
    return [square_grid(40), box_grid((23, 19, 17), extent=(1.0, 0.9, 0.8)),
            flared_tube(0.03, length=1.0, r0=0.06, growth=1.2)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("b", [2, 3, 4, 8])
def test_block_filter_matches_oracle(meshes, precision, b):
    p = meshes[1]
    tau = _tau(p)
    L = 80
    bands = [(6.0, 10.0), (14.0, 18.0)]
    alphas = np.stack([O.alpha_table(a, c, tau, L) for a, c in bands])
    R = start_vectors(p.n, b, 17)
    ref = O.filter_apply_multi(p.to_scipy(), p.m, R, tau, alphas)
    with K.Context(p, precision=precision, block_b=b) as c:
        K.kes_set_filters(c.handle, [a for a, _ in bands], [x for _, x in bands], tau, L)
        out = np.zeros((2, b, p.n))
        K.kes_filter_apply(c.handle, R, out, b)
    for f in range(2):
        err = filter_error(out[f], ref[f], R, p.m, alphas[f])
        assert err <= filter_tol(L, precision), (f, err)


def test_block_columns_equal_single_vector_runs(meshes):
    # every column of the SpMM step rounds like the single-vector kernel
    p = meshes[2]
    tau = _tau(p)
    R = start_vectors(p.n, 4, 2)
    with K.Context(p, block_b=4) as c:
        K.kes_set_filter(c.handle, 8.0, 12.0, tau, 60)
        blk = np.zeros((1, 4, p.n))
        K.kes_filter_apply(c.handle, R, blk, 4)
        for j in range(4):
            one = np.zeros((1, 1, p.n))
            K.kes_filter_apply(c.handle, R[j:j + 1], one, 1)
            np.testing.assert_array_equal(one[0, 0], blk[0, j])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 7, 30])
def test_block_accumulation_schedule_equals_single_vector_runs(meshes, precision, L):
    # the block kernels add the weighted terms every third step and at the last, the
    # single-vector kernels every step: the same terms in the same order with the same
    # operations, so every column of every weight table agrees bit for bit at any length
    p = meshes[2]
    tau = _tau(p)
    R = start_vectors(p.n, 4, 5 + L)
    with K.Context(p, precision=precision, block_b=4) as c:
        K.kes_set_filters(c.handle, [8.0, 14.0], [12.0, 18.0], tau, L)
        blk = np.zeros((2, 4, p.n))
        K.kes_filter_apply(c.handle, R, blk, 4)
        for j in range(4):
            one = np.zeros((2, 1, p.n))
            K.kes_filter_apply(c.handle, R[j:j + 1], one, 1)
            np.testing.assert_array_equal(one[:, 0], blk[:, j])
        cols = np.zeros((4, p.n))                  # columns 0-1 with table 0, 2-3 with table 1
        K.kes_filter_apply_columns(c.handle, R, cols, 4)
    np.testing.assert_array_equal(cols[:2], blk[0, :2])
    np.testing.assert_array_equal(cols[2:], blk[1, 2:])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("b", [2, 4, 8])
def test_every_block_launch_shape_rounds_identically(meshes, precision, b):
    # lane-per-row and two-lanes-per-row shapes, with and without L2 prefetch: every
    # column is the same FMA chain, so the filtered blocks agree bit for bit
    p = meshes[2]
    tau = _tau(p)
    R = start_vectors(p.n, b, 31)
    outs = []
    for v in range(K.kes_launch_shapes()[1]):
        with K.Context(p, precision=precision, block_b=b, blk_variant=v) as c:
            K.kes_set_filters(c.handle, [8.0, 14.0], [12.0, 18.0], tau, 30)
            o = np.zeros((2, b, p.n))
            K.kes_filter_apply(c.handle, R, o, b)
            cols = np.zeros((b, p.n))
            K.kes_filter_apply_columns(c.handle, R, cols, b)
            outs.append((o, cols))
    for o, cols in outs[1:]:
        np.testing.assert_array_equal(o, outs[0][0])
        np.testing.assert_array_equal(cols, outs[0][1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_meshes_filter_matches_oracle(meshes, precision):
    taus = np.array([_tau(p) for p in meshes])
    L = 70
    wmin = np.array([[10.0, 20.0], [5.0, 9.0], [4.0, 7.0]])
    wmax = np.array([[15.0, 26.0], [8.0, 13.0], [6.0, 9.0]])
    b = 2
    Rs = [start_vectors(p.n, b, 30 + j) for j, p in enumerate(meshes)]
    R = np.concatenate(Rs, axis=1)                       # (b, n_total)
    with K.Context(meshes, precision=precision, block_b=b) as c:
        assert K.kes_mesh_count(c.handle) == 3 and K.kes_size(c.handle) == R.shape[1]
        K.kes_set_filters_batch(c.handle, wmin, wmax, taus, L)
        out = np.zeros((2, b, R.shape[1]))
        K.kes_filter_apply(c.handle, R, out, b)
    off = 0
    for j, p in enumerate(meshes):
        alphas = np.stack([O.alpha_table(wmin[j, f], wmax[j, f], taus[j], L) for f in range(2)])
        ref = O.filter_apply_multi(p.to_scipy(), p.m, Rs[j], taus[j], alphas)
        for f in range(2):
            err = filter_error(out[f, :, off:off + p.n], ref[f], Rs[j], p.m, alphas[f])
            assert err <= filter_tol(L, precision), (j, f, err)
        off += p.n


def test_block_solver_b1_equals_single_vector_solver():
    p = square_grid(48)
    tau = _tau(p)
    r0 = start_vectors(p.n, 1, 0)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol = 40, 1e-8
    with K.Context(p) as c:
        K.kes_set_filter(c.handle, 15.0, 25.0, tau, 200)
        a = K.kes_krylov_solve(c.handle, r0[0], so)
        b = K.kes_block_krylov_solve(c.handle, r0, 1, so)[0]
    np.testing.assert_array_equal(a["ritz_omega2"], b["ritz_omega2"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_block_solver_resolves_multiplicity_like_the_oracle(precision):
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    exact = spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0)
    R = start_vectors(p.n, 2, 3)
    tol = 1e-8 if precision == "fp64" else 1e-5
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.want_vectors = 100, tol, 1
    with K.Context(p, precision=precision, block_b=2) as c:
        K.kes_set_filter(c.handle, 20.0, 30.0, tau, 300)
        res = K.kes_block_krylov_solve(c.handle, R, 2, so)[0]
    ores = O.block_krylov_solve(S, p.m, R, 20.0, 30.0, tau, 300, 100, tol)
    print(f"{precision}: GPU accepted {res['n_pairs']}, oracle {len(ores.omega2)}, exact {len(exact)}")
    for th in res["omega2"]:
        assert np.min(np.abs(exact - th)) <= EIG_REL[precision] * th
    if precision == "fp64":
        assert res["n_pairs"] == len(exact) == len(ores.omega2)
        np.testing.assert_allclose(np.sort(res["omega2"]), exact, rtol=1e-10)
    else:
        assert res["n_pairs"] >= len(exact) - 4
    for th, x in zip(res["omega2"], res["vectors"]):
        r = S @ x - th * p.m * x
        assert np.linalg.norm(r) <= tol * 1.01 * th * np.linalg.norm(p.m * x)


def test_batched_block_solver_per_mesh(meshes):
    sq, box = meshes[0], meshes[1]
    taus = np.array([_tau(sq), _tau(box)])
    wmin = np.array([[14.0], [7.0]])
    wmax = np.array([[20.0], [10.0]])
    b = 2
    Rs = [start_vectors(sq.n, b, 5), start_vectors(box.n, b, 6)]
    R = np.concatenate(Rs, axis=1)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol = 80, 1e-8
    with K.Context([sq, box], block_b=b) as c:
        K.kes_set_filters_batch(c.handle, wmin, wmax, taus, 250)
        res = K.kes_block_krylov_solve(c.handle, R, b, so)
    for j, (p, r) in enumerate(zip([sq, box], res)):
        exact = spectra.eigenvalues_in(p.cells, p.h, wmin[j, 0], wmax[j, 0])
        print(f"mesh {j}: accepted {r['n_pairs']} of {len(exact)}")
        assert r["n_pairs"] >= 1 and r["k_used"] <= 80
        for th in r["omega2"]:
            assert np.min(np.abs(exact - th)) <= 1e-10 * th
        oref = O.block_krylov_solve(p.to_scipy(), p.m, Rs[j], wmin[j, 0], wmax[j, 0], taus[j], 250, 80, 1e-8)
        assert abs(r["n_pairs"] - len(oref.omega2)) <= 2


@pytest.mark.parametrize("b,refine_L", [(1, 0), (2, 0), (1, 100)])
def test_fp32_solve_with_fp64_refinement_reaches_fp64_residuals(b, refine_L):
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    exact = spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0)
    R = start_vectors(p.n, b, 3)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.want_vectors, so.refine_sweeps, so.refine_L = 100, 1e-8, 1, 2, refine_L
    with K.Context(p, precision="fp32", block_b=b) as c:
        K.kes_set_filter(c.handle, 20.0, 30.0, tau, 300)
        res = K.kes_block_krylov_solve(c.handle, R, b, so)[0]
    assert res["refine_steps"] > 0 and res["refine_steps"] % (refine_L or 300) == 0
    distinct, _ = spectra.distinct(exact)
    found, _ = spectra.distinct(res["omega2"])
    print(f"b={b}: refined FP32 accepted {res['n_pairs']} pairs ({len(found)} of {len(distinct)} distinct) "
          f"after {res['refine_steps']} FP64 steps")
    assert res["refine_steps"] > 0
    assert len(found) >= len(distinct) - 1
    for th, x in zip(res["omega2"], res["vectors"]):
        assert np.min(np.abs(exact - th)) <= 1e-10 * th
        r = S @ x - th * p.m * x
        assert np.linalg.norm(r) <= 1.01e-8 * th * np.linalg.norm(p.m * x)



@pytest.mark.parametrize("b,block_b,refine_L", [(1, 8, 0), (2, 2, 0), (2, 4, 100)])
def test_fp32_pair_refinement_reaches_fp64_residuals(b, block_b, refine_L):
    # the refinement sweep's filter in FP32 pairs (double-float arithmetic on the FP32
    # units): the same pairs as the FP64 sweep, eigenvalues to 1e-10 of the closed form and
    # host-computed residuals within the 1e-8 acceptance
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    exact = spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0)
    R = start_vectors(p.n, b, 3)
    out = {}
    for prec in (K.KES_REFINE_FP64, K.KES_REFINE_F32X2):
        so = K.kes_solve_opts_default()
        so.kmax, so.tol, so.want_vectors, so.refine_sweeps, so.refine_L = 100, 1e-8, 1, 2, refine_L
        so.refine_precision = prec
        with K.Context(p, precision="fp32", block_b=block_b) as c:
            K.kes_set_filter(c.handle, 20.0, 30.0, tau, 300)
            out[prec] = K.kes_block_krylov_solve(c.handle, R, b, so)[0]
    r64, rx2 = out[K.KES_REFINE_FP64], out[K.KES_REFINE_F32X2]
    print(f"b={b}: FP64 sweep {r64['n_pairs']} pairs, FP32-pair sweep {rx2['n_pairs']} pairs")
    assert rx2["refine_steps"] == r64["refine_steps"] > 0
    assert abs(rx2["n_pairs"] - r64["n_pairs"]) <= 1 and rx2["n_pairs"] >= 1
    for th, x in zip(rx2["omega2"], rx2["vectors"]):
        assert np.min(np.abs(exact - th)) <= 1e-10 * th
        r = S @ x - th * p.m * x
        assert np.linalg.norm(r) <= 1.01e-8 * th * np.linalg.norm(p.m * x)
    for th in rx2["omega2"]:                       # the pairs both sweeps accept agree
        d = np.abs(r64["omega2"] - th)
        if d.size and d.min() <= 1e-9 * th:
            assert d.min() <= 1e-11 * th


def test_fp32_pair_refinement_needs_a_block_context():
    p = square_grid(16)
    tau = _tau(p)
    so = K.kes_solve_opts_default()
    so.kmax, so.refine_sweeps, so.refine_precision = 20, 1, K.KES_REFINE_F32X2
    with K.Context(p, precision="fp32", block_b=1) as c:
        K.kes_set_filter(c.handle, 20.0, 30.0, tau, 100)
        with pytest.raises(K.KesError) as e:
            K.kes_block_krylov_solve(c.handle, start_vectors(p.n, 1, 1), 1, so)
        assert e.value.status == -8
        so.refine_precision = 7
        with pytest.raises(K.KesError) as e:
            K.kes_block_krylov_solve(c.handle, start_vectors(p.n, 1, 1), 1, so)
        assert e.value.status == -1
    with K.Context(p, precision="fp64", block_b=1) as c:   # FP64 contexts refine in FP64
        K.kes_set_filter(c.handle, 20.0, 30.0, tau, 100)
        so.refine_precision = K.KES_REFINE_F32X2
        K.kes_block_krylov_solve(c.handle, start_vectors(p.n, 1, 1), 1, so)


def test_large_krylov_dimension_projects_and_certifies():
    # 800 basis vectors: the projection kernels then hold more than 48 KB of Ritz
    # coefficients per block (k x 8 doubles) and take the opted-in shared memory; the solve
    # must still return exact eigenvalues with host-verified residuals, and a Krylov
    # dimension beyond the kernels' limit is refused
    p = box_grid((21, 17, 15), extent=(1.0, 0.85, 0.75))      # 4,480 dofs
    S = p.to_scipy()
    tau = _tau(p)
    R = start_vectors(p.n, 8, 41)
    exact = spectra.eigenvalues_in(p.cells, p.h, 10.0, 14.0)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.check_every, so.want_vectors = 800, 1e-8, 800, 1
    with K.Context(p, precision="fp64", block_b=8) as c:
        K.kes_set_filter(c.handle, 10.0, 14.0, tau, 40)
        res = K.kes_block_krylov_solve(c.handle, R, 8, so)[0]
        so.kmax = 4000
        with pytest.raises(K.KesError) as e:
            K.kes_block_krylov_solve(c.handle, R, 8, so)
        assert e.value.status == -8
    assert res["k_used"] > 768 and res["n_pairs"] > 0
    for th, x in zip(res["omega2"], res["vectors"]):
        assert np.min(np.abs(exact - th)) <= 1e-10 * th
        assert np.linalg.norm(S @ x - th * p.m * x) <= 1.01e-8 * th * np.linalg.norm(p.m * x)


@pytest.mark.parametrize("extra", [0, 6])
def test_refinement_with_a_buffer_matches_oracle(extra):
    # FP64 block solve, then one refinement sweep over the in-interval Ritz vectors and
    # the `extra` nearest outside the interval (refine_extra): the refined subspace is
    # the oracle's up to rounding, so its in-interval Ritz values agree with the oracle's
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    lo, hi, L, kmax = 20.0, 30.0, 300, 100   # 36 eigenvalues (19 distinct), all accepted by kmax 100
    R = start_vectors(p.n, 2, 5)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.check_every, so.want_vectors = kmax, 1e-8, kmax, 1
    so.refine_sweeps, so.refine_extra = 1, extra
    with K.Context(p, precision="fp64", block_b=2) as c:
        K.kes_set_filter(c.handle, lo, hi, tau, L)
        res = K.kes_block_krylov_solve(c.handle, R, 2, so)[0]
    ref = O.multi_interval_krylov_solve(S, p.m, R, [(lo, hi)], tau, L, kmax, 1e-8, check_every=kmax,
                                        refine_sweeps=1, refine_extra=extra)
    inside = ~np.isnan(res["ritz_rel_res"])
    got = np.sort(res["ritz_omega2"][inside])
    exact = spectra.eigenvalues_in(p.cells, p.h, lo, hi)
    assert res["refine_steps"] > 0
    for th, x in zip(res["omega2"], res["vectors"]):
        assert np.min(np.abs(exact - th)) <= 1e-10 * th
        assert np.linalg.norm(S @ x - th * p.m * x) <= 1.01e-8 * th * np.linalg.norm(p.m * x)
    # the refined in-interval Ritz values: the oracle's refinement of the same selection
    _, _, _, th_ref, _ = O.refine_subspace(S, p.m, _selected_ritz_vectors(S, p.m, R, lo, hi, tau, L, kmax, extra),
                                           lo, hi, tau, L, 1e-8, 1, extra)
    th_ref = np.sort(th_ref)
    print(f"extra={extra}: {got.size} in-interval Ritz values (oracle {th_ref.size}), {res['n_pairs']} accepted, "
          f"{res['refine_steps']} refinement steps")
    assert got.size == th_ref.size
    np.testing.assert_allclose(got, th_ref, rtol=1e-9)
    assert abs(res["n_pairs"] - len(ref.omega2)) <= 1


def _selected_ritz_vectors(S, m, R, lo, hi, tau, L, kmax, extra):
    """The oracle's Ritz vectors that a refinement with `extra` buffer vectors filters."""
    r = O.block_krylov_solve(S, m, R, lo, hi, tau, L, kmax, 1e-8, check_every=kmax, keep_basis=True)
    theta, Y = O.rayleigh_ritz(S, r.basis)
    return (Y.T @ r.basis)[O.refine_selection(theta, lo, hi, extra)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("band", ["gaussian", "triangle"])
def test_band_weights_filter_and_solve(precision, band):
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    L = 300
    if band == "gaussian":
        alpha = O.alpha_table_gaussian(25.0, 2.5, tau, L)
    else:
        alpha = O.alpha_table_triangle(25.0, 5.0, tau, L)
    r = start_vectors(p.n, 1, 9)
    ref = O.filter_apply(S, p.m, r[0], tau, alpha)
    tol = 1e-8 if precision == "fp64" else 1e-5
    with K.Context(p, precision=precision) as ctx:
        K.kes_set_weights(ctx.handle, alpha[None, None, :], [[20.0]], [[30.0]], [tau], L)
        out = np.zeros((1, 1, p.n))
        K.kes_filter_apply(ctx.handle, r, out, 1)
        assert filter_error(out[0], ref, r, p.m, alpha) <= filter_tol(L, precision)
        so = K.kes_solve_opts_default()
        so.kmax, so.tol = 80, tol
        res = K.kes_krylov_solve(ctx.handle, start_vectors(p.n, 1, 0)[0], so)
    exact = spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0)
    print(f"{precision} {band} band: accepted {res['n_pairs']}")
    assert res["n_pairs"] >= 5
    for th in res["omega2"]:
        assert np.min(np.abs(exact - th)) <= EIG_REL[precision] * th


# ---------------------------------------------------------------- several intervals

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("F,b", [(2, 2), (2, 4), (3, 6), (4, 8)])
def test_filter_apply_columns_matches_oracle(meshes, precision, F, b):
    # column j is filtered with table j // (b // F) only; it rounds exactly like that
    # table's sum for that column in kes_filter_apply (b = 6 pads to 8 columns)
    p = meshes[1]
    tau = _tau(p)
    L = 80
    bands = [(4.0 + 3 * f, 6.5 + 3 * f) for f in range(F)]
    alphas = np.stack([O.alpha_table(a, c, tau, L) for a, c in bands])
    R = start_vectors(p.n, b, 40 + b)
    g = b // F
    with K.Context(p, precision=precision, block_b=b) as c:
        K.kes_set_filters(c.handle, [a for a, _ in bands], [x for _, x in bands], tau, L)
        cols = np.zeros((b, p.n))
        K.kes_filter_apply_columns(c.handle, R, cols, b)
        full = np.zeros((F, b, p.n))
        K.kes_filter_apply(c.handle, R, full, b)
    for j in range(b):
        ref = O.filter_apply(p.to_scipy(), p.m, R[j], tau, alphas[j // g])
        err = filter_error(cols[j:j + 1], ref[None, :], R[j:j + 1], p.m, alphas[j // g])
        assert err <= filter_tol(L, precision), (j, err)
        np.testing.assert_array_equal(cols[j], full[j // g, j])


def test_filter_apply_columns_rejects_bad_widths(meshes):
    p = meshes[0]
    with K.Context(p, block_b=4) as c:
        K.kes_set_filters(c.handle, [5.0, 9.0], [7.0, 11.0], _tau(p), 20)
        out = np.zeros((3, p.n))
        with pytest.raises(K.KesError):
            K.kes_filter_apply_columns(c.handle, start_vectors(p.n, 3, 0), out, 3)


# listed high band first, so that the merge into ascending order permutes the labels
MULTI_BANDS = [(36.0, 39.0), (20.0, 25.0)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multi_interval_solve_matches_oracle(precision):
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    R = start_vectors(p.n, 4, 3)
    tol = 1e-8 if precision == "fp64" else 1e-5
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.want_vectors = 120, tol, 1
    with K.Context(p, precision=precision, block_b=4) as c:
        K.kes_set_filters(c.handle, [a for a, _ in MULTI_BANDS], [x for _, x in MULTI_BANDS], tau, 300)
        res = K.kes_block_krylov_solve(c.handle, R, 4, so)[0]
    ores = O.multi_interval_krylov_solve(S, p.m, R, MULTI_BANDS, tau, 300, 120, tol)
    counts = [int(np.sum(res["interval"] == f)) for f in range(2)]
    print(f"{precision}: GPU accepted {counts} per interval, oracle "
          f"{[int(np.sum(ores.interval == f)) for f in range(2)]}")
    assert np.all(np.diff(res["omega2"]) >= 0)
    for f, (lo, hi) in enumerate(MULTI_BANDS):
        exact = spectra.eigenvalues_in(p.cells, p.h, lo, hi)
        got = res["omega2"][res["interval"] == f]
        assert np.all((np.sqrt(got) >= lo) & (np.sqrt(got) <= hi))
        for th in got:
            assert np.min(np.abs(exact - th)) <= EIG_REL[precision] * th
        if precision == "fp64":
            assert len(got) == len(exact) == int(np.sum(ores.interval == f))
            np.testing.assert_allclose(got, ores.omega2[ores.interval == f], rtol=1e-10)
        else:
            assert len(got) >= len(exact) - 4
    for th, x in zip(res["omega2"], res["vectors"]):
        assert np.linalg.norm(S @ x - th * p.m * x) <= tol * 1.01 * th * np.linalg.norm(p.m * x)


def test_multi_interval_solve_equals_separate_solves():
    # the intervals share the trajectory but nothing they compute: each interval's pairs
    # are bit for bit those of a separate block solve from its own start vectors
    p = square_grid(28)
    tau = _tau(p)
    R = start_vectors(p.n, 4, 11)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol = 60, 1e-8
    with K.Context(p, block_b=4) as c:
        K.kes_set_filters(c.handle, [a for a, _ in MULTI_BANDS], [x for _, x in MULTI_BANDS], tau, 250)
        both = K.kes_block_krylov_solve(c.handle, R, 4, so)[0]
    for f, (lo, hi) in enumerate(MULTI_BANDS):
        with K.Context(p, block_b=2) as c:
            K.kes_set_filter(c.handle, lo, hi, tau, 250)
            one = K.kes_block_krylov_solve(c.handle, R[2 * f:2 * f + 2], 2, so)[0]
        np.testing.assert_array_equal(both["omega2"][both["interval"] == f], one["omega2"])
        np.testing.assert_array_equal(both["rel_res"][both["interval"] == f], one["rel_res"])


def test_multi_interval_fp32_with_refinement():
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau(p)
    R = start_vectors(p.n, 4, 3)
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.want_vectors, so.refine_sweeps = 100, 1e-8, 1, 2
    with K.Context(p, precision="fp32", block_b=4) as c:
        K.kes_set_filters(c.handle, [a for a, _ in MULTI_BANDS], [x for _, x in MULTI_BANDS], tau, 300)
        res = K.kes_block_krylov_solve(c.handle, R, 4, so)[0]
    assert res["refine_steps"] > 0
    for f, (lo, hi) in enumerate(MULTI_BANDS):
        exact = spectra.eigenvalues_in(p.cells, p.h, lo, hi)
        got = res["omega2"][res["interval"] == f]
        d_exact, _ = spectra.distinct(exact)
        d_got, _ = spectra.distinct(got)
        print(f"interval {f}: refined FP32 accepted {len(got)} ({len(d_got)} of {len(d_exact)} distinct)")
        assert len(d_got) >= len(d_exact) - 1
        for th in got:
            assert np.min(np.abs(exact - th)) <= 1e-10 * th
    for th, x in zip(res["omega2"], res["vectors"]):
        assert np.linalg.norm(S @ x - th * p.m * x) <= 1.01e-8 * th * np.linalg.norm(p.m * x)


# ---------------------------------------------------------------- fourth-order stepper (Remark 2.4)

def _tau4(p):
    return 0.9 * 2 * math.sqrt(3) / O.power_iteration(p.to_scipy(), p.m, start_vectors(p.n, 1, 0)[0], 300)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("b", [1, 4])
def test_leapfrog4_filter_matches_oracle(meshes, precision, b):
    p = meshes[1]
    tau = _tau4(p)
    L = 80
    alpha = O.alpha_table(6.0, 10.0, tau, L)
    R = start_vectors(p.n, b, 23)
    with K.Context(p, precision=precision, block_b=b, stepper="leapfrog4") as c:
        K.kes_set_filter(c.handle, 6.0, 10.0, tau, L)
        out = np.zeros((1, b, p.n))
        K.kes_filter_apply(c.handle, R, out, b)
        st = K.kes_get_stats(c.handle)
    assert st["kernel_launches"] >= 2 * L      # a stage and a step per time step
    for j in range(b):
        ref = O.filter_apply_leapfrog4(p.to_scipy(), p.m, R[j], tau, alpha)
        err = filter_error(out[0, j], ref, R[j], p.m, alpha)
        print(f"{precision} b={b} column {j}: error {err:.2e} (tolerance {filter_tol_leapfrog4(L, precision):.2e})")
        assert err <= filter_tol_leapfrog4(L, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_leapfrog4_solve_finds_closed_form_eigenvalues(precision):
    p = square_grid(32)
    S = p.to_scipy()
    tau = _tau4(p)
    L = 175                                     # T close to the leapfrog tests' 300 steps of 0.9 * 2 / omega
    tol = 1e-8 if precision == "fp64" else 1e-5
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.want_vectors = 80, tol, 1
    with K.Context(p, precision=precision, stepper="leapfrog4") as c:
        K.kes_set_filter(c.handle, 20.0, 30.0, tau, L)
        res = K.kes_krylov_solve(c.handle, start_vectors(p.n, 1, 0)[0], so)
    exact = spectra.eigenvalues_in(p.cells, p.h, 20.0, 30.0)
    d_exact, _ = spectra.distinct(exact)
    d_got, _ = spectra.distinct(res["omega2"])
    print(f"{precision}: accepted {len(d_got)} of {len(d_exact)} distinct")
    assert len(d_got) >= len(d_exact) - (0 if precision == "fp64" else 4)
    for th, x in zip(res["omega2"], res["vectors"]):
        assert np.min(np.abs(exact - th)) <= EIG_REL[precision] * th
        assert np.linalg.norm(S @ x - th * p.m * x) <= tol * 1.01 * th * np.linalg.norm(p.m * x)


def test_leapfrog4_cfl_bound():
    p = square_grid(24)
    for stepper, ratio, ok in [("leapfrog", 2.5, False), ("leapfrog4", 2.5, True), ("leapfrog4", 3.5, False)]:
        with K.Context(p, stepper=stepper) as c:
            w, _ = K.kes_estimate_omega_max(c.handle, 300, start_vectors(p.n, 1, 0)[0])
            if ok:
                K.kes_set_filter(c.handle, 10.0, 20.0, ratio / w, 20)
            else:
                with pytest.raises(K.KesError):
                    K.kes_set_filter(c.handle, 10.0, 20.0, ratio / w, 20)


def test_meshes_times_intervals_equal_separate_solves(meshes):
    # two meshes of different sizes, two intervals each, in one solve: the batched
    # Gram-Schmidt stages serve all four processes with one launch per stage, and each
    # process's pairs must still be bit for bit those of its own separate solve
    sq, box = meshes[0], meshes[1]
    taus = np.array([_tau(sq), _tau(box)])
    wmin = np.array([[14.0, 22.0], [6.0, 11.0]])
    wmax = np.array([[19.0, 27.0], [9.0, 14.0]])
    Rs = [start_vectors(sq.n, 4, 41), start_vectors(box.n, 4, 42)]
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.check_every = 40, 1e-8, 8
    with K.Context([sq, box], block_b=4) as c:
        K.kes_set_filters_batch(c.handle, wmin, wmax, taus, 200)
        both = K.kes_block_krylov_solve(c.handle, np.concatenate(Rs, axis=1), 4, so)
    for j, p in enumerate([sq, box]):
        for f in range(2):
            with K.Context(p, block_b=2) as c:
                K.kes_set_filter(c.handle, wmin[j, f], wmax[j, f], taus[j], 200)
                one = K.kes_block_krylov_solve(c.handle, Rs[j][2 * f:2 * f + 2], 2, so)[0]
            sel = both[j]["interval"] == f
            print(f"mesh {j} interval {f}: {int(sel.sum())} pairs")
            np.testing.assert_array_equal(both[j]["omega2"][sel], one["omega2"])
            np.testing.assert_array_equal(both[j]["rel_res"][sel], one["rel_res"])


# ---------------------------------------------------------------- fixed-dimension iteration (Sec. 4)

@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32x2"])
def test_subspace_solve_matches_oracle(precision):
    # fp32x2: a context of the FP32 form whose sweeps filter in FP32 pairs: held to the
    # FP64 form's tolerances against the FP64 oracle
    p = square_grid(24)
    S = p.to_scipy()
    tau = _tau(p)
    lo, hi, L, dim, sweeps = 15.0, 22.0, 200, 36, 14
    X0 = start_vectors(p.n, dim, 5)
    x2, label = precision == "fp32x2", precision
    precision = "fp64" if x2 else precision       # the tolerances it is held to
    tol = 1e-8 if precision == "fp64" else 1e-5
    so = K.kes_solve_opts_default()
    so.kmax, so.tol, so.refine_sweeps, so.want_vectors = dim, tol, sweeps, 1
    so.refine_precision = K.KES_REFINE_F32X2 if x2 else K.KES_REFINE_FP64
    with K.Context(p, precision="fp32" if x2 else precision, block_b=8) as c:
        K.kes_set_filter(c.handle, lo, hi, tau, L)
        res = K.kes_subspace_solve(c.handle, X0, so)[0]
    th, rel, X, tha, rela = O.subspace_iteration(S, p.m, X0, lo, hi, tau, L, tol, sweeps)
    exact = spectra.eigenvalues_in(p.cells, p.h, lo, hi)
    print(f"{label}: GPU accepted {res['n_pairs']}, oracle {len(th)} of {len(exact)}; "
          f"{res['refine_steps']} steps")
    assert res["time_steps"] == 0 and res["refine_steps"] > 0 and res["k_used"] <= dim
    for t in res["omega2"]:
        assert np.min(np.abs(exact - t)) <= EIG_REL[precision] * t
    if precision == "fp64":
        # every oracle pair well inside the tolerance is found (pairs near it may land
        # on either side with a different rounding order)
        for t in th[rel <= tol / 10]:
            assert np.min(np.abs(res["omega2"] - t)) <= 1e-10 * t
        assert abs(res["n_pairs"] - len(th)) <= 2
    else:
        assert res["n_pairs"] >= len(th) - 3
    for t, x in zip(res["omega2"], res["vectors"]):
        assert np.linalg.norm(S @ x - t * p.m * x) <= tol * 1.01 * t * np.linalg.norm(p.m * x)


# ---------------------------------------------------------------- compact column index

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("b,stepper", [(1, "leapfrog"), (4, "leapfrog"), (1, "leapfrog4"), (4, "leapfrog4")])
def test_compact_column_index_rounds_identically(meshes, precision, b, stepper):
    # the 16-bit column - row index names the same columns as the int32 one: the filtered
    # blocks agree bit for bit, and the step moves 2 bytes less per stored entry
    p = meshes[1]
    tau = _tau4(p) if stepper == "leapfrog4" else _tau(p)
    R = start_vectors(p.n, b, 61)
    outs, steps = [], []
    for compact in (False, True):
        with K.Context(p, precision=precision, block_b=b, stepper=stepper, compact_cols=compact) as c:
            K.kes_set_filter(c.handle, 6.0, 10.0, tau, 40)
            o = np.zeros((1, b, p.n))
            K.kes_filter_apply(c.handle, R, o, b)
            outs.append(o)
            steps.append(K.kes_step_bytes(c.handle, 1, 1))
    np.testing.assert_array_equal(outs[0], outs[1])
    assert steps[1] == steps[0] - 2 * p.nnz * (2 if stepper == "leapfrog4" else 1)
