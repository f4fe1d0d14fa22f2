"""Host logic of bench.py that needs no GPU: the all-core oracle baseline (spawned
processes over one matrix mapped from disk, one job per process per round) and the
matching of accepted Ritz values to the exact spectrum with multiplicity."""
import numpy as np

import bench
import oracle as O
from fe_inputs import square_grid, start_vectors
from fe_inputs import spectra


def test_oracle_pool_runs_one_sample_per_process_and_matches_one_process():
    p = square_grid(24)
    r = start_vectors(p.n, 1, 3)[0]
    tau = 0.9 * 2 / np.sqrt(spectra.grid_omega2(p.cells, p.h).max())
    pool = bench.OraclePool(p, r, tau, (20.0, 30.0), 2)
    try:
        units, wall = pool.round(7)
        units5, _ = pool.round(5)
    finally:
        pool.close()
    assert units == 2 * p.n * 7 and units5 == 2 * p.n * 5 and wall > 0
    assert not any(pr.is_alive() for pr in pool.procs)
    # the worker ran the oracle on the same data as a plain call would
    assert np.isfinite(O.filter_apply(p.to_scipy(), p.m, r, tau, O.alpha_table(20.0, 30.0, tau, 5))).all()


def test_matched_pairs_counts_multiplicity_once_per_copy():
    exact = np.array([1.0, 2.0, 2.0, 2.0, 3.0])
    assert bench.matched_pairs(exact, [2.0, 2.0 * (1 + 1e-12), 3.0]) == 3
    assert bench.matched_pairs(exact, [2.0] * 5 + [1.0]) == 4          # at most the multiplicity
    assert bench.matched_pairs(exact, [2.5, 1.0 + 1e-6]) == 0          # not within 1e-8


def test_small_case_oracle_solve_reports_beside_the_gpu_fields():
    from fe_inputs import WORKLOADS
    wl = WORKLOADS["square64_fp64"]
    p = wl.build()
    tau = 0.9 * 2 / np.sqrt(spectra.grid_omega2(p.cells, p.h).max())
    exact = spectra.omega2_in(p.cells, p.h, wl.omega_min, wl.omega_max)
    small = {"workload": "square64_fp64", "dofs": p.n, "kmax": wl.kmax, "L": wl.L, "tau": tau,
             "gpu_s": 0.0, "gpu_accepted": 0, "gpu_omega2": []}
    assert bench.small_solve_oracle(None) is None
    out = bench.small_solve_oracle(small)
    assert "gpu_omega2" not in out and out["oracle_accepted"] >= 1 and out["oracle_s"] > 0
    assert out["accepted_by_both"] == 0 and out["max_rel_diff_of_pairs_both_accept"] is None
    small["gpu_omega2"] = [out["oracle_accepted_omega"][0] ** 2]   # a value the oracle accepts
    out = bench.small_solve_oracle(small)
    assert out["accepted_by_both"] == 1 and out["max_rel_diff_of_pairs_both_accept"] <= 1e-15
