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


def test_kernel_source_hash_ignores_comments_and_sees_code(tmp_path):
    # a committed profile's traffic figure stays attached to the kernel code it was taken on:
    # comment edits keep the hash, any code change alters it
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(int* p) {\n  p[0] = 1;  // store\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("// another header\n\n__global__ void k(int* p) {\n  p[0] = 1;\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("__global__ void k(int* p) {\n  p[0] = 2;\n}\n")
    assert bench.kernel_source_hash(str(a)) == bench.kernel_source_hash(str(b))
    assert bench.kernel_source_hash(str(a)) != bench.kernel_source_hash(str(c))


def test_committed_step_profiles_match_the_current_kernels():
    # the profiles the bench line's `traffic` comes from were taken on the current code
    assert bench.profiled_traffic("cube128_fp64", bench.STEP_KERNEL_SRC) is not None
    assert bench.profiled_traffic("cube128_fp32", bench.STEP_KERNEL_SRC) is not None
    assert bench.profiled_traffic("batch12_fp32", bench.BLOCK_KERNEL_SRC) is not None


def test_time_to_solution_forms_are_well_formed():
    names = [f[0] for f in bench.TTS_FORMS]
    assert len(names) == len(set(names))
    for name, prec, b, sweeps, frac, extra, rprec in bench.TTS_FORMS:
        assert prec in ("fp64", "fp32") and b in (1, 8) and 0 < frac <= 1.0 and extra >= 0
        assert (sweeps > 0) == (prec == "fp32")        # the FP32 forms are refined, FP64 ones not
        assert rprec in (0, 1) and ("x2" in name) == (rprec == 1)
