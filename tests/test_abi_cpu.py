"""C-ABI checks that need no GPU: the library loads, exports every function
include/kes.h declares, and its host-side logic (weights, filter response,
small symmetric eigensolver, input validation) is right."""
import math
import os

import numpy as np
import pytest

import paper_2402_08515_gb300 as K
import oracle as O  # noqa: E402
from fe_inputs import square_grid  # noqa: E402


def test_every_header_function_is_exported():
    names = K.header_functions()
    assert len(names) >= 15
    missing = [f for f in names if not hasattr(K.lib, f)]
    assert not missing, missing


def test_status_strings():
    for s in [0, 1, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert K.kes_strerror(s) and K.kes_strerror(s) != "unknown status"


def test_alpha_table_matches_oracle():
    for wmin, wmax, tau, L in [(20, 30, 0.0099467, 300), (40, 45, 0.0040598, 600), (0, 3, 0.0056, 300)]:
        np.testing.assert_allclose(K.kes_alpha_table(wmin, wmax, tau, L),
                                   O.alpha_table(wmin, wmax, tau, L), rtol=1e-13, atol=1e-17)


def test_filter_response_matches_oracle():
    tau, L = 0.0099467, 300
    w = np.linspace(0, 2 / tau * 0.999, 400)
    np.testing.assert_allclose(K.kes_filter_response(20, 30, tau, L, w),
                               O.beta_tilde(w, O.alpha_table(20, 30, tau, L), tau), rtol=0, atol=1e-11)


@pytest.mark.parametrize("k", [1, 2, 3, 7, 40, 120])
def test_sym_eig_random(k):
    rng = np.random.default_rng(k)
    A = rng.standard_normal((k, k))
    A = A + A.T
    w, V = K.kes_sym_eig(A)
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, np.abs(ref).max())
    np.testing.assert_allclose(w, ref, atol=1e-13 * scale * k)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-13 * k)
    np.testing.assert_allclose(A @ V, V * w, atol=1e-13 * scale * k)


def test_sym_eig_clusters_and_diagonal():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    d = np.repeat([1.0, 2.0, 2.0 + 1e-12, 5.0, 1e3], 6)
    A = (Q * d) @ Q.T
    A = 0.5 * (A + A.T)
    w, V = K.kes_sym_eig(A)
    np.testing.assert_allclose(w, np.sort(d), atol=1e-11)
    np.testing.assert_allclose(A @ V, V * w, atol=1e-11)
    D = np.diag([3.0, -1.0, 2.0])
    w, V = K.kes_sym_eig(D)
    np.testing.assert_array_equal(w, [-1.0, 2.0, 3.0])


def test_sym_eig_reads_lower_triangle_only():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((12, 12))
    A = A + A.T
    A_low = np.tril(A) + np.triu(np.full((12, 12), 1e300), 1)
    np.testing.assert_allclose(K.kes_sym_eig(A_low)[0], np.linalg.eigvalsh(A), atol=1e-12)


def test_create_validates_inputs_before_touching_the_gpu():
    p = square_grid(6)
    bad_m = p.m.copy()
    bad_m[3] = 0.0
    with pytest.raises(K.KesError) as e:
        K.kes_create(p.n, p.row_ptr, p.col, p.val, bad_m)
    assert e.value.status == -2
    bad_col = p.col.copy()
    bad_col[5] = p.n + 3
    with pytest.raises(K.KesError) as e:
        K.kes_create(p.n, p.row_ptr, bad_col, p.val, p.m)
    assert e.value.status == -1
    bad_val = p.val.copy()
    bad_val[0] = math.nan
    with pytest.raises(K.KesError) as e:
        K.kes_create(p.n, p.row_ptr, p.col, bad_val, p.m)
    assert e.value.status == -1


def test_host_helpers_reject_bad_arguments():
    with pytest.raises(K.KesError):
        K.kes_alpha_table(3.0, 2.0, 0.1, 10)
    with pytest.raises(K.KesError):
        K.kes_alpha_table(2.0, 3.0, -0.1, 10)
    with pytest.raises(K.KesError):
        K.kes_filter_response(2.0, 3.0, 0.1, 0, [1.0])


def test_gaussian_weights_match_oracle():
    for c, sigma, tau, L in [(25.0, 3.0, 0.0099, 300), (42.5, 1.5, 0.004, 600), (0.0, 2.0, 0.01, 50)]:
        np.testing.assert_allclose(K.kes_alpha_gaussian(c, sigma, tau, L), O.alpha_table_gaussian(c, sigma, tau, L),
                                   rtol=1e-13, atol=1e-16)
    with pytest.raises(K.KesError):
        K.kes_alpha_gaussian(1.0, -1.0, 0.1, 10)


def test_weights_response_matches_oracle():
    tau, L = 0.0099, 300
    w = np.linspace(0.0, 60.0, 97)
    for a in [O.alpha_table(20.0, 30.0, tau, L), O.alpha_table_gaussian(25.0, 3.0, tau, L),
              O.alpha_table_triangle(25.0, 5.0, tau, L)]:
        np.testing.assert_allclose(K.kes_weights_response(a, tau, w), O.beta_tilde(w, a, tau), rtol=1e-11, atol=1e-12)


def test_triangle_weights_match_oracle():
    for c, h, tau, L in [(25.0, 5.0, 0.0099, 300), (42.5, 2.5, 0.004, 600), (0.0, 2.0, 0.01, 50)]:
        np.testing.assert_allclose(K.kes_alpha_triangle(c, h, tau, L), O.alpha_table_triangle(c, h, tau, L),
                                   rtol=1e-13, atol=1e-16)
    with pytest.raises(K.KesError):
        K.kes_alpha_triangle(1.0, 0.0, 0.1, 10)


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of kes_opts, kes_solve_opts, kes_result and kes_stats must have
    # the C sizes and field offsets: compile a probe against include/kes.h
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"kes_opts": K.KesOpts, "kes_solve_opts": K.KesSolveOpts, "kes_result": K.KesResult,
               "kes_stats": K.KesStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kes.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, what, val = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if what == "size" else getattr(py, what).offset
        assert got == int(val), (cname, what, got, val)


def test_launch_shape_counts():
    n_step, n_block = K.kes_launch_shapes()
    assert n_step >= 8 and n_block >= 4


def test_sym_eig_threaded_size_is_accurate_and_independent_of_the_thread_count(tmp_path):
    # k >= 256 runs the Householder and rotation loops on OpenMP threads over independent
    # rows and columns: the result must be backward stable on a graded spectrum like that of
    # a projected stiffness matrix (eigenvalues from 0 to 2e5 with an interior cluster) and
    # bitwise the same with one thread as with several (the matrix is made once, here: the
    # BLAS that builds it rounds differently with other thread counts)
    import os
    import subprocess
    import sys
    k = 300
    rng = np.random.default_rng(7)
    lam = 2e5 * rng.random(k) ** 3
    lam[:20] = 1600 + 400 * rng.random(20)
    lam[20] = lam[0] * (1 + 1e-13)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    np.save(tmp_path / "A.npy", A)
    code = ("import numpy as np, sys\n"
            "import paper_2402_08515_gb300 as K\n"
            "w, V = K.kes_sym_eig(np.load(sys.argv[1]))\n"
            "np.save(sys.argv[2], np.concatenate([w, V.ravel()]))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for threads in ("1", "4"):
        path = tmp_path / f"t{threads}.npy"
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        subprocess.run([sys.executable, "-c", code, str(tmp_path / "A.npy"), str(path)], check=True, env=env,
                       cwd=root)
        out[threads] = np.load(path)
    np.testing.assert_array_equal(out["1"], out["4"])
    w, V = out["1"][:k], out["1"][k:].reshape(k, k)
    norm = np.abs(lam).max()
    assert np.abs(A @ V - V * w).max() <= 1e-13 * norm
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-12
    np.testing.assert_allclose(w, np.sort(lam), atol=1e-13 * norm)
