"""The allocation-free entry point kes_filter_apply_noalloc, called through the C ABI.

It serves callers that cannot call cudaMalloc (a program that reserves all its
device memory at start-up and forbids later allocation). Its output must agree
with the FP64 oracle's filter and with kes_filter_apply, the entry point that
owns a context, within the filter tolerance of the parity tests, on two calls in
a row (the second call reuses the scratch array the first one left behind), and
the second call must not change the device's free memory. One case fills the
library's fixed scratch array to its last row (n = KES_NOALLOC_MAX_N). This file
is collected last so that a run stopping at its first failure has run every
other test before it.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import paper_2402_08515_gb300 as K
from fe_inputs import box_grid, start_vectors
from tests.tolerances import filter_error, filter_tol

pytestmark = pytest.mark.gpu


def _device_csr(p, tau, dev):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(p.row_ptr, dtype=np.int64)).to(dev),
            torch.from_numpy(np.ascontiguousarray(p.col, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(p.val)).to(dev),
            torch.from_numpy(tau * tau / p.m).to(dev))


def test_noalloc_matches_oracle_and_context_entry_point_on_two_calls():
    import torch
    p = box_grid((37, 29, 23), extent=(1.0, 0.8, 0.7))        # 22,176 dofs: a ragged last warp
    tau = 0.9 * 2 / O.power_iteration(p.to_scipy(), p.m, start_vectors(p.n, 1, 0)[0], 300)
    wmin, wmax, L = 12.0, 20.0, 150
    alpha = O.alpha_table(wmin, wmax, tau, L)
    dev = torch.device("cuda", 0)
    row_ptr, col, val, tau2m = _device_csr(p, tau, dev)
    alpha_d = torch.from_numpy(alpha).to(dev)
    stream = torch.cuda.current_stream(dev)
    S = p.to_scipy()
    tol = filter_tol(L, "fp64")
    with K.Context(p) as c:
        K.kes_set_filter(c.handle, wmin, wmax, tau, L)
        free_after = []
        for seed in (21, 22):                                   # two calls in a row
            r = start_vectors(p.n, 1, seed)
            ctx_out = np.zeros((1, 1, p.n))
            K.kes_filter_apply(c.handle, r, ctx_out, 1)
            r_in = torch.from_numpy(r[0]).to(dev)
            r_out = torch.full((p.n,), float("nan"), dtype=torch.float64, device=dev)
            torch.cuda.synchronize(dev)
            free_before = torch.cuda.mem_get_info(dev)[0]
            K.kes_filter_apply_noalloc(p.n, row_ptr, col, val, tau2m, alpha_d, L, r_in, r_out,
                                       stream.cuda_stream)
            torch.cuda.synchronize(dev)
            free_after.append((free_before, torch.cuda.mem_get_info(dev)[0]))
            got = r_out.cpu().numpy()
            assert np.isfinite(got).all()
            ref = O.filter_apply(S, p.m, r[0], tau, alpha)
            assert filter_error(got, ref, r, p.m, alpha) <= tol, seed
            assert filter_error(got, ctx_out[0, 0], r, p.m, alpha) <= tol, seed
    # the first call may load the module that holds the scratch array; the second one
    # must leave the device's free memory as it found it
    assert free_after[1][0] == free_after[1][1]


def _chain(n, seed=5):
    """A weighted path graph Laplacian plus a positive diagonal (symmetric positive
    definite, 3 entries per row) with random lumped masses: seeded, synthetic."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, n - 1)
    d = rng.uniform(0.1, 1.0, n)
    main = d.copy()
    main[:-1] += w
    main[1:] += w
    S = sp.diags([-w, main, -w], [-1, 0, 1], format="csr").sorted_indices()
    m = rng.uniform(0.5, 2.0, n)
    return S, m


def test_noalloc_fills_its_scratch_array_to_the_last_row():
    import torch
    n = K.KES_NOALLOC_MAX_N
    S, m = _chain(n)
    gersh = float(np.max(np.asarray(abs(S).sum(axis=1)).ravel() / m))  # >= omega_max^2
    tau = 0.9 * 2 / np.sqrt(gersh)
    L = 40
    alpha = O.alpha_table(0.8, 1.6, tau, L)
    r = start_vectors(n, 1, 31)
    ref = O.filter_apply(S, m, r[0], tau, alpha)
    dev = torch.device("cuda", 0)
    row_ptr = torch.from_numpy(S.indptr.astype(np.int64)).to(dev)
    col = torch.from_numpy(S.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(S.data.astype(np.float64)).to(dev)
    tau2m = torch.from_numpy(tau * tau / m).to(dev)
    r_out = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    K.kes_filter_apply_noalloc(n, row_ptr, col, val, tau2m, torch.from_numpy(alpha).to(dev), L,
                               torch.from_numpy(r[0]).to(dev), r_out, torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize(dev)
    got = r_out.cpu().numpy()
    assert np.isfinite(got).all()
    assert filter_error(got, ref, r, m, alpha) <= filter_tol(L, "fp64")


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_tensors():
    import torch
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KesError) as e:
        K.kes_filter_apply_noalloc(K.KES_NOALLOC_MAX_N + 1, dummy, dummy, dummy, dummy, dummy, 10,
                                   dummy, dummy, None)
    assert e.value.status == -1
    # a float32 output or a short weight table is refused before anything is launched
    n, L = 3, 2
    row_ptr = torch.tensor([0, 1, 2, 3], dtype=torch.int64, device="cuda")
    col = torch.arange(3, dtype=torch.int32, device="cuda")
    v = torch.ones(3, dtype=torch.float64, device="cuda")
    for bad in ({"r_out": torch.zeros(3, dtype=torch.float32, device="cuda")},
                {"alpha": torch.zeros(L, dtype=torch.float64, device="cuda")},
                {"col": torch.arange(3, dtype=torch.int64, device="cuda")}):
        args = dict(row_ptr=row_ptr, col=col, val=v, tau2m=v, alpha=torch.zeros(L + 1, dtype=torch.float64,
                    device="cuda"), r_in=v, r_out=torch.zeros(3, dtype=torch.float64, device="cuda"))
        args.update(bad)
        with pytest.raises(K.KesError) as e:
            K.kes_filter_apply_noalloc(n, args["row_ptr"], args["col"], args["val"], args["tau2m"], args["alpha"],
                                       L, args["r_in"], args["r_out"], None)
        assert e.value.status == -1
