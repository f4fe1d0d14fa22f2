"""The allocation-free entry point kes_filter_apply_noalloc, called through the C ABI.

It serves callers that cannot call cudaMalloc (a program that reserves all its
device memory at start-up and forbids later allocation). Its output must agree
with kes_filter_apply, the entry point that owns a context, within the filter
tolerance of the parity tests, on two calls in a row (the second call reuses
the scratch array the first one left behind). This file is collected last so
that a run stopping at its first failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle as O
import paper_2402_08515_gb300 as K
from fe_inputs import box_grid, start_vectors
from tests.tolerances import filter_error, filter_tol

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_on_two_calls():
    import torch
    p = box_grid((37, 29, 23), extent=(1.0, 0.8, 0.7))        # 22,176 dofs: a ragged last warp
    tau = 0.9 * 2 / O.power_iteration(p.to_scipy(), p.m, start_vectors(p.n, 1, 0)[0], 300)
    wmin, wmax, L = 12.0, 20.0, 150
    alpha = K.kes_alpha_table(wmin, wmax, tau, L)
    dev = torch.device("cuda", 0)
    row_ptr = torch.from_numpy(p.row_ptr).to(dev)
    col = torch.from_numpy(p.col).to(dev)
    val = torch.from_numpy(p.val).to(dev)
    tau2m = torch.from_numpy(tau * tau / p.m).to(dev)
    alpha_d = torch.from_numpy(alpha).to(dev)
    stream = torch.cuda.current_stream(dev)
    with K.Context(p) as c:
        K.kes_set_filter(c.handle, wmin, wmax, tau, L)
        for seed in (21, 22):                                   # two calls in a row
            r = start_vectors(p.n, 1, seed)
            ref = np.zeros((1, 1, p.n))
            K.kes_filter_apply(c.handle, r, ref, 1)
            r_in = torch.from_numpy(r[0]).to(dev)
            r_out = torch.full((p.n,), float("nan"), dtype=torch.float64, device=dev)
            K.kes_filter_apply_noalloc(p.n, row_ptr, col, val, tau2m, alpha_d, L, r_in, r_out,
                                       stream.cuda_stream)
            torch.cuda.synchronize(dev)
            got = r_out.cpu().numpy()
            assert np.isfinite(got).all()
            err = filter_error(got, ref[0, 0], r, p.m, alpha)
            assert err <= filter_tol(L, "fp64"), (seed, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KesError) as e:
        K.kes_filter_apply_noalloc(K.KES_NOALLOC_MAX_N + 1, dummy, dummy, dummy, dummy, dummy, 10,
                                   dummy, dummy, None)
    assert e.value.status == -1
