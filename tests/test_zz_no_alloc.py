"""The no-allocation Lambda pass (cggm_lambda_sweep_noalloc) against the allocating one.

cggm_lambda_sweep_noalloc serves callers that cannot call cudaMalloc (code under an
allocator that owns all device memory, or loops that cannot afford cudaMalloc's implicit
synchronisation): it keeps its working memory in one array inside the library.  This
test calls it through the C ABI on device buffers and checks its direction against the
one cggm_lambda_sweep returns for the same inputs, on two calls in a row (the second on
other inputs, so left-over contents of the shared array would show), and that a size
beyond its stated maximum is refused.  The file runs last (name order), so a run that
stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_1509_04681_gb300")


def spd_inputs(q, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((q, q + 8)) / np.sqrt(q)
    Sigma = A @ A.T + np.eye(q)
    Bm = rng.standard_normal((q, 16)) / 4
    Psi = Bm @ Bm.T
    Syy = Sigma + 0.3 * (Bm[:, :1] @ Bm[:, :1].T) + 0.1 * np.eye(q)
    Lam = np.linalg.inv(Sigma)
    return Sigma, Psi, Syy, Lam


def active(q, rows, seed):
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(q)
    keep = (iu < rows) | (rng.uniform(size=iu.size) < 0.05) | (iu == ju)
    return iu[keep].astype(np.int32), ju[keep].astype(np.int32)


def call_noalloc(lib, Sigma, Psi, Syy, Lam, li, lj, lam, pen=1):
    q = Sigma.shape[0]
    dev = torch.device("cuda", 0)
    t = [torch.tensor(a, device=dev) for a in (Sigma, Psi, Syy, Lam)]
    ti = torch.tensor(li, device=dev)
    tj = torch.tensor(lj, device=dev)
    D = torch.full((q, q), float("nan"), device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    st = lib.cggm_lambda_sweep_noalloc(q, *[x.data_ptr() for x in t], len(li), ti.data_ptr(),
                                       tj.data_ptr(), float(lam), int(pen), D.data_ptr(),
                                       ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, D.cpu().numpy()


def test_noalloc_lambda_pass_matches_allocating_entry_point():
    from paper_1509_04681_gb300 import build
    build.build()
    lib = cg.cggm._lib()
    torch.cuda.set_device(0)
    with cg.Context(0) as ctx:
        for call, (q, rows, seed, lam) in enumerate([(200, 40, 1, 0.02), (131, 131, 2, 0.05)]):
            Sigma, Psi, Syy, Lam = spd_inputs(q, seed)
            li, lj = active(q, rows, seed)
            st, D = call_noalloc(lib, Sigma, Psi, Syy, Lam, li, lj, lam)
            assert st == 0, cg.cggm._lib().cggm_status_string(st)
            D_ref = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, lam,
                                          precision=cg.CGGM_FP64)
            assert np.all(np.isfinite(D))
            scale = max(1e-300, np.abs(D_ref).max())
            assert np.abs(D - D_ref).max() <= 1e-9 * scale, f"call {call}"
            np.testing.assert_array_equal(D, D.T)


def test_noalloc_at_its_maximum_size_and_empty_active_set():
    """q = CGGM_NOALLOC_MAX_Q with a near-full active set (the largest scratch layout), then
    m = 0 on a stream that the default stream does not wait for: the call must have written
    the zero direction before it returns."""
    lib = cg.cggm._lib()
    torch.cuda.set_device(0)
    q = 256
    Sigma, Psi, Syy, Lam = spd_inputs(q, 3)
    iu, ju = np.triu_indices(q)
    keep = np.random.default_rng(3).uniform(size=iu.size) < 0.9
    li, lj = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    with cg.Context(0) as ctx:
        st, D = call_noalloc(lib, Sigma, Psi, Syy, Lam, li, lj, 0.01)
        assert st == 0
        D_ref = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.01, precision=cg.CGGM_FP64)
        assert np.abs(D - D_ref).max() <= 1e-9 * max(1e-300, np.abs(D_ref).max())
    dev = torch.device("cuda", 0)
    t = [torch.tensor(a, device=dev) for a in (Sigma, Psi, Syy, Lam)]
    D0 = torch.full((q, q), float("nan"), device=dev, dtype=torch.float64)
    side = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    st = lib.cggm_lambda_sweep_noalloc(q, *[x.data_ptr() for x in t], 0, None, None, 0.01, 1,
                                       D0.data_ptr(), ctypes.c_void_p(side.cuda_stream))
    assert st == 0
    out = np.empty((q, q))
    # a plain copy, ordered after nothing on `side`: the call itself must have finished
    host = D0.to("cpu", non_blocking=False)
    out[:] = host.numpy()
    assert np.all(out == 0.0)


def test_noalloc_rejects_index_pairs_outside_the_matrix():
    lib = cg.cggm._lib()
    torch.cuda.set_device(0)
    q = 64
    Sigma, Psi, Syy, Lam = spd_inputs(q, 4)
    for li, lj in ([[0, 3], [1, 64]], [[0, 5], [1, 4]], [[-1, 0], [2, 2]]):
        st, _ = call_noalloc(lib, Sigma, Psi, Syy, Lam, np.array(li, np.int32),
                             np.array(lj, np.int32), 0.01)
        assert st == cg.CGGM_EINVAL, (li, lj, st)
    # the entry point still works after a refused call
    li, lj = active(q, 8, 4)
    st, D = call_noalloc(lib, Sigma, Psi, Syy, Lam, li, lj, 0.01)
    assert st == 0 and np.all(np.isfinite(D))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lib = cg.cggm._lib()
    q = 257  # CGGM_NOALLOC_MAX_Q + 1
    dev = torch.device("cuda", 0)
    M = torch.zeros((q, q), device=dev, dtype=torch.float64)
    idx = torch.zeros(1, device=dev, dtype=torch.int32)
    st = lib.cggm_lambda_sweep_noalloc(q, M.data_ptr(), M.data_ptr(), M.data_ptr(),
                                       M.data_ptr(), 1, idx.data_ptr(), idx.data_ptr(), 0.1, 1,
                                       M.data_ptr(), None)
    assert st == cg.CGGM_EINVAL
