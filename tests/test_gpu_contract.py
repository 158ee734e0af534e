"""Tensor-core contraction (cggm_contract, tcgen05 kind::tf32) against float64 products.

Error bound per entry: |C - C_ref|_ij <= tol * sum_k |A_ik B_jk| (+ the beta C term),
with tol = 3e-3 for one TF32 product (operands keep 10 mantissa bits) and 1e-5 for the
3xTF32 split (close to single precision).  Shapes cover exact tiles, ragged edges in M, N
and K, K shorter than one k-step, and more than one k-step ring cycle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_1509_04681_gb300")


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_04681_gb300 import build
    build.build()
    c = cg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape", [(128, 128, 32), (200, 130, 100), (64, 300, 4),
                                   (1000, 520, 1000), (257, 129, 288)])
@pytest.mark.parametrize("mode,tol", [(0, 3e-3), (1, 1e-5)])
def test_contract_matches_float64(ctx, shape, mode, tol):
    M, N, K = shape
    rng = np.random.default_rng(M + N + K + mode)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    alpha, beta = 0.5, 2.0
    dev = torch.device("cuda", 0)
    Ad, Bd, Cd = (torch.tensor(x, device=dev) for x in (A, B, C0))
    ctx.cggm_contract(Ad, Bd, Cd, alpha=alpha, beta=beta, mode=mode)
    torch.cuda.synchronize()
    C = Cd.cpu().numpy().astype(np.float64)
    ref = alpha * (A.astype(np.float64) @ B.astype(np.float64).T) + beta * C0.astype(np.float64)
    scale = alpha * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T) + \
        beta * np.abs(C0) * 1e-6 + 1e-30
    err = np.abs(C - ref) / scale
    assert err.max() <= tol, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_contract_rejects_unaligned_rows(ctx):
    dev = torch.device("cuda", 0)
    A = torch.zeros((10, 6), device=dev)  # row stride 6 floats: not a multiple of 4
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_contract(A, A)
    assert e.value.status == cg.CGGM_EINVAL
