"""The tensor-core complex products (tcgen05, TF32 in three passes) through
the C ABI's test hook, against complex128 products of the same complex64
inputs: C = beta C - A B for square blocks of several sizes, ragged against
the 128 x 128 output tiles and the 32-wide K stages.  The three-pass split
keeps about FP32 accuracy: the error is measured against max |A||B| and must
stay below 3e-7 times the inner dimension's square root, the size of FP32
rounding over the sum (one TF32 pass alone leaves about 1e-3)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_5003_gb300 import build
    build.build()
    from paper_1410_5003_gb300 import mlqp
    mlqp.load()
    return mlqp


@pytest.mark.parametrize("n,beta", [(64, 0), (96, 1), (240, 1), (512, 0), (512, 1)])
def test_tc_complex_product_matches_complex128(M, n, beta):
    g = torch.Generator(device="cpu").manual_seed(1000 + n + beta)
    mk = lambda: torch.complex(torch.randn(n, n, generator=g), torch.randn(n, n, generator=g))  # noqa: E731
    A, B, C = mk(), mk(), mk()
    ref = beta * C.to(torch.complex128) - A.to(torch.complex128) @ B.to(torch.complex128)
    for call in range(2):  # the operand planes are rewritten by every call
        out = M.tc_cgemm(A.cuda(), B.cuda(), C.cuda(), beta).cpu().to(torch.complex128)
        scale = float((A.abs().to(torch.float64) @ B.abs().to(torch.float64)).max())
        err = float((out - ref).abs().max()) / scale
        assert err < 3e-7 * np.sqrt(2 * n), (n, beta, call, err)


@pytest.mark.parametrize("rows,cols,K", [(64, 64, 16), (100, 130, 16), (700, 513, 16), (257, 65, 5),
                                         (512, 512, 60), (300, 170, 120)])
def test_fp64_tensor_core_update_matches_complex128(M, rows, cols, K):
    """The FP64 products on the tensor cores (seven 8-bit digit slices per
    operand row / column, BF16 products with exact FP32 sums): the block
    LU's rank-16 update (K <= 16) and the Schur updates' chunked product
    (K = 60 and 120, one scale per row and column over all of K): C - A B
    against complex128, to 4e-16 of max (|A||B|) times the inner dimension,
    the size of FP64 rounding over the sum.  One row of A
    spans 1e-12 .. 1 and one column of B contains zeros, and the tiles are
    ragged against the 64 x 64 output tiles."""
    g = torch.Generator(device="cpu").manual_seed(rows + cols + K)
    mk = lambda r, c: torch.complex(torch.randn(r, c, generator=g, dtype=torch.float64),  # noqa: E731
                                    torch.randn(r, c, generator=g, dtype=torch.float64))
    A, B, C = mk(rows, K), mk(K, cols), mk(rows, cols)
    A[3] *= torch.logspace(-12, 0, K, dtype=torch.float64)
    B[:, 2] = 0
    ref = C - A @ B
    out = M.oz_update(A.cuda(), B.cuda(), C.cuda()).cpu()
    scale = float((A.abs() @ B.abs()).max())
    err = float((out - ref).abs().max()) / scale
    assert err < 4e-16 * 2 * K, (rows, cols, K, err)
