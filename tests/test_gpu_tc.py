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
