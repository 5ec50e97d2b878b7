"""The tcgen05 kind::f16 MMA primitive (descriptors, tensor memory,
accumulator read-back) with bf16 and fp16 operands, against a float64 product
of the same 16-bit values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()


@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
@pytest.mark.parametrize("seed", [0, 1])
def test_tc_gemm_matches_float64(seed, dtype):
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    g = torch.Generator().manual_seed(seed)
    dt = torch.bfloat16 if dtype == "bf16" else torch.float16
    A = torch.randn(128, 128, generator=g).to(dt)
    B = torch.randn(32, 128, generator=g).to(dt)
    D = cg.ct_selftest_tc_gemm(A.cuda(), B.cuda()).cpu().numpy().astype(np.float64)
    ref = A.double().numpy() @ B.double().numpy().T
    scale = np.abs(A.double().numpy()) @ np.abs(B.double().numpy()).T
    assert np.all(np.abs(D - ref) <= 2.0 ** -20 * 128 * scale + 1e-30), float(np.max(np.abs(D - ref) / scale))


@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
def test_tc_gemm_structure(dtype):
    """Unit vectors locate every row/column/k position exactly."""
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    A = torch.zeros(128, 128)
    B = torch.zeros(32, 128)
    for r in range(128):
        A[r, (7 * r) % 128] = r + 1
    for c in range(32):
        B[c, (7 * (4 * c)) % 128] = 1.0      # matches A's row 4c
    dt = torch.bfloat16 if dtype == "bf16" else torch.float16
    D = cg.ct_selftest_tc_gemm(A.to(dt).cuda(), B.to(dt).cuda()).cpu().numpy()
    want = np.zeros((128, 32))
    for c in range(32):
        want[4 * c, c] = 4 * c + 1
    assert np.array_equal(D, want)


def test_tc_gemm_rejects_mixed_types():
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    with pytest.raises(ValueError):
        cg.ct_selftest_tc_gemm(torch.zeros(128, 128, dtype=torch.bfloat16).cuda(),
                               torch.zeros(32, 128, dtype=torch.float16).cuda())
