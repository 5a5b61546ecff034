"""The mixed path's FP64-accurate tensor-core GEMM (mpdo_gemm_tc: six 8-bit
slices per operand, exact tcgen05 slice products, error-free FP32
accumulation per 256 values of K) against numpy's FP64 product, for both
tensor kinds, on shapes spanning several 128 x 128 tiles with ragged tails,
K across accumulator drains, graded rows and non-finite entries."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()
    return t


def _bound(A, B):
    """|A_i|max |B_j|max sqrt(K): the scale of the slicing error of entry (i, j)."""
    return (np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :] * np.sqrt(A.shape[1]))


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
@pytest.mark.parametrize("M,N,K,grade", [(1, 1, 1, 0), (5, 7, 3, 0), (128, 128, 32, 0), (200, 300, 257, 0),
                                         (129, 1, 700, 3), (1024, 1024, 1024, 14), (300, 1100, 515, 6)])
def test_matches_fp64(torch, kind, M, N, K, grade):
    from paper_2203_05871_gb300 import MIXED_BF16X3, MIXED_TF32
    from paper_2203_05871_gb300.mpdo import gemm_tc
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)) * np.logspace(0, -grade, M)[:, None]
    B = rng.standard_normal((K, N)) * np.logspace(0, -grade / 2, N)[None, :]
    C = gemm_tc(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"),
                MIXED_TF32 if kind == "tf32" else MIXED_BF16X3).cpu().numpy()
    R = A @ B
    err = np.abs(C - R) / _bound(A, B)
    print(f"{kind} {M}x{N}x{K} grade {grade}: max err / (|A_i| |B_j| sqrt K) = {err.max():.2e}")
    assert err.max() <= 1e-12


def test_scaled_and_nonfinite_rows(torch):
    """Rows scaled by powers of two far apart keep their relative accuracy,
    and a NaN in A makes exactly its row of C NaN."""
    from paper_2203_05871_gb300 import MIXED_TF32
    from paper_2203_05871_gb300.mpdo import gemm_tc
    rng = np.random.default_rng(5)
    A = rng.standard_normal((260, 300)) * np.exp2(rng.integers(-300, 300, size=260))[:, None]
    B = rng.standard_normal((300, 140))
    C = gemm_tc(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), MIXED_TF32).cpu().numpy()
    assert (np.abs(C - A @ B) / _bound(A, B)).max() <= 1e-12
    A[17, 40] = np.nan
    C = gemm_tc(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), MIXED_TF32).cpu().numpy()
    assert np.all(np.isnan(C[17])) and np.all(np.isfinite(np.delete(C, 17, axis=0)))
