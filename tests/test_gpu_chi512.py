"""A 2048 x 2048 bond matrix, the size of the grid workload at chi_max = 512:
an N = 12 chain whose three middle bonds are 512 wide (the others narrow), so
the op on sites 5 and 6 truncates a (4 x 512) x (4 x 512) matrix back to 512:
QR over 2048 columns, Jacobi rows of 2048 (the FP32 pass's shared-memory path
on the mixed path).  One step against the
oracle at the GPU's ranks; the oracle takes its LAPACK SVD route at this size
(the route is pinned against its plain Jacobi one)."""
import numpy as np
import pytest

import workloads as W
from oracle import tebd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("tf32", 1e-5)])
def test_one_step_with_a_2048_bond_matrix(precision, tol):
    from paper_2203_05871_gb300 import FP64, MIXED_TF32, Solver
    n = 12
    dims = [1, 4, 16, 64, 256, 512, 512, 512, 256, 64, 16, 4, 1]
    tens = W.random_mpo_tensors(dims, seed=512, decay=0.01)
    wl = W.uniform_model("chain12_chi512", n, W.chain_bonds(n), chi_max=512, cutoff=1e-9, dt=0.05)
    s = Solver(n, batch=1, chi_cap=512, precision=FP64 if precision == "fp64" else MIXED_TF32)
    s.build_gates(wl)
    s.set_state(0, dims, tens)
    s.step(1)
    assert s.status()["status"][0] == 0
    log = [int(k) for k in s.rank_log(1)[0]]
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    o = tebd.TEBD(wl, 0, state=st, svd_impl="lapack").run(1, forced_k=log)
    gz, rz = s.measure_1q(range(n), "Z")[0], o.z()
    pairs = [(0, 11), (4, 7), (5, 6), (2, 9)]
    g, rg = s.measure_2q(pairs, "ZZ", connected=True)[0], o.zz_connected(pairs)
    scale = np.array([abs(o.state.expect_2q(i, j)) + abs(rz[i] * rz[j]) for (i, j) in pairs])
    ez = np.abs(gz - rz) / np.maximum(1.0, np.abs(rz))
    ezz = np.abs(g - rg) / np.maximum(1.0, scale)
    print(f"chi512 {precision}: ranks {log}, max rel |dZ| = {ez.max():.2e}, |dZZc| = {ezz.max():.2e}")
    assert max(log) > 256
    assert np.all(ez <= tol) and np.all(ezz <= tol)
