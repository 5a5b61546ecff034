"""Fourth-order Trotter steps (Suzuki's triple jump of the symmetric step,
the order App. B uses) through the C ABI, against the oracle: the MPO-TEBD at
the GPU's ranks (FP64 <= 1e-10, mixed <= 1e-5) and, untruncated, the dense
Trotter product of the same op list."""
import numpy as np
import pytest

import workloads as W
from oracle import dense, tebd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()


def _solver(wl, **kw):
    from paper_2203_05871_gb300 import Solver
    s = Solver(wl.n, batch=wl.batch, chi_cap=int(max(wl.chi_max)), trotter_order=4, **kw)
    s.build_gates(wl)
    return s


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("tf32", 1e-5)])
def test_order4_against_oracle(precision, tol):
    from paper_2203_05871_gb300 import FP64, MIXED_TF32
    wl = W.random_model(8, W.ring_bonds(8), 77, chi_max=24, cutoff=1e-11, dt=0.1)
    steps = 4
    s = _solver(wl, precision=FP64 if precision == "fp64" else MIXED_TF32)
    n_ops = s.op_counts()[0]
    s.step(steps)
    log = [int(k) for k in s.rank_log(steps)[0]]
    o = tebd.TEBD(wl, order=4).run(steps, forced_k=log)
    assert len(o.k_log) == steps * n_ops
    dz = np.abs(s.measure_1q(range(8), "Z")[0] - o.z()).max()
    pairs = [(i, j) for i in range(8) for j in range(i + 1, 8)]
    dzz = np.abs(s.measure_2q(pairs, "ZZ", connected=True)[0] - o.zz_connected(pairs)).max()
    print(f"order 4 {precision}: |dZ| = {dz:.2e}, |dZZc| = {dzz:.2e}")
    assert dz <= tol and dzz <= tol


def test_order4_untruncated_equals_dense_trotter():
    wl = W.random_model(6, W.chain_bonds(6), 78, chi_max=64, cutoff=0.0, dt=0.15)
    s = _solver(wl, force_trace=False)
    s.step(3)
    d = dense.DenseTrotter(wl, order=4).run(3)
    assert np.abs(s.measure_1q(range(6), "Z")[0] - d.z()).max() <= 1e-12
