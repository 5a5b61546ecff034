"""Global quantities of Sec. 2.3 through the C ABI (mpdo_renyi2, mpdo_osee)
against the oracle: the second Renyi entropy (Eq. (S_2)) and the operator
space entanglement entropy (Eq. (OSEE)) at every bond, FP64 path, <= 1e-10
on evolved states (the GPU's ranks replayed by the oracle) and on closed
forms."""
import numpy as np
import pytest

import workloads as W
from oracle import tebd

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()


def _solver(wl, **kw):
    from paper_2203_05871_gb300 import Solver
    s = Solver(wl.n, batch=wl.batch, chi_cap=int(max(wl.chi_max)), **kw)
    s.build_gates(wl)
    return s


def test_product_states_closed_forms():
    """All +z (pure product): S2 = 0 and OSEE = 0 at every bond; the
    (unnormalised) maximally mixed state: S2 = N ln 2."""
    n = 7
    wl = W.random_model(n, W.chain_bonds(n), 40, batch=2, chi_max=8)
    s = _solver(wl)
    s.set_state(1, [1] * (n + 1), [np.array([3.0, 0, 0, 0]).reshape(1, 4, 1)] * n)
    S2 = s.renyi2()
    assert abs(S2[0]) < 1e-14 and abs(S2[1] - n * np.log(2.0)) < 1e-13
    for bond in range(n - 1):
        assert np.all(np.abs(s.osee(bond)) < 1e-14)


@pytest.mark.parametrize("bonds_fn,n,batch", [(W.chain_bonds, 8, 1), (W.ring_bonds, 7, 3)])
def test_evolved_states_match_oracle(bonds_fn, n, batch):
    wl = W.random_model(n, bonds_fn(n), 41, batch=batch, chi_max=16, cutoff=1e-12, dt=0.1)
    if batch > 1:
        wl.chi_max[:] = [16, 8, 12]
    steps = 6
    s = _solver(wl)
    s.step(steps)
    S2 = s.renyi2()
    osee = np.array([s.osee(bond) for bond in range(n - 1)])   # [bond][b]
    log = s.rank_log(steps)
    for b in range(batch):
        o = tebd.TEBD(wl, b).run(steps, forced_k=[int(k) for k in log[b]])
        assert abs(S2[b] - o.state.renyi2()) <= TOL, b
        want = np.array([o.state.osee(bond) for bond in range(n - 1)])
        assert np.abs(osee[:, b] - want).max() <= TOL, (b, osee[:, b], want)
        assert want.max() > 1e-3   # the states are correlated


def test_saturated_random_state_chi128():
    """A seeded random MPO at chi = 128 (bond matrices of the size the
    benchmark truncates): S2 and the central OSEE against the oracle's QR
    canonicalisation, with the deviation printed."""
    n, chi = 10, 128
    wl = W.random_model(n, W.chain_bonds(n), 42, chi_max=chi, cutoff=1e-10)
    dims, tens = W.random_mpo_state(n, chi, seed=43, decay=0.02)
    s = _solver(wl)
    s.set_state(0, dims, tens)
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    dS2 = abs(s.renyi2()[0] - st.renyi2())
    got = [s.osee(bond)[0] for bond in (3, 4, 5)]
    want = [st.osee(bond) for bond in (3, 4, 5)]
    dO = max(abs(a - b) for a, b in zip(got, want))
    print(f"chi=128 random MPO: |dS2| = {dS2:.2e}, max|dOSEE| = {dO:.2e} (OSEE = {want})")
    assert dS2 <= TOL and dO <= 1e-9
