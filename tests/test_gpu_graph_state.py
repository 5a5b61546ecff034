"""Graph-state initial states (Sec. 2.2, Eq. (graph_state)) through the C
ABI: the state after mpdo_init_graph_state against the oracle's graph state
and the dense one (<X_i>, <Z_i>, <X_i Z_j>, <Z_i Z_j>, S2 = 0, OSEE), then
evolved by Trotter steps against the oracle started from the same state."""
import numpy as np
import pytest

import workloads as W
from oracle import dense, tebd

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()


CASES = [(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (0, 5), (1, 4)]), (7, [(0, 6), (2, 3), (1, 5)])]


@pytest.mark.parametrize("n,pairs", CASES)
def test_graph_state_matches_dense(n, pairs):
    from paper_2203_05871_gb300 import Solver
    wl = W.random_model(n, W.chain_bonds(n), 90, batch=2, chi_max=64, cutoff=1e-12)
    s = Solver(n, batch=2, chi_cap=64)
    s.build_gates(wl)
    s.init_graph_state(pairs)
    r = dense.rho_to_pauli(dense.graph_rho(n, pairs)).real
    nbr = {q: {j for (i, j) in pairs if i == q} | {i for (i, j) in pairs if j == q} for q in range(n)}
    for comp in "XYZ":
        got = s.measure_1q(range(n), comp)
        for q in range(n):
            c = [0] * n
            c[q] = "IXYZ".index(comp)
            want = dense.pauli_expect(r, n, c)
            assert np.all(np.abs(got[:, q] - want) <= TOL)
    # a leaf's stabiliser X_i Z_j is a two-qubit Pauli string: <X_i Z_j> = 1
    leaves = [(q, next(iter(nbr[q]))) for q in range(n) if len(nbr[q]) == 1]
    for (i, j) in leaves:
        assert np.all(np.abs(s.measure_2q([(i, j)], "XZ", connected=False)[:, 0] - 1.0) <= TOL)
    all_pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    zz = s.measure_2q(all_pairs, "ZZ", connected=False)
    for k, (i, j) in enumerate(all_pairs):
        c = [0] * n
        c[i] = c[j] = 3
        assert np.all(np.abs(zz[:, k] - dense.pauli_expect(r, n, c)) <= TOL)
    assert np.all(np.abs(s.renyi2()) <= 1e-10)
    st = tebd.graph_state(n, pairs, 64, 1e-12)
    for bond in range(n - 1):
        assert np.all(np.abs(s.osee(bond) - dense.osee(r, n, bond)) <= TOL)
        assert abs(st.osee(bond) - dense.osee(r, n, bond)) <= TOL


def test_graph_state_then_evolution():
    from paper_2203_05871_gb300 import Solver
    # chi_max 64 holds this graph state exactly: its Schmidt values are
    # degenerate, so a cut through them would keep an arbitrary subset of a
    # degenerate subspace (different on the two sides)
    n, pairs = CASES[0]
    wl = W.random_model(n, W.ring_bonds(n), 91, chi_max=64, cutoff=1e-11, dt=0.05)
    s = Solver(n, batch=1, chi_cap=64)
    s.build_gates(wl)
    s.init_graph_state(pairs)
    steps = 3
    s.step(steps)
    log = [int(k) for k in s.rank_log(steps)[0]]
    o = tebd.TEBD(wl, state=tebd.graph_state(n, pairs, 64, 1e-11)).run(steps, forced_k=log)
    all_pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    assert np.abs(s.measure_1q(range(n), "X")[0] - np.array([o.state.expect_1q(i, "X") for i in range(n)])).max() <= TOL
    assert np.abs(s.measure_2q(all_pairs, "ZZ", connected=True)[0] - o.zz_connected(all_pairs)).max() <= TOL
