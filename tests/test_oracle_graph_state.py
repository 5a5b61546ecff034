"""Pins of the graph-state initial state (Sec. 2.2, Eq. (graph_state)):
the stabilisers X_i prod_{j ~ i} Z_j of |G> have expectation 1 (evaluated on
the dense matrix with explicit operator products), the CZ superoperator is
a signed permutation of Pauli strings, and the oracle's MPO (CZ gates through
swaps) holds the dense coefficient vector exactly."""
import numpy as np
import pytest

from oracle import dense, model, tebd


def _pauli_string(n, ops):
    m = np.array([[1.0 + 0j]])
    for q in range(n):
        m = np.kron(m, ops.get(q, model.I2))
    return m


@pytest.mark.parametrize("n,pairs", [(5, [(0, 1), (1, 2), (2, 3), (3, 4)]), (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5),
                                                                              (0, 5), (1, 4)]),
                                     (4, [(0, 3)])])
def test_stabilisers_and_mpo(n, pairs):
    rho = dense.graph_rho(n, pairs)
    nbr = {q: set() for q in range(n)}
    for (i, j) in pairs:
        nbr[i].add(j)
        nbr[j].add(i)
    for q in range(n):
        ops = {q: model.X}
        ops.update({j: model.Z for j in nbr[q]})
        assert abs(np.trace(_pauli_string(n, ops) @ rho).real - 1.0) < 1e-12
        if nbr[q]:
            assert abs(np.trace(_pauli_string(n, {q: model.X}) @ rho).real) < 1e-12
    st = tebd.graph_state(n, pairs, chi_max=4 ** (n // 2), cutoff=0.0)
    assert np.abs(st.to_vector() - dense.rho_to_pauli(rho).real).max() < 1e-12
    assert abs(st.renyi2()) < 1e-12


def test_cz_is_a_signed_permutation():
    G = model.cz_matrix()
    assert np.allclose(np.abs(G).sum(axis=0), 1.0) and np.allclose(np.abs(G).sum(axis=1), 1.0)
    assert np.allclose(G @ G, np.eye(16))
    # X x I -> X x Z, Z x I -> Z x I, X x X -> Y x Y
    assert G[1 * 4 + 3, 1 * 4 + 0] == 1.0 and G[3 * 4 + 0, 3 * 4 + 0] == 1.0
    assert G[2 * 4 + 2, 1 * 4 + 1] == 1.0
