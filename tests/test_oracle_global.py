"""Pins of the oracle's global quantities (Sec. 2.3): the second Renyi
entropy S2 = -ln tr(rho^2) (Eq. (S_2)) and the operator space entanglement
entropy of |rho>> at a bond (Eq. (OSEE)).

Each is checked against facts that hold independently of the code under
test: closed forms on product states (S2 = sum of -ln((1 + |n_i|^2) / 2),
OSEE = 0), a pure state rho = |psi><psi| (S2 = 0, OSEE = 2 S_vN(psi), the
paper's own statement, with S_vN from LAPACK on psi itself), a mixed state
built from orthonormal vectors (tr rho^2 = sum_k w_k^2), and the MPO against
the dense matrix after an untruncated evolution."""
import numpy as np
import pytest

import workloads as W
from oracle import dense, tebd


def mps_from_vector(r, n):
    """Exact MPS of a 4^n coefficient vector by successive SVDs (no truncation)."""
    B = []
    rest = np.asarray(r, dtype=np.float64).reshape(1, -1)
    for p in range(n - 1):
        cl = rest.shape[0]
        M = rest.reshape(cl * 4, -1)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        k = max(1, int(np.sum(s > 1e-14 * s[0])))
        B.append(U[:, :k].reshape(cl, 4, k))
        rest = s[:k, None] * Vt[:k]
    B.append(rest.reshape(rest.shape[0], 4, 1))
    return tebd.MPOState(B, [np.ones(b.shape[2]) for b in B[:-1]])


def random_pure(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    return psi / np.linalg.norm(psi)


def svn(psi, n, bond):
    """Von Neumann entropy of the first bond+1 qubits of a pure state (LAPACK)."""
    s = np.linalg.svd(psi.reshape(2 ** (bond + 1), -1), compute_uv=False)
    p = s * s
    p = p[p > 1e-300]
    return float(-np.sum(p * np.log(p)))


@pytest.mark.parametrize("init", [["+z"] * 5, ["+x", "-y", "+z", "-z", "+x"]])
def test_pure_product_states(init):
    st = tebd.MPOState(*tebd.product_state(5, init))
    assert abs(st.renyi2()) < 1e-14
    for bond in range(4):
        assert abs(st.osee(bond)) < 1e-14


def test_mixed_product_closed_form():
    """Each qubit (I + l_i sigma^z) / 2: tr rho_i^2 = (1 + l_i^2) / 2, so
    S2 = sum_i -ln((1 + l_i^2) / 2); l_i = 0 everywhere is N ln 2."""
    ls = np.array([0.0, 0.3, 0.9, 0.5])
    B = [np.array([1.0, 0.0, 0.0, l]).reshape(1, 4, 1) / np.sqrt(2.0) for l in ls]
    st = tebd.MPOState(B, [np.ones(1)] * 3)
    assert abs(st.renyi2() - np.sum(-np.log((1 + ls ** 2) / 2))) < 1e-14
    mm = tebd.MPOState([np.array([1.0, 0, 0, 0]).reshape(1, 4, 1)] * 6, [np.ones(1)] * 5)
    assert abs(mm.renyi2() - 6 * np.log(2.0)) < 1e-13
    for bond in range(3):
        assert abs(st.osee(bond)) < 1e-14


def test_pure_state_osee_is_twice_the_entanglement():
    n = 6
    psi = random_pure(n, 11)
    rho = np.outer(psi, psi.conj())
    r = dense.rho_to_pauli(rho).real
    st = mps_from_vector(r, n)
    assert abs(st.renyi2()) < 1e-12
    assert abs(dense.renyi2(rho)) < 1e-12
    for bond in range(n - 1):
        want = 2.0 * svn(psi, n, bond)
        assert abs(st.osee(bond) - want) < 1e-11, bond
        assert abs(dense.osee(r, n, bond) - want) < 1e-11, bond


def test_mixed_state_purity_from_orthonormal_vectors():
    n = 5
    rng = np.random.default_rng(12)
    Q, _ = np.linalg.qr(rng.normal(size=(2 ** n, 2 ** n)) + 1j * rng.normal(size=(2 ** n, 2 ** n)))
    w = rng.uniform(size=7)
    w /= w.sum()
    rho = sum(wk * np.outer(Q[:, k], Q[:, k].conj()) for k, wk in enumerate(w))
    want = -np.log(np.sum(w ** 2))
    assert abs(dense.renyi2(rho) - want) < 1e-12
    st = mps_from_vector(dense.rho_to_pauli(rho).real, n)
    assert abs(st.renyi2() - want) < 1e-12
    r = dense.rho_to_pauli(rho).real
    for bond in range(n - 1):
        assert abs(st.osee(bond) - dense.osee(r, n, bond)) < 1e-11


def test_evolved_mpo_against_dense_trotter():
    """Untruncated MPO evolution (chi_max >= 4^(N/2)) and the dense Trotter
    product hold the same state: equal S2 and OSEE at every bond."""
    n = 6
    wl = W.random_model(n, W.chain_bonds(n), 21, chi_max=64, cutoff=0.0, dt=0.25)
    t = tebd.TEBD(wl, force_trace=False).run(8)
    d = dense.DenseTrotter(wl).run(8)
    r = d.vector()
    rho = dense.pauli_to_rho(r, n)
    assert abs(t.state.renyi2() - dense.renyi2(rho)) < 1e-11
    for bond in range(n - 1):
        assert abs(t.state.osee(bond) - dense.osee(r, n, bond)) < 1e-10
    assert t.state.osee(2) > 0.01   # the evolved state is correlated
