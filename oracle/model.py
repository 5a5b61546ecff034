"""Model of Sec. 2.1: Hamiltonian, dissipators and their superoperators.

Test infrastructure only (see ``oracle/__init__``).

Conventions (readings of the paper where it is silent or ambiguous):
* sigma^+ = (sigma^x + i sigma^y)/2 (Sec. 2.1) = |0><1| in the basis where
  sigma^z|0> = +|0>; D0 (Eq. (D0)) therefore relaxes towards sigma^z = +1.
* Eq. (K_def) is read with each *unordered* bond counted once, as in
  Eq. (K_drive): K_ij = (J/2)(XX + YY) + (Jz/2) ZZ.
* The on-site Hamiltonian is +1/2 (h_z Z + h_x X + h_y Y), Eq. (H0) literally.
* Pauli basis of Eq. (mpo_def), normalised: P_a / sqrt(2), a in (I, X, Y, Z),
  two-site index s1*4 + s2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = [I2, X, Y, Z]
SP = (X + 1j * Y) / 2.0          # sigma^+  (Sec. 2.1)
SM = (X - 1j * Y) / 2.0          # sigma^-


def comm(a, b):
    return a @ b - b @ a


def anti(a, b):
    return a @ b + b @ a


# ---------------------------------------------------------------------------
# local generators as maps on operators
# ---------------------------------------------------------------------------
def site_lindbladian_map(hx, hy, hz, g0, g1, g2):
    """rho -> L_i[rho] for one qubit: -i[H_i, rho] with H_i of Eq. (H0) plus
    D0, D1, D2 of Eqs. (D0)-(D2)."""
    H = 0.5 * (hz * Z + hx * X + hy * Y)

    def f(rho):
        out = -1j * comm(H, rho)
        out = out + g0 * (SP @ rho @ SM - 0.5 * anti(SM @ SP, rho))
        out = out + g1 * (SM @ rho @ SP - 0.5 * anti(SP @ SM, rho))
        out = out + g2 * (Z @ rho @ Z - rho)
        return out
    return f


def bond_lindbladian_map(J, Jz):
    """rho -> -i[K_ij, rho] on two qubits, K_ij = (J/2)(XX+YY) + (Jz/2)ZZ
    (Eq. (K_def), unordered bond counted once)."""
    K = 0.5 * J * (np.kron(X, X) + np.kron(Y, Y)) + 0.5 * Jz * np.kron(Z, Z)

    def f(rho):
        return -1j * comm(K, rho)
    return f


def pauli_basis(nsites):
    """Normalised Pauli-product basis P_a/sqrt(2)^n, index a = a1*4^(n-1)+..."""
    basis = []
    for idx in range(4 ** nsites):
        digits = [(idx // 4 ** (nsites - 1 - k)) % 4 for k in range(nsites)]
        op = np.array([[1.0 + 0j]])
        for d in digits:
            op = np.kron(op, PAULI[d] / np.sqrt(2.0))
        basis.append(op)
    return basis


def superop_in_pauli_basis(fmap, nsites):
    """Matrix of a superoperator in the normalised Pauli basis:
    M[a, b] = Tr(P_a^dagger f(P_b)).  Returns (real part, max |imag part|)."""
    basis = pauli_basis(nsites)
    d = len(basis)
    M = np.zeros((d, d), dtype=complex)
    for b in range(d):
        fb = fmap(basis[b])
        for a in range(d):
            M[a, b] = np.trace(basis[a].conj().T @ fb)
    return M.real.copy(), float(np.max(np.abs(M.imag)))


def site_generator(hx, hy, hz, g0, g1, g2):
    """4x4 Pauli-basis matrix of the single-qubit Liouvillian (real)."""
    M, im = superop_in_pauli_basis(site_lindbladian_map(hx, hy, hz, g0, g1, g2), 1)
    assert im < 1e-14
    return M


def bond_generator(J, Jz):
    """16x16 Pauli-basis matrix of the bond commutator superoperator (real)."""
    M, im = superop_in_pauli_basis(bond_lindbladian_map(J, Jz), 2)
    assert im < 1e-14
    return M


def op_generator(params, b, qa, qb, bond_index, weights):
    """Generator of one two-site gate acting on path positions (p, p+1) that
    hold qubits qa (left) and qb (right): the bond term plus the fraction
    w_q = 1/deg(q) of each qubit's on-site Liouvillian."""
    hx, hy, hz = params["h_x"][b], params["h_y"][b], params["h_z"][b]
    g0, g1, g2 = params["g0"][b], params["g1"][b], params["g2"][b]
    La = site_generator(hx[qa], hy[qa], hz[qa], g0[qa], g1[qa], g2[qa])
    Lb = site_generator(hx[qb], hy[qb], hz[qb], g0[qb], g1[qb], g2[qb])
    Lbond = bond_generator(params["J"][b][bond_index], params["Jz"][b][bond_index])
    return Lbond + weights[qa] * np.kron(La, np.eye(4)) + weights[qb] * np.kron(np.eye(4), Lb)


def cz_matrix():
    """Pauli-basis superoperator of the controlled-Z channel rho -> CZ rho CZ
    on two sites (Sec. 2.2, Eq. (graph_state)), by explicit traces:
    G[(a,b), (c,d)] = Tr[(P_a x P_b) CZ (P_c x P_d) CZ] / 4."""
    cz = np.diag([1.0, 1.0, 1.0, -1.0]).astype(complex)
    G = np.zeros((16, 16))
    for a in range(4):
        for b in range(4):
            Pab = np.kron(PAULI[a], PAULI[b])
            for c in range(4):
                for d in range(4):
                    Pcd = np.kron(PAULI[c], PAULI[d])
                    G[a * 4 + b, c * 4 + d] = np.trace(Pab @ cz @ Pcd @ cz).real / 4.0
    return G


def swap_matrix():
    """Pauli-basis SWAP of two sites: |a,b>> -> |b,a>>."""
    S = np.zeros((16, 16))
    for a in range(4):
        for b in range(4):
            S[b * 4 + a, a * 4 + b] = 1.0
    return S


# ---------------------------------------------------------------------------
# full 2^N operators (dense oracle)
# ---------------------------------------------------------------------------
def embed(op, i, n):
    """Sparse embedding of a single-qubit operator at qubit i (qubit 0 is the
    most significant kron factor)."""
    return sp.kron(sp.kron(sp.identity(2 ** i, format="csr"), sp.csr_matrix(op)),
                   sp.identity(2 ** (n - i - 1), format="csr"), format="csr")


def hamiltonian(n, bonds, hx, hy, hz, J, Jz):
    """Sparse H of Eq. (H0) with K of Eq. (K_def) (each bond once)."""
    H = sp.csr_matrix((2 ** n, 2 ** n), dtype=complex)
    for i in range(n):
        H = H + 0.5 * (hz[i] * embed(Z, i, n) + hx[i] * embed(X, i, n) + hy[i] * embed(Y, i, n))
    for k, (i, j) in enumerate(bonds):
        H = H + 0.5 * J[k] * (embed(X, i, n) @ embed(X, j, n) + embed(Y, i, n) @ embed(Y, j, n))
        H = H + 0.5 * Jz[k] * (embed(Z, i, n) @ embed(Z, j, n))
    return H.tocsr()


def jump_operators(n, g0, g1, g2):
    """Jump operators c_k with D[rho] = sum_k c rho c^+ - 1/2{c^+ c, rho}:
    sqrt(g0) sigma^+ (Eq. (D0)), sqrt(g1) sigma^- (Eq. (D1)),
    sqrt(g2) sigma^z (Eq. (D2): g2 (Z rho Z - rho))."""
    ops = []
    for i in range(n):
        if g0[i] != 0:
            ops.append(np.sqrt(g0[i]) * embed(SP, i, n))
        if g1[i] != 0:
            ops.append(np.sqrt(g1[i]) * embed(SM, i, n))
        if g2[i] != 0:
            ops.append(np.sqrt(g2[i]) * embed(Z, i, n))
    return ops


def liouvillian_superop(n, bonds, hx, hy, hz, J, Jz, g0, g1, g2):
    """Sparse 4^N x 4^N matrix of Eq. (dtrho) acting on row-major vec(rho):
    vec(A rho B) = kron(A, B^T) vec(rho)."""
    H = hamiltonian(n, bonds, hx, hy, hz, J, Jz)
    Id = sp.identity(2 ** n, format="csr", dtype=complex)
    L = -1j * (sp.kron(H, Id) - sp.kron(Id, H.T))
    for c in jump_operators(n, g0, g1, g2):
        cdc = (c.conj().T @ c).tocsr()
        L = L + sp.kron(c, c.conj()) - 0.5 * sp.kron(cdc, Id) - 0.5 * sp.kron(Id, cdc.T)
    return L.tocsr()


def lindblad_rhs(n, bonds, hx, hy, hz, J, Jz, g0, g1, g2):
    """rho -> L[rho] on a dense 2^N matrix (used to pin the superoperator)."""
    H = hamiltonian(n, bonds, hx, hy, hz, J, Jz)
    cs = jump_operators(n, g0, g1, g2)

    def f(rho):
        out = -1j * (H @ rho - (H.T @ rho.T).T)
        for c in cs:
            cdc = c.conj().T @ c
            out = out + c @ (c @ rho.conj().T).conj().T - 0.5 * (cdc @ rho + (cdc.T @ rho.T).T)
        return out
    return f
