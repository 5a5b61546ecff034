"""Dense oracles for small N.  Test infrastructure only.

(i)  ``exact_evolve``: the full 2^N x 2^N density matrix integrated exactly,
     rho(t) = exp(t L) rho(0), with L the sparse vectorised Lindbladian of
     Eq. (dtrho) and scipy's ``expm_multiply`` (the brute-force comparison the
     paper uses for N <= 10-11, App. B).
(ii) ``DenseTrotter``: the same op list and gates as the MPO oracle applied
     to the full 4^N Pauli-coefficient vector with no truncation.
Conversions between rho and its coefficients in the normalised Pauli basis
P_a/sqrt(2) per qubit (Eq. (mpo_def)).
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import expm_multiply

from . import model, schedule, tebd


def product_rho(n, init=None):
    """rho(t0) = |psi0><psi0|, |psi0> a product of Pauli eigenstates (Sec. 2.2)."""
    init = init or ["+z"] * n
    rho = np.array([[1.0 + 0j]])
    for q in range(n):
        sgn = 1.0 if init[q][0] == "+" else -1.0
        a = model.PAULI[tebd.PAULI_INDEX[init[q][1].upper()]]
        rho = np.kron(rho, 0.5 * (model.I2 + sgn * a))
    return rho


def exact_evolve(wl, b, times, rho0=None):
    """rho at each time in ``times`` (ascending) for instance b."""
    n = wl.n
    L = model.liouvillian_superop(n, wl.bonds, wl.h_x[b], wl.h_y[b], wl.h_z[b], wl.J[b], wl.Jz[b],
                                  wl.g0[b], wl.g1[b], wl.g2[b])
    rho = product_rho(n, wl.init) if rho0 is None else rho0
    v = rho.reshape(-1).astype(complex)
    out = []
    t_prev = 0.0
    for t in times:
        if t > t_prev:
            v = expm_multiply(L * (t - t_prev), v)
        t_prev = t
        out.append(v.reshape(2 ** n, 2 ** n).copy())
    return out


def _pauli_transform_matrix():
    """M[a, 2i+j] = (P_a)_{ji}/sqrt2, so sum_{ij} M[a,2i+j] rho_ij = Tr(P_a rho)/sqrt2."""
    M = np.zeros((4, 4), dtype=complex)
    for a in range(4):
        for i in range(2):
            for j in range(2):
                M[a, 2 * i + j] = model.PAULI[a][j, i] / np.sqrt(2.0)
    return M


def rho_to_pauli(rho):
    """r_a = Tr((P_a1/sqrt2 (x) ... (x) P_aN/sqrt2) rho); real for Hermitian rho."""
    n = int(round(np.log2(rho.shape[0])))
    t = rho.reshape([2] * (2 * n))
    perm = [x for q in range(n) for x in (q, n + q)]      # i1, j1, i2, j2, ...
    t = np.transpose(t, perm).reshape([4] * n)
    M = _pauli_transform_matrix()
    for q in range(n):
        t = np.moveaxis(np.tensordot(M, t, axes=([1], [q])), 0, q)
    return t.reshape(-1)


def pauli_to_rho(r, n):
    """Inverse of ``rho_to_pauli``."""
    rho = np.zeros((2 ** n, 2 ** n), dtype=complex)
    basis = None
    if n <= 6:
        basis = model.pauli_basis(n)
        for a in range(4 ** n):
            rho += r[a] * basis[a]
        return rho
    raise ValueError("pauli_to_rho only for n <= 6")


def expect_z(rho, i):
    n = int(round(np.log2(rho.shape[0])))
    Zi = model.embed(model.Z, i, n)
    return float(np.real(np.trace((Zi @ rho))) / np.real(np.trace(rho)))


def expect_zz(rho, i, j):
    n = int(round(np.log2(rho.shape[0])))
    Zij = model.embed(model.Z, i, n) @ model.embed(model.Z, j, n)
    return float(np.real(np.trace(Zij @ rho)) / np.real(np.trace(rho)))


def pauli_expect(r, n, comps):
    """<prod_i sigma^{c_i}> / tr rho from the coefficient vector."""
    t = r.reshape([4] * n)
    return float(t[tuple(comps)] / t[tuple([0] * n)])


class DenseTrotter:
    """Op list of ``schedule.step_layers`` applied to the 4^N vector."""

    def __init__(self, wl, b=0, r0=None, order=2):
        self.wl = wl
        self.n = wl.n
        self.layers = schedule.step_layers_order(wl.n, wl.bonds, order)
        self.gates = tebd.build_gates(wl, b, self.layers, wl.dt)
        if r0 is None:
            st = tebd.MPOState(*tebd.product_state(wl.n, wl.init))
            r0 = st.to_vector()
        self.r = np.array(r0, dtype=np.float64).reshape([4] * self.n)

    def step(self):
        for layer, gl in zip(self.layers, self.gates):
            for op, G in zip(layer, gl):
                p = op[1]
                G4 = G.reshape(4, 4, 4, 4)
                t = np.moveaxis(self.r, (p, p + 1), (0, 1))
                t = np.tensordot(G4, t, axes=([2, 3], [0, 1]))
                self.r = np.moveaxis(t, (0, 1), (p, p + 1))

    def run(self, steps):
        for _ in range(steps):
            self.step()
        return self

    def vector(self):
        return self.r.reshape(-1).copy()

    def z(self):
        out = []
        for i in range(self.n):
            c = [0] * self.n
            c[i] = 3
            out.append(pauli_expect(self.r.reshape(-1), self.n, c))
        return np.array(out)

    def zz(self, i, j):
        c = [0] * self.n
        c[i] = 3
        c[j] = 3
        return pauli_expect(self.r.reshape(-1), self.n, c)


def renyi2(rho):
    """Sec. 2.3 Eq. (S_2) on the dense matrix: S2 = -ln tr(rho^2) of rho / tr rho."""
    t = np.trace(rho).real
    return float(-np.log(np.trace(rho @ rho).real / (t * t)))


def osee(r, n, bond):
    """Sec. 2.3 Eq. (OSEE) from the dense coefficient vector r (4^n entries):
    singular values of r reshaped to (4^(bond+1), 4^(n-bond-1)) by LAPACK,
    then the entropy of their normalised squares."""
    s = np.linalg.svd(np.asarray(r).real.reshape(4 ** (bond + 1), -1), compute_uv=False)
    p = s * s / np.sum(s * s)
    p = p[p > 0.0]
    return float(-np.sum(p * np.log(p)))


def graph_rho(n, pairs):
    """rho = |G><G| of Eq. (graph_state): the state vector of |+x>^n with a
    controlled-Z (diag(1, 1, 1, -1)) on every listed pair, built directly on
    the 2^n amplitudes: CZ[j,k] flips the sign where bits j and k are 1."""
    psi = np.full(2 ** n, 2.0 ** (-n / 2.0), dtype=complex)
    idx = np.arange(2 ** n)
    for (j, k) in pairs:
        bj = (idx >> (n - 1 - j)) & 1
        bk = (idx >> (n - 1 - k)) & 1
        psi = np.where((bj & bk) == 1, -psi, psi)
    return np.outer(psi, psi.conj())
