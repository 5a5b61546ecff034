"""MPO time evolution with two-site Liouvillian gates.  Test infrastructure only.

State (App. A, Eq. (mpo_def)): the Pauli coefficients r_{a1..aN} of
rho = sum_a r_a  P_a1/sqrt2 (x) ... (x) P_aN/sqrt2 form an MPS with local
dimension 4:  r_{a1..aN} = B_0[a1] B_1[a2] ... B_{N-1}[aN], B_p of shape
(chi_{p-1}, 4, chi_p), chi_{-1} = chi_{N-1} = 1.  Next to the B's the state
keeps Schmidt weights lam_p on every inner bond (Vidal/Hastings form); the
B's alone represent the state, the weights only steer truncation.

One op on positions (p, p+1) with 16x16 gate G (App. B's compression is done
on |rho>>, per bond):
  Theta [l,s1,s2,r]  = sum_m B_p[l,s1,m] B_{p+1}[m,s2,r]        (merge)
  Theta'[l,s1',s2',r] = sum_{s1 s2} G[s1's2', s1s2] Theta[l,s1,s2,r]
  theta~ = diag(lam_{p-1}) Theta'  as a (4 chi_l) x (4 chi_r) matrix
  theta~ = U S V^T;  k from the truncation rule;  lam_p = S[:k]
  B_{p+1} <- V[:, :k]^T,   B_p <- Theta' V[:, :k]
Trace forcing (App. B, b_force_rho_trace): after each step
tr rho = 2^{N/2} * (product of the a=I slices) and B_0 /= tr rho.
Observables (Sec. 2.3): <sigma^a_i> = E(a at i)/E(all I) with E(string) the
product of the selected slices; the 2^{N/2} factors cancel.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np
import scipy.linalg as sla

from . import model, schedule, svd

PAULI_INDEX = {"I": 0, "X": 1, "Y": 2, "Z": 3}


def product_state(n: int, init: Optional[List[str]] = None):
    """Pauli product state of Sec. 2.2: rho_i = (I +- sigma^a)/2 per qubit.
    In the normalised basis the site vector is (1, +-1 at a)/sqrt(2)."""
    init = init or ["+z"] * n
    B = []
    for q in range(n):
        sgn = 1.0 if init[q][0] == "+" else -1.0
        a = PAULI_INDEX[init[q][1].upper()]
        v = np.zeros((1, 4, 1))
        v[0, 0, 0] = 1.0 / np.sqrt(2.0)
        v[0, a, 0] += sgn / np.sqrt(2.0)
        B.append(v)
    lam = [np.ones(1) for _ in range(n - 1)]
    return B, lam


class MPOState:
    def __init__(self, B, lam):
        self.B = [np.array(b, dtype=np.float64) for b in B]
        self.lam = [np.array(x, dtype=np.float64) for x in lam]

    @property
    def n(self):
        return len(self.B)

    def dims(self):
        return [b.shape[2] for b in self.B[:-1]]

    def copy(self):
        return MPOState([b.copy() for b in self.B], [x.copy() for x in self.lam])

    def to_vector(self):
        """Dense 4^N coefficient vector (small N only)."""
        v = self.B[0].reshape(4, -1)
        for b in self.B[1:]:
            v = np.einsum("am,msr->asr", v, b).reshape(-1, b.shape[2])
        return v.reshape(-1)

    # -- one two-site op -------------------------------------------------
    def apply(self, p, G, chi_max, cutoff, forced_k=None, tol=None, svd_impl="jacobi"):
        """One two-site op.  svd_impl = "jacobi" (the oracle's plain C
        one-sided Jacobi) or "lapack" (numpy's gesdd; CPU timing only)."""
        A, Bn = self.B[p], self.B[p + 1]
        cl, cr = A.shape[0], Bn.shape[2]
        theta = np.einsum("lsm,mtr->lstr", A, Bn)
        G4 = G.reshape(4, 4, 4, 4)
        thetap = np.einsum("abcd,lcdr->labr", G4, theta)
        lam_left = self.lam[p - 1] if p > 0 else np.ones(1)
        tt = (lam_left[:, None, None, None] * thetap).reshape(cl * 4, 4 * cr)
        s, Vt = svd.svd_right(tt, tol=tol) if svd_impl == "jacobi" else svd.svd_right_lapack(tt)
        k = svd.truncation_rank(s, chi_max, cutoff) if forced_k is None else int(forced_k)
        Yk = Vt[:k]
        self.B[p + 1] = Yk.reshape(k, 4, cr).copy()
        self.B[p] = (thetap.reshape(cl * 4, 4 * cr) @ Yk.T).reshape(cl, 4, k)
        self.lam[p] = s[:k].copy()
        return k, svd.discarded_weight(s, k)

    # -- global quantities -----------------------------------------------
    def chain(self, comps):
        """E(string): product over sites of the selected Pauli slices."""
        v = np.ones(1)
        for p, b in enumerate(self.B):
            v = v @ b[:, comps[p], :]
        return float(v[0])

    def trace(self):
        return 2.0 ** (self.n / 2.0) * self.chain([0] * self.n)

    def normalize_trace(self):
        t = self.trace()
        self.B[0] = self.B[0] / t
        return t

    def norm2(self):
        """<<rho|rho>> = sum_a r_a^2, the squared norm of the coefficient MPS:
        E_{p+1} = sum_s B_p[s]^T E_p B_p[s], E_0 = [[1]]."""
        E = np.ones((1, 1))
        for b in self.B:
            E = sum(b[:, s, :].T @ E @ b[:, s, :] for s in range(4))
        return float(E[0, 0])

    def renyi2(self):
        """Second Renyi entropy, Sec. 2.3 Eq. (S_2): S2 = -ln tr(rho^2) of the
        normalised rho.  The basis P_a/sqrt2 is orthonormal for the trace
        inner product, so tr(rho^2) = sum_a r_a^2 = norm2(), and normalising
        rho divides it by (tr rho)^2."""
        t = self.trace()
        return -np.log(self.norm2() / (t * t))

    def schmidt_values(self, bond):
        """Schmidt values of |rho>> for the cut between path positions bond
        and bond+1: canonicalise both sides with QR (numpy), then the SVD of
        the product of the two triangular factors."""
        R = np.ones((1, 1))
        for p in range(bond + 1):
            M = np.einsum("ij,jsr->isr", R, self.B[p])
            M = M.reshape(-1, M.shape[2])
            _, R = np.linalg.qr(M)
        Lf = np.ones((1, 1))
        for p in range(self.n - 1, bond, -1):
            M = np.einsum("lsr,rj->lsj", self.B[p], Lf)
            M = M.reshape(M.shape[0], -1)
            _, Rt = np.linalg.qr(M.T)
            Lf = Rt.T
        return np.linalg.svd(R @ Lf, compute_uv=False)

    def osee(self, bond):
        """Operator space entanglement entropy, Sec. 2.3 Eq. (OSEE): the von
        Neumann entropy of the normalised vectorised state |rho>> for the cut
        after path position bond, -sum_k p_k ln p_k with p_k = s_k^2 / sum s^2
        from the Schmidt values s_k."""
        s = self.schmidt_values(bond)
        p = s * s / np.sum(s * s)
        p = p[p > 0.0]
        return float(-np.sum(p * np.log(p)))

    def expect_1q(self, i, comp="Z"):
        c = [0] * self.n
        c[i] = PAULI_INDEX[comp]
        return self.chain(c) / self.chain([0] * self.n)

    def expect_2q(self, i, j, comps=("Z", "Z")):
        c = [0] * self.n
        c[i] = PAULI_INDEX[comps[0]]
        c[j] = PAULI_INDEX[comps[1]]
        return self.chain(c) / self.chain([0] * self.n)


def build_gates(wl, b, layers, dt):
    """16x16 gates of every op, instance b (scipy's expm)."""
    params = {"h_x": wl.h_x, "h_y": wl.h_y, "h_z": wl.h_z, "g0": wl.g0, "g1": wl.g1,
              "g2": wl.g2, "J": wl.J, "Jz": wl.Jz}
    w = schedule.onsite_weights(wl.n, wl.bonds)
    S = model.swap_matrix()
    out = []
    for layer in layers:
        gl = []
        for (kind, p, qa, qb, k, frac) in layer:
            if kind == "swap":
                gl.append(S)
            else:
                L = model.op_generator(params, b, qa, qb, k, w)
                gl.append(sla.expm(L * frac * dt))
        out.append(gl)
    return out


def graph_state_ops(n, pairs):
    """Op list that applies CZ to every listed pair (i, j) of path positions:
    for j > i + 1 swaps at j-1, ..., i+1 bring qubit j next to i, then CZ on
    (i, i+1), then the same swaps in reverse order.  Ops as (kind, p)."""
    ops = []
    for (i, j) in pairs:
        i, j = min(i, j), max(i, j)
        ops += [("swap", p) for p in range(j - 1, i, -1)]
        ops.append(("cz", i))
        ops += [("swap", p) for p in range(i + 1, j)]
    return ops


def graph_state(n, pairs, chi_max, cutoff):
    """The graph state of Sec. 2.2, Eq. (graph_state): every qubit +x, then a
    controlled-Z on every listed pair, applied as two-site gates (with the
    truncation rule of App. B) to the Pauli product state."""
    st = MPOState(*product_state(n, ["+x"] * n))
    S, CZ = model.swap_matrix(), model.cz_matrix()
    for kind, p in graph_state_ops(n, pairs):
        st.apply(p, CZ if kind == "cz" else S, chi_max, cutoff)
    return st


class TEBD:
    """Plain sequential MPO-TEBD for instance ``b`` of a workload."""

    def __init__(self, wl, b=0, state: Optional[MPOState] = None, force_trace=True, tol=None, order=2,
                 svd_impl="jacobi"):
        self.wl = wl
        self.b = b
        self.layers = schedule.step_layers_order(wl.n, wl.bonds, order)
        self.gates = build_gates(wl, b, self.layers, wl.dt)
        self.chi_max = int(wl.chi_max[b])
        self.cutoff = float(wl.cutoff[b])
        self.state = state if state is not None else MPOState(*product_state(wl.n, wl.init))
        self.force_trace = force_trace
        self.tol = tol
        self.svd_impl = svd_impl   # "lapack": numpy's gesdd route (large bond matrices)
        self.k_log: List[int] = []
        self.max_discarded = 0.0
        self.trace_log: List[float] = []

    def step(self, forced_k=None):
        """One second-order Trotter step.  ``forced_k`` (iterator of ints)
        replays a given rank sequence (frozen-rank mode)."""
        for layer, gl in zip(self.layers, self.gates):
            for op, G in zip(layer, gl):
                fk = next(forced_k) if forced_k is not None else None
                k, dw = self.state.apply(op[1], G, self.chi_max, self.cutoff, fk, self.tol, self.svd_impl)
                self.k_log.append(k)
                self.max_discarded = max(self.max_discarded, dw)
        if self.force_trace:
            self.trace_log.append(self.state.normalize_trace())

    def run(self, steps, forced_k=None):
        it = iter(forced_k) if forced_k is not None else None
        for _ in range(steps):
            self.step(it)
        return self

    def z(self):
        return np.array([self.state.expect_1q(i, "Z") for i in range(self.wl.n)])

    def zz_connected(self, pairs):
        z = self.z()
        return np.array([self.state.expect_2q(i, j) - z[i] * z[j] for (i, j) in pairs])
