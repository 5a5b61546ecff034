"""Host logic of the torch.autograd wrapper (no GPU): parameter packing and the
cotangent marshalling, with a stand-in solver whose observables are linear in
the parameters (so the exact gradient is known)."""
import numpy as np
import pytest

import workloads as W
from paper_2203_05871_gb300 import autograd as AG

torch = pytest.importorskip("torch")


def test_pack_with_params_roundtrip():
    wl = W.random_model(5, W.ring_bonds(5), 3, batch=2)
    p = AG.pack_params(wl)
    assert p.shape == (2, 6 * 5 + 2 * 5)
    w2 = AG.with_params(wl, p * 2.0)
    np.testing.assert_array_equal(AG.pack_params(w2), p * 2.0)
    np.testing.assert_array_equal(w2.g2, wl.g2 * 2.0)
    np.testing.assert_array_equal(wl.J, AG.pack_params(wl)[:, 30:35])   # original untouched
    with pytest.raises(ValueError):
        AG.with_params(wl, p[:, :-1])


def test_connected_matrix_and_pair_cotangent():
    n = 4
    vals = np.arange(6, dtype=float)[None, :] + 1.0
    C = AG.connected_matrix(vals, n)
    assert np.allclose(C, np.swapaxes(C, 1, 2)) and np.all(np.diagonal(C, axis1=1, axis2=2) == 0)
    assert C[0, 0, 1] == 1.0 and C[0, 2, 3] == 6.0
    g = np.zeros((1, n, n))
    g[0, 1, 0] = 2.0
    g[0, 0, 1] = 3.0
    w = AG.pair_cotangent(g)
    assert w[0, 0, 1] == 5.0 and w[0, 1, 0] == 0.0


class FakeSolver:
    """z = A p, conn_pairs = D p per instance: the backward must return A^T gz + D^T w."""

    def __init__(self, wl, seed=0):
        rng = np.random.default_rng(seed)
        self.n = wl.n
        P = 6 * wl.n + 2 * len(wl.bonds)
        self.A = rng.normal(size=(wl.n, P))
        self.D = rng.normal(size=(wl.n * (wl.n - 1) // 2, P))
        self.p = None

    def build_gates(self, w):
        self.p = AG.pack_params(w)

    def grad_forward(self, n_steps):
        pass

    def measure_1q(self, q, comp):
        return self.p @ self.A.T

    def measure_2q(self, pairs, comps, connected=True):
        return self.p @ self.D.T

    def grad_backward(self, zb, wb):
        n = self.n
        iu = np.triu_indices(n, 1)
        w = wb[:, iu[0], iu[1]]
        return zb @ self.A + w @ self.D, None


def test_function_marshals_cotangents():
    wl = W.random_model(4, W.chain_bonds(4), 9, batch=2)
    fs = FakeSolver(wl)
    p = torch.tensor(AG.pack_params(wl), dtype=torch.float64, requires_grad=True)
    z, C = AG.observables(p, fs, wl, 3)
    tz = torch.randn(z.shape, dtype=torch.float64)
    loss = ((z - tz) ** 2).sum() + (C ** 2).sum() * 0.5
    loss.backward()
    # reference: the same function written with plain torch ops
    p2 = p.detach().clone().requires_grad_(True)
    A = torch.tensor(fs.A)
    D = torch.tensor(fs.D)
    z2 = p2 @ A.T
    cp = p2 @ D.T
    loss2 = ((z2 - tz) ** 2).sum() + (cp ** 2).sum()   # C holds each pair twice
    loss2.backward()
    assert torch.allclose(p.grad, p2.grad, atol=1e-12)
