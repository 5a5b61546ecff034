"""Pins of the dense-Trotter gradient oracle (oracle/adjoint.py), no GPU.

Closed forms: for N = 2 with one bond, a second-order step is the single gate
exp(L dt) (the two half-steps of one generator merge exactly), so the dense
Trotter product is the exact solution and its derivatives are those of the
textbook two-level formulas.  Differentiated here with sympy from the closed
forms, not from the oracle's code.
"""
import numpy as np
import pytest
import sympy as sp

import workloads as W
from oracle import adjoint, dense

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def two_qubit(hx0=0.0, hz0=0.0, g00=0.0, J=0.0, init=("+z", "+z"), dt=0.05, steps=10):
    return W.uniform_model("two", 2, [(0, 1)], omega=[hz0, 0.0], Omega=hx0, J=J, g0=0.0, g2=0.0,
                           dt=dt, steps=steps, init=list(init)) if g00 == 0.0 else _with_decay(
        hx0, hz0, g00, J, init, dt, steps)


def _with_decay(hx0, hz0, g00, J, init, dt, steps):
    wl = W.uniform_model("two", 2, [(0, 1)], omega=[hz0, 0.0], Omega=hx0, J=J, g0=0.0, g2=0.0,
                         dt=dt, steps=steps, init=list(init))
    wl.g0[0][0] = g00
    return wl


def idx(wl, name, q):
    n, nb = wl.n, len(wl.bonds)
    names = ["h_x", "h_y", "h_z", "g0", "g1", "g2"]
    if name in names:
        return names.index(name) * n + q
    return 6 * n + (0 if name == "J" else nb) + q


def test_xy_transfer_derivative_in_J():
    """|1,0> under J (s+ s- + h.c.): <z_0> = -cos(2Jt), connected <z_0 z_1> =
    -sin^2(2Jt) (one excitation shared by two qubits)."""
    J0, t = 0.37, 0.5
    wl = two_qubit(J=J0, init=("-z", "+z"), dt=0.05, steps=10)
    Js, ts = sp.symbols("J t")
    z0 = -sp.cos(2 * Js * ts)
    conn = -sp.sin(2 * Js * ts) ** 2
    L, g = adjoint.dense_trotter_grad(wl, 0, 10, [1.0, 0.0], [[0, 0], [0, 0]])
    assert abs(L - float(z0.subs({Js: J0, ts: t}))) < 1e-12
    assert abs(g[idx(wl, "J", 0)] - float(sp.diff(z0, Js).subs({Js: J0, ts: t}))) < 1e-11
    L, g = adjoint.dense_trotter_grad(wl, 0, 10, [0.0, 0.0], [[0, 1.0], [0, 0]])
    assert abs(L - float(conn.subs({Js: J0, ts: t}))) < 1e-12
    assert abs(g[idx(wl, "J", 0)] - float(sp.diff(conn, Js).subs({Js: J0, ts: t}))) < 1e-11


def test_detuned_rabi_derivatives():
    """H = (Omega sigma_x + Delta sigma_z)/2 from +z:
    <z> = 1 - 2 (Omega/W)^2 sin^2(W t / 2), W = sqrt(Omega^2 + Delta^2)."""
    Om0, De0, t = 0.8, 0.45, 0.6
    wl = two_qubit(hx0=Om0, hz0=De0, dt=0.03, steps=20)
    O, D, T = sp.symbols("O D T")
    Wf = sp.sqrt(O ** 2 + D ** 2)
    z = 1 - 2 * (O / Wf) ** 2 * sp.sin(Wf * T / 2) ** 2
    sub = {O: Om0, D: De0, T: t}
    L, g = adjoint.dense_trotter_grad(wl, 0, 20, [1.0, 0.0], [[0, 0], [0, 0]])
    assert abs(L - float(z.subs(sub))) < 1e-12
    assert abs(g[idx(wl, "h_x", 0)] - float(sp.diff(z, O).subs(sub))) < 1e-11
    assert abs(g[idx(wl, "h_z", 0)] - float(sp.diff(z, D).subs(sub))) < 1e-11
    # qubit 1 is idle: nothing on it moves <z_0>
    for name in ["h_x", "h_y", "h_z", "g0", "g1", "g2"]:
        assert abs(g[idx(wl, name, 1)]) < 1e-13


def test_decay_derivative_in_g0():
    """sigma^- decay at rate g0 from -z: <z> = 1 - 2 exp(-g0 t)."""
    g00, t = 0.3, 0.8
    wl = two_qubit(g00=g00, init=("-z", "+z"), dt=0.04, steps=20)
    G, T = sp.symbols("G T")
    z = 1 - 2 * sp.exp(-G * T)
    L, g = adjoint.dense_trotter_grad(wl, 0, 20, [1.0, 0.0], [[0, 0], [0, 0]])
    assert abs(L - float(z.subs({G: g00, T: t}))) < 1e-12
    assert abs(g[idx(wl, "g0", 0)] - float(sp.diff(z, G).subs({G: g00, T: t}))) < 1e-11


def test_loss_cotangent_matches_finite_differences():
    rng = np.random.default_rng(5)
    n = 3
    r = rng.normal(size=4 ** n)
    r[0] += 3.0
    zb = rng.normal(size=n)
    wb = np.triu(rng.normal(size=(n, n)), 1)
    L0, g = adjoint.loss_and_cotangent(r, n, zb, wb)
    h = 1e-6
    for i in [0, 3, 12, 15, 48, 51, 60, 63, 5]:
        rp, rm = r.copy(), r.copy()
        rp[i] += h
        rm[i] -= h
        fd = (adjoint.loss_and_cotangent(rp, n, zb, wb)[0] - adjoint.loss_and_cotangent(rm, n, zb, wb)[0]) / (2 * h)
        assert abs(g.reshape(-1)[i] - fd) < 1e-8 * max(1.0, abs(fd))


def test_random_ring_gradient_matches_finite_differences():
    """Every parameter kind on a 4-qubit ring (swap-routed closing bond)."""
    wl = W.random_model(4, W.ring_bonds(4), 21, dt=0.07)
    steps = 3
    rng = np.random.default_rng(2)
    zb = rng.normal(size=4)
    wb = np.triu(rng.normal(size=(4, 4)), 1)
    L, g = adjoint.dense_trotter_grad(wl, 0, steps, zb, wb)
    assert abs(L - adjoint.dense_loss(wl, 0, steps, zb, wb)) < 1e-13
    n, nb = 4, len(wl.bonds)
    names = ["h_x", "h_y", "h_z", "g0", "g1", "g2"]
    h = 1e-6
    for k in range(6 * n + 2 * nb):
        wp = W.Workload(**{f: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v)
                           for f, v in wl.__dict__.items()})
        wm = W.Workload(**{f: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v)
                           for f, v in wl.__dict__.items()})
        if k < 6 * n:
            getattr(wp, names[k // n])[0][k % n] += h
            getattr(wm, names[k // n])[0][k % n] -= h
        elif k < 6 * n + nb:
            wp.J[0][k - 6 * n] += h
            wm.J[0][k - 6 * n] -= h
        else:
            wp.Jz[0][k - 6 * n - nb] += h
            wm.Jz[0][k - 6 * n - nb] -= h
        fd = (adjoint.dense_loss(wp, 0, steps, zb, wb) - adjoint.dense_loss(wm, 0, steps, zb, wb)) / (2 * h)
        assert abs(g[k] - fd) < 2e-8 * max(1.0, abs(fd)), (k, g[k], fd)


def test_dense_loss_is_the_trotter_observable():
    wl = W.random_model(4, W.chain_bonds(4), 3, dt=0.05)
    dt = dense.DenseTrotter(wl, 0).run(2)
    z = dt.z()
    zb = np.array([0.3, -1.0, 0.5, 2.0])
    wb = np.zeros((4, 4))
    wb[0, 2] = 1.5
    expect = zb @ z + 1.5 * (dt.zz(0, 2) - z[0] * z[2])
    assert abs(adjoint.dense_loss(wl, 0, 2, zb, wb) - expect) < 1e-13
