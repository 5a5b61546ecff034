"""Gradient of the dense Trotter product.  Test infrastructure only.

The paper computes no gradient.  This module gives the exact derivative of
the observables of ``dense.DenseTrotter`` (the op list of ``schedule`` applied
to the full 4^N Pauli-coefficient vector, no truncation) with respect to the
model parameters, by reverse mode written out plainly:

* loss at the final vector r (Sec. 2.3 observables, Eq. (mu), Eq. (etadef)):
      L = sum_i zbar_i <z_i> + sum_{i<j} wbar_ij (<z_i z_j> - <z_i><z_j>),
  <P> = r[P] / r[I..I]; its gradient dL/dr is taken entry by entry from
  this definition (only the entries I..I, Z at i, Z at i and j are touched);
* each op r' = G r on path positions (p, p+1), in reverse:
      G-bar += sum over the other indices of r'-bar (outer) r,
      r-bar  = G^T r'-bar;
* each gate G = exp(tau L_op) (tau = frac * dt): the cotangent of L_op is
  tau * (Frechet derivative of exp at (tau L_op)^T in the direction G-bar),
  evaluated by ``scipy.linalg.expm_frechet``;
* L_op is linear in the parameters, so dL/dtheta = <L_op-bar, L_op(unit theta)>,
  with L_op(unit theta) the generator ``model.op_generator`` builds when only
  theta is 1.

Parameters are packed as in the library: h_x[N], h_y[N], h_z[N], g0[N],
g1[N], g2[N], J[n_bonds], Jz[n_bonds].

Pinned by tests/test_oracle_adjoint.py: closed-form derivatives of
two-qubit solutions (XY transfer, Rabi with detuning, decay) and central
finite differences of ``DenseTrotter`` itself on a random ring.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import model, schedule, tebd

PARAM_NAMES = ["h_x", "h_y", "h_z", "g0", "g1", "g2"]


def _params(wl):
    return {"h_x": wl.h_x, "h_y": wl.h_y, "h_z": wl.h_z, "g0": wl.g0, "g1": wl.g1,
            "g2": wl.g2, "J": wl.J, "Jz": wl.Jz}


def unit_generator(wl, idx, qa, qb, bond, weights):
    """L_op of one op with parameter ``idx`` (packed index) = 1, all others 0."""
    n, nb = wl.n, len(wl.bonds)
    P = {k: [np.zeros(n)] for k in PARAM_NAMES}
    P["J"] = [np.zeros(nb)]
    P["Jz"] = [np.zeros(nb)]
    if idx < 6 * n:
        P[PARAM_NAMES[idx // n]][0][idx % n] = 1.0
    elif idx < 6 * n + nb:
        P["J"][0][idx - 6 * n] = 1.0
    else:
        P["Jz"][0][idx - 6 * n - nb] = 1.0
    return model.op_generator(P, 0, qa, qb, bond, weights)


def loss_and_cotangent(r, n, zbar, wbar):
    """L and dL/dr for the final coefficient vector r (4^N)."""
    t = np.asarray(r, dtype=np.float64).reshape([4] * n)
    I = tuple([0] * n)

    def idx(zs):
        c = [0] * n
        for q in zs:
            c[q] = 3
        return tuple(c)

    Z = t[I]
    e = np.array([t[idx([i])] / Z for i in range(n)])
    L = float(np.dot(zbar, e))
    g = np.zeros_like(t)
    # d e_i = (dE_i - e_i dZ) / Z
    for i in range(n):
        g[idx([i])] += zbar[i] / Z
        g[I] -= zbar[i] * e[i] / Z
    for i in range(n):
        for j in range(i + 1, n):
            w = wbar[i][j]
            if w == 0.0:
                continue
            eij = t[idx([i, j])] / Z
            L += w * (eij - e[i] * e[j])
            # d(e_ij - e_i e_j) = (dE_ij - e_ij dZ)/Z - e_j de_i - e_i de_j
            g[idx([i, j])] += w / Z
            g[I] -= w * eij / Z
            g[idx([i])] -= w * e[j] / Z
            g[I] += w * e[j] * e[i] / Z
            g[idx([j])] -= w * e[i] / Z
            g[I] += w * e[i] * e[j] / Z
    return L, g


def dense_trotter_grad(wl, b, steps, zbar, wbar):
    """Returns (L, grad) for instance b after ``steps`` dense Trotter steps."""
    n = wl.n
    layers = schedule.step_layers(n, wl.bonds)
    gates = tebd.build_gates(wl, b, layers, wl.dt)
    weights = schedule.onsite_weights(n, wl.bonds)
    st = tebd.MPOState(*tebd.product_state(n, wl.init))
    r = st.to_vector().reshape([4] * n)
    ops = [(op, G) for layer, gl in zip(layers, gates) for op, G in zip(layer, gl)]
    # forward, keeping the input of every op
    saved = []
    for _ in range(steps):
        for (op, G) in ops:
            p = op[1]
            saved.append(r)
            t = np.moveaxis(r, (p, p + 1), (0, 1))
            t = np.tensordot(G.reshape(4, 4, 4, 4), t, axes=([2, 3], [0, 1]))
            r = np.moveaxis(t, (0, 1), (p, p + 1))
    L, rbar = loss_and_cotangent(r, n, np.asarray(zbar, float), np.asarray(wbar, float))
    # reverse
    Gbar = [np.zeros((16, 16)) for _ in ops]
    for s in range(steps - 1, -1, -1):
        for o in range(len(ops) - 1, -1, -1):
            (op, G) = ops[o]
            p = op[1]
            r_in = saved[s * len(ops) + o]
            ob = np.moveaxis(rbar, (p, p + 1), (0, 1)).reshape(16, -1)
            ri = np.moveaxis(r_in, (p, p + 1), (0, 1)).reshape(16, -1)
            Gbar[o] += ob @ ri.T
            t = (G.T @ ob).reshape([4, 4] + [4] * (n - 2))
            rbar = np.moveaxis(t, (0, 1), (p, p + 1))
    # parameters
    P = _params(wl)
    nb = len(wl.bonds)
    grad = np.zeros(6 * n + 2 * nb)
    for o, (op, G) in enumerate(ops):
        kind, p, qa, qb, bond, frac = op
        if kind == "swap":
            continue
        tau = frac * wl.dt
        X = tau * model.op_generator(P, b, qa, qb, bond, weights)
        _, Xbar = sla.expm_frechet(X.T, Gbar[o])
        Lbar = tau * Xbar
        touched = [u * n + qa for u in range(6)] + [u * n + qb for u in range(6)] + [6 * n + bond, 6 * n + nb + bond]
        for idx in sorted(set(touched)):
            grad[idx] += float(np.sum(Lbar * unit_generator(wl, idx, qa, qb, bond, weights)))
    return L, grad


def dense_loss(wl, b, steps, zbar, wbar):
    """L of ``dense_trotter_grad`` without the gradient (for finite differences)."""
    from .dense import DenseTrotter
    r = DenseTrotter(wl, b).run(steps).vector()
    return loss_and_cotangent(r, wl.n, np.asarray(zbar, float), np.asarray(wbar, float))[0]
