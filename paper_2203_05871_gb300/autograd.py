"""torch.autograd.Function over libmpdo's adjoint: observables as a
differentiable function of the model parameters (argument marshalling only;
the evolution and its gradient run in the library's kernels).

    params  torch tensor [B, 6N + 2 n_bonds] (float64), packed as
            h_x[N], h_y[N], h_z[N], g0[N], g1[N], g2[N], J[n_bonds], Jz[n_bonds]
    returns (z, C): z [B, N] = <sigma^z_i>, C [B, N, N] = connected
            <sigma^z_i sigma^z_j> - <sigma^z_i><sigma^z_j> (symmetric, zero diagonal)
            after n_steps Trotter steps from the model's initial state.

Backward maps the cotangents of z and C to the parameters through
mpdo_grad_backward (the ranks of the forward run held fixed).  Typical use
(noise-model fitting): loss = ((z - z_measured) ** 2).sum(); loss.backward().
"""
from __future__ import annotations

import copy

import numpy as np

PARAM_FIELDS = ["h_x", "h_y", "h_z", "g0", "g1", "g2"]


def pack_params(wl) -> np.ndarray:
    """[B, 6N + 2 n_bonds] packed parameters of a workload-like object (fields
    h_x ... g2 of shape [B, N], J and Jz of shape [B, n_bonds])."""
    parts = [np.asarray(getattr(wl, f), dtype=np.float64) for f in PARAM_FIELDS]
    parts += [np.asarray(wl.J, dtype=np.float64), np.asarray(wl.Jz, dtype=np.float64)]
    return np.concatenate(parts, axis=1)


def with_params(wl, packed):
    """A shallow copy of wl whose parameter fields come from ``packed``."""
    packed = np.asarray(packed, dtype=np.float64)
    n, nb = wl.n, len(wl.bonds)
    if packed.shape != (wl.batch, 6 * n + 2 * nb):
        raise ValueError(f"params must have shape {(wl.batch, 6 * n + 2 * nb)}, got {packed.shape}")
    out = copy.copy(wl)
    for u, f in enumerate(PARAM_FIELDS):
        setattr(out, f, packed[:, u * n:(u + 1) * n].copy())
    out.J = packed[:, 6 * n:6 * n + nb].copy()
    out.Jz = packed[:, 6 * n + nb:].copy()
    return out


def connected_matrix(conn_pairs, n):
    """[B, n_pairs] values over pairs (i < j, row-major) -> symmetric [B, n, n]."""
    B = conn_pairs.shape[0]
    C = np.zeros((B, n, n))
    iu = np.triu_indices(n, 1)
    C[:, iu[0], iu[1]] = conn_pairs
    C[:, iu[1], iu[0]] = conn_pairs
    return C


def pair_cotangent(gC):
    """Cotangent of the symmetric C -> weights of the pairs i < j (upper triangle)."""
    g = np.asarray(gC, dtype=np.float64)
    return np.triu(g + np.swapaxes(g, 1, 2), 1)


def _function():
    import torch

    class LindbladObservables(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, solver, wl, n_steps):
            w = with_params(wl, params.detach().cpu().numpy())
            solver.build_gates(w)
            solver.grad_forward(int(n_steps))
            n = wl.n
            z = solver.measure_1q(range(n), "Z")
            pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
            C = connected_matrix(solver.measure_2q(pairs, "ZZ", connected=True), n)
            ctx.solver = solver
            return (torch.from_numpy(z).to(device=params.device, dtype=params.dtype),
                    torch.from_numpy(C).to(device=params.device, dtype=params.dtype))

        @staticmethod
        def backward(ctx, gz, gC):
            zb = None if gz is None else gz.detach().cpu().numpy().astype(np.float64)
            wb = None if gC is None else pair_cotangent(gC.detach().cpu().numpy())
            g, _ = ctx.solver.grad_backward(zb, wb)
            return torch.from_numpy(g).to(device=gz.device if gz is not None else gC.device,
                                          dtype=gz.dtype if gz is not None else gC.dtype), None, None, None

    return LindbladObservables


_FN = None


def observables(params, solver, wl, n_steps):
    """(z [B, N], C [B, N, N]) as differentiable functions of ``params``."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(params, solver, wl, n_steps)
