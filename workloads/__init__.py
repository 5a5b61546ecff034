"""Seeded synthetic inputs shared by the oracle, the tests and bench.py.

This module only *describes* workloads: coupling graphs (bond lists on the
MPO path), per-qubit / per-bond parameter draws and solver settings.  It holds
no step of the method (no Liouvillian, no gate, no contraction), so that the
CPU oracle and the CUDA path can both take their inputs from here without
sharing any arithmetic.

Parameter conventions follow the paper's model (Sec. 2.1, Eq. (H0), Eq. (K_def),
Eqs. (D0)-(D2)) in the rotating frame of Sec. 3.1 (Eq. (h_xi_hz_i)):
  h_z[i] = detuning omega_i, h_x[0] = Omega (drive on the edge qubit),
  J[b] = XY coupling of bond b, g0/g1/g2 = decay / excitation / dephasing.
Random draws use numpy ``Generator(PCG64(seed))`` in a fixed order:
J per bond (bond order), then Omega, then g0 per qubit, then g2 per qubit,
then chi_max per instance.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

Bond = Tuple[int, int]


# --------------------------------------------------------------------------
# geometry (bond lists in MPO-path positions; Sec. 2.5 maps any connectivity
# onto a 1D path with long-ranged bonds along it)
# --------------------------------------------------------------------------
def chain_bonds(n: int) -> List[Bond]:
    """Open chain 0-1-...-(n-1)."""
    return [(i, i + 1) for i in range(n - 1)]


def ring_bonds(n: int) -> List[Bond]:
    """Ring in natural order: the chain plus the closing bond (0, n-1)."""
    return chain_bonds(n) + [(0, n - 1)]


def snake_index(x: int, y: int, ly: int) -> int:
    """Path position of grid site (x, y) for a snake running up even columns
    and down odd columns (columns of ``ly`` sites)."""
    return ly * x + (y if x % 2 == 0 else ly - 1 - y)


def grid_snake_bonds(lx: int, ly: int) -> List[Bond]:
    """Nearest-neighbour bonds of an lx-by-ly grid, in snake-path positions.
    Vertical bonds first (column by column), then horizontal bonds."""
    bonds = []
    for x in range(lx):
        for y in range(ly - 1):
            a, b = snake_index(x, y, ly), snake_index(x, y + 1, ly)
            bonds.append((min(a, b), max(a, b)))
    for x in range(lx - 1):
        for y in range(ly):
            a, b = snake_index(x, y, ly), snake_index(x + 1, y, ly)
            bonds.append((min(a, b), max(a, b)))
    return bonds


# --------------------------------------------------------------------------
# a workload = one or more instances sharing a graph
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n: int
    bonds: List[Bond]
    # per-instance arrays, shape [B, n] or [B, n_bonds]
    h_x: np.ndarray
    h_y: np.ndarray
    h_z: np.ndarray
    g0: np.ndarray
    g1: np.ndarray
    g2: np.ndarray
    J: np.ndarray
    Jz: np.ndarray
    chi_max: np.ndarray      # [B] int
    cutoff: np.ndarray       # [B] float
    dt: float
    steps: int
    init: Optional[List[str]] = None   # per-qubit "+z", "-x", ...; None = all "+z"
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return int(self.h_z.shape[0])

    def instance(self, b: int) -> "Workload":
        """The single-instance workload b (arrays keep a leading axis of 1)."""
        sl = slice(b, b + 1)
        return Workload(self.name + f"[{b}]", self.n, list(self.bonds),
                        self.h_x[sl].copy(), self.h_y[sl].copy(), self.h_z[sl].copy(),
                        self.g0[sl].copy(), self.g1[sl].copy(), self.g2[sl].copy(),
                        self.J[sl].copy(), self.Jz[sl].copy(),
                        self.chi_max[sl].copy(), self.cutoff[sl].copy(),
                        self.dt, self.steps, None if self.init is None else list(self.init),
                        self.notes, dict(self.extra))

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


def _alternating(n: int) -> np.ndarray:
    return np.array([float(i % 2) for i in range(n)])


def uniform_model(name: str, n: int, bonds: List[Bond], *, omega=None, Omega=0.5,
                  drive_qubit=0, J=0.1, Jz=0.0, g0=0.01, g1=0.0, g2=0.02,
                  chi_max=32, cutoff=1e-12, dt=0.05, steps=40, batch=1, init=None,
                  notes="") -> Workload:
    """Deterministic model with one value per parameter kind (config-1 style)."""
    nb = len(bonds)
    hz = _alternating(n) if omega is None else np.asarray(omega, dtype=float)
    hx = np.zeros(n)
    hx[drive_qubit] = Omega
    rep = lambda v, k: np.tile(np.asarray(v, dtype=float).reshape(1, -1) * np.ones((1, k)), (batch, 1))
    return Workload(name, n, list(bonds),
                    rep(hx, n), rep(np.zeros(n), n), rep(hz, n),
                    rep(g0, n), rep(g1, n), rep(g2, n),
                    rep(J, nb), rep(Jz, nb),
                    np.full(batch, int(chi_max)), np.full(batch, float(cutoff)),
                    float(dt), int(steps), init, notes)


# --------------------------------------------------------------------------
# the five benchmark workloads
# --------------------------------------------------------------------------
def chain8_fp64() -> Workload:
    """N=8 open chain, chi_max=32, cutoff 1e-12, dt=0.05 x 40 steps;
    h_z alternating 0,1; J=0.1; Omega=0.5 on qubit 0; g0=0.01; g2=0.02."""
    return uniform_model("chain8_chi32", 8, chain_bonds(8), chi_max=32, cutoff=1e-12,
                         dt=0.05, steps=40)


def chain20_precision(seed: int = 2203058712, chi_max: int = 128) -> Workload:
    """N=20 open chain with seeded couplings: J_b~U[0.05,0.15], Omega~U[0.3,0.7],
    g0_i~U[0.005,0.02], g2_i~U[0.01,0.03]; h_z alternating 0,1;
    chi_max=128, cutoff 1e-10, dt=0.02 x 500 steps."""
    n = 20
    bonds = chain_bonds(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    J = rng.uniform(0.05, 0.15, size=len(bonds))
    Omega = rng.uniform(0.3, 0.7)
    g0 = rng.uniform(0.005, 0.02, size=n)
    g2 = rng.uniform(0.01, 0.03, size=n)
    hx = np.zeros(n)
    hx[0] = Omega
    one = lambda a: np.asarray(a, dtype=float).reshape(1, -1)
    return Workload("chain20_precision", n, bonds, one(hx), one(np.zeros(n)), one(_alternating(n)),
                    one(g0), one(np.zeros(n)), one(g2), one(J), one(np.zeros(len(bonds))),
                    np.array([chi_max]), np.array([1e-10]), 0.02, 500)


def batch64_chain16(batch: int = 64, seed0: int = 2203058713) -> Workload:
    """``batch`` independent N=16 open chains; instance b draws (seed seed0+b)
    J~U[0.05,0.2], Omega~U[0.1,1.0], g0~U[0.001,0.02], g2~U[0.005,0.05] (one
    value per instance, uniform over bonds/qubits) and chi_max from
    {32,64,128,256}; dt=0.05 x 200 steps; cutoff 1e-10."""
    n = 16
    bonds = chain_bonds(n)
    nb = len(bonds)
    cols = {k: [] for k in ("hx", "hz", "g0", "g2", "J", "chi")}
    for b in range(batch):
        rng = np.random.Generator(np.random.PCG64(seed0 + b))
        J = rng.uniform(0.05, 0.2)
        Omega = rng.uniform(0.1, 1.0)
        g0 = rng.uniform(0.001, 0.02)
        g2 = rng.uniform(0.005, 0.05)
        chi = int(rng.choice([32, 64, 128, 256]))
        hx = np.zeros(n)
        hx[0] = Omega
        cols["hx"].append(hx)
        cols["hz"].append(_alternating(n))
        cols["g0"].append(np.full(n, g0))
        cols["g2"].append(np.full(n, g2))
        cols["J"].append(np.full(nb, J))
        cols["chi"].append(chi)
    z = np.zeros((batch, n))
    return Workload("batch64_chain16", n, bonds, np.array(cols["hx"]), z.copy(), np.array(cols["hz"]),
                    np.array(cols["g0"]), z.copy(), np.array(cols["g2"]), np.array(cols["J"]),
                    np.zeros((batch, nb)), np.array(cols["chi"]), np.full(batch, 1e-10), 0.05, 200)


def ring24_adjoint() -> Workload:
    """N=24 ring in natural order (closing bond (0,23) routed by swap gates);
    J=0.1, Omega=0.5, g0=0.01, g2=0.02, h_z alternating; chi_max=256,
    cutoff 1e-10, dt=0.05 x 100 steps."""
    return uniform_model("ring24", 24, ring_bonds(24), chi_max=256, cutoff=1e-10, dt=0.05, steps=100)


def grid4x10_snake() -> Workload:
    """4x10 grid on a snake path (columns of 4), checkerboard h_z, J=0.1,
    Omega=0.5 on the corner qubit (path position 0), g0=0.01, g2=0.02;
    chi_max=512, cutoff 1e-9, dt=0.05 x 1000 steps."""
    lx, ly = 10, 4
    n = lx * ly
    hz = np.zeros(n)
    for x in range(lx):
        for y in range(ly):
            hz[snake_index(x, y, ly)] = float((x + y) % 2)
    return uniform_model("grid4x10", n, grid_snake_bonds(lx, ly), omega=hz, chi_max=512,
                         cutoff=1e-9, dt=0.05, steps=1000)


def random_model(n: int, bonds: List[Bond], seed: int, *, batch: int = 1, chi_max: int = 16,
                 cutoff: float = 0.0, dt: float = 0.05, steps: int = 4, with_all_terms=True,
                 init: Optional[List[str]] = None) -> Workload:
    """Small seeded model with every term of Eq. (H0)/(K_def)/(D0)-(D2) switched
    on (h_x, h_y, h_z, J, Jz, g0, g1, g2), for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = len(bonds)
    u = lambda lo, hi, shape: rng.uniform(lo, hi, size=shape)
    hx = u(-1.0, 1.0, (batch, n))
    hy = u(-1.0, 1.0, (batch, n)) if with_all_terms else np.zeros((batch, n))
    hz = u(-1.0, 1.0, (batch, n))
    g0 = u(0.0, 0.2, (batch, n))
    g1 = u(0.0, 0.1, (batch, n)) if with_all_terms else np.zeros((batch, n))
    g2 = u(0.0, 0.1, (batch, n))
    J = u(0.1, 0.6, (batch, nb))
    Jz = u(-0.3, 0.3, (batch, nb)) if with_all_terms else np.zeros((batch, nb))
    return Workload(f"random{n}_s{seed}", n, list(bonds), hx, hy, hz, g0, g1, g2, J, Jz,
                    np.full(batch, int(chi_max)), np.full(batch, float(cutoff)), float(dt),
                    int(steps), init)


def random_mpo_state(n: int, chi: int, seed: int, decay: float = 0.0):
    """Seeded random MPO site tensors B[p] of shape (chi_l, 4, chi_r) with the
    bond dimensions capped by 4^min(p+1, n-p-1) (the exact-representation
    bound of App. B) and entries N(0,1)/sqrt(4 chi_l) * exp(-decay * r) on
    right-bond index r.  decay = 0 gives a flat (worst-case) Schmidt spectrum;
    decay > 0 grades the bonds the way time-evolved states are graded (their
    Schmidt values fall off).  Used to start a benchmark at saturated bond
    dimension.  Returns (dims, tensors)."""
    dims = [1]
    for p in range(n - 1):
        dims.append(int(min(chi, 4 ** min(p + 1, n - p - 1))))
    dims.append(1)
    return dims, random_mpo_tensors(dims, seed, decay)


def random_mpo_tensors(dims, seed: int, decay: float = 0.0):
    """Site tensors of random_mpo_state for given bond dimensions dims[0..n]
    (dims[0] = dims[n] = 1; the caller keeps them within the 4^min(p, n-p)
    bound)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tensors = []
    for p in range(len(dims) - 1):
        cl, cr = dims[p], dims[p + 1]
        scale = np.exp(-decay * np.arange(cr)) if decay > 0 else np.ones(cr)
        tensors.append(rng.standard_normal((cl, 4, cr)) / np.sqrt(4.0 * cl) * scale[None, None, :])
    return tensors


ALL = {
    "chain8_chi32": chain8_fp64,
    "chain20_precision": chain20_precision,
    "batch64_chain16": batch64_chain16,
    "ring24": ring24_adjoint,
    "grid4x10": grid4x10_snake,
}
