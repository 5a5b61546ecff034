"""Op list of one second-order Trotter step.  Test infrastructure only.

The paper integrates with the W^II evolution MPO (Sec. 2.5) and is silent on a
two-site-gate schedule; this module takes the following reading:

* The qubits sit on a 1D path (Sec. 2.5); a bond (i, j) with j = i+1 is a
  nearest-neighbour (NN) bond, j > i+1 is long-ranged along the path.
* Forward half F, as a list of layers of disjoint ops:
  the layer of NN bonds with even left position, the layer of NN bonds with
  odd left position, then for each long-range bond (i, j) in bond order the
  swaps (j-1,j), (j-2,j-1), ..., (i+1,i+2) (one layer each, bringing qubit j
  next to i), the gate on (i, i+1), and the same swaps in reverse order.
* A step is F at dt/2 followed by reversed(F) at dt/2 (a symmetric, hence
  second-order, product).  Where the two halves meet, mirrored swap layers
  cancel (SWAP^2 = 1) and the meeting gate layer is applied once at dt.
* Each qubit's on-site Liouvillian is shared by its gates with weight
  1/deg(q), deg(q) = number of bonds at q; every qubit needs deg >= 1.

An op is the tuple (kind, p, qa, qb, bond, frac): kind 'gate' or 'swap', left
path position p, qubits qa at p and qb at p+1 before the op, bond index (-1 for
swaps) and the fraction of dt (0 for swaps).

Fourth order (the paper uses order 4 throughout, App. B; its W^II MPO is not
the blueprint here): Suzuki's symmetric triple jump of the second-order step,
S4(dt) = S2(w1 dt) S2(w0 dt) S2(w1 dt) with w1 = 1 / (2 - 2^(1/3)) and
w0 = 1 - 2 w1 (negative), i.e. the three op lists one after the other with
their gate fractions scaled.  Symmetric compositions have even order, so no
third-order variant is built.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

Op = Tuple[str, int, int, int, int, float]


def validate_bonds(n: int, bonds: Sequence[Tuple[int, int]]):
    if n < 2:
        raise ValueError("need at least two qubits")
    seen = set()
    deg = [0] * n
    for (i, j) in bonds:
        if not (0 <= i < n and 0 <= j < n) or i == j:
            raise ValueError(f"bad bond {(i, j)}")
        key = (min(i, j), max(i, j))
        if key in seen:
            raise ValueError(f"duplicate bond {key}")
        seen.add(key)
        deg[i] += 1
        deg[j] += 1
    if min(deg) == 0:
        raise ValueError("every qubit needs at least one bond")
    return deg


def onsite_weights(n, bonds):
    deg = validate_bonds(n, bonds)
    return [1.0 / d for d in deg]


def forward_layers(n: int, bonds: Sequence[Tuple[int, int]]) -> List[List[Op]]:
    validate_bonds(n, bonds)
    norm = [(min(i, j), max(i, j)) for (i, j) in bonds]
    even = sorted([(i, k) for k, (i, j) in enumerate(norm) if j == i + 1 and i % 2 == 0])
    odd = sorted([(i, k) for k, (i, j) in enumerate(norm) if j == i + 1 and i % 2 == 1])
    layers: List[List[Op]] = []
    if even:
        layers.append([("gate", i, i, i + 1, k, 0.5) for (i, k) in even])
    if odd:
        layers.append([("gate", i, i, i + 1, k, 0.5) for (i, k) in odd])
    at = list(range(n))                     # at[position] = qubit
    for k, (i, j) in enumerate(norm):
        if j == i + 1:
            continue
        swaps_in = list(range(j - 1, i, -1))   # left positions j-1, ..., i+1
        for p in swaps_in:
            layers.append([("swap", p, at[p], at[p + 1], -1, 0.0)])
            at[p], at[p + 1] = at[p + 1], at[p]
        layers.append([("gate", i, at[i], at[i + 1], k, 0.5)])
        for p in reversed(swaps_in):
            layers.append([("swap", p, at[p], at[p + 1], -1, 0.0)])
            at[p], at[p + 1] = at[p + 1], at[p]
    assert at == list(range(n))
    return layers


def _mirror_op(op: Op, at: List[int]) -> Op:
    kind, p, qa, qb, k, frac = op
    return (kind, p, at[p], at[p + 1], k, frac)


def step_layers(n: int, bonds: Sequence[Tuple[int, int]]) -> List[List[Op]]:
    """Layers of one full second-order step (see module docstring)."""
    F = forward_layers(n, bonds)
    R = list(reversed(F))
    # cancel mirrored swap layers at the junction
    while F and R and F[-1][0][0] == "swap" and R[0][0][0] == "swap" and \
            [o[1] for o in F[-1]] == [o[1] for o in R[0]]:
        F = F[:-1]
        R = R[1:]
    assert F and R and F[-1][0][0] == "gate"
    middle = [(kind, p, qa, qb, k, 1.0) for (kind, p, qa, qb, k, _f) in F[-1]]
    seq = F[:-1] + [middle] + R[1:]
    # recompute the qubits at each position along the whole step
    at = list(range(n))
    out = []
    for layer in seq:
        new = []
        for op in layer:
            new.append(_mirror_op(op, at))
        for op in layer:
            if op[0] == "swap":
                p = op[1]
                at[p], at[p + 1] = at[p + 1], at[p]
        out.append(new)
    assert at == list(range(n))
    return out


def count_ops(layers):
    g = sum(1 for L in layers for o in L if o[0] == "gate")
    s = sum(1 for L in layers for o in L if o[0] == "swap")
    return g, s


W1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
W0 = 1.0 - 2.0 * W1


def step_layers_order(n: int, bonds: Sequence[Tuple[int, int]], order: int = 2) -> List[List[Op]]:
    """Layers of one step of Trotter order 2 or 4 (module docstring)."""
    S = step_layers(n, bonds)
    if order == 2:
        return S
    if order != 4:
        raise ValueError("Trotter order must be 2 or 4")
    out = []
    for w in (W1, W0, W1):
        for layer in S:
            out.append([(kind, p, qa, qb, k, frac * w if kind == "gate" else frac)
                        for (kind, p, qa, qb, k, frac) in layer])
    return out
