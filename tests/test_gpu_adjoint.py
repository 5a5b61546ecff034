"""The adjoint (mpdo_grad_forward / mpdo_grad_backward) through the C ABI.

Checks, from the most to the least exact:
* closed forms (N = 3, the third qubit idle, so the MPO holds the exact
  two-qubit solution with no truncation): d<z_0>/dJ and d conn/dJ of the XY
  transfer, d<z_0>/dOmega and d<z_0>/dDelta of detuned Rabi, d<z_0>/dg0 of decay;
* central finite differences (h = 1e-6) of the GPU forward with the ranks held
  fixed, for every parameter kind, on a chain, a swap-routed ring and a batch;
* central finite differences of the CPU oracle's own MPO evolution (independent
  code) at the GPU's ranks;
* the dense oracle's exact Trotter gradient on an N = 8 ring: a truncated MPO
  with frozen ranks has a gradient that differs from the exact one where the
  tangent of the exact state points into discarded directions, and kept
  singular values near the cutoff (1e-10 of the largest here) amplify the
  rounding of the SVD; a CPU restatement of the same backward in numpy
  differs from the dense gradient by 2.3e-3 of its largest entry on this
  model, so the bound is 1e-2 while the loss itself agrees to 1e-9.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, tebd

pytestmark = pytest.mark.gpu

NAMES = ["h_x", "h_y", "h_z", "g0", "g1", "g2"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import build as B
    B.build()


def solver_for(wl, chi_cap=None, **kw):
    from paper_2203_05871_gb300 import Solver
    s = Solver(wl.n, batch=wl.batch, chi_cap=chi_cap or int(max(wl.chi_max)), **kw)
    s.build_gates(wl)
    return s


def copy_wl(wl):
    return W.Workload(**{f: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v)
                         for f, v in wl.__dict__.items()})


def shifted(wl, b, k, h):
    w = copy_wl(wl)
    n, nb = w.n, len(w.bonds)
    if k < 6 * n:
        getattr(w, NAMES[k // n])[b][k % n] += h
    elif k < 6 * n + nb:
        w.J[b][k - 6 * n] += h
    else:
        w.Jz[b][k - 6 * n - nb] += h
    return w


def gpu_loss(s, wl, steps, zb, wb, ranks):
    """L_b for every instance after `steps` steps at the given ranks."""
    s.build_gates(wl)
    s.force_ranks(ranks)
    s.step(steps)
    s.force_ranks(None)
    n = wl.n
    z = s.measure_1q(range(n), "Z")
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    conn = s.measure_2q(pairs, "ZZ", connected=True)
    out = np.einsum("bi,bi->b", zb, z)
    for k, (i, j) in enumerate(pairs):
        out = out + wb[:, i, j] * conn[:, k]
    return out


def grad_and_ranks(s, wl, steps, zb, wb):
    s.build_gates(wl)
    s.grad_forward(steps)
    ranks = s.rank_log(steps)
    g, L = s.grad_backward(zb, wb)
    return g, L, ranks


def weights(n, batch, seed):
    rng = np.random.default_rng(seed)
    zb = rng.normal(size=(batch, n))
    wb = np.triu(rng.normal(size=(batch, n, n)), 1)
    return zb, wb


def param_index(wl, name, q):
    n, nb = wl.n, len(wl.bonds)
    if name in NAMES:
        return NAMES.index(name) * n + q
    return 6 * n + (0 if name == "J" else nb) + q


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def three_qubits(init, **kw):
    wl = W.uniform_model("three", 3, W.chain_bonds(3), omega=kw.get("omega", [0.0, 0.0, 0.0]),
                         Omega=kw.get("Omega", 0.0), J=0.0, g0=0.0, g2=0.0, chi_max=16, cutoff=1e-12,
                         dt=kw.get("dt", 0.05), init=list(init))
    wl.J[0][0] = kw.get("J", 0.0)
    if "g0" in kw:
        wl.g0[0][0] = kw["g0"]
    return wl


def dcs(f, x):
    """Derivative of an analytic closed form by the complex step (exact to rounding)."""
    return float(np.imag(f(x + 1e-30j)) / 1e-30)


def test_closed_form_xy_transfer():
    J0, steps, dt = 0.37, 10, 0.05
    t = steps * dt
    wl = three_qubits(["-z", "+z", "+z"], J=J0, dt=dt)
    s = solver_for(wl)
    z0 = lambda J: -np.cos(2 * J * t)
    conn = lambda J: -np.sin(2 * J * t) ** 2
    g, L, _ = grad_and_ranks(s, wl, steps, np.array([[1.0, 0.0, 0.0]]), np.zeros((1, 3, 3)))
    assert abs(L[0] - z0(J0)) < 1e-12
    assert abs(g[0, param_index(wl, "J", 0)] - dcs(z0, J0)) < 1e-10
    wb = np.zeros((1, 3, 3))
    wb[0, 0, 1] = 1.0
    g, L, _ = grad_and_ranks(s, wl, steps, np.zeros((1, 3)), wb)
    assert abs(L[0] - conn(J0)) < 1e-12
    assert abs(g[0, param_index(wl, "J", 0)] - dcs(conn, J0)) < 1e-10


def test_closed_form_detuned_rabi_and_decay():
    Om0, De0, steps, dt = 0.8, 0.45, 20, 0.03
    t = steps * dt

    def z(O, D):
        W2 = O * O + D * D
        return 1 - 2 * (O * O / W2) * np.sin(np.sqrt(W2) * t / 2) ** 2

    wl = three_qubits(["+z", "+z", "+z"], Omega=Om0, omega=[De0, 0.0, 0.0], dt=dt)
    s = solver_for(wl)
    g, L, _ = grad_and_ranks(s, wl, steps, np.array([[1.0, 0.0, 0.0]]), np.zeros((1, 3, 3)))
    assert abs(L[0] - z(Om0, De0)) < 1e-12
    assert abs(g[0, param_index(wl, "h_x", 0)] - dcs(lambda O: z(O, De0), Om0)) < 1e-10
    assert abs(g[0, param_index(wl, "h_z", 0)] - dcs(lambda D: z(Om0, D), De0)) < 1e-10
    g00 = 0.3
    wl = three_qubits(["-z", "+z", "+z"], g0=g00, dt=0.04)
    s = solver_for(wl)
    zd = lambda G: 1 - 2 * np.exp(-G * 0.8)
    g, L, _ = grad_and_ranks(s, wl, 20, np.array([[1.0, 0.0, 0.0]]), np.zeros((1, 3, 3)))
    assert abs(L[0] - zd(g00)) < 1e-12
    assert abs(g[0, param_index(wl, "g0", 0)] - dcs(zd, g00)) < 1e-10


# ---------------------------------------------------------------------------
# finite differences
# ---------------------------------------------------------------------------
def check_fd(wl, steps, seed, params=None, tol=1e-6, **kw):
    s = solver_for(wl, **kw)
    zb, wb = weights(wl.n, wl.batch, seed)
    g, L, ranks = grad_and_ranks(s, wl, steps, zb, wb)
    assert np.all(np.isfinite(g))
    L0 = gpu_loss(s, wl, steps, zb, wb, ranks)
    assert np.abs(L0 - L).max() < 1e-12
    n, nb = wl.n, len(wl.bonds)
    params = range(6 * n + 2 * nb) if params is None else params
    h = 1e-6
    worst = 0.0
    for b in range(wl.batch):
        for k in params:
            fd = (gpu_loss(s, shifted(wl, b, k, h), steps, zb, wb, ranks)[b]
                  - gpu_loss(s, shifted(wl, b, k, -h), steps, zb, wb, ranks)[b]) / (2 * h)
            err = abs(g[b, k] - fd) / max(1.0, abs(fd))
            worst = max(worst, err)
            assert err < tol, (b, k, g[b, k], fd)
    return worst


def test_fd_chain_every_parameter():
    wl = W.random_model(6, W.chain_bonds(6), 31, chi_max=8, cutoff=1e-10, dt=0.05)
    check_fd(wl, 4, 1)


def test_fd_ring_swap_routed():
    wl = W.random_model(6, W.ring_bonds(6), 32, chi_max=12, cutoff=1e-10, dt=0.05)
    n, nb = 6, 6
    check_fd(wl, 3, 2, params=[0, 7, 14, 21, 28, 35, 6 * n, 6 * n + 5, 6 * n + nb + 5])


def test_fd_batched_uneven_chi():
    wl = W.random_model(5, W.chain_bonds(5), 33, batch=3, chi_max=8, cutoff=1e-10, dt=0.05)
    wl.chi_max[:] = [4, 6, 8]
    check_fd(wl, 3, 3, params=[1, 8, 12, 17, 24, 30, 33])


def test_batched_gradient_equals_single_instance():
    wl = W.random_model(5, W.chain_bonds(5), 34, batch=2, chi_max=8, cutoff=1e-10, dt=0.05)
    zb, wb = weights(5, 2, 4)
    s = solver_for(wl)
    g, L, _ = grad_and_ranks(s, wl, 3, zb, wb)
    for b in range(2):
        w1 = wl.instance(b)
        s1 = solver_for(w1)
        g1, L1, _ = grad_and_ranks(s1, w1, 3, zb[b:b + 1], wb[b:b + 1])
        assert np.abs(g1[0] - g[b]).max() <= 1e-12 * max(1.0, np.abs(g1).max())
        assert abs(L1[0] - L[b]) < 1e-13


def test_oracle_mpo_finite_differences():
    """FD of the CPU oracle's MPO-TEBD (its own SVD) at the GPU's ranks."""
    wl = W.random_model(5, W.ring_bonds(5), 35, chi_max=8, cutoff=1e-10, dt=0.05)
    steps = 3
    s = solver_for(wl)
    zb, wb = weights(5, 1, 5)
    g, L, ranks = grad_and_ranks(s, wl, steps, zb, wb)
    log = [int(k) for k in ranks[0]]

    def oracle_loss(w):
        o = tebd.TEBD(w, 0)
        o.run(steps, forced_k=log)
        st = o.state
        z = np.array([st.expect_1q(i) for i in range(5)])
        out = float(zb[0] @ z)
        for i in range(5):
            for j in range(i + 1, 5):
                out += wb[0, i, j] * (st.expect_2q(i, j) - z[i] * z[j])
        return out

    assert abs(oracle_loss(wl) - L[0]) < 1e-10
    h = 1e-6
    for k in [0, 6, 12, 18, 24, 29, 30, 34, 35, 39]:
        fd = (oracle_loss(shifted(wl, 0, k, h)) - oracle_loss(shifted(wl, 0, k, -h))) / (2 * h)
        assert abs(g[0, k] - fd) < 1e-6 * max(1.0, abs(fd)), (k, g[0, k], fd)


def test_dense_oracle_gradient_ring8():
    n = 8
    rng = np.random.default_rng(n)
    bonds = W.ring_bonds(n)
    wl = W.uniform_model("sector", n, bonds, omega=rng.uniform(-1, 1, n), Omega=0.0, J=0.1, g0=0.02,
                         g2=0.01, chi_max=64, cutoff=1e-20, dt=0.05, init=["-z"] + ["+z"] * (n - 1))
    wl.J[0] = rng.uniform(0.2, 0.5, len(bonds))
    wl.g0[0] = rng.uniform(0.01, 0.03, n)
    wl.g2[0] = rng.uniform(0.005, 0.02, n)
    steps = 6
    zb, wb = weights(n, 1, 6)
    s = solver_for(wl)
    g, L, _ = grad_and_ranks(s, wl, steps, zb, wb)
    Ld, gd = adjoint.dense_trotter_grad(wl, 0, steps, zb[0], wb[0])
    assert abs(L[0] - Ld) < 1e-9
    assert np.abs(g[0] - gd).max() <= 1e-2 * np.abs(gd).max()


# ---------------------------------------------------------------------------
# mixed precision and errors
# ---------------------------------------------------------------------------
def test_mixed_precision_gradient_close_to_fp64():
    from paper_2203_05871_gb300 import MIXED_TF32
    wl = W.random_model(6, W.chain_bonds(6), 36, chi_max=8, cutoff=1e-10, dt=0.05)
    zb, wb = weights(6, 1, 7)
    g64, L64, r64 = grad_and_ranks(solver_for(wl), wl, 3, zb, wb)
    s = solver_for(wl, precision=MIXED_TF32)
    s.build_gates(wl)
    s.force_ranks(r64)
    s.grad_forward(3)
    g32, L32 = s.grad_backward(zb, wb)
    assert abs(L32[0] - L64[0]) < 1e-5
    assert np.abs(g32 - g64).max() <= 1e-4 * max(1.0, np.abs(g64).max())


def test_grad_state_errors():
    from paper_2203_05871_gb300 import MpdoError
    wl = W.random_model(4, W.chain_bonds(4), 37, chi_max=4, cutoff=1e-10)
    s = solver_for(wl)
    with pytest.raises(MpdoError) as e:
        s.grad_backward(np.zeros((1, 4)), None)
    assert e.value.code == -8
    s.grad_forward(2)
    s.step(1)
    with pytest.raises(MpdoError) as e:
        s.grad_backward(np.zeros((1, 4)), None)
    assert e.value.code == -8
    s.grad_forward(2)
    bad = np.zeros((1, 4))
    bad[0, 1] = np.nan
    with pytest.raises(MpdoError) as e:
        s.grad_backward(bad, None)
    assert e.value.code == -1
    g, L = s.grad_backward(np.ones((1, 4)), None)
    assert np.all(np.isfinite(g))


def test_torch_autograd_function_matches_finite_differences():
    """A nonlinear fitting loss through the torch.autograd.Function."""
    torch = pytest.importorskip("torch")
    from paper_2203_05871_gb300 import autograd as AG
    wl = W.random_model(5, W.chain_bonds(5), 38, chi_max=8, cutoff=1e-10, dt=0.05)
    steps = 3
    s = solver_for(wl)
    p = torch.tensor(AG.pack_params(wl), dtype=torch.float64, requires_grad=True)
    target = torch.linspace(-0.5, 0.5, 5, dtype=torch.float64)[None]

    def loss_of(z, C):
        return ((z - target) ** 2).sum() + 0.5 * (C ** 2).sum()

    z, C = AG.observables(p, s, wl, steps)
    loss = loss_of(z, C)
    loss.backward()
    ranks = s.rank_log(steps)

    def L(pp):
        w = AG.with_params(wl, pp)
        s.build_gates(w)
        s.force_ranks(ranks)
        s.step(steps)
        s.force_ranks(None)
        zz = torch.from_numpy(s.measure_1q(range(5), "Z"))
        pairs = [(i, j) for i in range(5) for j in range(i + 1, 5)]
        CC = torch.from_numpy(AG.connected_matrix(s.measure_2q(pairs, "ZZ", connected=True), 5))
        return float(loss_of(zz, CC))

    p0 = AG.pack_params(wl)
    assert abs(L(p0) - float(loss)) < 1e-12
    h = 1e-6
    for k in [0, 7, 11, 16, 22, 27, 30, 33, 36]:
        pp, pm = p0.copy(), p0.copy()
        pp[0, k] += h
        pm[0, k] -= h
        fd = (L(pp) - L(pm)) / (2 * h)
        assert abs(float(p.grad[0, k]) - fd) < 1e-6 * max(1.0, abs(fd)), (k, float(p.grad[0, k]), fd)
