"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms of textbook problems, invariants, brute force and library
routines.  Each test names the oracle part that a plausible mistake would
break (dropped term, wrong sign, wrong index, transposed operand)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dense, model, schedule, svd, tebd


# ---------------------------------------------------------------------------
# single-qubit physics (Eq. (H0), Eqs. (D0)-(D2))
# ---------------------------------------------------------------------------
def bloch_steady_state(Delta, Omega, g0, g2):
    """Textbook Bloch-equation steady state of one qubit driven about x with
    detuning about z, T1 relaxation towards z=+1 (rate G1 = g0) and
    transverse decay G2 = g0/2 + 2 g2."""
    G1, G2 = g0, g0 / 2 + 2 * g2
    D = G1 * (G2 ** 2 + Delta ** 2) + Omega ** 2 * G2
    return np.array([Delta * Omega * G1 / D, -Omega * G1 * G2 / D, G1 * (G2 ** 2 + Delta ** 2) / D])


@pytest.mark.parametrize("Delta,Omega,g0,g2", [(0.0, 0.5, 0.01, 0.02), (1.0, 0.5, 0.01, 0.02),
                                               (-0.7, 1.3, 0.2, 0.05), (0.3, 0.2, 0.5, 0.0)])
def test_bloch_steady_state_dense_and_pauli(Delta, Omega, g0, g2):
    # dense 2x2 superoperator: null vector
    Ls = model.liouvillian_superop(1, [], [Omega], [0.0], [Delta], [], [], [g0], [0.0], [g2]).toarray()
    v = sla.null_space(Ls)[:, 0].reshape(2, 2)
    rho = v / np.trace(v)
    r = np.array([np.trace(rho @ P).real for P in (model.X, model.Y, model.Z)])
    np.testing.assert_allclose(r, bloch_steady_state(Delta, Omega, g0, g2), atol=1e-13)
    # Pauli-basis site generator used by the MPO oracle
    Lp = model.site_generator(Omega, 0.0, Delta, g0, 0.0, g2)
    c = sla.null_space(Lp)[:, 0]
    c = c / c[0]
    np.testing.assert_allclose(c[1:], bloch_steady_state(Delta, Omega, g0, g2), atol=1e-13)


def test_config1_bloch_values():
    # drive on qubit 0 of the N=8 chain at Delta=0 (values quoted to 8 digits)
    s = bloch_steady_state(0.0, 0.5, 0.01, 0.02)
    assert abs(s[1] - (-0.01996406)) < 5e-9 and abs(s[2] - 0.00179677) < 5e-9


def test_rabi_rotation_sense():
    """H = Omega/2 sigma^x from |0> (z=+1): <y> = -sin(Omega t), <z> = cos(Omega t)
    (right-handed rotation about x)."""
    Om = 0.9
    Lp = model.site_generator(Om, 0.0, 0.0, 0.0, 0.0, 0.0)
    for t in (0.3, 1.1, 2.5):
        c = sla.expm(Lp * t) @ np.array([1.0, 0, 0, 1.0])
        np.testing.assert_allclose(c[1:], [0.0, -np.sin(Om * t), np.cos(Om * t)], atol=1e-14)


def test_precession_and_decay_rates():
    """Free precession about z with h_z and the T1/T2 rates of D0, D1, D2."""
    hz, g0, g1, g2 = 0.7, 0.11, 0.05, 0.03
    Lp = model.site_generator(0.0, 0.0, hz, g0, g1, g2)
    t = 1.7
    c = sla.expm(Lp * t) @ np.array([1.0, 1.0, 0.0, 0.0])   # start along +x
    G2 = (g0 + g1) / 2 + 2 * g2
    np.testing.assert_allclose(c[1:3], np.exp(-G2 * t) * np.array([np.cos(hz * t), np.sin(hz * t)]),
                               atol=1e-14)
    c = sla.expm(Lp * t) @ np.array([1.0, 0.0, 0.0, -1.0])  # start at z=-1
    zinf = (g0 - g1) / (g0 + g1)
    np.testing.assert_allclose(c[3], zinf + (-1 - zinf) * np.exp(-(g0 + g1) * t), atol=1e-14)


# ---------------------------------------------------------------------------
# bond term (Eq. (K_def) read per unordered bond)
# ---------------------------------------------------------------------------
def test_xy_excitation_transfer():
    """Two qubits, |1>|0>, H = J(s+s- + h.c.): z0(t) = -cos(2Jt)."""
    J = 0.37
    wl = W.uniform_model("pair", 2, [(0, 1)], omega=[0, 0], Omega=0.0, J=J, g0=0.0, g2=0.0,
                         init=["-z", "+z"])
    ts = [0.4, 1.3, 2.9]
    rhos = dense.exact_evolve(wl, 0, ts)
    for t, rho in zip(ts, rhos):
        assert abs(dense.expect_z(rho, 0) + np.cos(2 * J * t)) < 1e-12
    # and through the Pauli-basis bond generator
    L = model.bond_generator(J, 0.0)
    r0 = tebd.MPOState(*tebd.product_state(2, ["-z", "+z"])).to_vector()
    for t in ts:
        r = sla.expm(L * t) @ r0
        assert abs(r[3 * 4 + 0] / r[0] + np.cos(2 * J * t)) < 1e-12


def test_zz_bond_phase():
    """Jz/2 ZZ rotates the x component of qubit 0 at rate 2*(Jz/2) when the
    other qubit sits in z=+1."""
    Jz = 0.45
    L = model.bond_generator(0.0, Jz)
    r0 = tebd.MPOState(*tebd.product_state(2, ["+x", "+z"])).to_vector()
    t = 0.8
    r = sla.expm(L * t) @ r0
    x0 = r[1 * 4 + 0] / r[0]
    assert abs(x0 - np.cos(Jz * t)) < 1e-13


# ---------------------------------------------------------------------------
# single-excitation sector (exact for XY + h_z + g0 + g2, Omega = g1 = Jz = 0)
# ---------------------------------------------------------------------------
def single_excitation(n, bonds, hz, J, g0, g2, a0, t):
    """R(t), the one-excitation block, from dR/dt = -i(Heff R - R Heff^+)
    - 2(g2_a + g2_b) R_ab (a != b), Heff = -diag(hz) + J_adj - i/2 diag(g0)."""
    Heff = -np.diag(hz).astype(complex)
    for k, (i, j) in enumerate(bonds):
        Heff[i, j] += J[k]
        Heff[j, i] += J[k]
    Heff -= 0.5j * np.diag(g0)
    Id = np.eye(n)
    # row-major vec: vec(A R B) = kron(A, B^T) vec(R)
    Lm = -1j * (np.kron(Heff, Id) - np.kron(Id, Heff.conj()))
    deph = np.array([[-2 * (g2[a] + g2[b]) if a != b else 0.0 for b in range(n)] for a in range(n)])
    Lm += np.diag(deph.reshape(-1))
    R0 = np.zeros((n, n), dtype=complex)
    R0[a0, a0] = 1.0
    return (sla.expm(Lm * t) @ R0.reshape(-1)).reshape(n, n)


def _sector_model(n, bonds, seed):
    rng = np.random.default_rng(seed)
    nb = len(bonds)
    wl = W.uniform_model("sector", n, bonds, omega=rng.uniform(-1, 1, n), Omega=0.0, J=0.1,
                         g0=0.0, g2=0.0, init=["+z"] * n)
    wl.J[0] = rng.uniform(0.2, 0.6, nb)
    wl.g0[0] = rng.uniform(0.0, 0.2, n)
    wl.g2[0] = rng.uniform(0.0, 0.1, n)
    return wl


def test_single_excitation_vs_dense_exact():
    n, bonds = 5, W.ring_bonds(5)
    wl = _sector_model(n, bonds, 3)
    wl.init = ["+z"] * n
    wl.init[2] = "-z"
    t = 1.9
    rho = dense.exact_evolve(wl, 0, [t])[0]
    R = single_excitation(n, bonds, wl.h_z[0], wl.J[0], wl.g0[0], wl.g2[0], 2, t).real
    for j in range(n):
        assert abs(dense.expect_z(rho, j) - (1 - 2 * R[j, j])) < 1e-12
    for i in range(n):
        for j in range(i + 1, n):
            zc = dense.expect_zz(rho, i, j) - dense.expect_z(rho, i) * dense.expect_z(rho, j)
            assert abs(zc - (-4 * R[i, i] * R[j, j])) < 1e-12


def test_single_excitation_pins_mpo_ring_with_swaps():
    """N=10 ring (swap-routed closing bond): the MPO oracle's Trotter error
    against the exact sector solution falls by ~4 when dt halves."""
    n, bonds = 10, W.ring_bonds(10)
    wl = _sector_model(n, bonds, 5)
    wl.init = ["+z"] * n
    wl.init[0] = "-z"
    T = 0.8
    R = single_excitation(n, bonds, wl.h_z[0], wl.J[0], wl.g0[0], wl.g2[0], 0, T).real
    zex = 1 - 2 * np.diag(R)
    errs = []
    for dt in (0.1, 0.05):
        w = wl.with_(dt=dt, chi_max=np.array([64]), cutoff=np.array([1e-14]))
        st = tebd.TEBD(w).run(int(round(T / dt)))
        errs.append(np.abs(st.z() - zex).max())
        assert max(st.state.dims()) <= 8       # excitation sector keeps chi small
    assert errs[0] < 5e-4
    assert 3.3 < errs[0] / errs[1] < 4.7


# ---------------------------------------------------------------------------
# invariants of the dense exact oracle
# ---------------------------------------------------------------------------
def test_dense_trace_hermiticity_and_rhs():
    wl = W.random_model(4, W.chain_bonds(4), 7)
    rho = dense.exact_evolve(wl, 0, [1.3])[0]
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.abs(rho - rho.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    # the sparse superoperator equals the operator-form right-hand side
    f = model.lindblad_rhs(4, wl.bonds, wl.h_x[0], wl.h_y[0], wl.h_z[0], wl.J[0], wl.Jz[0],
                           wl.g0[0], wl.g1[0], wl.g2[0])
    L = model.liouvillian_superop(4, wl.bonds, wl.h_x[0], wl.h_y[0], wl.h_z[0], wl.J[0], wl.Jz[0],
                                  wl.g0[0], wl.g1[0], wl.g2[0])
    rng = np.random.default_rng(1)
    A = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    np.testing.assert_allclose((L @ A.reshape(-1)).reshape(16, 16), f(A), atol=1e-13)


def test_edge_drive_x0_vanishes():
    """Resonant drive about x of qubit 0 (Delta=0, no dissipation): <X_0> = 0 at
    all times and <Y_0> turns negative (Sec. 3.2)."""
    n = 5
    wl = W.uniform_model("e1", n, W.chain_bonds(n), omega=np.zeros(n), Omega=2 * np.pi,
                         J=2 * np.pi, g0=0.0, g2=0.0)
    for rho in dense.exact_evolve(wl, 0, [0.05, 0.2, 0.7]):
        x0 = np.trace(model.embed(model.X, 0, n) @ rho).real
        y0 = np.trace(model.embed(model.Y, 0, n) @ rho).real
        assert abs(x0) < 1e-12 and y0 < 0


# ---------------------------------------------------------------------------
# Pauli-basis gates (trace preservation, reality, semigroup)
# ---------------------------------------------------------------------------
def test_gates_trace_preserving_and_semigroup():
    wl = W.random_model(4, W.ring_bonds(4), 11)
    layers = schedule.step_layers(4, wl.bonds)
    gates = tebd.build_gates(wl, 0, layers, 0.07)
    gates2 = tebd.build_gates(wl, 0, layers, 0.14)
    for layer, gl, gl2 in zip(layers, gates, gates2):
        for op, G, G2 in zip(layer, gl, gl2):
            if op[0] == "swap":
                continue
            e0 = np.zeros(16)
            e0[0] = 1
            np.testing.assert_allclose(G[0], e0, atol=1e-15)
            np.testing.assert_allclose(G @ G, G2, atol=1e-13)
    assert np.allclose(model.swap_matrix() @ model.swap_matrix(), np.eye(16))


def test_onsite_generator_matches_kron_of_dense():
    """Pauli-basis two-site generator vs the dense 2-qubit Liouvillian
    transformed into the Pauli basis (different construction routes)."""
    wl = W.random_model(2, [(0, 1)], 2)
    p = {k: getattr(wl, k) for k in ("h_x", "h_y", "h_z", "g0", "g1", "g2", "J", "Jz")}
    w = [1.0, 1.0]
    Lp = model.op_generator(p, 0, 0, 1, 0, w)
    Ld = model.liouvillian_superop(2, [(0, 1)], wl.h_x[0], wl.h_y[0], wl.h_z[0], wl.J[0], wl.Jz[0],
                                   wl.g0[0], wl.g1[0], wl.g2[0]).toarray()
    basis = model.pauli_basis(2)
    M = np.array([[np.trace(basis[a].conj().T @ (Ld @ basis[b].reshape(-1)).reshape(4, 4))
                   for b in range(16)] for a in range(16)])
    np.testing.assert_allclose(Lp, M.real, atol=1e-14)
    assert np.abs(M.imag).max() < 1e-14


# ---------------------------------------------------------------------------
# schedule
# ---------------------------------------------------------------------------
def test_schedule_counts():
    L = schedule.step_layers(8, W.chain_bonds(8))
    assert [len(x) for x in L] == [4, 3, 4]
    assert [o[5] for o in L[0]] == [0.5] * 4 and [o[5] for o in L[1]] == [1.0] * 3
    L = schedule.step_layers(24, W.ring_bonds(24))
    assert schedule.count_ops(L) == (47, 44)
    mid = [o for x in L for o in x if o[5] == 1.0]
    assert len(mid) == 1 and mid[0][1:4] == (0, 0, 23)
    L = schedule.step_layers(40, W.grid_snake_bonds(10, 4))
    g, s = schedule.count_ops(L)
    assert g == 131 and 420 <= s <= 440


def test_schedule_long_range_gate_targets():
    """Every physical gate acts on the two qubits of its bond."""
    bonds = W.grid_snake_bonds(4, 3)
    for (kind, p, qa, qb, k, f) in [o for x in schedule.step_layers(12, bonds) for o in x]:
        if kind == "gate":
            assert {qa, qb} == set(bonds[k])


def test_trotter_second_order():
    """Dense-Trotter vs exact: error ratio ~4 when dt halves (symmetric product)."""
    wl = W.random_model(5, W.ring_bonds(5), 4, dt=0.1)
    T = 0.8
    rho = dense.exact_evolve(wl, 0, [T])[0]
    zex = np.array([dense.expect_z(rho, i) for i in range(5)])
    e = []
    for dt in (0.1, 0.05, 0.025):
        d = dense.DenseTrotter(wl.with_(dt=dt)).run(int(round(T / dt)))
        e.append(np.abs(d.z() - zex).max())
    assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5


def test_trotter_fourth_order():
    """Suzuki's triple jump of the symmetric step: the error against the exact
    dense evolution falls by ~16 when dt halves, and is far below the
    second-order error at the same dt; the op list is three scaled copies."""
    wl = W.random_model(5, W.ring_bonds(5), 4, dt=0.1)
    T = 0.8
    rho = dense.exact_evolve(wl, 0, [T])[0]
    zex = np.array([dense.expect_z(rho, i) for i in range(5)])
    e = []
    for dt in (0.2, 0.1, 0.05):
        d = dense.DenseTrotter(wl.with_(dt=dt), order=4).run(int(round(T / dt)))
        e.append(np.abs(d.z() - zex).max())
    assert 13.0 < e[0] / e[1] < 19.0 and 13.0 < e[1] / e[2] < 19.0, e
    e2 = np.abs(dense.DenseTrotter(wl.with_(dt=0.1)).run(8).z() - zex).max()
    assert e[1] < 0.1 * e2
    L2 = schedule.step_layers(5, W.ring_bonds(5))
    L4 = schedule.step_layers_order(5, W.ring_bonds(5), 4)
    assert len(L4) == 3 * len(L2)
    fr = [o[5] for L in L4 for o in L if o[0] == "gate"]
    f2 = [o[5] for L in L2 for o in L if o[0] == "gate"]
    assert abs(sum(fr) - sum(f2)) < 1e-14      # total time per bond unchanged: w0 + 2 w1 = 1
    assert min(fr) < 0.0                       # the middle jump runs backwards


# ---------------------------------------------------------------------------
# SVD and truncation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(12, 12), (8, 20), (24, 8), (1, 4), (4, 1), (33, 17)])
def test_jacobi_svd_vs_lapack(m, n):
    rng = np.random.default_rng(m * 100 + n)
    # graded matrix (rows scaled over 10 decades), like diag(lambda) Theta'
    M = rng.standard_normal((m, n)) * np.logspace(0, -10, m)[:, None]
    s, Vt = svd.svd_right(M)
    s_ref = np.linalg.svd(M, compute_uv=False)
    np.testing.assert_allclose(s, s_ref, rtol=1e-12, atol=1e-15 * s_ref[0])
    r = min(m, n)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(r), atol=1e-12)
    # M V = U S with orthonormal U: ||M V_j|| = s_j and M = (M V) V^T when r = n
    MV = M @ Vt.T
    np.testing.assert_allclose(np.linalg.norm(MV, axis=0), s, rtol=1e-10, atol=1e-14)
    if r == n:
        np.testing.assert_allclose(MV @ Vt, M, atol=1e-13 * s_ref[0])


def test_jacobi_degenerate_and_zero():
    M = np.zeros((3, 5))
    s, Vt = svd.svd_right(M)
    assert np.all(s == 0)
    M = np.eye(4)[:, :4] * 2.0
    s, _ = svd.svd_right(M)
    np.testing.assert_allclose(s, [2, 2, 2, 2])


def test_truncation_rule_brute_force():
    s = np.array([1.0, 0.1, 0.01, 0.001])
    w = s ** 2
    for cutoff in (0.0, 1e-7, 1.5e-6, 1e-4, 2e-2, 1.0):
        for chi in (1, 2, 3, 4, 10):
            cands = [k for k in range(1, 5) if w[k:].sum() <= cutoff * w.sum()]
            assert svd.truncation_rank(s, chi, cutoff) == min(chi, min(cands))


# ---------------------------------------------------------------------------
# MPO oracle vs dense Trotter (untruncated) and special cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bonds_fn,n", [(W.chain_bonds, 6), (W.ring_bonds, 6),
                                        (lambda n: W.grid_snake_bonds(3, 2), 6)])
def test_mpo_vs_dense_trotter_untruncated(bonds_fn, n):
    wl = W.random_model(n, bonds_fn(n), 21, chi_max=4 ** (n // 2), cutoff=0.0, dt=0.07)
    d = dense.DenseTrotter(wl).run(3)
    t = tebd.TEBD(wl, force_trace=False).run(3)
    v = t.state.to_vector()
    np.testing.assert_allclose(v, d.vector(), atol=1e-12 * np.abs(d.vector()).max())


def test_mpo_trace_forcing_and_trace_invariant():
    wl = W.random_model(6, W.chain_bonds(6), 8, chi_max=64, cutoff=0.0)
    t = tebd.TEBD(wl).run(3)
    # gates are trace preserving: before forcing, tr rho stays 1 when nothing is discarded
    np.testing.assert_allclose(t.trace_log, 1.0, atol=1e-12)
    assert abs(t.state.trace() - 1.0) < 1e-13


def test_mpo_decoupled_chain_equals_single_qubit():
    """J = 0: every qubit evolves alone; chi stays 1 and <zz>_c = 0."""
    n = 12
    wl = W.uniform_model("dec", n, W.chain_bonds(n), omega=np.linspace(-1, 1, n), Omega=0.0,
                         J=0.0, g0=0.03, g2=0.02, chi_max=16, cutoff=1e-14, dt=0.1)
    wl.h_x[0] = np.linspace(0.2, 0.9, n)
    t = tebd.TEBD(wl).run(10)
    assert max(t.state.dims()) == 1
    for q in range(n):
        Lp = model.site_generator(wl.h_x[0][q], 0.0, wl.h_z[0][q], 0.03, 0.0, 0.02)
        c = sla.expm(Lp * 1.0) @ np.array([1.0, 0, 0, 1.0])
        assert abs(t.z()[q] - c[3]) < 1e-12
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    assert np.abs(t.zz_connected(pairs)).max() < 1e-13


def test_frozen_rank_replay_reproduces_run():
    wl = W.random_model(7, W.chain_bonds(7), 9, chi_max=6, cutoff=1e-8)
    t1 = tebd.TEBD(wl).run(3)
    t2 = tebd.TEBD(wl).run(3, forced_k=list(t1.k_log))
    np.testing.assert_allclose(t1.z(), t2.z(), atol=1e-14)
    assert t1.k_log == t2.k_log


def test_lapack_route_matches_jacobi_route():
    """The oracle's LAPACK SVD route (the CPU baseline of the paper's threaded
    LAPACK solver) keeps the same state as its plain Jacobi route."""
    wl = W.random_model(6, W.chain_bonds(6), 23, chi_max=8, cutoff=1e-12, dt=0.2)
    a = tebd.TEBD(wl)
    b = tebd.TEBD(wl)
    for _ in range(4):
        for layer, gl in zip(a.layers, a.gates):
            for op, G in zip(layer, gl):
                ka, _ = a.state.apply(op[1], G, 8, 1e-12)
                kb, _ = b.state.apply(op[1], G, 8, 1e-12, forced_k=ka, svd_impl="lapack")
        a.state.normalize_trace()
        b.state.normalize_trace()
    assert np.abs(a.z() - b.z()).max() < 1e-10
