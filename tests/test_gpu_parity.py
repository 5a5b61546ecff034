"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 path |delta| <= 1e-10 on every observable at equal chi_max and
cutoff (when both sides chose the same truncation ranks; otherwise the oracle
is replayed with the GPU's ranks), gates <= 1e-14."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dense, model, schedule, tebd

pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_MIXED = 1e-5     # mixed-precision path (FP32-preconditioned SVD) vs the FP64 oracle


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


def all_pairs(n):
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def oracle_run(wl, b, steps, forced=None):
    t = tebd.TEBD(wl, b)
    t.run(steps, forced_k=forced)
    return t


def compare_to_oracle(wl, steps, s, tol=TOL):
    """Run the GPU solver s for `steps` and compare z and connected zz of every
    instance with the oracle (frozen to the GPU's ranks if they differ)."""
    s.step(steps)
    gz = s.measure_1q(range(wl.n), "Z")
    pairs = all_pairs(wl.n)
    gzz = s.measure_2q(pairs, "ZZ", connected=True)
    log = s.rank_log(steps)
    worst = 0.0
    for b in range(wl.batch):
        o = oracle_run(wl, b, steps)
        if list(o.k_log) != [int(k) for k in log[b]]:
            o = oracle_run(wl, b, steps, forced=[int(k) for k in log[b]])
        dz = np.abs(o.z() - gz[b]).max()
        dzz = np.abs(o.zz_connected(pairs) - gzz[b]).max()
        worst = max(worst, dz, dzz)
        assert dz <= tol and dzz <= tol, (b, dz, dzz)
    return worst


# ---------------------------------------------------------------------------
def test_gates_match_oracle():
    wl = W.random_model(6, W.ring_bonds(6), 31, batch=2, chi_max=8)
    s = solver_for(wl)
    layers = schedule.step_layers(wl.n, wl.bonds)
    for b in range(2):
        ref = [G for gl in tebd.build_gates(wl, b, layers, wl.dt) for G in gl]
        got = s.gates(b)
        assert np.abs(np.array(ref) - got).max() <= 1e-14


@pytest.mark.parametrize("bonds_fn", [W.chain_bonds, W.ring_bonds, lambda n: W.grid_snake_bonds(3, 2)])
def test_untruncated_equals_dense_trotter(bonds_fn):
    n = 6
    wl = W.random_model(n, bonds_fn(n), 41, chi_max=64, cutoff=0.0, dt=0.07)
    s = solver_for(wl)
    s.step(3)
    d = dense.DenseTrotter(wl).run(3)
    gz = s.measure_1q(range(n), "Z")[0]
    assert np.abs(gz - d.z()).max() <= 1e-12
    pairs = all_pairs(n)
    gzz = s.measure_2q(pairs, "ZZ", connected=False)[0]
    assert np.abs(gzz - np.array([d.zz(i, j) for (i, j) in pairs])).max() <= 1e-12
    st = s.status()
    assert st["status"][0] == 0
    assert abs(st["trace_before"][0] - 1.0) < 1e-12


def test_chain8_chi32_forty_steps():
    wl = W.chain8_fp64()
    s = solver_for(wl)
    worst = compare_to_oracle(wl, wl.steps, s)
    assert worst <= TOL


@pytest.mark.parametrize("bonds,n", [(W.ring_bonds(8), 8), (W.grid_snake_bonds(3, 3), 9)])
def test_swap_routed_graphs(bonds, n):
    wl = W.random_model(n, bonds, 53, chi_max=16, cutoff=1e-10, dt=0.05, with_all_terms=False)
    s = solver_for(wl)
    compare_to_oracle(wl, 4, s)


def test_batched_uneven_chi():
    wl = W.random_model(8, W.chain_bonds(8), 61, batch=4, chi_max=32, cutoff=1e-11)
    wl.chi_max[:] = [4, 8, 16, 32]
    s = solver_for(wl, chi_cap=32)
    compare_to_oracle(wl, 5, s)


def test_x_y_components_and_mixed_pairs():
    wl = W.random_model(7, W.chain_bonds(7), 71, chi_max=64, cutoff=0.0)
    s = solver_for(wl)
    s.step(2)
    o = oracle_run(wl, 0, 2, forced=[int(k) for k in s.rank_log(2)[0]])
    for comp in "XYZ":
        g = s.measure_1q(range(7), comp)[0]
        ref = [o.state.expect_1q(i, comp) for i in range(7)]
        assert np.abs(g - ref).max() <= TOL
    pairs = [(0, 3), (5, 1), (2, 6), (4, 3)]
    g = s.measure_2q(pairs, "XY", connected=True)[0]
    for (i, j), v in zip(pairs, g):
        ref = o.state.expect_2q(i, j, ("X", "Y")) - o.state.expect_1q(i, "X") * o.state.expect_1q(j, "Y")
        assert abs(v - ref) <= TOL


def test_initial_pauli_states():
    wl = W.random_model(5, W.chain_bonds(5), 81, chi_max=16, cutoff=0.0,
                        init=["+x", "-y", "+z", "-z", "-x"])
    s = solver_for(wl)
    g = {c: s.measure_1q(range(5), c)[0] for c in "XYZ"}
    assert np.allclose(g["X"], [1, 0, 0, 0, -1]) and np.allclose(g["Y"], [0, -1, 0, 0, 0])
    assert np.allclose(g["Z"], [0, 0, 1, -1, 0])
    compare_to_oracle(wl, 2, s)


# ---------------------------------------------------------------------------
# full-size properties
# ---------------------------------------------------------------------------
def test_decoupled_grid40_chi512():
    """J = 0 on the 4x10 snake (swap routing, chi_cap 512): chi stays 1 and every
    qubit follows its own single-qubit evolution."""
    wl = W.grid4x10_snake()
    wl.J[:] = 0.0
    s = solver_for(wl, chi_cap=512)
    steps = 4
    s.step(steps)
    st = s.status()
    assert st["chi"].max() == 1 and st["status"][0] == 0
    z = s.measure_1q(range(wl.n), "Z")[0]
    for q in range(wl.n):
        Lp = model.site_generator(wl.h_x[0][q], 0.0, wl.h_z[0][q], wl.g0[0][q], 0.0, wl.g2[0][q])
        c = sla.expm(Lp * steps * wl.dt) @ np.array([1.0, 0, 0, 1.0])
        assert abs(z[q] - c[3]) < 1e-12


def test_observables_snake40_chi512_sampled():
    """Measurement at full size: the 4x10 snake (N = 40) holding a seeded random
    MPO at chi 512 (bonds saturated from position 4 inward).  Every <Z_i> and
    all 780 pairs (both orders, connected) are measured through the stacked
    all-pairs path; the <Z_i> and a sample of pairs are checked against the
    oracle's MPO traces.  The values are ratios of traces of a non-physical
    MPO, so the bound is relative to their size."""
    wl = W.grid4x10_snake()
    n = wl.n
    dims, tens = W.random_mpo_state(n, 512, seed=2203058712 + 3, decay=0.02)
    s = solver_for(wl, chi_cap=512, max_slots=1)
    s.set_state(0, dims, tens)
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    z = s.measure_1q(range(n), "Z")[0]
    rz = np.array([st.expect_1q(i) for i in range(n)])
    assert np.all(np.abs(z - rz) <= 1e-10 * np.maximum(1.0, np.abs(rz)))
    pairs = [(i, j) for i in range(n) for j in range(n) if i != j]
    g = s.measure_2q(pairs, "ZZ", connected=True)[0]
    rng = np.random.default_rng(5)
    sample = sorted(set(rng.choice(len(pairs), 120, replace=False).tolist()) |
                    {pairs.index(p) for p in [(0, 39), (39, 0), (0, 1), (38, 39), (19, 20), (20, 19)]})
    for k in sample:
        i, j = pairs[k]
        zz = st.expect_2q(min(i, j), max(i, j))
        ref = zz - rz[i] * rz[j]
        assert abs(g[k] - ref) <= 1e-10 * max(1.0, abs(zz) + abs(rz[i] * rz[j])), (i, j, g[k], ref)
    # mixed components: <X_i Z_j> = <Z_j X_i> through both orders of the pair
    xz = s.measure_2q([(3, 17), (17, 3)], "XZ", connected=False)[0]
    ref = st.expect_2q(3, 17, ("X", "Z"))
    assert abs(xz[0] - ref) <= 1e-10 * max(1.0, abs(ref))
    ref2 = st.expect_2q(3, 17, ("Z", "X"))
    assert abs(xz[1] - ref2) <= 1e-10 * max(1.0, abs(ref2))


def test_single_excitation_ring24_and_grid():
    from tests.test_oracle_pins import single_excitation
    for n, bonds in [(24, W.ring_bonds(24)), (40, W.grid_snake_bonds(10, 4))]:
        rng = np.random.default_rng(n)
        wl = W.uniform_model("sector", n, bonds, omega=rng.uniform(-1, 1, n), Omega=0.0, J=0.1, g0=0.02,
                             g2=0.01, chi_max=64, cutoff=1e-13, dt=0.02, init=["-z"] + ["+z"] * (n - 1))
        wl.J[0] = rng.uniform(0.2, 0.5, len(bonds))
        T = 0.4
        s = solver_for(wl)
        s.step(int(round(T / wl.dt)))
        R = single_excitation(n, bonds, wl.h_z[0], wl.J[0], wl.g0[0], wl.g2[0], 0, T).real
        z = s.measure_1q(range(n), "Z")[0]
        # second-order Trotter error at dt = 0.02: well below 1e-4 here
        assert np.abs(z - (1 - 2 * np.diag(R))).max() < 1e-4


def test_chi256_one_step_sampled():
    """N=10 chain from a seeded random MPO at chi = 256 (1024 x 1024 SVDs):
    one step on the GPU against the oracle on the same input."""
    wl = W.chain20_precision()
    n = 10
    wl = W.uniform_model("chain10_chi256", n, W.chain_bonds(n), chi_max=256, cutoff=1e-10, dt=0.02)
    dims, tens = W.random_mpo_state(n, 256, seed=7)
    s = solver_for(wl, chi_cap=256)
    s.set_state(0, dims, tens)
    s.step(1)
    log = [int(k) for k in s.rank_log(1)[0]]
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    o = tebd.TEBD(wl, 0, state=st)
    o.run(1, forced_k=log)
    gz = s.measure_1q(range(n), "Z")[0]
    assert np.abs(gz - o.z()).max() <= TOL
    pairs = [(0, 9), (3, 6), (4, 5), (1, 8)]
    g = s.measure_2q(pairs, "ZZ", connected=True)[0]
    assert np.abs(g - o.zz_connected(pairs)).max() <= TOL
    # the largest relative discarded weight of the step (a sum over the
    # discarded rows, whose mutual orthogonality the SVD does not need)
    md = s.status()["max_discarded"][0]
    assert o.max_discarded > 0.0 and abs(md - o.max_discarded) <= 1e-9 * o.max_discarded


# ---------------------------------------------------------------------------
# mixed-precision path: FP32 preconditioning Jacobi + FP64 finishing sweeps
# ---------------------------------------------------------------------------
def _mixed(kind="tf32"):
    from paper_2203_05871_gb300 import MIXED_BF16X3, MIXED_TF32
    return MIXED_TF32 if kind == "tf32" else MIXED_BF16X3


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_mixed_chain8_forty_steps(kind):
    wl = W.chain8_fp64()
    s = solver_for(wl, precision=_mixed(kind))
    worst = compare_to_oracle(wl, wl.steps, s, tol=TOL_MIXED)
    print(f"mixed {kind} chain8 x 40 steps: worst |d| = {worst:.2e}")
    assert worst <= TOL_MIXED


# qr "blocked": the opt-in blocked Householder QR of the preconditioner
# (panels of 16 columns, trailing updates as tensor-core slice products)
@pytest.mark.parametrize("qr", ["column", "blocked"])
@pytest.mark.parametrize("kind", ["tf32", "bf16"])
@pytest.mark.parametrize("bonds,n", [(W.ring_bonds(8), 8), (W.grid_snake_bonds(3, 3), 9)])
def test_mixed_swap_routed(bonds, n, kind, qr):
    wl = W.random_model(n, bonds, 57, chi_max=32, cutoff=1e-11, dt=0.05)
    s = solver_for(wl, precision=_mixed(kind), qr_blocked=(qr == "blocked"))
    compare_to_oracle(wl, 3, s, tol=TOL_MIXED)


def test_mixed_batched_uneven_chi():
    wl = W.random_model(8, W.chain_bonds(8), 63, batch=3, chi_max=32, cutoff=1e-11)
    wl.chi_max[:] = [8, 16, 32]
    s = solver_for(wl, chi_cap=32, precision=_mixed())
    compare_to_oracle(wl, 4, s, tol=TOL_MIXED)


# decay 0.045: a graded spectrum like the physical workloads'.  decay 0: a flat
# random spectrum cut from 1024 values to 256, where the gap at the cut is tiny
# and the kept subspace turns by (perturbation / gap): the contractions and the
# preconditioner products must be FP64-class (the tensor-core slice products
# are) for the mixed tolerance to hold there.
@pytest.mark.parametrize("qr", ["column", "blocked"])
@pytest.mark.parametrize("kind", ["tf32", "bf16"])
@pytest.mark.parametrize("decay,tol", [(0.0, TOL_MIXED), (0.045, TOL_MIXED)])
def test_mixed_chi256_one_step_sampled(decay, tol, kind, qr):
    n = 10
    wl = W.uniform_model("chain10_chi256", n, W.chain_bonds(n), chi_max=256, cutoff=1e-10, dt=0.02)
    dims, tens = W.random_mpo_state(n, 256, seed=11, decay=decay)
    s = solver_for(wl, chi_cap=256, precision=_mixed(kind), qr_blocked=(qr == "blocked"))
    s.set_state(0, dims, tens)
    s.step(1)
    log = [int(k) for k in s.rank_log(1)[0]]
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    o = tebd.TEBD(wl, 0, state=st)
    o.run(1, forced_k=log)
    # a random MPO is not a physical density matrix: its "expectation values"
    # are ratios of small traces and can exceed 1, so the bound is relative
    gz, rz = s.measure_1q(range(n), "Z")[0], o.z()
    pairs = [(0, 9), (3, 6), (4, 5), (1, 8)]
    # connected values are differences of terms that can be large here: bound by their size
    g, rg = s.measure_2q(pairs, "ZZ", connected=True)[0], o.zz_connected(pairs)
    scale = np.array([abs(o.state.expect_2q(i, j)) + abs(rz[i] * rz[j]) for (i, j) in pairs])
    ez = np.abs(gz - rz) / np.maximum(1.0, np.abs(rz))
    ezz = np.abs(g - rg) / np.maximum(1.0, scale)
    print(f"mixed {kind} {qr} QR chi256 decay {decay}: max rel |dZ| = {ez.max():.2e}, |dZZc| = {ezz.max():.2e}")
    assert np.all(ez <= tol) and np.all(ezz <= tol)
    md = s.status()["max_discarded"][0]
    assert o.max_discarded > 0.0 and abs(md - o.max_discarded) <= tol * o.max_discarded


def test_mixed_long_rows_chi300():
    """Rows longer than 1024: on an N=11 chain with a 300-wide bond 6 between
    16-wide bonds, the first layer's op on sites (4, 5) has 64 rows of
    4 * 300 = 1200 and takes the FP32 pass's shared-memory path; the other ops
    take its register path.  One step against the oracle at the GPU's ranks."""
    n = 11
    dims = [1, 4, 16, 16, 16, 16, 300, 16, 16, 16, 4, 1]
    tens = W.random_mpo_tensors(dims, seed=13, decay=0.02)
    wl = W.uniform_model("chain11_chi300", n, W.chain_bonds(n), chi_max=300, cutoff=1e-10, dt=0.02)
    s = solver_for(wl, chi_cap=300, precision=_mixed())
    s.set_state(0, dims, tens)
    s.step(1)
    assert s.status()["status"][0] == 0
    log = [int(k) for k in s.rank_log(1)[0]]
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    o = tebd.TEBD(wl, 0, state=st)
    o.run(1, forced_k=log)
    gz, rz = s.measure_1q(range(n), "Z")[0], o.z()
    assert np.all(np.abs(gz - rz) <= TOL_MIXED * np.maximum(1.0, np.abs(rz)))
    pairs = [(0, 10), (3, 6), (4, 5), (5, 6)]
    g, rg = s.measure_2q(pairs, "ZZ", connected=True)[0], o.zz_connected(pairs)
    scale = np.array([abs(o.state.expect_2q(i, j)) + abs(rz[i] * rz[j]) for (i, j) in pairs])
    assert np.all(np.abs(g - rg) <= TOL_MIXED * np.maximum(1.0, scale))


def test_mixed_vs_fp64_per_observable_error():
    """Precision comparison (N=20 chain, seeded couplings): the mixed path
    (3xTF32 tensor-core contractions, FP32-preconditioned FP64 SVD) against the
    FP64 path at equal chi_max and cutoff, every <Z_i> and connected <Z_i Z_j>."""
    from paper_2203_05871_gb300 import FP64
    wl = W.chain20_precision(chi_max=48)
    wl = wl.with_(dt=0.02, cutoff=np.array([1e-10]))
    steps = 25
    pairs = all_pairs(wl.n)
    res = {}
    for prec in (FP64, _mixed()):
        s = solver_for(wl, precision=prec)
        s.step(steps)
        res[prec] = (s.measure_1q(range(wl.n), "Z")[0], s.measure_2q(pairs, "ZZ", connected=True)[0],
                     s.rank_log(steps)[0])
    (z64, zz64, k64), (zm, zzm, km) = res[FP64], res[_mixed()]
    dz, dzz = np.abs(z64 - zm).max(), np.abs(zz64 - zzm).max()
    print(f"mixed vs fp64: max|dZ| = {dz:.2e}, max|dZZc| = {dzz:.2e}, ranks equal: {np.array_equal(k64, km)}")
    assert dz <= TOL_MIXED and dzz <= TOL_MIXED


def test_errors_are_codes_not_crashes():
    from paper_2203_05871_gb300 import MpdoError, Solver
    s = Solver(5, batch=1, chi_cap=8)
    with pytest.raises(MpdoError):
        s.step(1)                      # before build_gates
    wl = W.random_model(5, W.chain_bonds(5), 3, chi_max=16)
    with pytest.raises(MpdoError):
        s.build_gates(wl)              # chi_max > chi_cap
    wl = W.random_model(5, W.chain_bonds(5), 3, chi_max=8)
    wl.g0[0, 2] = -1.0
    with pytest.raises(MpdoError):
        s.build_gates(wl)              # negative rate
    wl.g0[0, 2] = 0.1
    s.build_gates(wl)
    with pytest.raises(MpdoError):
        s.measure_2q([(1, 1)])
    s.step(1)


def test_profile_counters():
    """Kernel timers and sweep counters (mpdo_profile_*): every kernel of the
    mixed step is timed, the SVDs' mean and critical-path sweeps are
    consistent, and a reset zeroes them."""
    wl = W.chain8_fp64()
    s = solver_for(wl, precision=_mixed())
    s.profile(True)
    s.step(3)
    p = s.profile_read(reset=True)
    for k in ["merge_gate", "qr", "jacobi_fp32", "precond_gemm", "jacobi_svd", "truncate", "reconstruct"]:
        assert p[k]["launches"] > 0 and p[k]["ms"] > 0.0, k
    j = p["jacobi_svd"]
    assert j["svds"] == 3 * s.op_counts()[0]
    assert j["chunks"] > 0
    # per chunk the slowest op needs at least one sweep and at most all the chunk's sweeps
    assert j["chunks"] <= j["critical_sweeps"] <= j["sweeps"]
    assert j["chunks"] <= j["critical_sweeps_fp32"] <= j["sweeps_fp32"]
    q = s.profile_read()
    assert q["jacobi_svd"]["svds"] == 0 and q["jacobi_svd"]["chunks"] == 0 and q["qr"]["launches"] == 0


# ---------------------------------------------------------------------------
# the step captured as a CUDA graph
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_step_equals_plain_step(precision):
    """Device-planned, graph-replayed steps reproduce the host-planned steps
    exactly (same ranks, same tensors): chain8 for 40 steps, and a batch of
    three instances with uneven chi_max on a swap-routed ring."""
    from paper_2203_05871_gb300 import FP64, MIXED_TF32
    prec = FP64 if precision == "fp64" else MIXED_TF32
    cases = [(W.chain8_fp64(), 40, None),
             (W.random_model(6, W.ring_bonds(6), 71, batch=3, chi_max=16, cutoff=1e-11), 5, [4, 8, 16])]
    for wl, steps, chis in cases:
        if chis:
            wl.chi_max[:] = chis
        a = solver_for(wl, precision=prec)
        b = solver_for(wl, precision=prec)
        a.step(steps)
        b.step(steps, graph=True)
        assert np.array_equal(a.rank_log(steps), b.rank_log(steps))
        for inst in range(wl.batch):
            da, ta = a.get_state(inst)
            db, tb = b.get_state(inst)
            assert da == db
            for x, y in zip(ta, tb):
                assert np.array_equal(x, y)
        # a second replay continues from the replayed state
        a.step(2)
        b.step(2, graph=True)
        assert np.abs(a.measure_1q(range(wl.n), "Z") - b.measure_1q(range(wl.n), "Z")).max() == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_blocks_keep_parity(precision):
    """The autotuner picks a power-of-two block per (chi_l, chi_r) class; steps
    with the tuned table still match the oracle, and the graph step still
    equals the host-planned step."""
    from paper_2203_05871_gb300 import FP64, MIXED_TF32
    from paper_2203_05871_gb300.mpdo import saturated_classes
    prec = FP64 if precision == "fp64" else MIXED_TF32
    wl = W.chain8_fp64()
    s = solver_for(wl, precision=prec)
    cls = saturated_classes(wl.n, int(wl.chi_max[0]))
    ch = s.autotune(cls)
    for (b64, b32) in ch:
        assert b64 >= 1 and b64 & (b64 - 1) == 0
        assert (b32 == 0) if precision == "fp64" else (b32 >= 1 and b32 & (b32 - 1) == 0)
    s.build_gates(wl)
    compare_to_oracle(wl, 12, s, tol=TOL if precision == "fp64" else TOL_MIXED)
    g = solver_for(wl, precision=prec)
    g.autotune(cls)
    g.build_gates(wl)
    s.build_gates(wl)
    s.step(6)
    g.step(6, graph=True)
    for x, y in zip(s.get_state(0)[1], g.get_state(0)[1]):
        assert np.array_equal(x, y)


def test_batched_instances_equal_single_instance_runs():
    """A batch of 8 independent N=16 chains (the batched workload's model,
    chi_max drawn per instance) against the same instances run one by one,
    and one instance against the oracle."""
    wl = W.batch64_chain16(batch=8)
    wl.chi_max[:] = [8, 16, 32, 64, 8, 16, 32, 64]
    steps = 6
    s = solver_for(wl, chi_cap=64)
    s.step(steps)
    pairs = [(0, 15), (3, 9), (7, 8)]
    z = s.measure_1q(range(wl.n), "Z")
    zz = s.measure_2q(pairs, "ZZ", connected=True)
    for b in range(wl.batch):
        w1 = wl.instance(b)
        s1 = solver_for(w1, chi_cap=64)
        s1.step(steps)
        assert np.abs(s1.measure_1q(range(wl.n), "Z")[0] - z[b]).max() <= 1e-12
        assert np.abs(s1.measure_2q(pairs, "ZZ", connected=True)[0] - zz[b]).max() <= 1e-12
    o = oracle_run(wl, 3, steps, forced=[int(k) for k in s.rank_log(steps)[3]])
    assert np.abs(o.z() - z[3]).max() <= TOL


# ---------------------------------------------------------------------------
# f32 site storage (the "complex64 storage" variant of the real Pauli basis)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_f32_storage_against_oracle(precision):
    """Sites stored as float: observables within the mixed tolerance of the
    FP64 oracle (each op rounds the new sites to float, ~6e-8 relative), and
    measurably different from FP64 storage (the float rounding is real)."""
    from paper_2203_05871_gb300 import FP64, MIXED_TF32, STORE_F32
    prec = FP64 if precision == "fp64" else MIXED_TF32
    wl = W.chain8_fp64()
    s32 = solver_for(wl, precision=prec, storage=STORE_F32)
    worst = compare_to_oracle(wl, wl.steps, s32, tol=TOL_MIXED)
    assert worst <= TOL_MIXED
    s64 = solver_for(wl, precision=prec)
    s64.step(wl.steps)
    d = np.abs(s64.measure_1q(range(wl.n), "Z") - s32.measure_1q(range(wl.n), "Z")).max()
    assert 0.0 < d < TOL_MIXED


def test_f32_storage_state_roundtrip_and_graph():
    from paper_2203_05871_gb300 import STORE_F32
    wl = W.random_model(6, W.ring_bonds(6), 72, chi_max=16, cutoff=1e-11)
    dims, tens = W.random_mpo_state(6, 16, seed=5)
    s = solver_for(wl, storage=STORE_F32)
    s.set_state(0, dims, tens)
    d2, t2 = s.get_state(0)
    assert d2 == list(dims)
    for x, y in zip(tens, t2):
        assert np.array_equal(np.asarray(x, np.float32).astype(np.float64), y)
    g = solver_for(wl, storage=STORE_F32)
    s.set_state(0, dims, tens)
    g.set_state(0, dims, tens)
    s.step(3)
    g.step(3, graph=True)
    for x, y in zip(s.get_state(0)[1], g.get_state(0)[1]):
        assert np.array_equal(x, y)
