"""The precision comparison at its stated size: N=20 open chain with seeded
couplings (J_b~U[0.05,0.15], Omega~U[0.3,0.7], g0_i~U[0.005,0.02],
g2_i~U[0.01,0.03], h_z alternating), chi_max = 128, cutoff 1e-10, dt = 0.02,
500 steps from all |0>.  The FP64 path, the TF32-slice and BF16-slice mixed
paths, and f32 site storage, each compared per observable (<Z_i>, connected
<Z_i Z_j>) with the FP64 path; the FP64 path compared with the oracle at the
GPU's ranks over the first 60 steps (a window the CPU oracle finishes in
seconds)."""
import numpy as np
import pytest

import workloads as W
from oracle import tebd

pytestmark = pytest.mark.gpu

STEPS = 500


@pytest.fixture(scope="module")
def runs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05871_gb300 import FP64, MIXED_BF16X3, MIXED_TF32, STORE_F32, Solver
    from paper_2203_05871_gb300 import build as B
    B.build()
    wl = W.chain20_precision(chi_max=128)
    pairs = [(i, j) for i in range(wl.n) for j in range(i + 1, wl.n)]
    out = {}
    for name, prec, store in [("fp64", FP64, 0), ("tf32", MIXED_TF32, 0), ("bf16", MIXED_BF16X3, 0),
                              ("fp64_f32store", FP64, STORE_F32), ("tf32_f32store", MIXED_TF32, STORE_F32)]:
        s = Solver(wl.n, batch=1, chi_cap=128, precision=prec, storage=store)
        s.build_gates(wl)
        s.step(STEPS)
        out[name] = {"z": s.measure_1q(range(wl.n), "Z")[0], "zz": s.measure_2q(pairs, "ZZ", connected=True)[0],
                     "chi": s.status()["chi"][0], "ranks": s.rank_log(STEPS)[0]}
        s.close()
    return wl, pairs, out


@pytest.mark.parametrize("name,tol", [("tf32", 1e-5), ("bf16", 1e-5), ("fp64_f32store", 1e-4),
                                      ("tf32_f32store", 1e-4)])
def test_per_observable_error_vs_fp64(runs, name, tol):
    wl, pairs, out = runs
    ref, got = out["fp64"], out[name]
    dz = np.abs(got["z"] - ref["z"])
    dzz = np.abs(got["zz"] - ref["zz"])
    worst_pair = pairs[int(np.argmax(dzz))]
    print(f"config 2, {name} vs fp64 after {STEPS} steps (t = {STEPS * wl.dt:g}): "
          f"max|dZ_i| = {dz.max():.2e} (qubit {int(np.argmax(dz))}), "
          f"max|dZZc_ij| = {dzz.max():.2e} (pair {worst_pair}), "
          f"ranks equal: {np.array_equal(got['ranks'], ref['ranks'])}, chi max {int(ref['chi'].max())}")
    print("  per qubit |dZ_i|:", " ".join(f"{x:.1e}" for x in dz))
    assert dz.max() <= tol and dzz.max() <= tol


def test_fp64_path_against_oracle_window():
    from paper_2203_05871_gb300 import Solver
    wl = W.chain20_precision(chi_max=128)
    steps = 60
    s = Solver(wl.n, batch=1, chi_cap=128)
    s.build_gates(wl)
    s.step(steps)
    log = [int(k) for k in s.rank_log(steps)[0]]
    o = tebd.TEBD(wl).run(steps, forced_k=log)
    pairs = [(i, j) for i in range(wl.n) for j in range(i + 1, wl.n)]
    dz = np.abs(s.measure_1q(range(wl.n), "Z")[0] - o.z()).max()
    dzz = np.abs(s.measure_2q(pairs, "ZZ", connected=True)[0] - o.zz_connected(pairs)).max()
    print(f"config 2 FP64 vs oracle, {steps} steps: |dZ| = {dz:.2e}, |dZZc| = {dzz:.2e}")
    assert dz <= 1e-10 and dzz <= 1e-10
