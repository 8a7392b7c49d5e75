"""Host-side harness rules shared by the benchmark and the tests (CPU)."""
import numpy as np
import pytest

from oracle import dg, rk
from paper_2003_08831_gb300 import inputs
from paper_2003_08831_gb300.solver import stable_dt


@pytest.mark.parametrize("mu", [0.0, 1.0 / 1600.0, 0.05])
def test_stable_dt_matches_the_oracle_rule(mu):
    """The package's fixed-time-step rule (used by the benchmark on host arrays) and the
    oracle's agree: the same reading of the unstated CFL condition."""
    mesh = dg.Mesh(3, (4, 3, 5), (0.0, 0.0, 0.0), (2 * np.pi, 2.0, 3.0))
    x, y, z = mesh.coords()
    U = inputs.tgv_state(x, y, z, mach=0.3)
    phys = dg.Physics(1.4, mu=mu, Pr=0.72)
    ref = rk.stable_dt(mesh, U, phys, 0.5)
    got = stable_dt(mesh.flat(U), 3, list(mesh.h), 0.5, mu=mu, Pr=0.72)
    assert abs(got - ref) <= 1e-15 * ref


def test_roofline_model_bytes_flops_and_bound():
    """The benchmark's per-kernel roofline model (bench.kernel_work / kernel_rooflines) on a
    2^3-element p = 2 mesh, checked against the counts written out by hand: bytes of each
    kernel's inputs and outputs averaged over a BS3 step, the split of its flops by
    arithmetic, and the bound that sets the roofline time."""
    import bench
    K, p = 8, 2
    Np, P2 = 27, 9
    nodes = K * Np
    w = bench.kernel_work(p, K, precision=0)
    # k_prep, FP64 (tf = 8): stage 1 reads u (40) + pending d (40) and writes u (40) and the
    # parameter vector (6 x 8); stages 2, 3 read u and one earlier stage (40 + 40), write
    # the parameter vector and the entropy increments (48 + 40)
    prep_bytes = nodes * ((40 + 80 + 48) + 2 * (40 + 40 + 48 + 40)) / 3
    assert w["prep"][1] == pytest.approx(prep_bytes)
    prep_flops = nodes * (3 * 22 + 10 + (10 + 122) * 2) / 3
    assert w["prep"][0] == pytest.approx({"f64": prep_flops})
    # k_face: 3 K P2 face-node pairs, 17 flux-precision values each
    assert w["face"][1] == 3 * K * P2 * 17 * 8
    assert w["face"][0] == {"f64": 3 * K * P2 * 111}
    # k_relax: u and d (80 B per node); the cubic starting coefficient on the FP32 pipe
    assert w["relax"][1] == 80 * nodes
    assert w["relax"][0] == pytest.approx({"f64": nodes * (65 + 75), "f32": nodes * 20})
    # mixed modes: the flux in FP32, the estimate parts in FP64 (ES_MIXED) or float-float
    wm, wf = bench.kernel_work(p, K, precision=1), bench.kernel_work(p, K, precision=3)
    assert set(wm["face"][0]) == {"f32"} and set(wm["relax"][0]) == {"f64", "f32"}
    assert set(wf["relax"][0]) == {"ff", "f32"} and wf["face"][1] == 3 * K * P2 * 17 * 4
    # bound and fraction: a 1 ms launch of k_face at 1 TFLOP/s FP64 needs
    # 3 K P2 111 / 1e12 s of the FP64 pipe; with that the larger roofline time
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 64.0}
    prof = {k: (1.0, 1) for k in ("prep", "face", "volume", "relax")}
    r = bench.kernel_rooflines(p, K, 0, prof, peaks)
    t64 = 3 * K * P2 * 111 / 1e12
    assert r["face"]["frac_fp64"] == pytest.approx(t64 / 1e-3)
    assert r["face"]["bound"] in ("fp64", "hbm")
    assert r["face"]["frac"] == pytest.approx(max(r["face"]["frac_fp64"], r["face"]["frac_hbm"]))
    # float-float work occupies the FP32 pipe at 2 x FF_INSTR_PER_OP flops per operation
    rf = bench.kernel_rooflines(p, K, 3, prof, peaks)
    wr = bench.kernel_work(p, K, precision=3)["relax"][0]
    assert rf["relax"]["frac_fp32"] == pytest.approx((wr["f32"] + 2 * bench.FF_INSTR_PER_OP * wr["ff"]) / 64e12 / 1e-3)
