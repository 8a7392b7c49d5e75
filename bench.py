#!/usr/bin/env python
"""Throughput of the locally relaxed entropy-stable RK step on GB300.

Metric: DOF.RK-stage updates/s = LGL nodes x RK stages x steps / time, one
"step" being one full relaxed RK step (every stage's right-hand side and the
per-element gamma_kappa solve with the relaxed update) over the whole mesh.

Default workload: 3D compressible Euler Taylor--Green vortex, Mach 0.1,
periodic [0, 2 pi]^3, 32^3 hexahedra, p = 3 (2,097,152 nodes), BS3 (3 stages),
local relaxation, CFL 0.5, FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own instance (independent
problems, no data-path collective: weak scaling); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on the host on a bounded sample of
the same workload (rank 0 only).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

TWO_PI = 2.0 * math.pi
METRIC = "DOF·RK-stage updates/s (RHS+local relaxation), FP64 vs mixed; % of roofline"
UNIT = "DOF*stage/s"

WORKLOADS = {
    # the metric's configuration: Euler TGV 32^3 p=3 FP64, 200 steps
    "tgv_euler_p3_32^3_fp64": dict(p=3, n=32, mu=0.0, precision=0, ic="tgv", steps=200),
    "tgv_euler_p3_32^3_mixed": dict(p=3, n=32, mu=0.0, precision=1, ic="tgv", steps=200),
    "tgv_euler_p3_32^3_fp64x": dict(p=3, n=32, mu=0.0, precision=2, ic="tgv", steps=200),
    "tgv_euler_p3_32^3_mixed_ff": dict(p=3, n=32, mu=0.0, precision=3, ic="tgv", steps=200),
    "tgv_ns_re1600_p4_32^3_fp64x": dict(p=4, n=32, mu=1.0 / 1600.0, precision=2, ic="tgv", steps=200),
    "tgv_ns_re1600_p4_32^3_fp64": dict(p=4, n=32, mu=1.0 / 1600.0, precision=0, ic="tgv", steps=200),
    "tgv_ns_re1600_p4_32^3_mixed_noise": dict(p=4, n=32, mu=1.0 / 1600.0, precision=1, ic="tgv_noise", steps=200),
    "tgv_ns_re1600_p4_32^3_mixed_ff_noise": dict(p=4, n=32, mu=1.0 / 1600.0, precision=3, ic="tgv_noise",
                                                 steps=200),
    "vortex_euler_p3_4^3_fp64": dict(p=3, n=4, mu=0.0, precision=0, ic="vortex", steps=20),
}
MAIN = "tgv_euler_p3_32^3_fp64"
PRECISION_LABEL = {0: "FP64",
                   1: "mixed (FP32 fluxes/SATs/viscous terms; FP64 state, stage states, entropy increments, "
                      "estimate sums and gamma solve)",
                   2: "FP64X (float-float fluxes/SATs/viscous terms on the FP32 pipe, ~2^-47 per operation; "
                      "FP64 state/estimate/gamma)",
                   3: "mixed float-float (FP32 fluxes/SATs/viscous terms; stage states, entropy increments, "
                      "estimate sums and gamma solve in float-float on the FP32 pipe; FP64 state)"}
DTYPE = {0: "f64", 1: "f64+f32", 2: "f64+f32x2", 3: "f64+f32+f32x2"}
STAGES = 3  # BS3: b_4 = 0


# ---------------------------------------------------------------------------------------
# algorithmic work of the volume kernel (the dominant one), counted from its source:
# two-point flux 56 flops (FMA = 2, one division = 1), scatter to both nodes 20;
# interface terms 20 per line; per-direction write-back 25 (p+1)^3 per element;
# relaxation term (stages 2, 3) 12 per node; BR1 divergence 4 (2 (p+1)^2 + 8) per line.
def volume_flops_per_element(p, ns=False, with_A=False):
    P1 = p + 1
    lines = 3 * P1 * P1
    pairs = P1 * (P1 - 1) // 2
    f = lines * (pairs * 76 + 20) + 25 * P1 ** 3
    if with_A:
        f += 12 * P1 ** 3
    if ns:
        f += lines * 4 * (2 * P1 * P1 + 8) + lines * 4 * P1
    return f


# Algorithmic work of the other kernels per unit, counted from their FP64 sources the same
# way (FMA = 2; reciprocal, rsqrt, log each 1; the series logarithms by their terms):
# k_face per face node: Ismail--Roe flux 56 + Rusanov dissipation 55 (two conserved
#   states from z 2 x 19, lambda 2, 5 jump terms 15);
# k_prep per node: parameter vector 22 + 10 per earlier stage combined (+10 for the pending
#   update in the first stage); entropy-variable increments 122 in stages 2 and 3 (one
#   division for 1/rho, 1/rho', 1/p and one for beta/(1+y), log1p(z) - z counted as 1);
# k_relax per node and step: setup 65 in the solve's arithmetic (primitive state 35, X0 Y0 V2
#   25, a 5) and the cubic starting coefficient 20, which both solves take in FP32, + 75 per
#   Bregman evaluation (one for a smooth step from the cubic start).
# k_grad per node (Navier--Stokes): entropy variables from z 4; per direction the D product
#   8 (p+1), the metric 4 and the face lifting 12 on the 2/(p+1) face nodes; chain rule 90
#   (velocity 3, 1/w_5 1, velocity gradients 27, temperature gradients 9, divergence 2,
#   stresses 27, energy fluxes 21).
FACE_FLOPS_PER_FACE_NODE = 56 + 55
PREP_FLOPS_Z, PREP_FLOPS_PER_STAGE, PREP_FLOPS_PENDING, PREP_FLOPS_DW = 22, 10, 10, 122
RELAX_FLOPS_SETUP, RELAX_FLOPS_CUBIC, RELAX_FLOPS_EVAL = 65, 20, 75


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the k_volume launches of one
# step of the default workload (stages 1, 2, 3; FP64, tile variant 1), from the ncu capture
# summarised in profiles/; the roofline reports their mean, per launch like `achieved`.
# It is reported only while the kernel sources hash to the value the capture was taken with.
VOLUME_TRAFFIC = {"source_sha1": "9ead7ce83383f973f27e285f991389a131516fd2",
                  "bytes_per_stage": [148340480 + 48874752, 232487680 + 55985664, 400438528 + 65617408]}


def kernel_source_sha1():
    h = hashlib.sha1()
    for f in ("es_kernels.cuh", "es_device.cuh", "es_ff.cuh"):
        with open(os.path.join(ROOT, "paper_2003_08831_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def fp_peak_tflops(precision, sm_mhz):
    """ALU peak from unit counts x clock: 152 SMs, FP64 2 DFMA/clk/SM, FP32 128 FFMA/clk/SM."""
    per_clk = 4.0 if precision == 0 else 256.0
    return 152 * per_clk * sm_mhz * 1e6 / 1e12


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the
    recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json copy bandwidth)"
    except Exception:
        return 6800.0, "fallback (no MEASURED_PEAKS.json)"


def measure_alu_peaks(gpu_index=None):
    """FP64 and FP32 FMA-chain throughput of this GPU (es_fma_peak), with the SM clock
    sampled while the probe runs."""
    from paper_2003_08831_gb300 import _binding as B
    sampler = ClockSampler(gpu_index).start() if gpu_index is not None else None
    fp64 = max(B.es_fma_peak(True) for _ in range(2))
    fp32 = max(B.es_fma_peak(False) for _ in range(2))
    clk = sampler.stop() if sampler is not None else None
    return {"fp64_tflops": fp64, "fp32_tflops": fp32, "sm_mhz": clk["sm_mhz"] if clk else None,
            "how": "es_fma_peak: independent FMA chains, 8 per thread, 64 warps per SM, best of 2 x 5 launches"}


# Arithmetic of each part of each kernel per precision mode: "f64", "f32" or "ff"
# (float-float on the FP32 pipe).  ES_MIXED keeps the stage combination, the entropy
# increments, d and the sums and the gamma solve in FP64; ES_MIXED_FF and ES_FP64X form
# them in float-float; the parameter vector is float-float in every mode but FP64.
ARITH = {
    0: {"z": "f64", "comb": "f64", "dw": "f64", "flux": "f64", "sums": "f64", "relax": "f64"},
    1: {"z": "ff", "comb": "f64", "dw": "f64", "flux": "f32", "sums": "f64", "relax": "f64"},
    2: {"z": "ff", "comb": "ff", "dw": "ff", "flux": "ff", "sums": "ff", "relax": "ff"},
    3: {"z": "ff", "comb": "ff", "dw": "ff", "flux": "f32", "sums": "ff", "relax": "ff"},
}
# FP32 instructions per float-float operation, counted from es_ff.cuh: a sum is a TwoSum
# (6) + 2 additions + a Fast2Sum (3) = 11, a product 1 + 3 fmas + a Fast2Sum = 7, the
# accumulating product 12; the flux and thermodynamics mix sums and products about
# evenly: 9.  A float-float operation occupies the FP32 pipe like 9 FFMAs, i.e. 18 of
# the peak's flops.
FF_INSTR_PER_OP = 9.0
TF_BYTES = {0: 8, 1: 4, 2: 8, 3: 4}


def kernel_work(p, n_el, precision, ns=False, stages=3):
    """Per kernel kind, averaged over the launches of one BS3 step: algorithmic flops split
    by arithmetic ({"f64": .., "f32": .., "ff": ..}) and the bytes the kernel must move
    (its inputs and outputs in this design: state and d in FP64, stage values,
    parameter vector and face fluxes in the flux precision)."""
    P1 = p + 1
    Np = P1 ** 3
    nodes = n_el * Np
    tf = TF_BYTES[precision]
    ar = ARITH[precision]
    nprev = [0, 1, 1]                       # BS3: a21, a32 (a31 = 0)
    dw_stage = [False, True, True]          # entropy increments where b_i != 0, i > 1
    out = {}

    def add(d, kind, val):
        d[kind] = d.get(kind, 0.0) + val

    # k_prep
    fl, by = {}, 0.0
    for i in range(stages):
        add(fl, ar["z"], nodes * PREP_FLOPS_Z)
        add(fl, ar["comb"], nodes * (PREP_FLOPS_PER_STAGE * nprev[i] + (PREP_FLOPS_PENDING if i == 0 else 0)))
        if dw_stage[i]:
            add(fl, ar["dw"], nodes * PREP_FLOPS_DW)
        by += nodes * (40 + 5 * tf * nprev[i] + 6 * tf + (80 if i == 0 else 0) + (40 if dw_stage[i] else 0))
    out["prep"] = ({k: v / stages for k, v in fl.items()}, by / stages)
    # k_face: 3 K P1^2 face-node pairs, both sides' z and 1/z1 read, the flux written
    fn = 3 * n_el * P1 * P1
    out["face"] = ({ar["flux"]: fn * FACE_FLOPS_PER_FACE_NODE}, fn * 17 * tf)
    # k_volume
    fl, by = {}, 0.0
    for i in range(stages):
        wa = dw_stage[i]
        f = volume_flops_per_element(p, ns, wa) * n_el
        sums = (12 * Np * n_el if wa else 0) + (10 * 2 * Np * n_el if i == stages - 1 else 0)
        add(fl, ar["flux"], f - (12 * Np * n_el if wa else 0))
        add(fl, ar["sums"], sums)
        b = nodes * 5 * tf + n_el * 30 * P1 * P1 * tf + (40 * nodes if wa else 0)
        b += (40 + 2 * 5 * tf) * nodes if i == stages - 1 else 5 * tf * nodes
        if ns:
            b += 12 * tf * nodes
        by += b
    out["volume"] = ({k: v / stages for k, v in fl.items()}, by / stages)
    out["relax"] = ({ar["relax"]: nodes * (RELAX_FLOPS_SETUP + RELAX_FLOPS_EVAL), "f32": nodes * RELAX_FLOPS_CUBIC},
                    80.0 * nodes)
    if ns:
        out["grad"] = ({ar["flux"]: nodes * (4 + 3 * (8 * P1 + 4 + 24.0 / P1) + 90)}, nodes * (5 + 12) * tf)
    return out


def kernel_rooflines(p, n_el, precision, prof, peaks, ns=False):
    """Per kernel kind: the time its algorithmic work needs at the measured peaks --
    the FP64 pipe (FP64 flops) and the FP32 pipe (FP32 flops, float-float operations at
    FF_INSTR_PER_OP instructions each) run side by side, HBM at the measured copy
    bandwidth -- against its average event-timed launch; frac = roofline time / launch
    time and bound = the unit that sets the roofline time."""
    hbm, _ = hbm_peak_gbs()
    out = {}
    for k, (fl, by) in kernel_work(p, n_el, precision, ns).items():
        ms, n = prof.get(k, (0.0, 0))
        if not n:
            continue
        t = ms / n * 1e-3
        t64 = fl.get("f64", 0.0) / (peaks["fp64_tflops"] * 1e12)
        t32 = (fl.get("f32", 0.0) + 2.0 * FF_INSTR_PER_OP * fl.get("ff", 0.0)) / (peaks["fp32_tflops"] * 1e12)
        tb = by / (hbm * 1e9)
        troof = max(t64, t32, tb)
        bound = "fp64" if troof == t64 else ("fp32" if troof == t32 else "hbm")
        out[k] = {"avg_launch_ms": ms / n, "flops": {a: v for a, v in fl.items()}, "bytes": by,
                  "frac_fp64": t64 / t, "frac_fp32": t32 / t, "frac_hbm": tb / t,
                  "bound": bound, "frac": troof / t}
    return out


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
def workload_config(name):
    """The config object both arms report for workload `name`."""
    wl = WORKLOADS[name]
    P1 = wl["p"] + 1
    K = wl["n"] ** 3
    return {"workload": name, "elements": K, "p": wl["p"], "nodes": K * P1 ** 3, "rk": "BS3 (3 stages)",
            "relaxation": "local", "cfl": 0.5, "interface": "EC + Rusanov",
            "physics": "Navier-Stokes Re 1600 Pr 0.72" if wl["mu"] > 0 else "Euler",
            "precision": PRECISION_LABEL[wl["precision"]],
            "l2": "inputs larger than L2 (state + 3 stage buffers + aux > 500 MB), no flush"}


def aggregate(ms_local, units_local, dist=None, device="cpu"):
    """Weak-scaling aggregation over ranks: the slowest rank's time and the units of
    work of all ranks (no data-path collective; this runs once after the timed
    region).  Returns (max ms, total units)."""
    if dist is None:
        return float(ms_local), float(units_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shard(count, rank, world):
    """Indices of `count` independent instances owned by `rank` (round robin)."""
    return list(range(rank, count, world))


def initial_state(solver, wl, gamma_gas=1.4):
    from paper_2003_08831_gb300 import inputs
    xyz = solver.coords()
    x, y, z = xyz[0], xyz[1], xyz[2]
    if wl["ic"] == "tgv":
        return inputs.tgv_state(x, y, z, mach=0.1, gamma=gamma_gas)
    if wl["ic"] == "tgv_noise":
        return inputs.perturbed_tgv_state(x.reshape(-1), y.reshape(-1), z.reshape(-1), mach=0.1,
                                          gamma=gamma_gas).reshape(5, solver.K, solver.Np)
    return inputs.vortex_state(x, y, 0.0, centre=(5.0, 5.0))


def make_solver(wl):
    from paper_2003_08831_gb300.solver import Solver
    n = wl["n"]
    if wl["ic"] == "vortex":
        lo, hi = (0.0, 0.0, 0.0), (10.0, 10.0, 10.0)
    else:
        lo, hi = (0.0, 0.0, 0.0), (TWO_PI, TWO_PI, TWO_PI)
    return Solver(wl["p"], (n, n, n), lo, hi, mu=wl["mu"], Pr=0.72, precision=wl["precision"])


def state_error(q, ref):
    """Relative L2 over all conserved variables and per-variable max error relative to the
    variable's max |ref| (floored at 1e-3 of the largest), of a state against a reference."""
    q = np.asarray(q, dtype=np.float64).reshape(5, -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(5, -1)
    d = q - ref
    scale = np.maximum(np.max(np.abs(ref), axis=1), 1e-3 * np.max(np.abs(ref)))
    return {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
            "max_rel_per_var": [float(v) for v in np.max(np.abs(d), axis=1) / scale]}


def error_vs_fp64(wl, steps=20):
    """The form's state after `steps` relaxed steps against the FP64 path (which matches
    the oracle to 1e-12) from the same initial state and time step."""
    from paper_2003_08831_gb300.solver import stable_dt
    out = {}
    for prec in (0, wl["precision"]):
        w = dict(wl, precision=prec)
        s = make_solver(w)
        q0 = initial_state(s, w)
        h = [(s.hi[m] - s.lo[m]) / s.n[m] for m in range(3)]
        dt = stable_dt(q0, s.p, h, 0.5, mu=w["mu"])
        q = s.to_device(q0)
        s.advance(q, steps, dt)
        if s.status() != 0:
            raise RuntimeError("device status %d in the precision comparison" % s.status())
        out[prec] = q.cpu().numpy()
        s.close()
        del q
    r = state_error(out[wl["precision"]], out[0])
    r["steps"] = steps
    r["reference"] = "FP64 path, same initial state and dt"
    return r


def measure_device(wl, steps, warmup, dist=None, clocks_gpu=None):
    """Device-resident timing of `steps` relaxed steps (CUDA events on the launching stream)."""
    import torch
    from paper_2003_08831_gb300.solver import stable_dt
    s = make_solver(wl)
    q0 = initial_state(s, wl)
    h = [(s.hi[m] - s.lo[m]) / s.n[m] for m in range(3)]
    dt = stable_dt(q0, s.p, h, 0.5, mu=wl["mu"])
    q = s.to_device(q0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    s.autotune(q)   # volume-kernel tile for this workload (stage RHS timings; q unchanged)
    s.advance(q, warmup, dt, t, want_hist=False, want_gamma_elem=False)
    torch.cuda.synchronize()
    rc = s.status()
    if rc != 0:
        raise RuntimeError("device status %d after warm-up" % rc)
    hist = torch.empty(steps, dtype=torch.float64, device="cuda")
    n0 = s.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(clocks_gpu).start() if clocks_gpu is not None else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    from paper_2003_08831_gb300 import _binding as B
    B.es_advance(s.ctx, q, steps, dt, t, hist, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop() if sampler is not None else None
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - n0
    rc = s.status()
    if rc != 0:
        raise RuntimeError("device status %d after the timed region" % rc)
    g = hist.cpu().numpy()
    res = {"ms": ms, "launches": launches, "dt": dt, "gamma_min": float(g.min()), "gamma_max": float(g.max()),
           "nodes": s.N, "solver": s, "q": q, "t": t, "clocks": clocks}
    return res


def measure_batch(precision, steps, warmup, count=256, ref_states=None, keep_states=False):
    """Batched form: `count` independent isentropic-vortex instances (seeded n in 4..12,
    p in 2..5, centre, strength, Mach), per-instance dt at CFL 0.5, all advanced
    together by CUDA-graph replay after the volume tiles are autotuned."""
    import torch
    from paper_2003_08831_gb300 import inputs
    from paper_2003_08831_gb300.solver import BatchSolver, stable_dt
    params = inputs.batch_instances(count)
    insts = [dict(p=d["p"], n=(d["n"],) * 3, lo=(0.0, 0.0, 0.0), hi=(d["box"],) * 3) for d in params]
    b = BatchSolver(insts, precision=precision)
    dts = []
    for i, d in enumerate(params):
        xyz = b.coords(i)
        q0 = inputs.vortex_state(xyz[0], xyz[1], 0.0, eps=d["eps"], mach=d["mach"], centre=d["centre"],
                                 period=d["box"])
        b.set_state(i, q0)
        dts.append(stable_dt(q0, d["p"], [d["box"] / d["n"]] * 3, 0.5))
    b.set_dt(dts)
    b.autotune()   # stage right-hand sides only: the states are unchanged
    b.advance(warmup)
    torch.cuda.synchronize()
    st0 = b.status()
    if st0 not in (0, -4):   # -4: an element without a positive root was flagged (left unconstrained)
        raise RuntimeError("batch status %d after warm-up" % st0)
    stream = torch.cuda.current_stream()
    n0 = b.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.advance(steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = b.status()
    if st1 not in (0, -4):
        raise RuntimeError("batch status %d after the timed region" % st1)
    t, g = b.times()
    nodes = b.nodes()
    out = {"value": nodes * STAGES * steps / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
           "instances": count, "nodes": int(nodes), "kernels_per_step": int((b.launch_count() - n0) / steps),
           "graph_launches_per_step": 1, "gamma_range": [float(g.min()), float(g.max())],
           "degrees": {str(p): sum(1 for d in params if d["p"] == p) for p in range(2, 6)},
           "no_root_flagged": bool(st0 == -4 or st1 == -4)}
    states = None
    if keep_states or ref_states is not None:
        states = [b.get_state(i) for i in range(count)]
    if ref_states is not None:
        # same instances, initial states, dt and number of steps (warm-up + timed) as the FP64 run
        out["error_vs_fp64"] = state_error(np.concatenate([st.reshape(5, -1) for st in states], axis=1),
                                           np.concatenate([st.reshape(5, -1) for st in ref_states], axis=1))
        out["error_vs_fp64"]["steps"] = warmup + steps
        out["error_vs_fp64"]["reference"] = "FP64 batch, same instances, states, dt and steps"
    b.close()
    if keep_states:
        return out, states
    return out


def degree_rates(precision, steps=10, warmup=3, target_nodes=2_000_000):
    """Relaxed-step throughput of one large isentropic-vortex instance per LGL degree
    (p = 2..5, about target_nodes nodes each, the batch's box and vortex, tiles
    autotuned): the rate each degree's kernels reach when the GPU is full of them."""
    import torch
    from paper_2003_08831_gb300 import inputs
    from paper_2003_08831_gb300.solver import Solver, stable_dt
    out = {}
    for p in range(2, 6):
        n = max(4, int(round((target_nodes / (p + 1) ** 3) ** (1.0 / 3.0))))
        s = Solver(p, (n, n, n), (0.0,) * 3, (10.0,) * 3, precision=precision)
        xyz = s.coords()
        q0 = inputs.vortex_state(xyz[0], xyz[1], 0.0, eps=4.5, mach=0.3, centre=(5.0, 5.0), period=10.0)
        dt = stable_dt(q0, p, [10.0 / n] * 3, 0.5)
        q = s.to_device(q0)
        s.autotune(q)
        s.advance(q, warmup, dt, want_hist=False, want_gamma_elem=False)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        s.advance(q, steps, dt, want_hist=False, want_gamma_elem=False)
        e1.record()
        torch.cuda.synchronize()
        out[p] = {"elements": n ** 3, "nodes": s.N, "value": s.N * STAGES * steps / (e0.elapsed_time(e1) / 1e3)}
        s.close()
    return out


def degree_mix(form, params, precision):
    """The batch against its degree mix: the rate predicted from the single-instance rate
    of each degree (the batch's nodes of degree p take nodes_p / rate_p), and the
    batch's measured rate as a fraction of that prediction."""
    rates = degree_rates(precision)
    nodes = {p: sum(d["n"] ** 3 * (p + 1) ** 3 for d in params if d["p"] == p) for p in range(2, 6)}
    total = sum(nodes.values())
    pred = total / sum(nodes[p] / rates[p]["value"] for p in nodes if nodes[p])
    return {"single_instance_rate_per_degree": {str(p): rates[p]["value"] for p in rates},
            "batch_nodes_per_degree": {str(p): nodes[p] for p in nodes},
            "predicted_from_degree_mix": pred, "measured_over_predicted": form["value"] / pred}


def measure_shock(precision, steps=50, warmup=3, n=25, p=3):
    """Section 4.1.2 form: the moving viscous shock on n^3 elements of [-0.5, 0.5]^3 (M 2.5,
    Re 10, Pr 3/4), Dirichlet-penalty boundaries on the x1 faces (exterior state evaluated on
    the device at every stage time), RK(4,4), dt = 0.03 h^2; CUDA events around `steps` steps,
    and the density error against the exact solution at the end."""
    import torch
    from paper_2003_08831_gb300 import inputs, _binding as B
    from paper_2003_08831_gb300.solver import Solver
    prm = inputs.viscous_shock_parameters(2.5, 10.0, 0.75)
    s = Solver(p, (n, n, n), (-0.5,) * 3, (0.5,) * 3, mu=prm["mu"], Pr=0.75, rk=B.ES_RK_RK4, precision=precision)
    s.set_boundary(0, B.ES_BC_VISCOUS_SHOCK, [2.5, 10.0, 0.75, -1.0])
    xyz = s.coords()
    q = s.to_device(inputs.viscous_shock_state(xyz[0], 0.0, prm))
    dt = 0.03 / n ** 2
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.advance(q, warmup, dt, t, want_hist=False, want_gamma_elem=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance(q, steps, dt, t, want_hist=False, want_gamma_elem=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if s.status() != 0:
        raise RuntimeError("device status %d in the viscous-shock form" % s.status())
    err = q.cpu().numpy().reshape(5, -1)[0] - inputs.viscous_shock_state(xyz[0], t.item(), prm)[0].reshape(-1)
    nodes = s.N
    s.close()
    return {"value": nodes * 4 * steps / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps, "nodes": int(nodes),
            "elements": n ** 3, "p": p, "rk": "RK(4,4) (4 stages)", "boundaries": "Dirichlet penalty on x1 (exact solution)",
            "t_end": t.item(), "density_rel_l2_error_vs_exact": float(np.linalg.norm(err) / np.linalg.norm(
                inputs.viscous_shock_state(xyz[0], t.item(), prm)[0]))}


def kernel_profile(res, steps):
    """Second pass with per-launch CUDA events: time per kernel kind."""
    import torch
    s, q, t = res["solver"], res["q"], res["t"]
    s.profile(True)
    s.advance(q, steps, res["dt"], t, want_hist=False, want_gamma_elem=False)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    return prof


def measure_e2e(wl, steps, warmup):
    """End to end through the C ABI on pinned HOST buffers: per step H2D of the state,
    one relaxed step, D2H of the state, t and gamma (es_advance_host)."""
    import torch
    from paper_2003_08831_gb300.solver import stable_dt
    s = make_solver(wl)
    q0 = initial_state(s, wl)
    h = [(s.hi[m] - s.lo[m]) / s.n[m] for m in range(3)]
    dt = stable_dt(q0, s.p, h, 0.5, mu=wl["mu"])
    qh = torch.from_numpy(np.ascontiguousarray(q0.reshape(5, -1))).pin_memory()
    th = torch.zeros(1, dtype=torch.float64).pin_memory()
    gh = torch.zeros(1, dtype=torch.float64).pin_memory()
    qn, tn, gn = qh.numpy(), th.numpy(), gh.numpy()
    for _ in range(warmup):
        s.advance_host(qn, 1, dt, tn, gn)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.advance_host(qn, 1, dt, tn, gn)
    el = time.perf_counter() - t0
    if s.status() != 0:
        raise RuntimeError("device status after e2e run")
    nodes = s.N
    s.close()
    return {"value": nodes * STAGES * steps / el, "unit": UNIT,
            "h2d_bytes_per_step": int(5 * nodes * 8 + 8), "d2h_bytes_per_step": int(5 * nodes * 8 + 16),
            "ms_per_step": 1e3 * el / steps}


# ---------------------------------------------------------------------------------------
def oracle_setup(ne=6):
    """A periodic ne^3-element sub-box of the TGV workload (same p, element size and
    state): (mesh, U, phys, dt)."""
    from oracle import dg, rk
    from paper_2003_08831_gb300 import inputs
    p, N = 3, 32
    h = TWO_PI / N
    mesh = dg.Mesh(p, (ne, ne, ne), (0.0, 0.0, 0.0), (ne * h, ne * h, ne * h))
    x, y, z = mesh.coords()
    U = inputs.tgv_state(x, y, z, mach=0.1)
    phys = dg.Physics(1.4, diss=1)
    return mesh, U, phys, rk.stable_dt(mesh, U, phys, 0.5)


_BARRIER = None


def _oracle_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(job):
    """One host core: `warmup` untimed steps, then (after every worker is ready) full
    relaxed BS3 steps for `amount` seconds (by_time) or steps; returns (steps, seconds,
    nodes)."""
    amount, by_time, warmup, ne = job
    from oracle import rk
    mesh, U, phys, dt = oracle_setup(ne)
    for _ in range(warmup):
        U = rk.rk_step(mesh, U, dt, phys, rk.BS3).U
    _BARRIER.wait()
    n = 0
    t0 = time.perf_counter()
    while True:
        U = rk.rk_step(mesh, U, dt, phys, rk.BS3).U
        n += 1
        el = time.perf_counter() - t0
        if (by_time and el >= amount) or (not by_time and n >= amount):
            break
    return n, el, mesh.K * mesh.Np


def oracle_parallel(amount, by_time=True, warmup=1, ne=6, cores=None):
    """The FP64 CPU oracle, as it stands, on every host core: one spawned process per core,
    each advancing its own independent periodic ne^3-element sub-box of the TGV workload;
    the timed loops start together.  Returns (DOF*stage/s summed over the cores, total
    steps, longest timed loop in s, nodes per sub-box, cores)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=ctx, initializer=_oracle_init,
                                initargs=(barrier,)) as ex:
        res = list(ex.map(_oracle_worker, [(amount, by_time, warmup, ne)] * cores))
    nodes = res[0][2]
    rate = sum(nodes * STAGES * n / el for n, el, _ in res)
    return rate, sum(n for n, _, _ in res), max(el for _, el, _ in res), nodes, cores


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    value, n, el, nodes, cores = oracle_parallel(args.steps, by_time=False, warmup=args.warmup)
    sample = ("%d independent periodic 6^3-element sub-boxes (%d nodes each) of the 32^3 p=3 Euler TGV, one per "
              "host core, %d full relaxed BS3 steps each" % (cores, nodes, args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (closed-form Taylor-Green vortex, Mach 0.1)",
        "config": workload_config(MAIN),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=MAIN, choices=sorted(WORKLOADS))
    ap.add_argument("--no-forms", action="store_true", help="skip the extra precision/physics forms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--quick", action="store_true",
                    help="timed region only (no kernel-event pass, e2e, forms or CPU baseline): for profilers")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_full(args, rank, world, local_rank)


def compact(form):
    """The few numbers of a form that the end of the JSON line repeats."""
    out = {"value": form["value"], "ms_per_step": form["ms_per_step"]}
    kr = form.get("kernel_roofline") or {}
    if "volume" in kr:
        out["volume_frac"] = round(kr["volume"]["frac"], 3)
        out["volume_bound"] = kr["volume"]["bound"]
    if "speedup_vs_fp64_same_physics" in form:
        out["speedup_vs_fp64"] = round(form["speedup_vs_fp64_same_physics"], 3)
    if "error_vs_fp64" in form:
        out["rel_l2_vs_fp64"] = form["error_vs_fp64"]["rel_l2"]
    if "degree_mix" in form:
        out["predicted_from_degree_mix"] = form["degree_mix"]["predicted_from_degree_mix"]
        out["measured_over_predicted"] = round(form["degree_mix"]["measured_over_predicted"], 3)
    return out


def run_full(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    __graft_entry__.build()
    wl = WORKLOADS[args.workload]
    peaks = None if args.quick else measure_alu_peaks(local_rank)
    res = measure_device(wl, args.steps, args.warmup, dist=dist, clocks_gpu=local_rank)
    ms, units = aggregate(res["ms"], res["nodes"] * STAGES * args.steps, dist, "cuda")
    clocks = res.pop("clocks", None)
    value = units / (ms / 1e3)
    if args.quick:
        res["solver"].close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                              "quick": True, "config": {"workload": args.workload}}), flush=True)
        if dist is not None:
            dist.barrier()
        return 0
    prof = kernel_profile(res, min(args.steps, 50))
    res["solver"].close()
    del res["q"], res["t"], res["solver"]
    if rank != 0:
        if dist is not None:
            dist.barrier()
        return 0
    p = wl["p"]
    K = wl["n"] ** 3
    ns = wl["mu"] > 0
    # average over the 3 stages: the A term is accumulated in stages 2 and 3
    fl = K * (volume_flops_per_element(p, ns, False) + 2 * volume_flops_per_element(p, ns, True)) / 3.0
    vol_ms, vol_n = prof["volume"]
    avg_ms = vol_ms / max(vol_n, 1)
    achieved = fl / (avg_ms * 1e-3) / 1e12
    sm_mhz = clocks["sm_mhz"] if clocks else 2070.0
    peak = fp_peak_tflops(wl["precision"], sm_mhz)
    peak_meas = peaks["fp64_tflops"] if wl["precision"] == 0 else peaks["fp32_tflops"]
    tot = sum(v[0] for v in prof.values())
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[wl["precision"]],
        "data": "synthetic (closed-form Taylor-Green vortex, Mach 0.1)",
        "config": workload_config(args.workload),
        "dt": res["dt"], "gamma_range": [res["gamma_min"], res["gamma_max"]],
        "gpu_launches": int(res["launches"]),
        "roofline": {"bound": "alu", "kernel": "k_volume (flux differencing + SATs)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (sum(VOLUME_TRAFFIC["bytes_per_stage"]) / 3.0
                                 if VOLUME_TRAFFIC["source_sha1"] == kernel_source_sha1() and wl is WORKLOADS[MAIN]
                                 else None),
                     "traffic_unit": "bytes per launch, mean of the step's three launches (ncu, same kernel "
                                     "sources)",
                     "peak_source": "%s ALU peak from unit counts x median SM clock (%.0f MHz): 152 SMs x %s"
                                    % ("FP64" if wl["precision"] == 0 else "FP32", sm_mhz,
                                       "2 DFMA/clk" if wl["precision"] == 0 else "128 FFMA/clk"),
                     "peak_measured": peak_meas, "frac_of_measured": achieved / peak_meas,
                     "peak_measured_source": "FMA-chain throughput in this run (es_fma_peak)",
                     "flops_per_launch": fl, "avg_launch_ms": avg_ms},
        "kernel_share": {k: round(v[0] / tot, 4) for k, v in prof.items() if v[1] > 0},
        "kernel_roofline": kernel_rooflines(p, K, wl["precision"], prof, peaks, ns),
        "clocks": clocks,
        "peaks_measured": dict(peaks, hbm_gbs=hbm_peak_gbs()[0], hbm_source=hbm_peak_gbs()[1]),
    }
    if world == 1 and not args.no_cpu:
        v, nsteps, el, nn, cores = oracle_parallel(10.0)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "%d independent periodic 6^3-element sub-boxes (%d nodes each) of the "
                                         "workload's mesh and state, one per host core, %d full relaxed BS3 steps "
                                         "in total in %.1f s" % (cores, nn, nsteps, el)}
    out["e2e"] = measure_e2e(wl, min(args.steps, 20), 3)
    if world == 1 and not args.no_forms:
        forms = {}
        for name in ["tgv_euler_p3_32^3_mixed", "tgv_euler_p3_32^3_mixed_ff", "tgv_euler_p3_32^3_fp64x",
                     "tgv_ns_re1600_p4_32^3_fp64", "tgv_ns_re1600_p4_32^3_fp64x",
                     "tgv_ns_re1600_p4_32^3_mixed_noise", "tgv_ns_re1600_p4_32^3_mixed_ff_noise"]:
            w2 = WORKLOADS[name]
            steps2 = 50
            r2 = measure_device(w2, steps2, 3)
            p2 = kernel_profile(r2, 20)
            r2["solver"].close()
            t2 = sum(v[0] for v in p2.values())
            err = error_vs_fp64(w2) if w2["precision"] != 0 else None
            forms[name] = {"value": r2["nodes"] * STAGES * steps2 / (r2["ms"] / 1e3),
                           "ms_per_step": r2["ms"] / steps2, "steps": steps2,
                           "gamma_range": [r2["gamma_min"], r2["gamma_max"]], "launches": int(r2["launches"]),
                           "kernel_share": {k: round(v[0] / t2, 4) for k, v in p2.items() if v[1] > 0},
                           "kernel_roofline": kernel_rooflines(w2["p"], w2["n"] ** 3, w2["precision"], p2, peaks,
                                                               w2["mu"] > 0),
                           "speedup_vs_fp64_same_physics": None}
            if err is not None:
                forms[name]["error_vs_fp64"] = err
            del r2
        forms["viscous_shock_ns_p3_25^3_fp64"] = measure_shock(0)
        forms["viscous_shock_ns_p3_25^3_fp64x"] = measure_shock(2)
        forms["batched_vortex_256_fp64"], ref = measure_batch(0, 20, 3, keep_states=True)
        for prec, name in [(1, "batched_vortex_256_mixed"), (3, "batched_vortex_256_mixed_ff"),
                           (2, "batched_vortex_256_fp64x")]:
            forms[name] = measure_batch(prec, 20, 3, ref_states=ref)
        del ref
        from paper_2003_08831_gb300 import inputs as _inp
        bparams = _inp.batch_instances(256)
        for prec, name in [(0, "batched_vortex_256_fp64"), (3, "batched_vortex_256_mixed_ff")]:
            forms[name]["degree_mix"] = degree_mix(forms[name], bparams, prec)
        fp = {"tgv_euler_p3_32^3_mixed": value, "tgv_euler_p3_32^3_mixed_ff": value,
              "tgv_euler_p3_32^3_fp64x": value,
              "tgv_ns_re1600_p4_32^3_fp64x": forms["tgv_ns_re1600_p4_32^3_fp64"]["value"],
              "tgv_ns_re1600_p4_32^3_mixed_noise": forms["tgv_ns_re1600_p4_32^3_fp64"]["value"],
              "tgv_ns_re1600_p4_32^3_mixed_ff_noise": forms["tgv_ns_re1600_p4_32^3_fp64"]["value"],
              "batched_vortex_256_mixed": forms["batched_vortex_256_fp64"]["value"],
              "batched_vortex_256_mixed_ff": forms["batched_vortex_256_fp64"]["value"],
              "batched_vortex_256_fp64x": forms["batched_vortex_256_fp64"]["value"],
              "viscous_shock_ns_p3_25^3_fp64x": forms["viscous_shock_ns_p3_25^3_fp64"]["value"]}
        for k, base in fp.items():
            forms[k]["speedup_vs_fp64_same_physics"] = forms[k]["value"] / base
        for k in forms:
            if forms[k].get("speedup_vs_fp64_same_physics", 0) is None:
                del forms[k]["speedup_vs_fp64_same_physics"]
        out["forms"] = forms
        # the FP64 vs mixed pair on the largest single-instance workload (Navier--Stokes TGV,
        # 32^3, p = 4) and the other forms, repeated compactly at the end of the line
        out["ns_fp64"] = compact(forms["tgv_ns_re1600_p4_32^3_fp64"])
        out["ns_mixed"] = compact(forms["tgv_ns_re1600_p4_32^3_mixed_noise"])
        out["ns_mixed_ff"] = compact(forms["tgv_ns_re1600_p4_32^3_mixed_ff_noise"])
        out["ns_fp64x"] = compact(forms["tgv_ns_re1600_p4_32^3_fp64x"])
        out["euler_mixed"] = compact(forms["tgv_euler_p3_32^3_mixed"])
        out["euler_mixed_ff"] = compact(forms["tgv_euler_p3_32^3_mixed_ff"])
        out["euler_fp64x"] = compact(forms["tgv_euler_p3_32^3_fp64x"])
        out["batch_fp64"] = compact(forms["batched_vortex_256_fp64"])
        out["batch_mixed_ff"] = compact(forms["batched_vortex_256_mixed_ff"])
    out["headline_volume_frac"] = {"of_unit_count_peak": round(achieved / peak, 3),
                                   "of_measured_fma_peak": round(achieved / peak_meas, 3)}
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
