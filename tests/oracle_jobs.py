"""Oracle runs shared by the GPU parity tests (test infrastructure, not a test module).

* ``gamma_sensitivity`` -- how far each step's gamma and each gamma_kappa of the oracle
  move when every right-hand-side evaluation is perturbed at a rounding level
  (2 eps times the magnitude of the summed terms per node, oracle.dg.rhs_term_magnitude).
  gamma_kappa is the root of a second-order quantity, so this is the scale at which
  two correct implementations (different summation orders, FMA contraction) differ.
* ``tgv_job`` / ``start_jobs`` -- independent oracle advances of the 32^3 Taylor--Green
  workloads in worker processes.  The pool uses the spawn start method (a pool forked
  after the parent has initialised CUDA can hang), each worker rebuilds its mesh and
  initial state from the closed forms, and the perturbed runs for the sensitivities
  run beside the unperturbed one, so a full-size comparison costs the time of one
  oracle run.  The oracle's arithmetic is untouched: a perturbed run only passes
  rk.advance a right-hand side with added noise.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from oracle import dg, relax, rk
from paper_2003_08831_gb300 import inputs

G = 1.4
EPS = 2.0 ** -52


def noisy_rhs(seed, eps, state_eps=0.0):
    """dg.rhs plus 2 eps x term magnitude x N(0, 1) per value (seeded).  With state_eps the
    right-hand side is also evaluated on the stage state perturbed by
    2 state_eps x |U| x N(0, 1) per value: a rounding of the state (the FP32 parameter
    vector of the mixed modes) moves all fluxes of a node together, which independent
    noise on the summed right-hand side does not reproduce."""
    rng = np.random.default_rng(1000 + seed)

    def f(m_, U_, p_, t=0.0):
        V = U_ + 2 * state_eps * np.abs(U_) * rng.standard_normal(U_.shape) if state_eps else U_
        R = dg.rhs(m_, V, p_, t)
        T = dg.rhs_term_magnitude(m_, U_, p_, t)
        return R + 2 * eps * T * rng.standard_normal(R.shape)
    return f


def gamma_sensitivity(mesh, U, dt, nsteps, phys, tab, mode, hist, seeds=4, eps=EPS, delta_floor=relax.DELTA_FLOOR):
    """Largest relative change, over `seeds` perturbed runs, of each step's gamma and of
    the last step's gamma_kappa (elements finite in both runs)."""
    g0 = np.array([h.gamma for h in hist])
    gk0 = np.asarray(hist[-1].gamma_kappa).reshape(-1)
    dg_, dgk = np.zeros(nsteps), np.zeros(gk0.size)
    for seed in range(seeds):
        _, _, h2 = rk.advance(mesh, U, dt, nsteps, phys, tab, mode=mode, rhs=noisy_rhs(seed, eps),
                              delta_floor=delta_floor)
        dg_ = np.maximum(dg_, np.abs(np.array([h.gamma for h in h2]) - g0) / g0)
        gk2 = np.asarray(h2[-1].gamma_kappa).reshape(-1)
        fin = np.isfinite(gk0) & np.isfinite(gk2)
        dgk[fin] = np.maximum(dgk[fin], np.abs(gk2[fin] - gk0[fin]) / gk0[fin])
    return dg_, dgk


def tgv_mesh(p, N=32):
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    return dg.Mesh(p, (N, N, N), lo, hi), lo, hi


def tgv_initial(mesh, noise):
    x, y, z = mesh.coords()
    if noise:
        return inputs.perturbed_tgv_state(x.reshape(-1), y.reshape(-1), z.reshape(-1)).reshape(mesh.shape)
    return inputs.tgv_state(x, y, z)


def tgv_job(job):
    """One oracle advance of the Taylor--Green workload described by `job` (dict: p, N,
    mu, noise, nsteps, dt, seed (None: unperturbed), eps, state_eps (optional), floor,
    want_state).  Returns
    t, each step's gamma, gamma_kappa and delta_kappa (the element's RMS relative
    change, sqrt(2 a / sum P rho)) and, if asked, the final state."""
    mesh, _, _ = tgv_mesh(job["p"], job["N"])
    U = tgv_initial(mesh, job["noise"])
    phys = dg.Physics(G, mu=job["mu"], Pr=0.72, diss=1)
    rhs = None if job["seed"] is None else noisy_rhs(job["seed"], job["eps"], job.get("state_eps", 0.0))
    P = np.broadcast_to(mesh.mass().reshape(1, -1), (mesh.K, mesh.Np))
    t = 0.0
    gam, gks, deltas = [], [], []
    for _ in range(job["nsteps"]):
        r = rk.rk_step(mesh, U, job["dt"], phys, rk.BS3, delta_floor=job["floor"], rhs=rhs, t=t)
        uf, df = mesh.flat(U), mesh.flat(r.d)
        a = 0.5 * np.sum(P * relax.hessian_form(uf, df, G), axis=-1)
        deltas.append(np.sqrt(2.0 * a / np.sum(P * uf[0], axis=-1)))
        gam.append(r.gamma)
        gks.append(np.asarray(r.gamma_kappa).reshape(-1))
        U = r.U
        t = t + r.gamma * job["dt"]
    out = {"t": t, "gamma": np.array(gam), "gk": np.stack(gks), "delta": np.stack(deltas)}
    if job.get("want_state"):
        out["U"] = U
    return out


def _available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def start_jobs(jobs, bytes_per_job):
    """Submit every job to a spawn pool sized by the cores and the memory available for
    the largest job (bytes_per_job: a number, or a list per job); returns (executor,
    futures) in the order of `jobs`."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")    # one thread per worker: the workers are the parallelism
    worst = max(bytes_per_job) if isinstance(bytes_per_job, (list, tuple)) else bytes_per_job
    by_mem = max(1, int(0.6 * _available_bytes() // max(worst, 1)))
    workers = max(1, min(len(jobs), os.cpu_count() or 1, by_mem))
    ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    return ex, [ex.submit(tgv_job, j) for j in jobs]
