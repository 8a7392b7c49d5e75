"""Convenience layer over the C ABI: one context, torch device buffers, numpy host I/O.

Argument marshalling and bookkeeping only; all arithmetic of the scheme runs in
libes.so.  ``stable_dt`` is the harness' time-step rule (computed once from the
initial state, then fixed).
"""
import json

import numpy as np

from . import _binding as B

CHECKPOINT_MAGIC = "es-relax-checkpoint-v1"


def save_checkpoint(path, q, meta):
    """Raw little-endian FP64 state [5][K][Np] followed by nothing else, plus a JSON
    header file path + '.json' holding meta (config, t, step, dt, ...).  The step is
    deterministic (fixed reduction orders, order-free min), so resuming from a
    checkpoint reproduces an uninterrupted run bit for bit."""
    q = np.ascontiguousarray(np.asarray(q, dtype="<f8"))
    header = dict(meta)
    header["magic"] = CHECKPOINT_MAGIC
    header["shape"] = list(q.shape)
    with open(path, "wb") as f:
        f.write(q.tobytes())
    with open(path + ".json", "w") as f:
        json.dump(header, f, indent=1, sort_keys=True)


def load_checkpoint(path):
    with open(path + ".json") as f:
        header = json.load(f)
    if header.get("magic") != CHECKPOINT_MAGIC:
        raise ValueError("not a checkpoint: %s" % path)
    q = np.fromfile(path, dtype="<f8")
    shape = tuple(header["shape"])
    if q.size != int(np.prod(shape)):
        raise ValueError("checkpoint %s is truncated" % path)
    return q.reshape(shape).astype(np.float64), header


class Solver:
    def __init__(self, p, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma_gas=1.4, mu=0.0, Pr=0.72, R=1.0,
                 interface_diss=1, relax=B.ES_RELAX_LOCAL, rk=B.ES_RK_BS3, precision=B.ES_FP64,
                 delta_floor=0.0, device="cuda", visc_diss=0.0, root_rtol=0.0):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.p, self.n = int(p), tuple(int(a) for a in n)
        self.lo, self.hi = tuple(map(float, lo)), tuple(map(float, hi))
        self.gamma_gas, self.mu, self.Pr, self.R = gamma_gas, mu, Pr, R
        self.P1 = self.p + 1
        self.Np = self.P1 ** 3
        self.K = self.n[0] * self.n[1] * self.n[2]
        self.N = self.K * self.Np
        self.cfg = B.make_config(p, n, lo, hi, gamma_gas, mu, Pr, R, interface_diss, relax, rk, precision,
                                 delta_floor, visc_diss, root_rtol)
        with torch.cuda.device(self.device):
            self.ctx = B.es_create(self.cfg)

    def close(self):
        if self.ctx is not None:
            B.es_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers -------------------------------------------------------------------------
    def empty_state(self):
        return self.torch.empty((5, self.K, self.Np), dtype=self.torch.float64, device=self.device)

    def to_device(self, q):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(5, self.K, self.Np))
        return self.torch.from_numpy(q).to(self.device)

    def coords(self):
        xyz = np.empty((3, self.K, self.Np))
        B.es_node_coords(self.ctx, xyz)
        return xyz

    # -- C ABI calls -------------------------------------------------------------------------
    def rhs(self, q, want_E=False, stream=None):
        dq = self.empty_state()
        E = self.torch.empty(self.K, dtype=self.torch.float64, device=self.device) if want_E else None
        B.es_rhs(self.ctx, q, dq, E, stream)
        return (dq, E) if want_E else dq

    def entropy(self, q, stream=None):
        eta = self.torch.empty(self.K, dtype=self.torch.float64, device=self.device)
        B.es_entropy(self.ctx, q, eta, stream)
        return eta

    def relax_step(self, u_old, u_new, d_eta, stream=None):
        gk = self.torch.empty(self.K, dtype=self.torch.float64, device=self.device)
        g = self.torch.empty(1, dtype=self.torch.float64, device=self.device)
        out = self.empty_state()
        B.es_relax_step(self.ctx, u_old, u_new, d_eta, gk, g, out, stream)
        return gk, g, out

    def advance(self, q, nsteps, dt, t=None, want_hist=True, want_gamma_elem=True, stream=None):
        torch = self.torch
        if t is None:
            t = torch.zeros(1, dtype=torch.float64, device=self.device)
        hist = torch.empty(max(nsteps, 1), dtype=torch.float64, device=self.device) if want_hist else None
        gk = torch.empty(self.K, dtype=torch.float64, device=self.device) if want_gamma_elem else None
        B.es_advance(self.ctx, q, nsteps, dt, t, hist, gk, stream)
        return t, hist, gk

    def step_estimate(self, q, dt, t=None, stream=None):
        """One relaxed step (in place on q) returning the per-element quantities of the
        local entropy inequality: dict of device tensors eta_old, deta, eta_new, gamma_elem
        and the step's gamma (es_step_estimate)."""
        torch = self.torch
        out = {k: torch.empty(self.K, dtype=torch.float64, device=self.device)
               for k in ("eta_old", "deta", "eta_new", "gamma_elem")}
        out["gamma"] = torch.empty(1, dtype=torch.float64, device=self.device)
        if t is None:
            t = torch.zeros(1, dtype=torch.float64, device=self.device)
        B.es_step_estimate(self.ctx, q, dt, t, out["gamma"], out["gamma_elem"], out["eta_old"], out["deta"],
                           out["eta_new"], stream)
        out["t"] = t
        return out

    def advance_host(self, q_host, nsteps, dt, t_host, hist_host=None, stream=None):
        B.es_advance_host(self.ctx, q_host, nsteps, dt, t_host, hist_host, stream)

    def status(self, stream=None):
        return B.es_status(self.ctx, stream)

    def launch_count(self):
        return B.es_launch_count(self.ctx)

    def config_dict(self):
        c = self.cfg
        return {"p": c.p, "n": [c.nx, c.ny, c.nz], "lo": list(c.lo), "hi": list(c.hi), "gamma_gas": c.gamma_gas,
                "mu": c.mu, "Pr": c.Pr, "R": c.R, "interface_diss": c.interface_diss, "relax": c.relax,
                "rk": c.rk, "precision": c.precision, "delta_floor": c.delta_floor, "visc_diss": c.visc_diss,
                "root_rtol": c.root_rtol, "tableau": getattr(self, "tableau", None)}

    def checkpoint(self, path, q, t, step, dt):
        """Write the device state q, time t (float) and step counter to path (see save_checkpoint)."""
        save_checkpoint(path, q.detach().cpu().numpy(),
                        {"config": self.config_dict(), "t": float(t), "step": int(step), "dt": float(dt)})

    @classmethod
    def resume(cls, path, device="cuda"):
        """(solver, q on the device, t, step, dt) from a checkpoint."""
        q, h = load_checkpoint(path)
        c = h["config"]
        s = cls(c["p"], tuple(c["n"]), tuple(c["lo"]), tuple(c["hi"]), c["gamma_gas"], c["mu"], c["Pr"], c["R"],
                c["interface_diss"], c["relax"], c["rk"], c["precision"], c["delta_floor"], device=device,
                visc_diss=c.get("visc_diss", 0.0), root_rtol=c.get("root_rtol", 0.0))
        if c.get("tableau"):
            s.set_tableau(c["tableau"]["A"], c["tableau"]["b"], c["tableau"]["c"])
        return s, s.to_device(q), h["t"], h["step"], h["dt"]

    def set_boundary(self, direction, kind, params=None):
        """Dirichlet-penalty boundaries on the faces of `direction` (ES_BC_STATE with the two
        exterior states, ES_BC_VISCOUS_SHOCK with (Mach, Re, Pr, speed)); ES_BC_PERIODIC resets."""
        B.es_set_boundary(self.ctx, direction, kind, params)

    def set_time(self, t):
        """Time at which rhs() evaluates prescribed boundary states."""
        B.es_set_time(self.ctx, t)

    def set_tableau(self, A, b, c):
        """Explicit Runge--Kutta tableau (up to 10 stages) for the following steps; it is
        stored with checkpoints."""
        B.es_set_tableau(self.ctx, A, b, c)
        self.tableau = {"A": [list(map(float, row)) for row in A], "b": list(map(float, b)),
                        "c": list(map(float, c))}

    def autotune(self, q, stream=None):
        B.es_autotune(self.ctx, q, stream)

    def volume_variant(self):
        return B.es_volume_variant(self.ctx)

    def set_volume_variant(self, variant):
        """0..2: k_prep + k_face + k_volume tiles; 3..5: the fused stage kernel (FP32
        fluxes, periodic Euler); every variant gives the same bits."""
        B.es_set_volume_variant(self.ctx, variant)

    def profile(self, enable):
        B.es_profile_enable(self.ctx, enable)

    def profile_read(self):
        return B.es_profile_read(self.ctx)


def stable_dt(q, p, h, cfl, gamma_gas=1.4, mu=0.0, Pr=0.72):
    """Host-side harness rule, fixed for the run: the sum of the directional
    Courant numbers, dt = cfl / ((2p+1) max_n sum_m (|v_m| + c)/h_m), and for
    mu > 0 also dt <= cfl rho_min / (mu max(4/3, gamma/Pr) sum_m ((2p+1)/h_m)^2)."""
    q = np.asarray(q).reshape(5, -1)
    rho = q[0]
    v = q[1:4] / rho
    pr = (gamma_gas - 1.0) * (q[4] - 0.5 * rho * np.sum(v * v, axis=0))
    c = np.sqrt(gamma_gas * pr / rho)
    lam = np.max(sum((np.abs(v[m]) + c) / h[m] for m in range(3)))
    dt = cfl / ((2 * p + 1) * lam)
    if mu > 0.0:
        k2 = sum(((2 * p + 1) / h[m]) ** 2 for m in range(3))
        dt = min(dt, cfl * float(np.min(rho)) / (mu * max(4.0 / 3.0, gamma_gas / Pr) * k2))
    return dt


class BatchSolver:
    """Many independent instances (possibly different degrees and element counts)."""

    def __init__(self, instances, gamma_gas=1.4, mu=0.0, Pr=0.72, R=1.0, interface_diss=1,
                 relax=B.ES_RELAX_LOCAL, rk=B.ES_RK_BS3, precision=B.ES_FP64, delta_floor=0.0, visc_diss=0.0,
                 root_rtol=0.0):
        """instances: list of dicts with p, n (nx, ny, nz), lo, hi."""
        self.cfgs = [B.make_config(d["p"], d["n"], d.get("lo", (0.0, 0.0, 0.0)), d.get("hi", (1.0, 1.0, 1.0)),
                                   gamma_gas, mu, Pr, R, interface_diss, relax, rk, precision, delta_floor,
                                   visc_diss, root_rtol)
                     for d in instances]
        self.instances = instances
        self.count = len(instances)
        self.b = B.es_batch_create(self.cfgs)

    def close(self):
        if self.b is not None:
            B.es_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, i):
        d = self.instances[i]
        P1 = d["p"] + 1
        return (5, d["n"][0] * d["n"][1] * d["n"][2], P1 ** 3)

    def nodes(self, i=-1):
        return B.es_batch_nodes(self.b, i)

    def coords(self, i):
        sh = self.shape(i)
        xyz = np.empty((3, sh[1], sh[2]))
        B.es_batch_node_coords(self.b, i, xyz)
        return xyz

    def set_state(self, i, q):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(self.shape(i)))
        B.es_batch_set_state(self.b, i, q)

    def get_state(self, i):
        q = np.empty(self.shape(i))
        B.es_batch_get_state(self.b, i, q)
        return q

    def set_dt(self, dt):
        B.es_batch_set_dt(self.b, np.ascontiguousarray(np.asarray(dt, dtype=np.float64)))

    def autotune(self, stream=None):
        B.es_batch_autotune(self.b, stream)

    def set_tableau(self, A, b, c):
        """Explicit Runge--Kutta tableau (up to 10 stages) for every instance."""
        B.es_batch_set_tableau(self.b, A, b, c)

    def advance(self, nsteps, stream=None):
        B.es_batch_advance(self.b, nsteps, stream)

    def step_estimate(self, stream=None):
        """One relaxed step of every instance keeping the local entropy inequality's
        quantities (es_batch_step_estimate); read them with get_estimate(i)."""
        B.es_batch_step_estimate(self.b, stream)

    def get_estimate(self, i):
        """dict of host arrays eta_old, deta, eta_new, gamma_elem of instance i."""
        K = self.shape(i)[1]
        out = {k: np.empty(K) for k in ("eta_old", "deta", "eta_new", "gamma_elem")}
        B.es_batch_get_estimate(self.b, i, out["eta_old"], out["deta"], out["eta_new"], out["gamma_elem"])
        return out

    def times(self):
        t = np.zeros(self.count)
        g = np.zeros(self.count)
        B.es_batch_times(self.b, t, g)
        return t, g

    def status(self, stream=None):
        return B.es_batch_status(self.b, stream)

    def launch_count(self):
        return B.es_batch_launch_count(self.b)
