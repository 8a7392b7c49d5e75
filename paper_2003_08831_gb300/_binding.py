"""ctypes binding of libes.so (include/es.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors
(device memory, streams) and numpy arrays (host buffers) to the plain pointers
and sizes of the C ABI and raises on non-zero return codes.  If libes.so is
missing or fails to load, every call raises: there is no fallback path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libes.so")

ES_OK = 0
ES_ERR_INVALID = -1
ES_ERR_CUDA = -2
ES_ERR_NONPHYSICAL = -3
ES_ERR_NO_ROOT = -4
ES_ERR_NOMEM = -6
ES_ERR_TOO_LARGE = -7
ES_RK_BS3, ES_RK_RK4, ES_RK_RK65 = 0, 1, 2
ES_FP64, ES_MIXED, ES_FP64X, ES_MIXED_FF = 0, 1, 2, 3
ES_RELAX_NONE, ES_RELAX_LOCAL, ES_RELAX_GLOBAL = 0, 1, 2
ES_BC_PERIODIC, ES_BC_STATE, ES_BC_VISCOUS_SHOCK = 0, 1, 2

EXPORTS = ["es_create", "es_destroy", "es_rhs", "es_entropy", "es_relax_step", "es_advance",
           "es_advance_host", "es_node_coords", "es_status", "es_launch_count", "es_strerror",
           "es_profile_enable", "es_profile_read", "es_rhs_noalloc", "es_rhs_noalloc_scratch_bytes",
           "es_autotune", "es_batch_create", "es_batch_destroy", "es_batch_nodes", "es_batch_node_coords",
           "es_batch_set_state", "es_batch_get_state", "es_batch_set_dt", "es_batch_autotune",
           "es_batch_volume_variant", "es_batch_advance", "es_batch_times", "es_batch_status",
           "es_batch_launch_count", "es_reciprocal", "es_set_boundary", "es_set_time", "es_set_tableau",
           "es_batch_set_tableau", "es_step_estimate", "es_batch_step_estimate", "es_batch_get_estimate", "es_fma_peak", "es_volume_variant",
           "es_set_volume_variant"]
KERNEL_KINDS = ["prep", "face", "grad", "volume", "relax", "other"]


class es_config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("gamma_gas", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("R", ctypes.c_double), ("interface_diss", ctypes.c_int), ("relax", ctypes.c_int),
                ("rk", ctypes.c_int), ("precision", ctypes.c_int), ("delta_floor", ctypes.c_double),
                ("visc_diss", ctypes.c_double), ("root_rtol", ctypes.c_double)]


class ESError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, strerror(code), code))
        self.code = code


_lib = None


def load(path=None):
    """Load libes.so once; raise if it is absent (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libes.so not found at %s: build it with paper_2003_08831_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    lib.es_create.argtypes = [ctypes.POINTER(es_config), ctypes.POINTER(vp)]
    lib.es_create.restype = i
    lib.es_destroy.argtypes = [vp]
    lib.es_destroy.restype = None
    lib.es_rhs.argtypes = [vp, vp, vp, vp, vp]
    lib.es_rhs.restype = i
    lib.es_entropy.argtypes = [vp, vp, vp, vp]
    lib.es_entropy.restype = i
    lib.es_relax_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.es_relax_step.restype = i
    lib.es_advance.argtypes = [vp, vp, i, d, vp, vp, vp, vp]
    lib.es_advance.restype = i
    lib.es_advance_host.argtypes = [vp, vp, i, d, vp, vp, vp]
    lib.es_advance_host.restype = i
    lib.es_node_coords.argtypes = [vp, vp]
    lib.es_node_coords.restype = i
    lib.es_status.argtypes = [vp, vp]
    lib.es_status.restype = i
    lib.es_launch_count.argtypes = [vp]
    lib.es_launch_count.restype = ctypes.c_longlong
    lib.es_profile_enable.argtypes = [vp, i]
    lib.es_profile_enable.restype = i
    lib.es_profile_read.argtypes = [vp, vp, vp]
    lib.es_profile_read.restype = i
    lib.es_rhs_noalloc.argtypes = [ctypes.POINTER(es_config), vp, vp, vp, vp]
    lib.es_rhs_noalloc.restype = i
    lib.es_rhs_noalloc_scratch_bytes.argtypes = [ctypes.POINTER(es_config)]
    lib.es_rhs_noalloc_scratch_bytes.restype = ctypes.c_size_t
    lib.es_autotune.argtypes = [vp, vp, vp]
    lib.es_autotune.restype = i
    lib.es_batch_create.argtypes = [ctypes.POINTER(es_config), i, ctypes.POINTER(vp)]
    lib.es_batch_create.restype = i
    lib.es_batch_destroy.argtypes = [vp]
    lib.es_batch_destroy.restype = None
    lib.es_batch_nodes.argtypes = [vp, i]
    lib.es_batch_nodes.restype = ctypes.c_longlong
    lib.es_batch_node_coords.argtypes = [vp, i, vp]
    lib.es_batch_node_coords.restype = i
    lib.es_batch_set_state.argtypes = [vp, i, vp]
    lib.es_batch_set_state.restype = i
    lib.es_batch_get_state.argtypes = [vp, i, vp]
    lib.es_batch_get_state.restype = i
    lib.es_batch_set_dt.argtypes = [vp, vp]
    lib.es_batch_set_dt.restype = i
    lib.es_batch_autotune.argtypes = [vp, vp]
    lib.es_batch_autotune.restype = i
    lib.es_batch_volume_variant.argtypes = [vp, i]
    lib.es_batch_volume_variant.restype = i
    lib.es_batch_advance.argtypes = [vp, i, vp]
    lib.es_batch_advance.restype = i
    lib.es_batch_times.argtypes = [vp, vp, vp]
    lib.es_batch_times.restype = i
    lib.es_batch_status.argtypes = [vp, vp]
    lib.es_batch_status.restype = i
    lib.es_batch_launch_count.argtypes = [vp]
    lib.es_batch_launch_count.restype = ctypes.c_longlong
    lib.es_reciprocal.argtypes = [vp, vp, ctypes.c_longlong, vp]
    lib.es_reciprocal.restype = i
    lib.es_set_boundary.argtypes = [vp, i, i, vp, i]
    lib.es_set_boundary.restype = i
    lib.es_set_time.argtypes = [vp, d]
    lib.es_set_time.restype = i
    lib.es_set_tableau.argtypes = [vp, i, vp, vp, vp]
    lib.es_set_tableau.restype = i
    lib.es_batch_set_tableau.argtypes = [vp, i, vp, vp, vp]
    lib.es_batch_set_tableau.restype = i
    lib.es_step_estimate.argtypes = [vp, vp, d, vp, vp, vp, vp, vp, vp, vp]
    lib.es_step_estimate.restype = i
    lib.es_batch_step_estimate.argtypes = [vp, vp]
    lib.es_batch_step_estimate.restype = i
    lib.es_batch_get_estimate.argtypes = [vp, i, vp, vp, vp, vp]
    lib.es_batch_get_estimate.restype = i
    lib.es_volume_variant.argtypes = [vp]
    lib.es_volume_variant.restype = i
    lib.es_set_volume_variant.argtypes = [vp, i]
    lib.es_set_volume_variant.restype = i
    lib.es_fma_peak.argtypes = [i, vp, vp]
    lib.es_fma_peak.restype = i
    lib.es_strerror.argtypes = [i]
    lib.es_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code):
    try:
        return load().es_strerror(int(code)).decode()
    except Exception:
        return "error %d" % code


def _check(rc, where):
    if rc != ES_OK:
        raise ESError(rc, where)


def _ptr(t):
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array")


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_config(p, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma_gas=1.4, mu=0.0, Pr=0.72, R=1.0,
                interface_diss=1, relax=ES_RELAX_LOCAL, rk=ES_RK_BS3, precision=ES_FP64, delta_floor=0.0,
                visc_diss=0.0, root_rtol=0.0):
    c = es_config()
    c.p = p
    c.nx, c.ny, c.nz = n
    c.lo = (ctypes.c_double * 3)(*lo)
    c.hi = (ctypes.c_double * 3)(*hi)
    c.gamma_gas, c.mu, c.Pr, c.R = gamma_gas, mu, Pr, R
    c.interface_diss, c.relax, c.rk, c.precision = interface_diss, relax, rk, precision
    c.delta_floor = delta_floor
    c.visc_diss = visc_diss
    c.root_rtol = root_rtol
    return c


# ---- the C ABI under the same names -------------------------------------------------------

def es_create(cfg):
    ctx = ctypes.c_void_p()
    _check(load().es_create(ctypes.byref(cfg), ctypes.byref(ctx)), "es_create")
    return ctx


def es_destroy(ctx):
    load().es_destroy(ctx)


def es_rhs(ctx, q, dqdt, E_elem=None, stream=None):
    _check(load().es_rhs(ctx, _ptr(q), _ptr(dqdt), _ptr(E_elem), _stream(stream)), "es_rhs")


def es_entropy(ctx, q, eta_elem, stream=None):
    _check(load().es_entropy(ctx, _ptr(q), _ptr(eta_elem), _stream(stream)), "es_entropy")


def es_set_boundary(ctx, direction, kind, params=None):
    """params: host sequence of doubles (10 for ES_BC_STATE, 4 for ES_BC_VISCOUS_SHOCK)."""
    n = 0 if params is None else len(params)
    buf = (ctypes.c_double * max(n, 1))(*([] if params is None else [float(v) for v in params]))
    _check(load().es_set_boundary(ctx, int(direction), int(kind), ctypes.cast(buf, ctypes.c_void_p) if n else None, n),
           "es_set_boundary")


def es_set_time(ctx, t):
    _check(load().es_set_time(ctx, float(t)), "es_set_time")


def _tableau_arrays(A, b, c):
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    s = b.size
    if A.shape != (s, s) or c.size != s:
        raise ValueError("tableau shapes: A (s, s), b (s,), c (s,)")
    return s, A, b, c


def es_set_tableau(ctx, A, b, c):
    """A (s x s, strictly lower triangular), b, c: host sequences of floats."""
    s, A, b, c = _tableau_arrays(A, b, c)
    _check(load().es_set_tableau(ctx, s, A.ctypes.data, b.ctypes.data, c.ctypes.data), "es_set_tableau")


def es_batch_set_tableau(batch, A, b, c):
    s, A, b, c = _tableau_arrays(A, b, c)
    _check(load().es_batch_set_tableau(batch, s, A.ctypes.data, b.ctypes.data, c.ctypes.data),
           "es_batch_set_tableau")


def es_relax_step(ctx, u_old, u_new, d_eta, gamma_elem, gamma, u_out, stream=None):
    _check(load().es_relax_step(ctx, _ptr(u_old), _ptr(u_new), _ptr(d_eta), _ptr(gamma_elem), _ptr(gamma),
                                _ptr(u_out), _stream(stream)), "es_relax_step")


def es_advance(ctx, q, nsteps, dt, t, gamma_hist=None, gamma_elem=None, stream=None):
    _check(load().es_advance(ctx, _ptr(q), int(nsteps), float(dt), _ptr(t), _ptr(gamma_hist), _ptr(gamma_elem),
                             _stream(stream)), "es_advance")


def es_step_estimate(ctx, q, dt, t=None, gamma=None, gamma_elem=None, eta_old=None, deta=None, eta_new=None,
                     stream=None):
    _check(load().es_step_estimate(ctx, _ptr(q), float(dt), _ptr(t), _ptr(gamma), _ptr(gamma_elem), _ptr(eta_old),
                                   _ptr(deta), _ptr(eta_new), _stream(stream)), "es_step_estimate")


def es_advance_host(ctx, q_host, nsteps, dt, t_host, gamma_hist_host=None, stream=None):
    _check(load().es_advance_host(ctx, _ptr(q_host), int(nsteps), float(dt), _ptr(t_host), _ptr(gamma_hist_host),
                                  _stream(stream)), "es_advance_host")


def es_node_coords(ctx, xyz_host):
    _check(load().es_node_coords(ctx, _ptr(xyz_host)), "es_node_coords")


def es_status(ctx, stream=None):
    return load().es_status(ctx, _stream(stream))


def es_launch_count(ctx):
    return int(load().es_launch_count(ctx))


def es_strerror(code):
    return strerror(code)


def es_profile_enable(ctx, enable):
    _check(load().es_profile_enable(ctx, int(bool(enable))), "es_profile_enable")


def es_profile_read(ctx):
    """{kind: (ms, launches)} since the last read."""
    import numpy as np
    ms = np.zeros(len(KERNEL_KINDS))
    n = np.zeros(len(KERNEL_KINDS), dtype=np.int64)
    _check(load().es_profile_read(ctx, _ptr(ms), _ptr(n)), "es_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def es_rhs_noalloc(cfg, q, dqdt, E_elem=None, stream=None):
    """Right-hand side through the allocation-free entry point (no context)."""
    _check(load().es_rhs_noalloc(ctypes.byref(cfg), _ptr(q), _ptr(dqdt), _ptr(E_elem), _stream(stream)),
           "es_rhs_noalloc")


def es_rhs_noalloc_scratch_bytes(cfg):
    return int(load().es_rhs_noalloc_scratch_bytes(ctypes.byref(cfg)))


def es_volume_variant(ctx):
    return int(load().es_volume_variant(ctx))


def es_set_volume_variant(ctx, variant):
    _check(load().es_set_volume_variant(ctx, int(variant)), "es_set_volume_variant")


def es_autotune(ctx, q, stream=None):
    _check(load().es_autotune(ctx, _ptr(q), _stream(stream)), "es_autotune")


# ---- batches ---------------------------------------------------------------------------------

def es_batch_create(cfgs):
    arr = (es_config * len(cfgs))(*cfgs)
    b = ctypes.c_void_p()
    _check(load().es_batch_create(arr, len(cfgs), ctypes.byref(b)), "es_batch_create")
    return b


def es_batch_destroy(b):
    load().es_batch_destroy(b)


def es_batch_nodes(b, inst=-1):
    return int(load().es_batch_nodes(b, int(inst)))


def es_batch_node_coords(b, inst, xyz_host):
    _check(load().es_batch_node_coords(b, int(inst), _ptr(xyz_host)), "es_batch_node_coords")


def es_batch_set_state(b, inst, q_host):
    _check(load().es_batch_set_state(b, int(inst), _ptr(q_host)), "es_batch_set_state")


def es_batch_get_state(b, inst, q_host):
    _check(load().es_batch_get_state(b, int(inst), _ptr(q_host)), "es_batch_get_state")


def es_batch_set_dt(b, dt_host):
    _check(load().es_batch_set_dt(b, _ptr(dt_host)), "es_batch_set_dt")


def es_batch_autotune(b, stream=None):
    _check(load().es_batch_autotune(b, _stream(stream)), "es_batch_autotune")


def es_batch_volume_variant(b, inst):
    return int(load().es_batch_volume_variant(b, int(inst)))


def es_batch_advance(b, nsteps, stream=None):
    _check(load().es_batch_advance(b, int(nsteps), _stream(stream)), "es_batch_advance")


def es_batch_step_estimate(b, stream=None):
    _check(load().es_batch_step_estimate(b, _stream(stream)), "es_batch_step_estimate")


def es_batch_get_estimate(b, inst, eta_old_host=None, deta_host=None, eta_new_host=None, gamma_elem_host=None):
    _check(load().es_batch_get_estimate(b, int(inst), _ptr(eta_old_host), _ptr(deta_host), _ptr(eta_new_host),
                                        _ptr(gamma_elem_host)), "es_batch_get_estimate")


def es_batch_times(b, t_host=None, gamma_host=None):
    _check(load().es_batch_times(b, _ptr(t_host), _ptr(gamma_host)), "es_batch_times")


def es_batch_status(b, stream=None):
    return load().es_batch_status(b, _stream(stream))


def es_batch_launch_count(b):
    return int(load().es_batch_launch_count(b))


def es_fma_peak(fp64, stream=None):
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 if fp64 else FP32)."""
    out = ctypes.c_double(0.0)
    _check(load().es_fma_peak(int(bool(fp64)), ctypes.byref(out), _stream(stream)), "es_fma_peak")
    return out.value


def es_reciprocal(x, out, stream=None):
    _check(load().es_reciprocal(_ptr(x), _ptr(out), int(x.numel()), _stream(stream)), "es_reciprocal")
