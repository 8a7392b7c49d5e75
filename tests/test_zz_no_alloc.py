"""The allocation-free right-hand side (es_rhs_noalloc) against es_rhs.

es_rhs_noalloc serves callers that cannot allocate device memory: it takes
only inputs and outputs and keeps its scratch in a fixed array compiled into
the library.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process
as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_08831_gb300 import _binding as B
from paper_2003_08831_gb300 import inputs

TOL = 1e-12


def test_scratch_size_limit_is_checked_on_the_host():
    """Sizes beyond the fixed scratch are rejected before any GPU work (no GPU needed)."""
    import __graft_entry__
    __graft_entry__.build()
    lib = B.load()
    small = B.make_config(3, (4, 4, 4))
    big = B.make_config(5, (40, 40, 40), mu=0.01)
    assert 0 < B.es_rhs_noalloc_scratch_bytes(small) <= 32 * 1024 * 1024
    assert B.es_rhs_noalloc_scratch_bytes(big) > 32 * 1024 * 1024
    rc = lib.es_rhs_noalloc(ctypes.byref(big), ctypes.c_void_p(16), ctypes.c_void_p(32), None, None)
    assert rc == B.ES_ERR_TOO_LARGE
    assert "scratch" in B.strerror(rc)


@pytest.mark.gpu
@pytest.mark.parametrize("p,n,mu,precision,visc", [(3, (5, 4, 3), 0.0, 0, 0.0), (4, (3, 3, 4), 0.01, 0, 0.0),
                                                   (3, (4, 3, 5), 0.0, 1, 0.0), (4, (3, 4, 3), 0.01, 3, 0.0),
                                                   (2, (3, 4, 3), 0.02, 0, 0.5), (3, (4, 5, 3), 0.01, 2, 0.0)])
def test_rhs_noalloc_matches_es_rhs_on_two_calls(p, n, mu, precision, visc):
    """An ES_FP64X config (precision 2) runs on the FP64 kernels here, so its reference is
    es_rhs of an ES_FP64 context on the same mesh; the other modes compare with es_rhs of
    a context of the same precision."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_08831_gb300.solver import Solver
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    ref_precision = B.ES_FP64 if precision == B.ES_FP64X else precision
    s = Solver(p, n, lo, hi, mu=mu, precision=ref_precision, visc_diss=visc)
    xyz = s.coords()
    cfg = B.make_config(p, n, lo, hi, mu=mu, precision=precision, visc_diss=visc)
    rng = np.random.default_rng(p)
    for call in range(2):   # two calls in a row: the shared scratch keeps the last contents
        q0 = inputs.tgv_state(xyz[0] + 0.3 * call, xyz[1], xyz[2], mach=0.3)
        q0 = q0 * (1 + 1e-3 * rng.uniform(-1, 1, q0.shape))
        q = s.to_device(q0)
        ref, Eref = s.rhs(q, want_E=True)
        out = torch.full_like(ref, float("nan"))
        E = torch.full((s.K,), float("nan"), dtype=torch.float64, device="cuda")
        B.es_rhs_noalloc(cfg, q, out, E)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy().reshape(5, -1), ref.cpu().numpy().reshape(5, -1)
        scale = np.maximum(np.max(np.abs(b), axis=1), 1e-3 * np.max(np.abs(b)))
        assert np.all(np.max(np.abs(a - b), axis=1) <= TOL * scale)
        Ea, Eb = E.cpu().numpy(), Eref.cpu().numpy()
        assert np.all(np.abs(Ea - Eb) <= TOL * np.max(np.abs(Eb)))
    s.close()
