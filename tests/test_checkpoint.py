"""Checkpoint / resume: the file format round-trips (CPU) and a resumed run is
bit-identical to an uninterrupted one (GPU)."""
import numpy as np
import pytest

from paper_2003_08831_gb300 import inputs
from paper_2003_08831_gb300.solver import load_checkpoint, save_checkpoint


def test_checkpoint_file_round_trip(tmp_path):
    q = np.random.default_rng(0).normal(size=(5, 12, 27))
    meta = {"t": 0.125, "step": 7, "dt": 1e-3, "config": {"p": 2}}
    path = str(tmp_path / "ck.bin")
    save_checkpoint(path, q, meta)
    q2, h = load_checkpoint(path)
    assert np.array_equal(q, q2)
    assert h["step"] == 7 and h["t"] == 0.125 and h["config"]["p"] == 2
    with open(path, "r+b") as f:          # a truncated file is rejected
        f.truncate(100)
    with pytest.raises(ValueError):
        load_checkpoint(path)


@pytest.mark.gpu
@pytest.mark.parametrize("tableau", [None, "RK65"])
def test_resume_is_bit_identical(tmp_path, tableau):
    """Also with a tableau loaded through set_tableau, which the checkpoint carries."""
    import torch

    from oracle import rk

    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_08831_gb300.solver import Solver, stable_dt
    lo, hi = (0.0, 0.0, 0.0), (10.0, 10.0, 10.0)
    s = Solver(3, (4, 3, 5), lo, hi)
    if tableau:
        tab = rk.TABLEAUX[tableau]
        s.set_tableau(tab["A"], tab["b"], tab["c"])
    xyz = s.coords()
    q0 = inputs.vortex_state(xyz[0], xyz[1], 0.0, centre=(5.0, 5.0), period=10.0)
    dt = stable_dt(q0, 3, [2.5, 10 / 3, 2.0], 0.5)
    q = s.to_device(q0)
    t, _, _ = s.advance(q, 10, dt)
    full = q.cpu().numpy()
    q = s.to_device(q0)
    t1, _, _ = s.advance(q, 4, dt)
    path = str(tmp_path / "ck.bin")
    s.checkpoint(path, q, t1.item(), 4, dt)
    s.close()
    s2, q2, tr, step, dt2 = Solver.resume(path)
    assert step == 4 and dt2 == dt
    t2 = torch.tensor([tr], dtype=torch.float64, device="cuda")
    s2.advance(q2, 6, dt2, t2)
    assert np.array_equal(q2.cpu().numpy(), full)
    assert t2.item() == t.item()
    s2.close()
