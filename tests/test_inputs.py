"""Pins of the seeded synthetic input generators shared by the oracle and the CUDA path
(paper_2003_08831_gb300/inputs.py): they hold none of the method's arithmetic, but every
parity case starts from them.

* SplitMix64 (Steele, Lea & Flood 2014): the first outputs for seed 1234567 are the
  reference sequence printed with Vigna's reference implementation.
* Taylor--Green initial state: divergence-free velocity, and the pressure solves the
  incompressible pressure Poisson equation lap p = -rho0 div((v.grad) v) (rho0 = V0 = 1),
  checked by central differences at random points (a wrong factor or sign in the
  pressure leaves an O(1) residual).
* The seeded noise of the perturbed Taylor--Green state and the batch-instance draws:
  deterministic, within their stated ranges, and seed-dependent.
"""
import numpy as np

from paper_2003_08831_gb300 import inputs


def test_splitmix64_reference_sequence():
    out = inputs.splitmix64(1234567, np.arange(5, dtype=np.uint64))
    assert [int(v) for v in out] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                     4593380528125082431, 16408922859458223821]


def test_uniform_range_and_mean():
    u = inputs.uniform(inputs.SEED, np.arange(200000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1.0 / 12 / u.size)
    assert abs(np.var(u) - 1.0 / 12) < 2e-3


def _fd(f, X, k, h):
    e = np.zeros(3)
    e[k] = h
    return (f(*(X + e)) - f(*(X - e))) / (2 * h)


def test_tgv_divergence_free_and_pressure_poisson():
    rng = np.random.default_rng(4)
    h = 1e-3

    def vel(x, y, z):
        _, u, v, w, _ = inputs.tgv_primitives(np.array(x), np.array(y), np.array(z), mach=0.1)
        return np.array([u, v, w])

    def pres(x, y, z):
        return inputs.tgv_primitives(np.array(x), np.array(y), np.array(z), mach=0.1)[4]

    def conv(x, y, z):
        X = np.array([x, y, z])
        v = vel(*X)
        return sum(v[k] * _fd(vel, X, k, h) for k in range(3))

    for X in rng.uniform(0.0, 2 * np.pi, (40, 3)):
        div = sum(_fd(vel, X, k, h)[k] for k in range(3))
        assert abs(div) < 1e-9
        lap = sum((pres(*(X + h * np.eye(3)[k])) - 2 * pres(*X) + pres(*(X - h * np.eye(3)[k]))) / h ** 2
                  for k in range(3))
        divconv = sum(_fd(conv, X, k, h)[k] for k in range(3))
        assert abs(lap + divconv) < 1e-5 * max(1.0, abs(lap))


def test_tgv_mach_and_isothermal_start():
    x = np.linspace(0, 2 * np.pi, 7)
    rho, u, v, w, p = inputs.tgv_primitives(x, 0.3 * x, 0.7 * x, mach=0.1, gamma=1.4)
    p0 = 1.0 / (1.4 * 0.01)
    assert np.allclose(rho, p / p0) and np.all(w == 0.0)
    # the sound speed of the mean state is 1/Mach times the velocity scale V0 = 1
    assert np.isclose(np.sqrt(1.4 * p0 / 1.0), 10.0)


def test_perturbed_tgv_noise_bounded_and_seeded():
    rng = np.random.default_rng(1)
    x, y, z = (rng.uniform(0, 2 * np.pi, 5000) for _ in range(3))
    base = inputs.tgv_state(x, y, z)
    a = inputs.perturbed_tgv_state(x, y, z)
    assert np.array_equal(a, inputs.perturbed_tgv_state(x, y, z))
    assert not np.array_equal(a, inputs.perturbed_tgv_state(x, y, z, seed=inputs.SEED + 1))
    rel = a[0] / base[0] - 1.0
    assert np.max(np.abs(rel)) <= 1e-3 * (1 + 1e-12) and np.max(np.abs(rel)) > 9e-4
    dv = a[1:4] / a[0] - base[1:4] / base[0]
    assert np.max(np.abs(dv)) <= 1e-3 * (1 + 1e-9)
    assert abs(np.mean(rel)) < 5 * 1e-3 / np.sqrt(3 * rel.size)


def test_batch_instances_ranges():
    insts = inputs.batch_instances(256)
    assert insts == inputs.batch_instances(256)
    assert insts != inputs.batch_instances(256, seed=inputs.SEED + 1)
    ps = {d["p"] for d in insts}
    ns = [d["n"] for d in insts]
    assert ps == {2, 3, 4, 5}
    assert min(ns) >= 4 and max(ns) <= 12 and len(set(ns)) >= 6
    for d in insts:
        assert 3.0 <= d["eps"] <= 6.0 and 0.1 <= d["mach"] <= 0.5
        assert all(0.0 <= c <= d["box"] for c in d["centre"])
