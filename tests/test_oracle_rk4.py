"""Pins for the oracle's Lorenz hyperchaotic iteration (Eq. (1), RK4 reading).

* the origin is an equilibrium of Eq. (1): RK4 must keep it exactly;
* on the invariant z-axis Eq. (1) reduces to z' = -beta z, where one RK4 step
  is multiplication by the degree-4 Taylor polynomial of exp(-beta h);
* against an independent high-accuracy integrator (scipy DOP853), the error is
  O(h^4): halving h divides it by about 16.  A dropped term, wrong sign or
  swapped variable in Eq. (1), or a wrong RK4 weight, breaks one of these.
* a Python-float transcription with the same operation order is bit-identical
  (this one only detects fused multiply-add contraction in the C build)."""
import math

import numpy as np
import pytest

import oracle

SIGMA, RHO, BETA = 10.0, 28.0, 8.0 / 3.0


def rhs(t, s, gamma):
    x, y, z, w = s
    return [SIGMA * (y - x) + w, RHO * x - y - x * z, x * y - BETA * z, -y * z + gamma * w]


def test_origin_is_fixed():
    s = oracle.rk4_trajectory([0.0, 0.0, 0.0, 0.0], -1.0, 100)
    assert np.all(s == 0.0)


@pytest.mark.parametrize("z0", [1.0, 37.5, 1e-3])
@pytest.mark.parametrize("h", [0.001, 0.01, 0.1])
def test_z_axis_reduces_to_linear_decay(z0, h):
    s = oracle.rk4_step([0.0, 0.0, z0, 0.0], -0.7, h)
    assert s[0] == 0.0 and s[1] == 0.0 and s[3] == 0.0
    a = -BETA * h
    expect = z0 * (1 + a + a * a / 2 + a ** 3 / 6 + a ** 4 / 24)
    assert abs(s[2] - expect) <= 8 * math.ulp(expect)


def test_fourth_order_convergence_against_dop853():
    scipy_integrate = pytest.importorskip("scipy.integrate")
    gamma = -1.0
    s0 = np.array([1.3, -2.2, 18.0, 4.5])
    T = 0.04
    ref = scipy_integrate.solve_ivp(rhs, (0.0, T), s0, method="DOP853", rtol=1e-13, atol=1e-13, args=(gamma,)).y[:, -1]
    errs = []
    for h in (0.004, 0.002, 0.001):
        steps = int(round(T / h))
        s = oracle.rk4_trajectory(s0, gamma, steps, h)[-1]
        errs.append(np.max(np.abs(s - ref)))
    assert errs[-1] < 1e-9
    for a, b in zip(errs, errs[1:]):
        assert 10.0 < a / b < 24.0, errs


def test_every_term_of_eq1_matters():
    # Near-zero error against DOP853 for the true field, large error for a
    # field with any one term removed: the oracle integrates Eq. (1) itself.
    scipy_integrate = pytest.importorskip("scipy.integrate")
    gamma = -0.5
    s0 = np.array([2.0, 3.0, 15.0, -6.0])
    T = 0.05
    got = oracle.rk4_trajectory(s0, gamma, 50, 0.001)[-1]

    def solve(f):
        return scipy_integrate.solve_ivp(f, (0.0, T), s0, method="DOP853", rtol=1e-12, atol=1e-12).y[:, -1]

    assert np.max(np.abs(got - solve(lambda t, s: rhs(t, s, gamma)))) < 1e-9
    mutants = [
        lambda t, s: [SIGMA * (s[1] - s[0]), RHO * s[0] - s[1] - s[0] * s[2], s[0] * s[1] - BETA * s[2], -s[1] * s[2] + gamma * s[3]],
        lambda t, s: [SIGMA * (s[1] - s[0]) + s[3], RHO * s[0] - s[1] + s[0] * s[2], s[0] * s[1] - BETA * s[2], -s[1] * s[2] + gamma * s[3]],
        lambda t, s: [SIGMA * (s[1] - s[0]) + s[3], RHO * s[0] - s[1] - s[0] * s[2], s[0] * s[3] - BETA * s[2], -s[1] * s[2] + gamma * s[3]],
        lambda t, s: [SIGMA * (s[1] - s[0]) + s[3], RHO * s[0] - s[1] - s[0] * s[2], s[0] * s[1] - BETA * s[2], s[1] * s[2] + gamma * s[3]],
    ]
    for m in mutants:
        assert np.max(np.abs(got - solve(m))) > 1e-4


def _py_rk4(s, gamma, h):
    # Same operation order as the oracle (contraction detector only).
    def f(x, y, z, w):
        return (SIGMA * (y - x) + w, (RHO * x - y) - x * z, x * y - BETA * z, gamma * w - y * z)
    hh, h6 = h / 2.0, h / 6.0
    k1 = f(*s)
    k2 = f(*[s[v] + hh * k1[v] for v in range(4)])
    k3 = f(*[s[v] + hh * k2[v] for v in range(4)])
    k4 = f(*[s[v] + h * k3[v] for v in range(4)])
    return [s[v] + h6 * (((k1[v] + 2.0 * k2[v]) + 2.0 * k3[v]) + k4[v]) for v in range(4)]


def test_no_fma_contraction_in_build():
    s = [7.123456789, -3.3, 21.5, 1.25]
    gamma = -1.1
    traj = oracle.rk4_trajectory(s, gamma, 2000, 0.001)
    for t in range(2000):
        s = _py_rk4(s, gamma, 0.001)
        assert list(traj[t]) == s, t


def test_trajectories_stay_bounded():
    import synth_inputs as si
    for seed in range(6):
        ic = oracle.key_to_ic(si.key(seed))
        traj = oracle.rk4_trajectory(ic[:4], ic[4], 20000)
        assert np.all(np.isfinite(traj))
        assert np.max(np.abs(traj)) < 1e3
