"""Analysis models (Sec. 3 and Appendix B of arXiv 2408.15115): the Clift-
Gauvin terminal velocity against its force balance and the Stokes limit, the
Basset-Boussinesq-Oseen and Feuillebois-Lasek integrators against their exact
Laplace-transform solutions (first-order convergence in dt), and the
frequency estimator on a synthetic oscillation."""
import math

import numpy as np

from paper_2408_15115_gb300 import analysis as A


def test_cg71_terminal_velocity_balance_and_stokes_limit():
    d, nu, kappa = 8.0, 0.05, 2.5
    for g in (1e-7, 1e-5, 1e-4):
        v = A.cg71_terminal_velocity(d, nu, kappa, g)
        weight = (kappa - 1.0) * math.pi * d ** 3 / 6.0 * g
        drag = A.cg71_cd(v * d / nu) * math.pi * d * d / 8.0 * v * v
        assert abs(drag / weight - 1.0) < 1e-10
    # Re ~ 0.01: Stokes, v = (kappa - 1) g d^2 / (18 nu) up to the 0.15 Re^0.687 correction
    g = 1e-7
    v = A.cg71_terminal_velocity(d, nu, kappa, g)
    vs = (kappa - 1.0) * g * d * d / (18.0 * nu)
    re = v * d / nu
    assert re < 0.01
    assert abs(v / vs - 1.0 / (1.0 + 0.15 * re ** 0.687)) < 1e-3


def test_bbo_exact_solution_limits():
    r, nu, kappa, G = 4.0, 0.05, 2.5, 1.5e-5
    uT = A.stokes_terminal_velocity(r, nu, G)
    t = np.array([1e-6, 1e5, 1e14])
    u = A.bbo_settling_exact(r, nu, kappa, G, t)
    # from rest the initial acceleration is G / (kappa + 1/2); at long times u -> uT
    assert abs(u[0] / (G / (kappa + 0.5) * 1e-6) - 1.0) < 1e-2
    assert abs(u[2] / uT - 1.0) < 1e-5 and u[1] < u[2]  # the Basset tail decays as t^(-1/2)


def test_bbo_integrator_converges_to_exact_solution():
    r, nu, kappa, G = 4.0, 0.05, 2.5, 1.5e-5
    uT = A.stokes_terminal_velocity(r, nu, G)
    errs = []
    for dt in (1.0, 0.5, 0.25):
        t, u = A.bbo_settling(r, nu, kappa, G, 600.0, dt)
        ue = A.bbo_settling_exact(r, nu, kappa, G, t)
        errs.append(np.abs(u - ue).max() / uT)
    assert errs[-1] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4  # first order
    # without the history force: the exponential approach
    t, u = A.bbo_settling(r, nu, kappa, G, 600.0, 0.05, history=False)
    tau = (kappa + 0.5) * r * r / (4.5 * nu)
    assert np.abs(u - uT * (1.0 - np.exp(-t / tau))).max() / uT < 1e-3
    # the history force slows the approach
    t, uh = A.bbo_settling(r, nu, kappa, G, 600.0, 0.25)
    assert np.all(uh[1:] < u[::5][1:] + 1e-15)


def test_fl78_integrator_converges_to_exact_solution():
    r, nu, kappa, T = 4.0, 0.05, 2.5, 1e-3
    wT = T / (8.0 * math.pi * nu * r ** 3)
    errs = []
    for dt in (2.0, 1.0, 0.5):
        t, w = A.fl78_rotation(r, nu, kappa, T, 400.0, dt, quad=16)
        we = A.fl78_rotation_exact(r, nu, kappa, T, t)
        errs.append(np.abs(w - we).max() / wT)
    assert errs[-1] < 5e-3
    assert 1.5 < errs[0] / errs[1] < 2.5 and 1.5 < errs[1] / errs[2] < 2.5
    # exact solution: initial angular acceleration T / I, terminal value T / (8 pi nu r^3)
    I = 0.4 * kappa * 4.0 / 3.0 * math.pi * r ** 5
    we = A.fl78_rotation_exact(r, nu, kappa, T, np.array([1e-6, 1e14]))
    assert abs(we[0] / (T / I * 1e-6) - 1.0) < 1e-2
    assert abs(we[1] / wT - 1.0) < 1e-3
    # without history terms: exponential with time constant I / (8 pi nu r^3)
    t, w = A.fl78_rotation(r, nu, kappa, T, 400.0, 0.05, history=False)
    tc = I / (8.0 * math.pi * nu * r ** 3)
    assert np.abs(w - wT * (1.0 - np.exp(-t / tc))).max() / wT < 1e-3


def test_oscillation_frequency_of_a_synthetic_signal():
    t = np.arange(4000) * 0.7
    f0 = 0.013 / 0.7 * 1.37  # not on an FFT bin
    x = 0.3 * np.sin(2 * math.pi * f0 * t + 0.4) + 1e-4 * t + 2.0
    f = A.oscillation_frequency(t, x)
    assert abs(f / f0 - 1.0) < 2e-3
    assert abs(A.strouhal(f, 8.0, 0.02) - f * 8.0 / 0.02) < 1e-15


def test_fl78_with_a_given_inertia():
    # `inertia` replaces 2 m r^2 / 5 (a body whose hydrodynamic radius differs
    # from its mass distribution's): the default value reproduces the default
    # solution, and the initial angular acceleration is T / I for any I
    r, nu, kappa, T = 4.0, 0.05, 2.5, 1e-3
    I0 = 0.4 * kappa * 4.0 / 3.0 * math.pi * r ** 5
    t = np.array([1e-6, 10.0, 100.0, 1000.0])
    assert np.allclose(A.fl78_rotation_exact(r, nu, kappa, T, t, inertia=I0),
                       A.fl78_rotation_exact(r, nu, kappa, T, t), rtol=1e-9, atol=0.0)
    for I in (0.5 * I0, 3.0 * I0):
        w = A.fl78_rotation_exact(r, nu, kappa, T, np.array([1e-6]), inertia=I)
        assert abs(w[0] / (T / I * 1e-6) - 1.0) < 1e-2
        # the integrator agrees with the exact solution for the same inertia
        tt, wn = A.fl78_rotation(r, nu, kappa, T, 200.0, 0.25, quad=16, inertia=I)
        we = A.fl78_rotation_exact(r, nu, kappa, T, tt, inertia=I)
        assert np.abs(wn - we).max() < 1e-2 * T / (8.0 * math.pi * nu * r ** 3)
