"""Analysis models used to read settling runs (host side, lattice or SI units,
rho_f = 1 unless stated).

* Clift & Gauvin (1971) drag curve (Eq. 28) and the terminal velocity it
  gives for a sphere, v_T^R (Sec. 3.1).
* The settling transient of a sphere from rest by the Basset-Boussinesq-Oseen
  equation (Appendix B, Eq. B.1): added mass, Stokes drag and the Basset
  history force, integrated with piecewise-linear velocity (the history
  integral of each interval is exact for a linear velocity), plus its exact
  solution for a constant driving force by Laplace transform.
* The angular velocity of a sphere under a constant torque by the Feuillebois
  & Lasek (1978) relation quoted in Appendix B (Eq. B.2), integrated the same
  way.
* The dominant oscillation frequency of a trajectory signal and the Strouhal
  number f d / v.
* The split of a surface force into pressure and viscous parts is computed on
  the GPU (query_particle_state: F, Fp).

Readings (the appendix is partly garbled): the driving term of Eq. B.1 is
passed in as an acceleration `g_drive` (with the buoyancy reading of the
step, (kappa - 1) g; with the printed form, kappa g), so B.1 reads
(kappa + 1/2) du/dt = g_drive - (9/2) nu u / r^2 - (9/2) sqrt(nu / pi) / r
int_0^t u'(s) (t - s)^(-1/2) ds.
"""
import math

import numpy as np


def cg71_cd(re):
    """Drag coefficient of a sphere at Reynolds number re (Eq. 28)."""
    return 24.0 / re * (1.0 + 0.15 * re ** 0.687) + 0.42 / (1.0 + 4.25e4 * re ** -1.16)


def cg71_terminal_velocity(d, nu, kappa, g):
    """Terminal velocity of a sphere of diameter d with the Eq. 28 drag:
    (kappa - 1) (pi d^3 / 6) g = C_D(Re) (pi d^2 / 8) v^2, Re = v d / nu,
    solved by bisection on log v (the residual is increasing in v)."""
    weight = (kappa - 1.0) * math.pi * d ** 3 / 6.0 * g

    def resid(v):
        return cg71_cd(v * d / nu) * math.pi * d * d / 8.0 * v * v - weight

    lo, hi = 1e-12, 1.0
    while resid(hi) < 0.0:
        hi *= 10.0
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if resid(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def _bbo_coeffs(r, nu, kappa):
    A = kappa + 0.5
    a = 4.5 * nu / (r * r)
    b = 4.5 * math.sqrt(nu / math.pi) / r
    return A, a, b


def bbo_settling(r, nu, kappa, g_drive, t_end, dt, history=True):
    """Velocity u(t_n), t_n = n dt, of a sphere of radius r released from rest
    under the driving acceleration g_drive, by Eq. B.1.  Each step is implicit
    in the new velocity: with u piecewise linear, the history integral up to
    t_{n+1} is sum_j (u_{j+1} - u_j) / dt * 2 (sqrt(t_{n+1} - t_j) -
    sqrt(t_{n+1} - t_{j+1})), whose last term holds the unknown u_{n+1}; the
    Stokes term is taken at t_{n+1}.  Returns (t, u)."""
    A, a, b = _bbo_coeffs(r, nu, kappa)
    n = int(round(t_end / dt))
    t = dt * np.arange(n + 1)
    u = np.zeros(n + 1)
    du = np.zeros(n)  # u_{j+1} - u_j
    c_last = 2.0 * math.sqrt(dt) / dt  # weight of du_n in the history integral at t_{n+1}
    for k in range(n):
        hist = 0.0
        if history and k > 0:
            tk = t[k + 1]
            j = np.arange(k)
            w = 2.0 * (np.sqrt(tk - t[j]) - np.sqrt(tk - t[j + 1])) / dt
            hist = float(np.dot(w, du[:k]))
        # A du/dt + a (u_k + du) + b (hist + c_last du) = g_drive
        bb = b if history else 0.0
        du[k] = (g_drive - a * u[k] - bb * hist) / (A / dt + a + bb * c_last)
        u[k + 1] = u[k] + du[k]
    return t, u


def bbo_settling_exact(r, nu, kappa, g_drive, t):
    """Exact solution of Eq. B.1 from rest for a constant driving force.  By
    Laplace transform U(s) = G / (s (A s + b sqrt(pi s) + a)); with
    A p^2 + b sqrt(pi) p + a = A (p + l1)(p + l2), p = sqrt(s), and
    L^-1[1 / (s (sqrt(s) + l))] = (1 - exp(l^2 t) erfc(l sqrt(t))) / l,
    u(t) = G / (A (l2 - l1)) [(1 - E(l1, t)) / l1 - (1 - E(l2, t)) / l2],
    E(l, t) = exp(l^2 t) erfc(l sqrt(t)) = w(i l sqrt(t)) (Faddeeva w; the
    roots may be complex)."""
    from scipy.special import wofz
    A, a, b = _bbo_coeffs(r, nu, kappa)
    disc = complex((b * math.sqrt(math.pi) / A) ** 2 - 4.0 * a / A)
    s = np.sqrt(disc)
    l1 = (b * math.sqrt(math.pi) / A - s) / 2.0
    l2 = (b * math.sqrt(math.pi) / A + s) / 2.0
    t = np.asarray(t, dtype=np.float64)
    rt = np.sqrt(t)
    E1 = wofz(1j * l1 * rt)
    E2 = wofz(1j * l2 * rt)
    u = g_drive / (A * (l2 - l1)) * ((1.0 - E1) / l1 - (1.0 - E2) / l2)
    return u.real


def stokes_terminal_velocity(r, nu, g_drive):
    """Terminal velocity of Eq. B.1: g_drive r^2 / (4.5 nu) (Stokes drag)."""
    return g_drive * r * r / (4.5 * nu)


def _fl78_coeffs(r, nu, kappa, inertia=None):
    m = kappa * 4.0 / 3.0 * math.pi * r ** 3
    I = 0.4 * m * r * r if inertia is None else float(inertia)
    c0 = 8.0 * math.pi * nu * r ** 3
    return I, c0, c0 * r / (3.0 * math.sqrt(math.pi * nu)), c0 / 3.0


def fl78_rotation(r, nu, kappa, torque, t_end, dt, quad=8, history=True, inertia=None):
    """Angular velocity w(t_n) of a sphere of radius r at rest under a
    constant torque (per unit fluid density), by the relation of Eq. B.2:
      I dw/dt = T - 8 pi nu r^3 w - 8 pi nu r^3 r / (3 sqrt(pi nu))
                int w'(s) (t - s)^(-1/2) ds
              + (8/3) pi nu r^3 int w'(s) exp(nu (t - s) / r^2)
                erfc(sqrt(nu (t - s) / r^2)) ds,
    I = 2 m r^2 / 5 with m = kappa (4/3) pi r^3 (rho_f = 1) unless `inertia`
    gives it (a body whose hydrodynamic radius r differs from the radius of
    its mass distribution).  Piecewise-linear
    w; the first history kernel is integrated exactly per interval, the
    second (bounded) one by Gauss-Legendre with `quad` nodes; implicit in the
    new angular velocity.  Terminal value T / (8 pi nu r^3).  Returns (t, w)."""
    from scipy.special import erfcx
    I, c0, c1, c2 = _fl78_coeffs(r, nu, kappa, inertia)
    if not history:
        c1 = c2 = 0.0
    xg, wg = np.polynomial.legendre.leggauss(quad)

    def k2(tau):  # exp(x) erfc(sqrt(x)), x = nu tau / r^2: erfcx(sqrt(x))
        return erfcx(np.sqrt(nu * np.maximum(tau, 0.0) / (r * r)))

    n = int(round(t_end / dt))
    t = dt * np.arange(n + 1)
    w = np.zeros(n + 1)
    dw = np.zeros(n)
    for k in range(n):
        tk = t[k + 1]
        # weights of dw_j / dt in both history integrals at t_{k+1}, j = 0..k
        j = np.arange(k + 1)
        wa = 2.0 * (np.sqrt(tk - t[j]) - np.sqrt(tk - t[j + 1])) / dt
        # int_{t_j}^{t_{j+1}} K2(tk - s) ds by Gauss-Legendre
        mid, half = 0.5 * (t[j] + t[j + 1]), 0.5 * dt
        s = mid[:, None] + half * xg[None, :]
        wb = (k2(tk - s) * wg[None, :]).sum(1) * half / dt
        h_old = c1 * float(np.dot(wa[:k], dw[:k])) - c2 * float(np.dot(wb[:k], dw[:k]))
        # I dw/dt + c0 (w_k + dw) + h_old + (c1 wa_k - c2 wb_k) dw = T
        dw[k] = (torque - c0 * w[k] - h_old) / (I / dt + c0 + c1 * wa[k] - c2 * wb[k])
        w[k + 1] = w[k] + dw[k]
    return t, w


def fl78_rotation_exact(r, nu, kappa, torque, t, inertia=None):
    """Exact solution of Eq. B.2 from rest for a constant torque.  With
    q = sqrt(nu) / r, L[exp(q^2 t) erfc(q sqrt(t))] = 1 / (sqrt(s)(sqrt(s) + q)),
    so W(s) = T (p + q) / (s P(p)), p = sqrt(s), with the cubic
    P(p) = (I p^2 + c1 sqrt(pi) p + c0)(p + q) - c2 p; by partial fractions over
    its roots p_i, w(t) = T sum_i R_i (1 - E(-p_i, t)) / (-p_i),
    R_i = (p_i + q) / P'(p_i), E(l, t) = exp(l^2 t) erfc(l sqrt(t)).
    `inertia` as in fl78_rotation."""
    from scipy.special import wofz
    I, c0, c1, c2 = _fl78_coeffs(r, nu, kappa, inertia)
    q = math.sqrt(nu) / r
    c1p = c1 * math.sqrt(math.pi)
    P = np.array([I, I * q + c1p, c1p * q + c0 - c2, c0 * q])
    roots = np.roots(P)
    dP = np.polyder(P)
    t = np.asarray(t, dtype=np.float64)
    rt = np.sqrt(t)
    w = np.zeros_like(t, dtype=complex)
    for pi_ in roots:
        R = (pi_ + q) / np.polyval(dP, pi_)
        lam = -pi_
        w += R * (1.0 - wofz(1j * lam * rt)) / lam
    return (torque * w).real


def oscillation_frequency(t, x):
    """Dominant frequency of a uniformly sampled signal x(t): the mean and
    linear trend removed, a Hann window, and the FFT magnitude peak refined by
    a parabola through the three bins around it (log magnitudes)."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    dt = (t[-1] - t[0]) / (n - 1)
    x = x - np.polyval(np.polyfit(t, x, 1), t)
    X = np.abs(np.fft.rfft(x * np.hanning(n)))
    k = int(np.argmax(X[1:])) + 1
    if 1 <= k < X.size - 1:
        y0, y1, y2 = np.log(X[k - 1] + 1e-300), np.log(X[k] + 1e-300), np.log(X[k + 1] + 1e-300)
        den = y0 - 2.0 * y1 + y2
        delta = 0.5 * (y0 - y2) / den if den != 0.0 else 0.0
    else:
        delta = 0.0
    return (k + delta) / (n * dt)


def strouhal(freq, d, v):
    """Strouhal number f d / v."""
    return freq * d / v
