"""Closed-form initial / exact states at physical points x of shape (n, 3).

Each function returns conserved variables (rho, rho u, rho v, rho w, E) of
shape (n, 5).  They are inputs, not part of the FR method.
"""
import numpy as np


def _cons(rho, u, v, w, p, gamma):
    out = np.empty(np.shape(rho) + (5,))
    out[..., 0] = rho
    out[..., 1] = rho * u
    out[..., 2] = rho * v
    out[..., 3] = rho * w
    out[..., 4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return out


def isentropic_vortex(x, t=0.0, gamma=1.4, beta=5.0, centre=(5.0, 5.0),
                      period=10.0, adv=(1.0, 1.0)):
    """Isentropic vortex in the xy plane, extruded along z, advected by
    ``adv``; the exact solution at time t is the initial one shifted by
    adv * t (taken modulo the period, nearest image)."""
    dx = x[:, 0] - centre[0] - adv[0] * t
    dy = x[:, 1] - centre[1] - adv[1] * t
    dx = dx - period * np.round(dx / period)
    dy = dy - period * np.round(dy / period)
    r2 = dx * dx + dy * dy
    e = np.exp(0.5 * (1.0 - r2))
    u = adv[0] - beta / (2 * np.pi) * dy * e
    v = adv[1] + beta / (2 * np.pi) * dx * e
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8 * gamma * np.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _cons(rho, u, v, np.zeros_like(u), p, gamma)


def taylor_green(x, mach=0.1, gamma=1.4):
    """Taylor-Green vortex: u = sin x cos y cos z, v = -cos x sin y cos z,
    p = p0 + (cos 2x + cos 2y)(2 + cos 2z)/16, rho = p / p0,
    p0 = 1 / (gamma Ma^2)."""
    p0 = 1.0 / (gamma * mach ** 2)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (2 + np.cos(2 * Z)) / 16.0
    rho = p / p0
    return _cons(rho, u, v, np.zeros_like(u), p, gamma)


def flow3d(x, mach=0.3, gamma=1.4):
    """Smooth, fully three-dimensional state, periodic on the unit box: the
    Taylor-Green velocity of X = 2 pi x plus w = sin(X + 0.3) cos Y
    sin(Z + 0.7) / 2, density 1 + sin(X + Y) cos Z / 10 and pressure
    p0 (1 + cos X cos(Y + Z) / 20), p0 = 1 / (gamma Ma^2).  Every conserved
    variable varies in all three directions, so no component of a
    right-hand side vanishes by symmetry."""
    p0 = 1.0 / (gamma * mach ** 2)
    X, Y, Z = (2 * np.pi * x[:, k] for k in range(3))
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = 0.5 * np.sin(X + 0.3) * np.cos(Y) * np.sin(Z + 0.7)
    rho = 1.0 + 0.1 * np.sin(X + Y) * np.cos(Z)
    p = p0 * (1.0 + 0.05 * np.cos(X) * np.cos(Y + Z))
    return _cons(rho, u, v, w, p, gamma)


def perturbed_uniform(x, mach=0.2, gamma=1.4, amp=0.05, nmodes=4, kmax=3,
                      seed=20240829):
    """rho = 1, p = 1/(gamma Ma^2), velocity (1,0,0) plus ``amp`` times the
    mean of ``nmodes`` seeded Fourier modes a_m sin(2 pi k_m . x + phi_m)
    with integer wave vectors |k_m| <= kmax and unit directions a_m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vel = np.zeros((len(x), 3))
    vel[:, 0] = 1.0
    m = 0
    while m < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not 0 < np.linalg.norm(k) <= kmax:
            continue
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        phi = rng.uniform(0, 2 * np.pi)
        vel += (amp / nmodes) * np.outer(np.sin(2 * np.pi * x @ k + phi), a)
        m += 1
    rho = np.ones(len(x))
    p = np.full(len(x), 1.0 / (gamma * mach ** 2))
    return _cons(rho, vel[:, 0], vel[:, 1], vel[:, 2], p, gamma)


SHU_OSHER_POST = (3.857142857, 2.629369, 10.33333)


def shu_osher(x, gamma=1.4, x_shock=-4.0):
    """Mach 3 shock at x_shock moving into rho = 1 + 0.2 sin(5x), u = 0,
    p = 1; post-shock state (3.857142857, 2.629369, 10.33333)."""
    X = x[:, 0]
    post = X < x_shock
    rho = np.where(post, SHU_OSHER_POST[0], 1.0 + 0.2 * np.sin(5.0 * X))
    u = np.where(post, SHU_OSHER_POST[1], 0.0)
    p = np.where(post, SHU_OSHER_POST[2], 1.0)
    z = np.zeros_like(X)
    return _cons(rho, u, z, z, p, gamma)


def shear(x, p0=1.0, gamma=1.4):
    """Steady shear u = (y, 0, 0), rho = 1, p = p0 (exact steady Euler
    solution; with viscosity mu its energy equation gains +mu)."""
    y = x[:, 1]
    one = np.ones_like(y)
    return _cons(one, y, 0 * y, 0 * y, p0 * one, gamma)


def uniform(x, rho=1.0, vel=(0.3, -0.2, 0.5), p=1.0, gamma=1.4):
    one = np.ones(len(x))
    return _cons(rho * one, vel[0] * one, vel[1] * one, vel[2] * one,
                 p * one, gamma)
