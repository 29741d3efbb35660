"""Stencil operators of the benchmark workloads as library descriptors.

Each function returns a list of terms ``(dx, dy, dz, in, coef, out, w)``
for ``binding.do_all`` / ``binding.do_reduce`` (Section 3: fixed-offset reads
around the core element, writes at the core element, optional returned
value, which is how Section 5.2 fuses the sweep and the convergence test).
"""
from __future__ import annotations

VALUE, NONE = 254, 255

X6 = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
X4 = X6[:4]


def jacobi5_2d():
    """2D Jacobi averaging for Laplace: u' = (u(i+-1, j) + u(i, j+-1)) / 4."""
    return [(dx, dy, 0, 0, NONE, 0, 0.25) for dx, dy, _ in X4]


def difference():
    """Returned value u_a - u_b (inputs 0, 1): the infinity-norm convergence test."""
    return [(0, 0, 0, 0, NONE, VALUE, 1.0), (0, 0, 0, 1, NONE, VALUE, -1.0)]


def heat7(lam, with_f=True):
    """Damped Jacobi / heat sweep u' = (1 - 6 lam) u + lam (sum6 + f): one FMA per input."""
    t = [(0, 0, 0, 0, NONE, 0, 1.0 - 6.0 * lam)]
    t += [(dx, dy, dz, 0, NONE, 0, lam) for dx, dy, dz in X6]
    if with_f:
        t.append((0, 0, 0, 1, NONE, 0, lam))
    return t


def heat7_fused(lam, with_f=True):
    """The same sweep fused with its residual: value r = sum6 - 6u (+ f), u' = u + lam r."""
    t = [(dx, dy, dz, 0, NONE, VALUE, 1.0) for dx, dy, dz in X6]
    t.append((0, 0, 0, 0, NONE, VALUE, -6.0))
    if with_f:
        t.append((0, 0, 0, 1, NONE, VALUE, 1.0))
    t += [(0, 0, 0, 0, NONE, 0, 1.0), (0, 0, 0, VALUE, NONE, 0, lam)]
    return t


def residual7():
    """Returned value r = f - A u = sum6 - 6u + f (inputs 0 = u, 1 = f)."""
    t = [(dx, dy, dz, 0, NONE, VALUE, 1.0) for dx, dy, dz in X6]
    return t + [(0, 0, 0, 0, NONE, VALUE, -6.0), (0, 0, 0, 1, NONE, VALUE, 1.0)]


def poisson_jacobi():
    """Poisson Jacobi u' = (sum6 + f) / 6 (inputs 0 = u, 1 = f)."""
    return [(dx, dy, dz, 0, NONE, 0, 1.0 / 6.0) for dx, dy, dz in X6] + [(0, 0, 0, 1, NONE, 0, 1.0 / 6.0)]


def poisson_sor(omega):
    """SOR update of the Poisson equation 6u - sum6 = f in place, for red-black
    colouring: u' = (1 - omega) u + omega (sum6 + f) / 6 (inputs 0 = u,
    1 = f); omega = 1 is Gauss-Seidel, the Jacobi operator applied per colour."""
    if omega == 1.0:
        return poisson_jacobi()
    return ([(0, 0, 0, 0, NONE, 0, 1.0 - omega)] + [(dx, dy, dz, 0, NONE, 0, omega / 6.0) for dx, dy, dz in X6]
            + [(0, 0, 0, 1, NONE, 0, omega / 6.0)])


def fig1b():
    """The operator printed in Fig. 1b: v = (6 u - sum6) / 36."""
    return [(0, 0, 0, 0, NONE, 0, 6.0 / 36.0)] + [(dx, dy, dz, 0, NONE, 0, -1.0 / 36.0) for dx, dy, dz in X6]


# 13-point biharmonic (centre 20, axial-1 -8, diagonal 2, axial-2 1)
_BIHARM = ([((0, 0), 20.0)] + [((a, b), -8.0) for a, b in ((1, 0), (-1, 0), (0, 1), (0, -1))]
           + [((a, b), 2.0) for a, b in ((1, 1), (1, -1), (-1, 1), (-1, -1))]
           + [((a, b), 1.0) for a, b in ((2, 0), (-2, 0), (0, 2), (0, -2))])


def climate(dt=1.0, dz=1.0):
    """Inputs q0, q1, q2, kappa, w, t0, t1, t2 -> outputs q0', q1', q2':
    q' = q + dt (-kappa D4h(q) - w (q(k+1) - q(k-1)) / (2 dz) + t)."""
    terms = []
    for m in range(3):
        terms.append((0, 0, 0, m, NONE, m, 1.0))
        terms += [(a, b, 0, m, 3, m, -dt * c) for (a, b), c in _BIHARM]
        terms.append((0, 0, 1, m, 4, m, -dt / (2.0 * dz)))
        terms.append((0, 0, -1, m, 4, m, dt / (2.0 * dz)))
        terms.append((0, 0, 0, 5 + m, NONE, m, dt))
    return terms
