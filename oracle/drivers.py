"""Oracle drivers for the five benchmark workloads, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).  Each driver writes its stencil
operator in the paper's terms (Section 3: fixed-offset reads around the core
element, writes only at the core element, an optional returned value) and runs
the iteration-space loop of Section 5.2: ``do_all`` into the second grid of a
ping-pong pair, swap, repeat, with ``do_reduce`` for the convergence measure.

The operators are the readings of the workloads stated in the design notes:

* 2D Jacobi averaging (Laplace):  u'(i,j) = 1/4 (sum of the 4 axial neighbours).
* 3D damped Jacobi / heat:        r = sum6(u) - 6u + f,  u' = u + lam * r.
* 4th-order horizontal diffusion with centred vertical advection, per field m:
      q_m' = q_m + dt * ( -kappa * D4h(q_m) - w * (q_m(k+1) - q_m(k-1)) / (2 dz) + t_m )
  with D4h the 13-point biharmonic (centre 20, axial-1 -8, diagonal 2, axial-2 1).
* Poisson Jacobi:                 u' = (sum6(u) + f) / 6, residual r = f - A u, A u = 6u - sum6(u).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

V, N = O.VALUE, O.NONE

AXIAL_2D = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
AXIAL_3D = AXIAL_2D + [(0, 0, 1), (0, 0, -1)]


def jacobi2d_terms():
    """u'(i,j) = 1/4 (u(i-1,j) + u(i+1,j) + u(i,j-1) + u(i,j+1)); input 0 = u, output 0 = u'."""
    return [(dx, dy, dz, 0, N, 0, 0.25) for dx, dy, dz in AXIAL_2D]


def difference_terms():
    """Returned value u_a(p) - u_b(p) for inputs (u_a, u_b): the convergence check of Section 5.2."""
    return [(0, 0, 0, 0, N, V, 1.0), (0, 0, 0, 1, N, V, -1.0)]


def fig1b_terms():
    """The operator printed in Fig. 1b: v = 1/36 (6 u - sum of the 6 axial neighbours)."""
    return [(0, 0, 0, 0, N, 0, 6.0 / 36.0)] + [(dx, dy, dz, 0, N, 0, -1.0 / 36.0)
                                                for dx, dy, dz in AXIAL_3D]


def heat_terms(lam, with_f=True):
    """Fused damped-Jacobi/heat operator: value r = sum6(u) - 6u (+ f); output u + lam * r.

    Inputs: 0 = u, 1 = f (when ``with_f``).  The value is the residual of the
    iterate being read, so a ``do_reduce`` with this operator both advances
    the grid and measures the residual in one scan (Section 5.2's fused
    diffusion + convergence).
    """
    t = [(dx, dy, dz, 0, N, V, 1.0) for dx, dy, dz in AXIAL_3D]
    t.append((0, 0, 0, 0, N, V, -6.0))
    if with_f:
        t.append((0, 0, 0, 1, N, V, 1.0))
    t.append((0, 0, 0, 0, N, 0, 1.0))
    t.append((0, 0, 0, V, N, 0, lam))
    return t


BIHARMONIC_13 = ([((0, 0), 20.0)]
                 + [((dx, dy), -8.0) for dx, dy in [(1, 0), (-1, 0), (0, 1), (0, -1)]]
                 + [((dx, dy), 2.0) for dx, dy in [(1, 1), (1, -1), (-1, 1), (-1, -1)]]
                 + [((dx, dy), 1.0) for dx, dy in [(2, 0), (-2, 0), (0, 2), (0, -2)]])


def climate_terms(dt=1.0, dz=1.0):
    """8 inputs (q0, q1, q2, kappa, w, t0, t1, t2) -> 3 outputs (q0', q1', q2')."""
    terms = []
    for m in range(3):
        q, kappa, w, tend = m, 3, 4, 5 + m
        terms.append((0, 0, 0, q, N, m, 1.0))
        for (ox, oy), c in BIHARMONIC_13:
            terms.append((ox, oy, 0, q, kappa, m, -dt * c))
        terms.append((0, 0, 1, q, w, m, -dt / (2.0 * dz)))
        terms.append((0, 0, -1, q, w, m, dt / (2.0 * dz)))
        terms.append((0, 0, 0, tend, N, m, dt))
    return terms


def poisson_jacobi_terms():
    """u' = (sum6(u) + f) / 6 with inputs 0 = u, 1 = f; the value is sum6(u) + f."""
    t = [(dx, dy, dz, 0, N, V, 1.0) for dx, dy, dz in AXIAL_3D]
    t.append((0, 0, 0, 1, N, V, 1.0))
    t.append((0, 0, 0, V, N, 0, 1.0 / 6.0))
    return t


def residual_terms():
    """Returned value r = f - A u = sum6(u) - 6u + f for inputs 0 = u, 1 = f; no output."""
    t = [(dx, dy, dz, 0, N, V, 1.0) for dx, dy, dz in AXIAL_3D]
    t.append((0, 0, 0, 0, N, V, -6.0))
    t.append((0, 0, 0, 1, N, V, 1.0))
    return t


def jacobi2d_run(u0: O.Grid, sweeps: int):
    """Ping-pong Jacobi from u0; both grids carry u0's halo.  Returns
    (u_N, u_{N-1}, max |u_N - u_{N-1}|), the last being Section 5.2's infinity-norm test."""
    a, b = u0.copy(), u0.copy()
    terms = jacobi2d_terms()
    for _ in range(sweeps):
        O.do_all(terms, [a], [b])
        a, b = b, a
    res = O.do_reduce(O.MAXABS, difference_terms(), [a, b]) if sweeps >= 1 else float("nan")
    return a, b, res


def heat_run(u0: O.Grid, f: O.Grid | None, lam: float, sweeps: int, every: int = 0):
    """Damped Jacobi / heat sweeps.  Every ``every`` sweeps (counting from
    sweep 0) the sweep is a fused do_reduce returning the L2 norm of the
    residual of the iterate it reads: residuals of u_0, u_every, u_2every, ..."""
    with_f = f is not None
    terms = heat_terms(lam, with_f)
    a, b = u0.copy(), u0.copy()
    residuals = []
    for s in range(sweeps):
        ins = [a, f] if with_f else [a]
        if every and s % every == 0:
            residuals.append(O.do_reduce(O.L2, terms, ins, [b]))
        else:
            O.do_all(terms, ins, [b])
        a, b = b, a
    return a, residuals


def climate_run(q, kappa, w, t, sweeps: int):
    """Multi-grid operator, 8 inputs -> 3 outputs, ping-pong on the three q grids."""
    cur = [g.copy() for g in q]
    nxt = [g.copy() for g in q]
    terms = climate_terms()
    for _ in range(sweeps):
        O.do_all(terms, cur + [kappa, w] + list(t), nxt)
        cur, nxt = nxt, cur
    return cur


def poisson_residual(u: O.Grid, f: O.Grid):
    """(||f - A u||_2, ||f||_2) over the interior."""
    r = O.do_reduce(O.L2, residual_terms(), [u, f])
    fn = O.do_reduce(O.L2, [], [f])
    return r, fn


def poisson_jacobi_solve(f: O.Grid, tol: float, max_sweeps: int, check_every: int = 10):
    """Plain FP64 Jacobi from u = 0 (zero halo) until ||f - A u||_2 / ||f||_2 <= tol."""
    a = O.zeros(f.n, f.halo)
    b = O.zeros(f.n, f.halo)
    terms = poisson_jacobi_terms()
    fn = O.do_reduce(O.L2, [], [f])
    s = 0
    while s < max_sweeps:
        if s % check_every == 0:
            r = O.do_reduce(O.L2, residual_terms(), [a, f])
            if r <= tol * fn:
                return a, s
        O.do_all(terms, [a, f], [b])
        a, b = b, a
        s += 1
    return a, s


def np_grid(arr: np.ndarray, halo) -> O.Grid:
    """Wraps a dense array with halo (any float dtype, widened exactly to FP64)."""
    return O.Grid(np.ascontiguousarray(arr, dtype=np.float64), tuple(halo))
