"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself:
closed forms, telescoping invariants, exact (math.fsum) sums, a library sparse
solve, brute-force dense matrices assembled independently, and the operator
printed in Fig. 1b (tests/golden/fig1b_operator.txt)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import drivers as D
from oracle import oracle as O

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_from(fun, n, halo):
    """Grid whose every cell (halo included) holds fun(i, j, k) in interior coordinates."""
    g = O.zeros(n, halo)
    hx, hy, hz = halo
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(-hz, nz + hz), np.arange(-hy, ny + hy), np.arange(-hx, nx + hx),
                          indexing="ij")
    g.a[...] = fun(i.astype(np.float64), j.astype(np.float64), k.astype(np.float64))
    return g


def laplacian_terms(dim):
    """Sum of axial neighbours minus 2*dim times the centre, written per axis."""
    t = []
    for ax in range(dim):
        for s in (1, -1):
            o = [0, 0, 0]
            o[ax] = s
            t.append((o[0], o[1], o[2], 0, O.NONE, 0, 1.0))
    t.append((0, 0, 0, 0, O.NONE, 0, -2.0 * dim))
    return t


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("coef", [(1, 2, -1, 3, -2, 5, 7), (-2, 1, 2, 0, 1, -1, -3)])
def test_quadratic_laplacian_3d_exact(coef):
    a, b, c, d, e, f, g0 = coef
    n, h = (9, 7, 6), (1, 1, 1)
    u = grid_from(lambda i, j, k: a * i * i + b * j * j + c * k * k + d * i + e * j + f * k + g0, n, h)
    out = O.zeros(n, h)
    O.do_all(laplacian_terms(3), [u], [out])
    assert np.all(out.interior() == 2.0 * (a + b + c))


def test_quadratic_laplacian_2d_exact():
    n, h = (11, 5, 1), (1, 1, 0)
    u = grid_from(lambda i, j, k: 2 * i * i - j * j + 3 * i - 4 * j + 1, n, h)
    out = O.zeros(n, h)
    O.do_all(laplacian_terms(2), [u], [out])
    assert np.all(out.interior() == 2.0 * (2 - 1))


def sine_mode(n, p):
    def fun(i, j, k):
        v = np.sin(p[0] * math.pi * (i + 1) / (n[0] + 1)) * np.sin(p[1] * math.pi * (j + 1) / (n[1] + 1))
        if n[2] > 1:
            v = v * np.sin(p[2] * math.pi * (k + 1) / (n[2] + 1))
        return v
    h = (1, 1, 1) if n[2] > 1 else (1, 1, 0)
    g = grid_from(fun, n, h)
    # the eigenmode vanishes on the halo up to the rounding of sin(m pi); make it exact
    inner = g.interior().copy()
    g.a[...] = 0.0
    g.interior()[...] = inner
    return g


@pytest.mark.parametrize("p", [(1, 1, 1), (2, 3, 1), (5, 1, 4)])
def test_heat_sine_eigenmode_factor(p):
    n = (12, 10, 9)
    lam = 1.0 / 8.0
    u = sine_mode(n, p)
    factor = 1.0 + 2.0 * lam * sum(math.cos(p[d] * math.pi / (n[d] + 1)) - 1.0 for d in range(3))
    sweeps = 7
    last, _ = D.heat_run(u, None, lam, sweeps)
    expect = u.interior() * factor ** sweeps
    assert np.max(np.abs(last.interior() - expect)) <= 1e-13 * np.max(np.abs(u.interior()))


@pytest.mark.parametrize("p", [(1, 1, 1), (3, 2, 1)])
def test_jacobi2d_sine_eigenmode_factor(p):
    n = (14, 9, 1)
    u = sine_mode(n, p)
    mu = 0.5 * (math.cos(p[0] * math.pi / (n[0] + 1)) + math.cos(p[1] * math.pi / (n[1] + 1)))
    last, prev, _ = D.jacobi2d_run(u, 5)
    assert np.max(np.abs(last.interior() - u.interior() * mu ** 5)) <= 1e-14
    assert np.max(np.abs(prev.interior() - u.interior() * mu ** 4)) <= 1e-14


def test_poisson_jacobi_sine_eigenmode_factor():
    n = (8, 8, 8)
    u = sine_mode(n, (1, 2, 3))
    f = O.zeros(n, (1, 1, 1))
    out = O.zeros(n, (1, 1, 1))
    O.do_all(D.poisson_jacobi_terms(), [u, f], [out])
    mu = sum(math.cos(q * math.pi / 9) for q in (1, 2, 3)) / 3.0
    assert np.max(np.abs(out.interior() - mu * u.interior())) <= 1e-15


def test_laplace2d_discrete_harmonic_fixed_point():
    """u = sin(pi x) cosh(beta (y - 1/2)) / cosh(beta / 2) with cosh(beta h) = 2 - cos(pi h)
    solves the 5-point equation exactly and equals sin(pi x) on both y edges."""
    m = 40
    hgrid = 1.0 / (m + 1)
    beta = math.acosh(2.0 - math.cos(math.pi * hgrid)) / hgrid

    def fun(i, j, k):
        x, y = (i + 1) * hgrid, (j + 1) * hgrid
        return np.sin(math.pi * x) * np.cosh(beta * (y - 0.5)) / math.cosh(beta / 2)

    u = grid_from(fun, (m, m, 1), (1, 1, 0))
    last, prev, res = D.jacobi2d_run(u, 1)
    assert np.max(np.abs(last.interior() - u.interior())) <= 1e-14
    assert res <= 1e-14


# ------------------------------------------------------------- biharmonic, advection
def climate_grids(n, q_fun, kappa_fun, w_fun, t_val):
    h = (2, 2, 1)
    q = [grid_from(q_fun, n, h) for _ in range(3)]
    kappa = grid_from(kappa_fun, n, h)
    w = grid_from(w_fun, n, h)
    t = [grid_from(lambda i, j, k: np.full_like(i, t_val), n, h) for _ in range(3)]
    return q, kappa, w, t


@pytest.mark.parametrize("q_fun,expect", [
    (lambda i, j, k: i ** 4, lambda i, j, k: -24.0),
    (lambda i, j, k: j ** 4 - i ** 4, lambda i, j, k: 0.0),
    (lambda i, j, k: i * i * j * j, lambda i, j, k: -8.0),
    (lambda i, j, k: 3 * i ** 3 - 2 * i * i * j + i * j * j + 5 * j ** 3 + 2 * i - 7, lambda i, j, k: 0.0),
])
def test_biharmonic_polynomials_exact(q_fun, expect):
    n = (9, 8, 4)
    q, kappa, w, t = climate_grids(n, q_fun, lambda i, j, k: np.ones_like(i), lambda i, j, k: 0 * i, 0.0)
    out = D.climate_run(q, kappa, w, t, 1)
    ref = grid_from(lambda i, j, k: q_fun(i, j, k) + expect(i, j, k), n, (2, 2, 1))
    for m in range(3):
        assert np.all(out[m].interior() == ref.interior())


def test_coefficient_read_at_core_element():
    """kappa enters at the core element: with q = i^4 and kappa = 1 + i the update is -24 (1 + i)."""
    n = (9, 6, 3)
    q, kappa, w, t = climate_grids(n, lambda i, j, k: i ** 4, lambda i, j, k: 1.0 + i,
                                   lambda i, j, k: 0 * i, 0.0)
    out = D.climate_run(q, kappa, w, t, 1)
    ref = grid_from(lambda i, j, k: i ** 4 - 24.0 * (1.0 + i), n, (2, 2, 1))
    assert np.all(out[1].interior() == ref.interior())


def test_vertical_advection_and_tendency_exact():
    """Centred difference of k^2 is 4k, halved by 2 dz: q' = k^2 - 2k w + t."""
    n = (5, 4, 7)
    q, kappa, w, t = climate_grids(n, lambda i, j, k: k * k, lambda i, j, k: 0 * i,
                                   lambda i, j, k: 1.0 + 0 * i, 3.0)
    out = D.climate_run(q, kappa, w, t, 1)
    ref = grid_from(lambda i, j, k: k * k - 2.0 * k + 3.0, n, (2, 2, 1))
    assert np.all(out[2].interior() == ref.interior())


# ---------------------------------------------------------------------- invariants
def test_flux_invariant_telescoping():
    """sum over the interior of (sum6 - 6u) equals the sum over the six faces of
    (halo value - adjacent interior value)."""
    rng = np.random.default_rng(7)
    n, h = (10, 7, 6), (1, 1, 1)
    u = O.zeros(n, h)
    u.a[...] = rng.integers(-50, 50, size=u.a.shape).astype(np.float64)
    f = O.zeros(n, h)
    got = O.do_reduce(O.SUM, D.residual_terms(), [u, f])
    a = u.a
    I = a[1:-1, 1:-1, 1:-1]
    flux = (a[1:-1, 1:-1, 0].sum() - I[:, :, 0].sum() + a[1:-1, 1:-1, -1].sum() - I[:, :, -1].sum()
            + a[1:-1, 0, 1:-1].sum() - I[:, 0, :].sum() + a[1:-1, -1, 1:-1].sum() - I[:, -1, :].sum()
            + a[0, 1:-1, 1:-1].sum() - I[0, :, :].sum() + a[-1, 1:-1, 1:-1].sum() - I[-1, :, :].sum())
    assert got == flux


def test_fused_sweep_and_residual_equal_two_passes():
    """Section 5.2: the fused operator and two separate scans are algorithmically equivalent."""
    rng = np.random.default_rng(3)
    n, h = (8, 9, 7), (1, 1, 1)
    u = O.zeros(n, h)
    f = O.zeros(n, h)
    u.a[...] = rng.uniform(-1, 1, u.a.shape)
    f.a[...] = rng.uniform(-1, 1, f.a.shape)
    fused_out, plain_out = O.zeros(n, h), O.zeros(n, h)
    r_fused = O.do_reduce(O.L2, D.heat_terms(0.125), [u, f], [fused_out])
    O.do_all(D.heat_terms(0.125), [u, f], [plain_out])
    r_two = O.do_reduce(O.L2, D.residual_terms(), [u, f])
    assert np.array_equal(fused_out.a[1:-1, 1:-1, 1:-1], plain_out.a[1:-1, 1:-1, 1:-1])
    assert r_fused == r_two


def test_heat_first_residual_is_norm_of_rhs():
    rng = np.random.default_rng(11)
    n, h = (6, 5, 7), (1, 1, 1)
    u0 = O.zeros(n, h)
    f = O.zeros(n, h)
    f.interior()[...] = rng.uniform(-1, 1, (7, 5, 6))
    _, res = D.heat_run(u0, f, 0.125, 20, every=10)
    assert len(res) == 2
    exact = math.sqrt(math.fsum((f.interior() ** 2).ravel()))
    assert abs(res[0] - exact) <= 4 * EPS * exact


# -------------------------------------------------------------------- brute force
def dense_operator(terms, ins, n_out):
    """Dense matrices (one per output) acting on the concatenation of all flattened
    input arrays, assembled row by row by enumerating each term's offset."""
    n = ins[0].n
    sizes = [g.a.size for g in ins]
    base = np.concatenate([[0], np.cumsum(sizes)])
    rows = n[0] * n[1] * n[2]
    value = np.zeros((rows, base[-1]))
    outs = [np.zeros((rows, base[-1])) for _ in range(n_out)]
    r = 0
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                for phase in ("value", "out"):
                    for (dx, dy, dz, a, c, m, w) in terms:
                        if (phase == "value") != (m == O.VALUE):
                            continue
                        coef = 1.0
                        if c != O.NONE:
                            gc = ins[c]
                            coef = gc.a[k + gc.halo[2], j + gc.halo[1], i + gc.halo[0]]
                        target = value if m == O.VALUE else outs[m]
                        if a == O.VALUE:
                            target[r] += w * coef * value[r]
                        else:
                            g = ins[a]
                            col = np.ravel_multi_index((k + dz + g.halo[2], j + dy + g.halo[1],
                                                        i + dx + g.halo[0]), g.a.shape)
                            target[r, base[a] + col] += w * coef
                r += 1
    return value, outs


def random_terms(rng, n_in, n_out, halos, count):
    terms = []
    for t in range(count):
        a = int(rng.integers(0, n_in))
        hx, hy, hz = halos[a]
        o = [int(rng.integers(-hx, hx + 1)), int(rng.integers(-hy, hy + 1)), int(rng.integers(-hz, hz + 1))]
        c = int(rng.integers(0, n_in)) if rng.random() < 0.3 else O.NONE
        m = O.VALUE if rng.random() < 0.25 else int(rng.integers(0, n_out))
        terms.append((o[0], o[1], o[2], a, c, m, float(rng.uniform(-2, 2))))
    terms.append((0, 0, 0, O.VALUE, O.NONE, 0, 0.75))
    return terms


@pytest.mark.parametrize("n,halos,seed", [
    ((8, 8, 8), [(1, 1, 1), (2, 2, 1), (0, 0, 0)], 1),
    ((7, 5, 6), [(2, 1, 2), (1, 1, 1), (1, 0, 1)], 2),
    ((8, 8, 1), [(1, 1, 0), (2, 2, 0), (0, 0, 0)], 3),
])
def test_bruteforce_dense_matrix(n, halos, seed):
    rng = np.random.default_rng(seed)
    ins = [O.zeros(n, h) for h in halos]
    for g in ins:
        g.a[...] = rng.uniform(-1, 1, g.a.shape)
    n_out = 2
    terms = random_terms(rng, len(ins), n_out, halos, 14)
    outs = [O.zeros(n, (1, 1, 0)) for _ in range(n_out)]
    val = O.do_all(terms, ins, outs, want_value=True)
    Vm, Om = dense_operator(terms, ins, n_out)
    x = np.concatenate([g.a.ravel() for g in ins])
    scale = np.abs(np.concatenate([g.a.ravel() for g in ins])).max() * sum(abs(t[6]) for t in terms) * 4
    assert np.max(np.abs(val.ravel() - Vm @ x)) <= 1e-13 * scale
    for m in range(n_out):
        assert np.max(np.abs(outs[m].interior().ravel() - Om[m] @ x)) <= 1e-13 * scale


# ------------------------------------------------- absolute stencil S(p) (abs_mode)
def distinct_read_terms(rng, n_in, n_out, halos):
    """A random operator in which no two terms read the same element of the
    same grid at the same core element (distinct (input, offset) pairs), each
    output has at most one term reading the returned value, and coefficient
    grids appear on direct and value terms alike."""
    pairs = set()
    terms = []
    while len(terms) < 13:
        a = int(rng.integers(0, n_in))
        hx, hy, hz = halos[a]
        o = (int(rng.integers(-hx, hx + 1)), int(rng.integers(-hy, hy + 1)), int(rng.integers(-hz, hz + 1)))
        if (a, o) in pairs:
            continue
        pairs.add((a, o))
        c = int(rng.integers(0, n_in)) if rng.random() < 0.4 else O.NONE
        m = O.VALUE if len(terms) % 3 == 0 else int(rng.integers(0, n_out))
        terms.append((*o, a, c, m, float(rng.choice([-1.0, 1.0]) * rng.uniform(0.25, 2.0))))
    for m in range(n_out):
        terms.append((0, 0, 0, O.VALUE, int(rng.integers(0, n_in)) if m == 0 else O.NONE, m,
                      float(rng.uniform(-2.0, -0.5))))
    return terms


@pytest.mark.parametrize("n,halos,seed", [
    ((6, 5, 4), [(1, 1, 1), (2, 1, 1), (1, 0, 1)], 11),
    ((7, 6, 1), [(1, 1, 0), (2, 2, 0), (0, 0, 0)], 12),
])
def test_abs_stencil_is_abs_matrix_times_abs_input(n, halos, seed):
    """S(p) = sum_t |w_t| |X_t(p)| |C_t(p)| (with the value's own S for terms that
    read the value).  For a linear operator whose terms read distinct
    elements, that is the row of |A| (the element-wise absolute value of the
    dense matrix assembled independently above) times |x|: no two terms share
    a matrix entry, and a value term's entries are the value row scaled by
    w C.  Inputs and coefficients take both signs, so a missing absolute
    value on any factor changes S."""
    rng = np.random.default_rng(seed)
    ins = [O.zeros(n, h) for h in halos]
    for g in ins:
        g.a[...] = rng.uniform(-1, 1, g.a.shape)
        g.a[np.abs(g.a) < 0.05] = -0.5
    n_out = 2
    terms = distinct_read_terms(rng, len(ins), n_out, halos)
    outs = [O.zeros(n, (0, 0, 0)) for _ in range(n_out)]
    O.do_all(terms, ins, outs, abs_mode=True)
    val = O.do_all(terms, ins, [O.zeros(n, (0, 0, 0)) for _ in range(n_out)], abs_mode=True, want_value=True)
    Vm, Om = dense_operator(terms, ins, n_out)
    ax = np.abs(np.concatenate([g.a.ravel() for g in ins]))
    want_v = np.abs(Vm) @ ax
    assert np.allclose(val.ravel(), want_v, rtol=32 * EPS, atol=0.0)
    for m in range(n_out):
        want = np.abs(Om[m]) @ ax
        assert np.allclose(outs[m].interior().ravel(), want, rtol=32 * EPS, atol=0.0), m
    # S bounds |operator| at every element (triangle inequality), with equality
    # only where no cancellation occurs
    plain = [O.zeros(n, (0, 0, 0)) for _ in range(n_out)]
    O.do_all(terms, ins, plain)
    for m in range(n_out):
        assert np.all(np.abs(plain[m].interior()) <= outs[m].interior() * (1 + 32 * EPS))


def test_abs_stencil_on_constant_grids():
    """Closed form: every input constant c_a (negative), so S_value = sum over the
    value's terms of |w| |c_in| |c_coef|, and S_m adds |w| S_value |c_coef| for
    the terms of output m that read the value."""
    n, halos = (5, 4, 3), [(1, 1, 1), (1, 1, 1), (0, 0, 0)]
    consts = [-2.0, -0.5, -3.0]
    ins = [O.zeros(n, h) for h in halos]
    for g, c in zip(ins, consts):
        g.a[...] = c
    V, N = O.VALUE, O.NONE
    terms = [(1, 0, 0, 0, N, V, 1.5), (0, 0, -1, 1, 2, V, -0.25), (0, 0, 0, 0, 1, 0, -1.0),
             (0, 0, 0, V, 2, 0, 0.5), (0, 1, 0, 1, N, 1, 2.0), (0, 0, 0, V, N, 1, -4.0)]
    s_val = 1.5 * 2.0 + 0.25 * 0.5 * 3.0
    s0 = 1.0 * 2.0 * 0.5 + 0.5 * s_val * 3.0
    s1 = 2.0 * 0.5 + 4.0 * s_val
    outs = [O.zeros(n, (0, 0, 0)) for _ in range(2)]
    val = O.do_all(terms, ins, outs, abs_mode=True, want_value=True)
    assert np.all(val == s_val)
    assert np.all(outs[0].interior() == s0) and np.all(outs[1].interior() == s1)


# ------------------------------------------------------------- paper's operator
def load_fig1b():
    rows = []
    with open(os.path.join(GOLDEN, "fig1b_operator.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                dx, dy, dz, num, den = line.split()
                rows.append(((int(dx), int(dy), int(dz)), float(num) / float(den)))
    return rows


def test_fig1b_spike_response_matches_printed_operator():
    """A single 1 at p0 makes out(p0 - o) = w_o for each printed offset o and 0 elsewhere."""
    golden = load_fig1b()
    assert len(golden) == 7
    n, h = (7, 6, 5), (1, 1, 1)
    p0 = (3, 2, 2)
    u = O.zeros(n, h)
    u.a[p0[2] + 1, p0[1] + 1, p0[0] + 1] = 1.0
    out = O.zeros(n, h)
    O.do_all(D.fig1b_terms(), [u], [out])
    expect = np.zeros((n[2], n[1], n[0]))
    for (dx, dy, dz), w in golden:
        expect[p0[2] - dz, p0[1] - dy, p0[0] - dx] = w
    assert np.array_equal(out.interior(), expect)


def test_fig1b_on_quadratic():
    """Fig. 1b is -1/36 times the 7-point Laplacian, so on a quadratic it gives -2(a+b+c)/36."""
    n, h = (6, 6, 6), (1, 1, 1)
    u = grid_from(lambda i, j, k: 3 * i * i + j * j - 2 * k * k + i, n, h)
    out = O.zeros(n, h)
    O.do_all(D.fig1b_terms(), [u], [out])
    S = O.zeros(n, h)
    O.do_all(D.fig1b_terms(), [u], [S], abs_mode=True)
    assert np.all(np.abs(out.interior() + 2.0 * (3 + 1 - 2) / 36.0) <= 8 * EPS * S.interior())


# --------------------------------------------------------------------- reductions
def test_sum_is_compensated_against_exact_fsum():
    rng = np.random.default_rng(5)
    n, h = (17, 9, 5), (1, 1, 1)
    g = O.zeros(n, h)
    big = rng.choice([1e16, -1e16, 1e8, -1e8], size=g.interior().shape)
    g.interior()[...] = big + rng.uniform(-1, 1, big.shape)
    exact = math.fsum(g.interior().ravel())
    got = O.do_reduce(O.SUM, [], [g])
    bound = 2 * EPS * abs(exact) + g.interior().size * EPS * EPS * np.abs(g.interior()).sum()
    assert abs(got - exact) <= bound
    naive = float(np.cumsum(g.interior().ravel())[-1])
    assert abs(naive - exact) > abs(got - exact)


def test_neumaier_catches_large_then_small():
    n, h = (4, 1, 1), (0, 0, 0)
    g = O.zeros(n, h)
    g.a[0, 0, :] = [1.0, 1e100, 1.0, -1e100]
    assert O.do_reduce(O.SUM, [], [g]) == 2.0


def test_maxabs_and_nan_propagation():
    rng = np.random.default_rng(9)
    n, h = (13, 4, 3), (1, 1, 1)
    g = O.zeros(n, h)
    g.a[...] = 1e9  # halo must not count
    g.interior()[...] = rng.uniform(-5, 5, (3, 4, 13))
    assert O.do_reduce(O.MAXABS, [], [g]) == np.max(np.abs(g.interior()))
    g.interior()[1, 2, 3] = np.nan
    for op in (O.SUM, O.MAXABS, O.L2):
        assert math.isnan(O.do_reduce(op, [], [g]))


def test_l2_against_fsum_and_subrange():
    rng = np.random.default_rng(13)
    n, h = (11, 10, 9), (1, 1, 1)
    g = O.zeros(n, h)
    g.a[...] = rng.uniform(-3, 3, g.a.shape)
    lo, hi = (2, 1, 3), (9, 10, 7)
    sub = g.a[1 + lo[2]:1 + hi[2], 1 + lo[1]:1 + hi[1], 1 + lo[0]:1 + hi[0]]
    exact = math.sqrt(math.fsum((sub * sub).ravel()))
    got = O.do_reduce(O.L2, [], [g], lo=lo, hi=hi)
    assert abs(got - exact) <= 4 * EPS * exact
    assert O.do_reduce(O.SUM, [], [g], lo=lo, hi=hi) == pytest.approx(math.fsum(sub.ravel()), rel=1e-14)


def test_empty_range_reductions():
    g = O.zeros((4, 4, 4), (1, 1, 1))
    assert O.do_reduce(O.SUM, [], [g], lo=(2, 0, 0), hi=(2, 4, 4)) == 0.0
    assert O.do_reduce(O.MAXABS, [], [g], lo=(0, 0, 3), hi=(4, 4, 3)) == 0.0


# ------------------------------------------------------------------ checks, solve
def test_rejects_reads_outside_halo_and_bad_ranges():
    g = O.zeros((5, 5, 5), (1, 1, 1))
    o = O.zeros((5, 5, 5), (1, 1, 1))
    with pytest.raises(ValueError):
        O.do_all([(2, 0, 0, 0, O.NONE, 0, 1.0)], [g], [o])
    with pytest.raises(ValueError):
        O.do_all([(0, 0, 0, 0, O.NONE, 0, 1.0)], [g], [o], lo=(0, 0, 0), hi=(6, 5, 5))
    with pytest.raises(ValueError):
        O.do_all([(0, 0, 0, 0, O.NONE, 0, 1.0)], [g], [g])
    # a sub-range leaves room: offset 2 is fine when the range stops one short of the edge
    O.do_all([(2, 0, 0, 0, O.NONE, 0, 1.0)], [g], [o], lo=(0, 0, 0), hi=(4, 5, 5))


def poisson_matrix(n):
    """7-point -Laplacian with zero Dirichlet halo, assembled with scipy.sparse kron."""
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    return (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsc()


def test_poisson_jacobi_solution_matches_sparse_direct_solve():
    n = 6
    rng = np.random.default_rng(17)
    f = O.zeros((n, n, n), (1, 1, 1))
    f.interior()[...] = rng.uniform(-1, 1, (n, n, n))
    u, sweeps = D.poisson_jacobi_solve(f, 1e-12, 20000)
    exact = spla.spsolve(poisson_matrix(n), f.interior().ravel())
    assert sweeps < 20000
    assert np.max(np.abs(u.interior().ravel() - exact)) <= 1e-10 * np.max(np.abs(exact))
    r, fn = D.poisson_residual(u, f)
    assert r <= 1e-12 * fn


def test_within_reduction_is_the_logical_and_of_the_pointwise_tests():
    """Section 5.2's convergence test do_reduce(fuse(diff, conv), logical_and),
    checked by brute force on small grids: numpy's all(|a - b| <= eps) decides
    the same for eps below, at and above the largest difference, for a planted
    NaN and for an empty range."""
    rng = np.random.default_rng(7)
    n, h = (9, 7, 5), (1, 1, 1)
    a = np.zeros((n[2] + 2, n[1] + 2, n[0] + 2))
    b = np.zeros_like(a)
    a[1:-1, 1:-1, 1:-1] = rng.uniform(-1, 1, size=(n[2], n[1], n[0]))
    b[1:-1, 1:-1, 1:-1] = a[1:-1, 1:-1, 1:-1] + rng.uniform(-1e-3, 1e-3, size=(n[2], n[1], n[0]))
    d = np.abs(a[1:-1, 1:-1, 1:-1] - b[1:-1, 1:-1, 1:-1])
    terms = D.difference_terms()
    for eps in (0.0, 0.5 * d.max(), d.max(), 2.0 * d.max()):
        got = O.do_reduce_within(eps, terms, [O.Grid(a, h), O.Grid(b, h)])
        assert got == (1.0 if np.all(d <= eps) else 0.0)
    a2 = a.copy()
    a2[3, 4, 5] = np.nan
    assert O.do_reduce_within(1.0, terms, [O.Grid(a2, h), O.Grid(b, h)]) == 0.0
    assert O.do_reduce_within(0.0, terms, [O.Grid(a, h), O.Grid(b, h)], lo=(2, 2, 2), hi=(2, 5, 5)) == 1.0
    with pytest.raises(ValueError):
        O.do_reduce_within(-1.0, terms, [O.Grid(a, h), O.Grid(b, h)])


# ---------------------------------------------------------------- ordered iteration spaces
def _column_grids(n, h, seed):
    rng = np.random.default_rng(seed)
    shape = (n[2] + 2 * h[2], n[1] + 2 * h[1], n[0] + 2 * h[0])
    f = np.zeros(shape)
    f[h[2]:h[2] + n[2], h[1]:h[1] + n[1], h[0]:h[0] + n[0]] = rng.integers(-50, 50, size=(n[2], n[1], n[0]))
    return f


@pytest.mark.parametrize("order,axis,rev", [(O.K_INC, 0, False), (O.K_DEC, 0, True),
                                            (O.J_INC, 1, False), (O.J_DEC, 1, True),
                                            (O.I_INC, 2, False), (O.I_DEC, 2, True)])
def test_ordered_recurrence_is_a_running_sum(order, axis, rev):
    """do_*_inc / _dec (Section 3) with out = out(previous) + f, the output
    bound also as the input it reads one step back: a running sum along the
    ordered axis (numpy cumsum, reversed for _dec), starting from the halo."""
    n, h = (6, 5, 7), (1, 1, 1)
    f = _column_grids(n, h, 11)
    x = np.zeros_like(f)
    step = {O.I_INC: (-1, 0, 0), O.I_DEC: (1, 0, 0), O.J_INC: (0, -1, 0), O.J_DEC: (0, 1, 0),
            O.K_INC: (0, 0, -1), O.K_DEC: (0, 0, 1)}[order]
    terms = [(step[0], step[1], step[2], 0, 255, 0, 1.0), (0, 0, 0, 1, 255, 0, 1.0)]
    X = O.Grid(x, h)
    O.do_ordered(order, terms, [X, O.Grid(f, h)], [X])
    core = f[1:-1, 1:-1, 1:-1]
    want = np.flip(np.cumsum(np.flip(core, axis), axis=axis), axis) if rev else np.cumsum(core, axis=axis)
    assert np.array_equal(x[1:-1, 1:-1, 1:-1], want)
    assert np.all(x[0] == 0) and np.all(x[-1] == 0)  # halos untouched


def test_ordered_bidiagonal_forward_substitution():
    """do_k_inc solving L x = g per (i, j) column, L unit lower bidiagonal
    with sub-diagonal m(k): x(k) = g(k) - m(k) x(k-1), the coefficient grid
    m multiplying the previous element.  Checked against a dense triangular
    solve of every column (scipy)."""
    import scipy.linalg as sla
    n, h = (4, 3, 9), (0, 0, 1)
    rng = np.random.default_rng(5)
    shape = (n[2] + 2, n[1], n[0])
    g = np.zeros(shape)
    m = np.zeros(shape)
    g[1:-1] = rng.uniform(-1, 1, size=(n[2], n[1], n[0]))
    m[1:-1] = rng.uniform(-0.9, 0.9, size=(n[2], n[1], n[0]))
    x = np.zeros(shape)
    X = O.Grid(x, h)
    terms = [(0, 0, 0, 1, 255, 0, 1.0), (0, 0, -1, 0, 2, 0, -1.0)]
    O.do_ordered(O.K_INC, terms, [X, O.Grid(g, h), O.Grid(m, h)], [X])
    for j in range(n[1]):
        for i in range(n[0]):
            L = np.eye(n[2]) + np.diag(m[2:-1, j, i], -1)
            want = sla.solve_triangular(L, g[1:-1, j, i], lower=True)
            assert np.allclose(x[1:-1, j, i], want, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ red-black colouring
AXIAL6 = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def sor_terms(omega=1.0):
    """In-place SOR update of the 7-point Poisson equation 6u - sum6 = f:
    u <- (1 - omega) u + omega (sum6 + f) / 6; omega = 1 is Gauss-Seidel."""
    t = [(dx, dy, dz, 0, O.NONE, 0, omega / 6.0) for dx, dy, dz in AXIAL6]
    t.append((0, 0, 0, 1, O.NONE, 0, omega / 6.0))
    if omega != 1.0:
        t.append((0, 0, 0, 0, O.NONE, 0, 1.0 - omega))
    return t


def poisson_residual_np(u, f):
    """f - (6u - sum6 u) on the interior, by array slicing (halo width 1)."""
    a = u.a
    lap = (6.0 * a[1:-1, 1:-1, 1:-1] - a[2:, 1:-1, 1:-1] - a[:-2, 1:-1, 1:-1] - a[1:-1, 2:, 1:-1]
           - a[1:-1, :-2, 1:-1] - a[1:-1, 1:-1, 2:] - a[1:-1, 1:-1, :-2])
    return f.interior() - lap


def colour_of(n):
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return (i + j + k) % 2


def test_redblack_half_sweep_solves_its_colour():
    """Gauss-Seidel on one colour solves the equation exactly at every element
    of that colour (its neighbours are all of the other colour and do not
    change), and leaves the other colour and the halo untouched."""
    n, h = (7, 6, 5), (1, 1, 1)
    rng = np.random.default_rng(31)
    u, f = O.zeros(n, h), O.zeros(n, h)
    u.a[...] = rng.uniform(-1, 1, u.a.shape)        # the halo holds Dirichlet values
    f.interior()[...] = rng.uniform(-1, 1, n[::-1])
    col = colour_of(n)
    halo0 = u.a.copy()
    for colour in (0, 1, 0, 1):
        before = u.interior().copy()
        O.do_colored(colour, sor_terms(), [u, f], [u])
        r = poisson_residual_np(u, f)
        assert np.max(np.abs(r[col == colour])) <= 1e-14 * 16
        assert np.array_equal(u.interior()[col != colour], before[col != colour])
        assert np.abs(r[col != colour]).max() > 1e-6    # the other colour is not solved yet
        inner = np.zeros(u.a.shape, bool)
        inner[1:-1, 1:-1, 1:-1] = True
        assert np.array_equal(u.a[~inner], halo0[~inner])


def sor_rate(omega, mu):
    """Spectral radius of SOR for a consistently ordered matrix whose Jacobi
    iteration has spectral radius mu, for omega up to the optimum (Young):
    the largest root of (lambda + omega - 1)^2 = lambda omega^2 mu^2."""
    s = (omega * mu + math.sqrt(omega * omega * mu * mu - 4.0 * (omega - 1.0))) / 2.0
    return s * s


@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_redblack_sor_asymptotic_rate(omega):
    """Red-black ordering makes the 7-point matrix consistently ordered, so
    red-black Gauss-Seidel contracts the error by mu^2 per iteration and SOR
    by the root above, with mu = cos(pi / (n + 1)) the Jacobi radius of the
    n^3 Dirichlet problem."""
    n, h = (8, 8, 8), (1, 1, 1)
    rng = np.random.default_rng(32)
    u, f = O.zeros(n, h), O.zeros(n, h)
    u.interior()[...] = rng.uniform(-1, 1, n)
    terms = sor_terms(omega)
    norms = []
    for _ in range(160):
        O.do_colored(0, terms, [u, f], [u])
        O.do_colored(1, terms, [u, f], [u])
        norms.append(np.linalg.norm(u.interior()))
    rate = norms[-1] / norms[-2]
    want = sor_rate(omega, math.cos(math.pi / 9))
    assert abs(rate - want) <= 2e-4 * want, (rate, want)


def test_redblack_gauss_seidel_converges_to_direct_solve():
    n = 6
    rng = np.random.default_rng(33)
    u, f = O.zeros((n, n, n), (1, 1, 1)), O.zeros((n, n, n), (1, 1, 1))
    f.interior()[...] = rng.uniform(-1, 1, (n, n, n))
    for _ in range(200):
        O.do_colored(0, sor_terms(), [u, f], [u])
        O.do_colored(1, sor_terms(), [u, f], [u])
    exact = spla.spsolve(poisson_matrix(n), f.interior().ravel())
    assert np.max(np.abs(u.interior().ravel() - exact)) <= 1e-11 * np.max(np.abs(exact))


def test_colored_rejects_bad_colour_and_ranges():
    u, f = O.zeros((4, 4, 4), (1, 1, 1)), O.zeros((4, 4, 4), (1, 1, 1))
    with pytest.raises(ValueError):
        O.do_colored(2, sor_terms(), [u, f], [u])
    with pytest.raises(ValueError):
        O.do_colored(0, [(2, 0, 0, 0, O.NONE, 0, 1.0)], [u, f], [u])


# ------------------------------------------------------------------ do_diamond
def sat_terms():
    """Summed-area table: x = f + x(i-1, j) + x(i, j-1) - x(i-1, j-1) (x input 0, f input 1)."""
    return [(0, 0, 0, 1, O.NONE, 0, 1.0), (-1, 0, 0, 0, O.NONE, 0, 1.0), (0, -1, 0, 0, O.NONE, 0, 1.0),
            (-1, -1, 0, 0, O.NONE, 0, -1.0)]


@pytest.mark.parametrize("n,h", [((13, 9, 1), (1, 1, 0)), ((7, 6, 3), (1, 1, 1))])
def test_diamond_summed_area_table(n, h):
    """With (i-1, j) and (i, j-1) done before (i, j), the recurrence builds the
    2D prefix sum of f in each plane: numpy's cumsum along both axes, exactly
    on integer data."""
    rng = np.random.default_rng(41)
    x, f = O.zeros(n, h), O.zeros(n, h)
    f.interior()[...] = rng.integers(-20, 20, size=n[::-1])
    O.do_diamond(sat_terms(), [x, f], [x])
    want = np.cumsum(np.cumsum(f.interior(), axis=2), axis=1)
    assert np.array_equal(x.interior(), want)


def diamond_by_antidiagonals(terms, arrays, h, n):
    """do_diamond computed another way: every anti-diagonal i + j = t at once,
    t ascending (numpy), each element from the arrays as they stand; outputs
    are input 0 (in place)."""
    hx, hy, hz = h
    a = [x.copy() for x in arrays]
    for k in range(n[2]):
        for t in range(n[0] + n[1] - 1):
            j = np.arange(max(0, t - n[0] + 1), min(n[1], t + 1))
            i = t - j
            acc = np.zeros(len(j))
            for dx, dy, dz, src, coef, out, w in terms:
                xv = a[src][k + hz + dz, j + hy + dy, i + hx + dx]
                cv = 1.0 if coef == O.NONE else a[coef][k + hz, j + hy, i + hx]
                acc = acc + (w * xv) * cv
            a[0][k + hz, j + hy, i + hx] = acc
    return a[0]


def test_diamond_is_independent_of_the_wavefront_order():
    """Reads of the output at offsets with dx, dy <= 0 see updated elements and
    at dx, dy >= 0 old ones, whichever order respects the diamond: the
    lexicographic loop equals a sweep by anti-diagonals."""
    n, h = (11, 8, 2), (1, 1, 1)
    rng = np.random.default_rng(42)
    x0 = rng.uniform(-1, 1, (n[2] + 2, n[1] + 2, n[0] + 2))
    f0 = rng.uniform(-1, 1, x0.shape)
    terms = [(-1, 0, 0, 0, O.NONE, 0, 0.3), (0, -1, 0, 0, O.NONE, 0, 0.2), (-1, -1, 0, 0, O.NONE, 0, -0.1),
             (1, 0, 0, 0, O.NONE, 0, 0.15), (0, 1, 0, 0, O.NONE, 0, 0.25), (1, 1, 0, 0, 1, 0, 0.05),
             (0, 0, 0, 0, O.NONE, 0, -0.4), (0, 0, 1, 1, O.NONE, 0, 0.5)]
    x = O.Grid(x0.copy(), h)
    O.do_diamond(terms, [x, O.Grid(f0.copy(), h)], [x])
    want = diamond_by_antidiagonals(terms, [x0, f0], h, n)
    assert np.array_equal(x.a, want)


def test_diamond_lexicographic_gauss_seidel_rate():
    """Gauss-Seidel in the natural order on the 5-point Laplacian, in place:
    the matrix is consistently ordered, so the error contracts by
    cos^2(pi / (n + 1)) per sweep (n x n Dirichlet problem)."""
    n, h = (10, 10, 1), (1, 1, 0)
    rng = np.random.default_rng(43)
    u = O.zeros(n, h)
    u.interior()[...] = rng.uniform(-1, 1, (1, 10, 10))
    terms = [(1, 0, 0, 0, O.NONE, 0, 0.25), (-1, 0, 0, 0, O.NONE, 0, 0.25), (0, 1, 0, 0, O.NONE, 0, 0.25),
             (0, -1, 0, 0, O.NONE, 0, 0.25)]
    norms = []
    for _ in range(150):
        O.do_diamond(terms, [u], [u])
        norms.append(np.linalg.norm(u.interior()))
    rate = norms[-1] / norms[-2]
    want = math.cos(math.pi / 11) ** 2
    assert abs(rate - want) <= 2e-4 * want, (rate, want)


# ------------------------------------------------------------------ run-time point operators
HEAT_BODY = ("out0 = 0.25 * in0(0,0,0) + 0.125 * (in0(1,0,0) + in0(-1,0,0) + in0(0,1,0) + in0(0,-1,0)"
             " + in0(0,0,1) + in0(0,0,-1)) + 0.125 * in1(0,0,0);")


def test_program_linear_body_equals_the_term_list():
    """The heat operator written as a body gives what the term-list oracle
    gives (a separate implementation), up to the order of the additions."""
    n, h = (9, 7, 6), (1, 1, 1)
    rng = np.random.default_rng(51)
    u, f = O.zeros(n, h), O.zeros(n, h)
    u.a[...] = rng.uniform(-1, 1, u.a.shape)
    f.a[...] = rng.uniform(-1, 1, f.a.shape)
    a, b = O.zeros(n, h), O.zeros(n, h)
    O.Program(HEAT_BODY, 2, 1).run([u, f], [a])
    terms = ([(0, 0, 0, 0, O.NONE, 0, 0.25)] + [(dx, dy, dz, 0, O.NONE, 0, 0.125) for dx, dy, dz in AXIAL6]
             + [(0, 0, 0, 1, O.NONE, 0, 0.125)])
    O.do_all(terms, [u, f], [b])
    assert np.max(np.abs(a.a - b.a)) <= 8 * EPS


def test_program_index_and_products_exact():
    """The index query of a stateful operator and a product of reads, on
    integer data: exact."""
    n, h = (6, 5, 4), (1, 1, 1)
    u = grid_from(lambda i, j, k: i - 2 * j + 3 * k, n, h)
    a, b = O.zeros(n, h), O.zeros(n, h)
    O.Program("out0 = (real)(i + 10 * j + 100 * k); out1 = in0(0,0,0) * in0(1,0,0);", 1, 2).run([u], [a, b])
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    assert np.array_equal(a.interior(), i + 10 * j + 100 * k)
    assert np.array_equal(b.interior(), (i - 2 * j + 3 * k) * (i + 1 - 2 * j + 3 * k))


def test_program_laplacian_of_a_quadratic_is_constant():
    n, h = (7, 6, 5), (1, 1, 1)
    u = grid_from(lambda i, j, k: 2 * i * i - j * j + 3 * k * k + i * j, n, h)
    a = O.zeros(n, h)
    body = ("out0 = in0(1,0,0) + in0(-1,0,0) + in0(0,1,0) + in0(0,-1,0) + in0(0,0,1) + in0(0,0,-1)"
            " - 6.0 * in0(0,0,0);")
    O.Program(body, 1, 1).run([u], [a])
    assert np.all(a.interior() == 2 * (2 - 1 + 3))


def test_program_reads_beyond_the_reach_are_refused():
    n, h = (5, 4, 3), (2, 2, 2)
    u = grid_from(lambda i, j, k: i + j + k + 1.0, n, h)
    a = O.zeros(n, h)
    p = O.Program("out0 = in0(2,0,0) + in0(0,0,0);", 1, 1, reach=(1, 1, 1))
    p.run([u], [a])
    assert p.outside == 5 * 4 * 3
    assert np.array_equal(a.interior(), u.interior())


def test_program_value_is_the_term_list_value():
    """The body's `value` (the heat residual written as a body) is the value the
    term-list oracle returns for the same operator, element by element."""
    n, h = (8, 6, 5), (1, 1, 1)
    rng = np.random.default_rng(52)
    u, f = O.zeros(n, h), O.zeros(n, h)
    u.a[...] = rng.uniform(-1, 1, u.a.shape)
    f.a[...] = rng.uniform(-1, 1, f.a.shape)
    body = ("value = in0(1,0,0) + in0(-1,0,0) + in0(0,1,0) + in0(0,-1,0) + in0(0,0,1) + in0(0,0,-1)"
            " - 6.0 * in0(0,0,0) + in1(0,0,0);")
    got = O.Program(body, 2, 0).run([u, f], [], lo=(1, 0, 1), hi=(8, 5, 4), want_value=True)
    terms = ([(dx, dy, dz, 0, O.NONE, O.VALUE, 1.0) for dx, dy, dz in AXIAL6]
             + [(0, 0, 0, 0, O.NONE, O.VALUE, -6.0), (0, 0, 0, 1, O.NONE, O.VALUE, 1.0)])
    want = O.do_all(terms, [u, f], [], lo=(1, 0, 1), hi=(8, 5, 4), want_value=True)
    assert got.shape == want.shape == (3, 5, 7)
    assert np.max(np.abs(got - want)) <= 16 * EPS
