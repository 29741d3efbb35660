"""IEEE FP64 sweeps of the star / heat family with equal neighbour weights.

When the six axial weights are bit-identical the compiled kernel evaluates
w * (((x+ + x-) + (y+ + y-)) + (z+ + z-)) with the first two pair sums done
as exact IEEE additions on the integer pipe (fp64_int.cuh), and adds it
after the other terms of its destination.  These tests pin
that path bit for bit: with weights 2, 1, 1 every product is exact, so each
FMA is one correctly rounded addition and numpy can restate both evaluation
orders exactly, over data that reaches every branch of the integer adder
(subnormals, exact cancellations, overflow to infinity, infinities, NaNs,
signed zeros, wide exponent gaps).  GSCL_FP64_INT_ADD=0 turns the path off:
the kernel then takes one FMA per term in table order (+x, -x, +y, -y, +z,
-z), which the same data checks too.  The oracle-parity tests of the heat
operators (equal weights) run through this path as well."""
import numpy as np
import pytest

from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu

H = (1, 1, 1)
W0, W, WF = 2.0, 1.0, 1.0


def heat_op(w0=W0, w=W, wf=WF):
    t = [(0, 0, 0, 0, S.NONE, 0, w0)]
    t += [(dx, dy, dz, 0, S.NONE, 0, w) for dx, dy, dz in S.X6]
    t.append((0, 0, 0, 1, S.NONE, 0, wf))
    return t


def special_field(seed, n, halo, frac=0.3):
    """Values of every class: normals over a wide exponent range, subnormals,
    huge values whose pair sums overflow, infinities, NaNs, signed zeros and
    neighbours that cancel exactly."""
    rng = np.random.default_rng(seed)
    shape = I.padded_shape(n, halo)
    a = rng.uniform(-1.0, 1.0, size=shape) * np.exp2(rng.integers(-60, 61, size=shape).astype(np.float64))
    pick = rng.random(shape)
    cls = rng.integers(0, 8, size=shape)
    special = pick < frac
    sub = np.frombuffer(rng.integers(1, 1 << 52, size=a.size, dtype=np.uint64).tobytes(), dtype=np.float64)
    sub = sub.reshape(shape) * np.where(rng.random(shape) < 0.5, -1.0, 1.0)
    vals = [sub,                                            # subnormal
            np.where(rng.random(shape) < 0.5, -1.0, 1.0) * 1.6e308 * rng.uniform(0.7, 1.0, size=shape),  # huge
            np.full(shape, np.inf), np.full(shape, -np.inf), np.full(shape, np.nan),
            np.zeros(shape), np.full(shape, -0.0),
            np.exp2(rng.integers(-1074, -1020, size=shape).astype(np.float64))]  # tiny: subnormal sums
    for c in range(8):
        m = special & (cls == c)
        a[m] = vals[c][m]
    # exact cancellations: some x+ neighbours are minus their x- partner
    flip = rng.random(shape) < 0.05
    a[:, :, 2:][flip[:, :, 2:]] = -a[:, :, :-2][flip[:, :, 2:]]
    return a


def shifted(a, n, halo, dx, dy, dz):
    nx, ny, nz = n
    hx, hy, hz = halo
    return a[hz + dz:hz + dz + nz, hy + dy:hy + dy + ny, hx + dx:hx + dx + nx]


def expected(u, f, n, axial_sum, w0=W0, w=W, wf=WF):
    """The kernel's evaluation order restated in numpy (exact products)."""
    c = shifted(u, n, H, 0, 0, 0)
    nb = [shifted(u, n, H, *d) for d in S.X6]
    fc = shifted(f, n, H, 0, 0, 0)
    with np.errstate(all="ignore"):
        v = 0.0 + w0 * c
        if axial_sum:
            v = v + wf * fc
            s = ((nb[0] + nb[1]) + (nb[2] + nb[3])) + (nb[4] + nb[5])
            v = v + w * s
        else:
            for x in nb:
                v = v + w * x
            v = v + wf * fc
    return v


def sweep(u, f, n, op):
    gu, gf = B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)
    go = B.Grid(n, H, "f64").upload(np.zeros(I.padded_shape(n, H)))
    B.do_all(op, [gu, gf], [go])
    B.sync()
    return I.interior_view(go.download().numpy(), n, H)


def same_bits(got, want):
    """Bit-identical, NaNs anywhere both have one (any payload)."""
    nan_g, nan_w = np.isnan(got), np.isnan(want)
    ok = (nan_g == nan_w) & (nan_g | (got.view(np.uint64) == want.view(np.uint64)))
    return ok


@pytest.fixture
def compiled(monkeypatch):
    monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    monkeypatch.delenv("GSCL_FP64_ARITH", raising=False)
    monkeypatch.delenv("GSCL_FP64_INT_ADD", raising=False)
    return monkeypatch


@pytest.mark.parametrize("n", [(70, 45, 23), (64, 16, 3), (5, 3, 2), (257, 33, 9)])
@pytest.mark.parametrize("frac", [0.0, 0.3])
def test_axial_sum_bit_exact_over_every_value_class(compiled, n, frac):
    u = special_field(400 + n[0], n, H, frac)
    f = special_field(401 + n[0], n, H, frac * 0.3)
    got = sweep(u, f, n, heat_op())
    ok = same_bits(got, expected(u, f, n, True))
    assert ok.all(), (int((~ok).sum()), np.argwhere(~ok)[:3].tolist())


@pytest.mark.parametrize("n", [(70, 45, 23), (5, 3, 2)])
def test_switch_off_gives_table_order(compiled, n):
    compiled.setenv("GSCL_FP64_INT_ADD", "0")
    u = special_field(500 + n[0], n, H, 0.3)
    f = special_field(501 + n[0], n, H, 0.1)
    got = sweep(u, f, n, heat_op())
    ok = same_bits(got, expected(u, f, n, False))
    assert ok.all(), (int((~ok).sum()), np.argwhere(~ok)[:3].tolist())


def test_unequal_weights_keep_table_order(compiled):
    """One neighbour weight of 2 among weights of 1 keeps one FMA per term in
    table order (normal data: no product overflows)."""
    n = (70, 45, 23)
    u = special_field(600, n, H, 0.0)
    f = special_field(601, n, H, 0.0)
    op = heat_op()
    op[3] = op[3][:6] + (2.0,)
    got = sweep(u, f, n, op)
    v = 0.0 + W0 * shifted(u, n, H, 0, 0, 0)
    for t in op[1:7]:
        v = v + t[6] * shifted(u, n, H, *t[:3])
    v = v + WF * shifted(f, n, H, 0, 0, 0)
    assert same_bits(got, v).all()


@pytest.mark.parametrize("lam", [0.125, 1.0 / 6.0, 0.1])
def test_heat_within_tolerance_of_both_orders(compiled, lam):
    """Random data, the benchmark's heat weights: the axial-sum result and the
    table-order result differ by a few roundings of the absolute stencil
    (each is within 7 roundings of the exact sum)."""
    n = (96, 40, 17)
    u = I.random_interior(700, n, H, -1.0, 1.0, halo_value=0.25)
    f = I.random_interior(701, n, H, -1.0, 1.0)
    op = S.heat7(lam)
    a = sweep(u, f, n, op)
    compiled.setenv("GSCL_FP64_INT_ADD", "0")
    b = sweep(u, f, n, op)
    absst = abs(1 - 6 * lam) * np.abs(shifted(u, n, H, 0, 0, 0)) + lam * np.abs(shifted(f, n, H, 0, 0, 0))
    for d in S.X6:
        absst = absst + lam * np.abs(shifted(u, n, H, *d))
    assert np.all(np.abs(a - b) <= 16 * 2.0 ** -53 * absst)


def fused_op(wc, lam):
    """The fused heat sweep's structure (value r = sum6 + wc u + f, u' = u +
    lam r) with weights whose products are exact."""
    t = [(dx, dy, dz, 0, S.NONE, S.VALUE, 1.0) for dx, dy, dz in S.X6]
    t += [(0, 0, 0, 0, S.NONE, S.VALUE, wc), (0, 0, 0, 1, S.NONE, S.VALUE, 1.0)]
    return t + [(0, 0, 0, 0, S.NONE, 0, 1.0), (0, 0, 0, S.VALUE, S.NONE, 0, lam)]


def test_fused_residual_sweep_bit_exact(compiled):
    """The fused sweep with its L2 norm: the value's axial group takes the
    same path; u' bit for bit, the norm within the reduction's tolerance."""
    n = (70, 45, 23)
    u = special_field(800, n, H, 0.0)
    f = special_field(801, n, H, 0.0)
    gu, gf = B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)
    go = B.Grid(n, H, "f64").upload(np.zeros(I.padded_shape(n, H)))
    res = B.do_reduce(B.L2, fused_op(-4.0, 0.125), [gu, gf], [go])
    B.sync()
    got = I.interior_view(go.download().numpy(), n, H)
    c = shifted(u, n, H, 0, 0, 0)
    nb = [shifted(u, n, H, *d) for d in S.X6]
    r = 0.0 + (-4.0) * c
    r = r + shifted(f, n, H, 0, 0, 0)
    r = r + (((nb[0] + nb[1]) + (nb[2] + nb[3])) + (nb[4] + nb[5]))
    want = (0.0 + c) + 0.125 * r
    assert same_bits(got, want).all()
    norm = float(np.sqrt(np.sum(r * r)))
    assert abs(res - norm) <= 1e-12 * norm


def test_batch_matches_single_grid(compiled):
    """A batch of the same operator takes the same path as gscl_do_all alone."""
    shapes = [(33, 40, 35), (64, 17, 50), (7, 5, 3)]
    insts, singles = [], []
    for k, n in enumerate(shapes):
        u = special_field(900 + k, n, H, 0.1)
        f = special_field(950 + k, n, H, 0.0)
        gu, gf = B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)
        go = B.Grid(n, H, "f64").upload(np.zeros(I.padded_shape(n, H)))
        insts.append(([gu, gf], [go]))
        singles.append(sweep(u, f, n, heat_op()))
    bt = B.Batch(heat_op(), insts)
    bt.run(1)
    B.sync()
    for (ins, outs), n, want in zip(insts, shapes, singles):
        got = I.interior_view(outs[0].download().numpy(), n, H)
        assert same_bits(got, want).all()


def colour_mask(n, color):
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((i + j + k) & 1) == color


@pytest.mark.parametrize("compact", ["1", "0"])
@pytest.mark.parametrize("n", [(70, 45, 23), (5, 3, 2)])
def test_colored_sweep_bit_exact(compiled, compact, n):
    """Red-black sweeps in place (the colour-compacted kernel and the
    colour-predicated one): the colour's points take the axial-sum value of
    the grid as it was, the other colour keeps its bits."""
    compiled.setenv("GSCL_COLOR_COMPACT", compact)
    u = special_field(1000 + n[0], n, H, 0.2)
    f = special_field(1001 + n[0], n, H, 0.1)
    gu, gf = B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)
    cur = u.copy()
    for color in (1, 0):
        B.do_colored(heat_op(), [gu, gf], [gu], color=color)
        B.sync()
        v = expected(cur, f, n, True)
        inner = I.interior_view(cur, n, H)
        inner[...] = np.where(colour_mask(n, color), v, inner)
        ok = same_bits(I.interior_view(gu.download().numpy(), n, H), inner)
        assert ok.all(), (color, int((~ok).sum()), np.argwhere(~ok)[:3].tolist())


def test_colored_batch_mixed_weights_equals_each_instance_alone(compiled):
    """A coloured batch whose instances have equal and unequal neighbour
    weights: each instance takes the evaluation its single call takes (a flag
    per instance), bit for bit."""
    sides = [(70, 21, 19), (33, 64, 12), (5, 3, 2)]
    ops = [heat_op(), heat_op(), heat_op()]
    ops[1][3] = ops[1][3][:6] + (2.0,)  # unequal: table order
    us = [special_field(1100 + k, n, H, 0.0) for k, n in enumerate(sides)]
    fs = [special_field(1150 + k, n, H, 0.0) for k, n in enumerate(sides)]
    alone = []
    for op, n, u, f in zip(ops, sides, us, fs):
        gu, gf = B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)
        B.do_colored(op, [gu, gf], [gu], color=0, half_sweeps=3)
        alone.append(gu.download().numpy())
    grids = [(B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)) for n, u, f in zip(sides, us, fs)]
    batch = B.ColoredBatch(ops, [([gu, gf], [gu]) for gu, gf in grids])
    batch.run_colored(0, 3)
    B.sync()
    for k, ((gu, _), want) in enumerate(zip(grids, alone)):
        assert same_bits(gu.download().numpy(), want).all(), k


HC = (2, 2, 1)
BIH = ([((0, 0), 20.0)] + [((a, b), -8.0) for a, b in ((1, 0), (-1, 0), (0, 1), (0, -1))]
       + [((a, b), 2.0) for a, b in ((1, 1), (1, -1), (-1, 1), (-1, -1))]
       + [((a, b), 1.0) for a, b in ((2, 0), (-2, 0), (0, 2), (0, -2))])


def climate_expected(q, kap, w, t, n, groups):
    """The climate operator (dt = dz = 1) in the kernel's order, with exact
    products (kappa and w powers of two): per output, the unit term, the
    biharmonic run times kappa (its rings of four summed as (x0 + x1) +
    (x2 + x3) when grouped), the vertical pair times w (differenced when
    grouped), the tendency."""
    outs = []
    kc, wc = shifted(kap, n, HC, 0, 0, 0), shifted(w, n, HC, 0, 0, 0)
    with np.errstate(all="ignore"):
        for m in range(3):
            def x(dx, dy, dz=0):
                return shifted(q[m], n, HC, dx, dy, dz)
            v = 0.0 + x(0, 0)
            g = -BIH[0][1] * x(0, 0)
            for k in (1, 5, 9):
                ring = BIH[k:k + 4]
                if groups:
                    s = (x(*ring[0][0]) + x(*ring[1][0])) + (x(*ring[2][0]) + x(*ring[3][0]))
                    g = g + (-ring[0][1]) * s
                else:
                    for off, c in ring:
                        g = g + (-c) * x(*off)
            v = v + kc * g
            if groups:
                g2 = -0.5 * (x(0, 0, 1) - x(0, 0, -1))
            else:
                g2 = -0.5 * x(0, 0, 1)
                g2 = g2 + 0.5 * x(0, 0, -1)
            v = v + wc * g2
            outs.append(v + shifted(t[m], n, HC, 0, 0, 0))
    return outs


@pytest.mark.parametrize("int_add", ["1", "0"])
@pytest.mark.parametrize("n", [(70, 45, 9), (5, 3, 2)])
def test_climate_groups_bit_exact(compiled, int_add, n):
    """The 8 -> 3 climate operator: its biharmonic rings of four equal
    weights summed with one integer-pipe addition each and its vertical pair
    differenced on the integer pipe (GSCL_FP64_INT_ADD=0: one FMA per term),
    bit for bit against numpy in the same order."""
    compiled.setenv("GSCL_FP64_INT_ADD", int_add)
    rng = np.random.default_rng(1200 + n[0])
    shape = I.padded_shape(n, HC)
    q = [special_field(1210 + m, n, HC, 0.0) for m in range(3)]
    t = [special_field(1220 + m, n, HC, 0.0) for m in range(3)]
    kap = np.exp2(rng.integers(-10, -2, size=shape).astype(np.float64))
    w = np.where(rng.random(shape) < 0.5, -1.0, 1.0) * np.exp2(rng.integers(-6, 0, size=shape).astype(np.float64))
    ins = [B.Grid(n, HC, "f64").upload(a) for a in (q[0], q[1], q[2], kap, w, t[0], t[1], t[2])]
    outs = [B.Grid(n, HC, "f64").upload(np.zeros(shape)) for _ in range(3)]
    B.do_all(S.climate(), ins, outs)
    B.sync()
    want = climate_expected(q, kap, w, t, n, int_add == "1")
    for m in range(3):
        ok = same_bits(I.interior_view(outs[m].download().numpy(), n, HC), want[m])
        assert ok.all(), (m, int((~ok).sum()), np.argwhere(~ok)[:3].tolist())


def fma0(w, x):
    """fma(w, x, +0) for a power of two w: the rounded product (numpy rounds
    to nearest even, keeping the sign of a product that underflows to zero),
    and +0 where x is a zero."""
    with np.errstate(all="ignore"):
        p = w * x
    return np.where(x == 0.0, 0.0, p)


@pytest.mark.parametrize("w0", [0.25, 1.0, -0.5, 2.0 ** -600])
@pytest.mark.parametrize("n", [(70, 45, 23), (5, 3, 2)])
def test_power_of_two_first_term_bit_exact(compiled, w0, n):
    """A first weight that is a power of two of magnitude at most 1 (the heat
    sweep's 1 - 6 lam = 1/4): the chain opens with fma(w0, u, +0), whose bits
    include products that underflow into subnormals or to a signed zero; a
    batch gives the same bits."""
    u = special_field(1400 + n[0], n, H, 0.3)
    f = special_field(1401 + n[0], n, H, 0.1)
    op = heat_op(w0=w0)
    got = sweep(u, f, n, op)
    c = shifted(u, n, H, 0, 0, 0)
    nb = [shifted(u, n, H, *d) for d in S.X6]
    with np.errstate(all="ignore"):
        v = fma0(w0, c)
        v = v + WF * shifted(f, n, H, 0, 0, 0)
        v = v + W * (((nb[0] + nb[1]) + (nb[2] + nb[3])) + (nb[4] + nb[5]))
    ok = same_bits(got, v)
    assert ok.all(), (int((~ok).sum()), np.argwhere(~ok)[:3].tolist())
    gu, gf = B.Grid(n, H, "f64").upload(u), B.Grid(n, H, "f64").upload(f)
    go = B.Grid(n, H, "f64").upload(np.zeros(I.padded_shape(n, H)))
    B.Batch(op, [([gu, gf], [go])]).run(1)
    B.sync()
    assert same_bits(I.interior_view(go.download().numpy(), n, H), got).all()
