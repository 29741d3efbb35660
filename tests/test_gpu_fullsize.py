"""The benchmark configurations of the widened rows at their full sizes and
launch configurations, checked against the oracle on what it computes in
seconds: the 256 x 256 x 80 bidiagonal solve (sampled columns), one red-black
SOR iteration on 256^3, one natural-order Gauss-Seidel sweep on 64 planes of
512^2 (sampled planes), and the 256^3 heat body compiled at run time in FP32
(the staged kernel; sampled planes)."""
import math

import numpy as np
import pytest

from gpu_common import as_storage
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu


def test_bidiagonal_solve_256x256x80_sampled_columns():
    n, h = (256, 256, 80), (1, 1, 1)
    g = I.random_interior(606, n, h, -1.0, 1.0)
    m = I.random_interior(607, n, h, -0.9, 0.9)
    x = I.random_interior(608, n, h, 0.0, 0.0)
    terms = [(0, 0, 0, 1, B.NONE, 0, 1.0), (0, 0, -1, 0, 2, 0, -1.0)]
    gg = [B.Grid(n, h).upload(a) for a in (x, g, m)]
    assert B.ordered_specialization(B.K_INC, terms, gg, gg[:1]) == 2
    B.do_ordered(B.K_INC, terms, gg, gg[:1])
    got = gg[0].download().numpy()
    og = [O.Grid(a.copy(), h) for a in (x, g, m)]
    for i0, j0 in ((0, 0), (131, 77), (255, 255), (64, 200)):
        O.do_ordered(O.K_INC, terms, og, og[:1], lo=(i0, j0, 0), hi=(i0 + 1, j0 + 1, 80))
        a = got[1:-1, j0 + 1, i0 + 1]
        b = og[0].a[1:-1, j0 + 1, i0 + 1]
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


def test_redblack_sor_iteration_256():
    n, h = (256, 256, 256), (1, 1, 1)
    omega = 2.0 / (1.0 + math.sin(math.pi / 257))
    terms = S.poisson_sor(omega)
    u0 = I.random_interior(709, n, h, -1.0, 1.0)
    f0 = I.random_interior(707, n, h, -1.0, 1.0)
    gu, gf = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f0)
    B.do_colored(terms, [gu, gf], [gu], color=0, half_sweeps=2)
    got = gu.download().numpy()
    ou, of = O.Grid(u0.copy(), h), O.Grid(f0.copy(), h)
    O.do_colored(0, terms, [ou, of], [ou])
    O.do_colored(1, terms, [ou, of], [ou])
    assert np.max(np.abs(got - ou.a)) <= 1e-13 * np.max(np.abs(ou.a))


def test_diamond_gauss_seidel_64_planes_of_512_sampled():
    n, h = (512, 512, 64), (1, 1, 1)
    terms = [(1, 0, 0, 0, B.NONE, 0, 0.25), (-1, 0, 0, 0, B.NONE, 0, 0.25), (0, 1, 0, 0, B.NONE, 0, 0.25),
             (0, -1, 0, 0, B.NONE, 0, 0.25), (0, 0, 0, 1, B.NONE, 0, 0.25)]
    u0 = I.random_interior(808, n, h, -1.0, 1.0, halo_value=0.5)
    f0 = I.random_interior(809, n, h, -1.0, 1.0)
    gu, gf = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f0)
    B.do_diamond(terms, [gu, gf], [gu])
    got = gu.download().numpy()
    ou, of = O.Grid(u0.copy(), h), O.Grid(f0.copy(), h)
    for k in (0, 31, 63):
        O.do_diamond(terms, [ou, of], [ou], lo=(0, 0, k), hi=(512, 512, k + 1))
        assert np.max(np.abs(got[k + 1] - ou.a[k + 1])) <= 1e-13


def test_heat_body_256_fp32_staged_sampled_planes():
    n, h = (256, 256, 256), (1, 1, 1)
    body = ("out0 = (real)0.25 * in0(0,0,0) + (real)0.125 * (in0(1,0,0) + in0(-1,0,0) + in0(0,1,0)"
            " + in0(0,-1,0) + in0(0,0,1) + in0(0,0,-1)) + (real)0.125 * in1(0,0,0);")
    u0 = I.random_interior(202, n, h, -1.0, 1.0)
    f0 = I.random_interior(203, n, h, -1.0, 1.0)
    gi = [B.Grid(n, h, "f32").upload(a) for a in (u0, f0)]
    go = B.Grid(n, h, "f32").upload(np.zeros(I.padded_shape(n, h)))
    B.Program(body, 2, 1, "f32").run(gi, [go])
    got = go.download().double().numpy()
    oi = [O.Grid(as_storage(a, "f32"), h) for a in (u0, f0)]
    oo = O.Grid(np.zeros(I.padded_shape(n, h)), h)
    prog = O.Program(body, 2, 1)
    for k in (0, 128, 255):
        prog.run(oi, [oo], lo=(0, 0, k), hi=(256, 256, k + 1))
        assert np.max(np.abs(got[k + 1] - oo.a[k + 1])) <= 1e-6
