"""CPU-only checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-side layout and validation logic behave as
documented.  No call here touches a GPU."""
import ctypes

import pytest

from paper_1207_1746_b300 import binding as B


@pytest.fixture(scope="module")
def L():
    return B.lib()


def test_exports_every_declared_symbol(L):
    names = B.declared_symbols()
    assert "gscl_do_all" in names and "gscl_do_reduce" in names
    for name in names:
        assert hasattr(L, name), name


@pytest.mark.parametrize("dtype,elem", [("f64", 8), ("f32", 4), ("bf16", 2)])
@pytest.mark.parametrize("n,halo,ndim", [((256, 256, 256), (1, 1, 1), 3), ((17, 13, 11), (2, 2, 1), 3),
                                         ((256, 256, 1), (1, 1, 0), 2), ((1, 1, 1), (0, 0, 0), 3),
                                         ((33, 7, 5), (4, 3, 2), 3)])
def test_layout_alignment(dtype, elem, n, halo, ndim):
    pitch, off, nbytes = B.layout(n, halo, dtype, ndim)
    assert (pitch * elem) % 128 == 0
    assert ((off + halo[0]) * elem) % 128 == 0
    assert pitch >= off + n[0] + 2 * halo[0]
    assert pitch - (off + n[0] + 2 * halo[0]) < 128 // elem
    assert nbytes == pitch * (n[1] + 2 * halo[1]) * (n[2] + 2 * halo[2]) * elem


@pytest.mark.parametrize("args", [
    (4, (8, 8, 8), (1, 1, 1), "f64"),
    (3, (0, 8, 8), (1, 1, 1), "f64"),
    (3, (8, 8, 8), (5, 1, 1), "f64"),
    (2, (8, 8, 2), (1, 1, 0), "f64"),
    (2, (8, 8, 1), (1, 1, 1), "f64"),
])
def test_layout_rejects_bad_shapes(args):
    ndim, n, halo, dtype = args
    with pytest.raises(B.GsclError) as e:
        B.layout(n, halo, dtype, ndim)
    assert e.value.status == 1


class FakeGrid:
    """A handle over a fake (never dereferenced) aligned address: enough to
    exercise host-side validation without a GPU."""
    _next = 1 << 20

    def __init__(self, n, halo, dtype="f64", ndim=3):
        _, _, nbytes = B.layout(n, halo, dtype, ndim)
        FakeGrid._next += (nbytes + 4095) // 4096 * 4096 + 4096
        h = ctypes.c_uint64()
        B.check(B.lib().gscl_grid_create(ndim, (ctypes.c_int64 * 3)(*n), (ctypes.c_int32 * 3)(*halo),
                                         B._DTYPES[dtype][0], ctypes.c_void_p(FakeGrid._next), nbytes,
                                         ctypes.byref(h)))
        self.handle = h.value


def do_all_status(terms, ins, outs, rng=None, sweeps=1):
    st = B.Stencil(terms)
    return B.lib().gscl_do_all(ctypes.byref(st.c), B._handles(ins), len(ins), B._handles(outs), len(outs),
                               B._range(rng), sweeps, None)


def test_handles_create_destroy_stale(L):
    g = FakeGrid((8, 8, 8), (1, 1, 1))
    d = B.GridDesc()
    assert L.gscl_grid_info(g.handle, ctypes.byref(d)) == 0
    assert d.n[0] == 8 and d.halo[2] == 1
    assert L.gscl_grid_destroy(g.handle) == 0
    assert L.gscl_grid_destroy(g.handle) == 8          # GSCL_ERR_STATE
    assert L.gscl_grid_info(g.handle, ctypes.byref(d)) == 8
    g2 = FakeGrid((8, 8, 8), (1, 1, 1))                 # reuses the slot, new generation
    assert g2.handle != g.handle
    assert L.gscl_grid_info(g.handle, ctypes.byref(d)) == 8
    assert L.gscl_grid_info(0, ctypes.byref(d)) == 8


def test_create_rejects_misaligned_and_small_buffers(L):
    n, halo = (8, 8, 8), (1, 1, 1)
    _, _, nbytes = B.layout(n, halo)
    h = ctypes.c_uint64()
    args = (3, (ctypes.c_int64 * 3)(*n), (ctypes.c_int32 * 3)(*halo), 0)
    assert L.gscl_grid_create(*args, ctypes.c_void_p(0x10040), nbytes, ctypes.byref(h)) == 1
    assert L.gscl_grid_create(*args, ctypes.c_void_p(0x10000), nbytes - 1, ctypes.byref(h)) == 6


def test_swap_exchanges_storage_and_checks_layout(L):
    a, b = FakeGrid((8, 8, 8), (1, 1, 1)), FakeGrid((8, 8, 8), (1, 1, 1))
    c = FakeGrid((8, 8, 9), (1, 1, 1))
    da, db = B.GridDesc(), B.GridDesc()
    L.gscl_grid_info(a.handle, ctypes.byref(da))
    L.gscl_grid_info(b.handle, ctypes.byref(db))
    pa, pb = da.dev_buf, db.dev_buf
    ha, hb, hc = ctypes.c_uint64(a.handle), ctypes.c_uint64(b.handle), ctypes.c_uint64(c.handle)
    assert L.gscl_swap(ctypes.byref(ha), ctypes.byref(hb)) == 0
    L.gscl_grid_info(a.handle, ctypes.byref(da))
    assert da.dev_buf == pb
    assert L.gscl_swap(ctypes.byref(ha), ctypes.byref(hb)) == 0
    L.gscl_grid_info(a.handle, ctypes.byref(da))
    assert da.dev_buf == pa                             # swap twice == identity
    assert L.gscl_swap(ctypes.byref(ha), ctypes.byref(hc)) == 5   # GSCL_ERR_SHAPE


def test_do_all_validation_errors():
    u, v = FakeGrid((16, 8, 8), (1, 1, 1)), FakeGrid((16, 8, 8), (1, 1, 1))
    w2 = FakeGrid((16, 8, 8), (2, 2, 1))
    f32 = FakeGrid((16, 8, 8), (1, 1, 1), "f32")
    other = FakeGrid((16, 8, 7), (1, 1, 1))
    ok_terms = [(1, 0, 0, 0, B.NONE, 0, 1.0)]
    # read beyond the halo
    assert do_all_status([(2, 0, 0, 0, B.NONE, 0, 1.0)], [u], [v]) == 2
    # ... allowed when read from a grid with a wider halo
    assert do_all_status([(2, 0, 0, 0, B.NONE, 0, 1.0)], [w2], [v]) != 2
    # range outside the interior
    assert do_all_status(ok_terms, [u], [v], rng=((0, 0, 0), (17, 8, 8))) == 2
    # output read at a non-zero offset (do_all promises no order)
    assert do_all_status(ok_terms, [u], [u]) == 3
    # the same output twice
    assert do_all_status([(0, 0, 0, 0, B.NONE, 0, 1.0), (0, 0, 0, 0, B.NONE, 1, 1.0)], [u], [v, v]) == 3
    # dtype and shape mismatch
    assert do_all_status(ok_terms, [u], [f32]) == 4
    assert do_all_status(ok_terms, [u], [other]) == 5
    # bad codes
    assert do_all_status([(0, 0, 0, 3, B.NONE, 0, 1.0)], [u], [v]) == 1
    assert do_all_status([(0, 0, 0, 0, B.NONE, 2, 1.0)], [u], [v]) == 1
    assert do_all_status([(1, 0, 0, B.VALUE, B.NONE, 0, 1.0)], [u], [v]) == 1
    assert do_all_status([(0, 0, 0, 0, 5, 0, 1.0)], [u], [v]) == 1
    assert do_all_status(ok_terms, [u], [v], sweeps=0) == 1
    # too many terms
    assert do_all_status([(0, 0, 0, 0, B.NONE, 0, 1.0)] * 65, [u], [v]) == 10
    # stale handle
    B.lib().gscl_grid_destroy(v.handle)
    assert do_all_status(ok_terms, [u], [v]) == 8
    # an empty range is accepted and enqueues nothing (no GPU needed)
    assert do_all_status(ok_terms, [u], [w2], rng=((0, 0, 3), (16, 8, 3))) == 0


def test_reduce_validation_errors():
    u = FakeGrid((16, 8, 8), (1, 1, 1))
    L = B.lib()
    res = ctypes.c_double()
    st = B.Stencil([(0, 0, 0, 0, B.NONE, 0, 1.0)])  # no value term
    ws = ctypes.c_void_p(1 << 30)

    def args(op, wsb):
        return (op, ctypes.byref(st.c), B._handles([u]), 1, B._handles([u]), 1, None,
                ctypes.byref(res), 1, ws, wsb, None)

    assert L.gscl_do_reduce(*args(7, 1 << 22)) == 1
    assert L.gscl_do_reduce(*args(0, 16)) == 6
    assert L.gscl_do_reduce(*args(0, 1 << 22)) == 1
    assert L.gscl_reduce_workspace_bytes() >= 256


def test_status_strings(L):
    for s in range(11):
        assert L.gscl_status_str(s)
    assert b"unknown" in L.gscl_status_str(99)


def test_workload_operators_map_to_compiled_structures(monkeypatch):
    from paper_1207_1746_b300 import stencils as S
    cases = [(S.heat7(0.125), 2, 1, 0), (S.heat7(0.125, with_f=False), 1, 1, 1), (S.poisson_jacobi(), 2, 1, 2),
             (S.jacobi5_2d(), 1, 1, 3), (S.climate(), 8, 3, 4), (S.heat7_fused(0.125), 2, 1, 5),
             (S.heat7_fused(0.125, with_f=False), 1, 1, 6), (S.residual7(), 2, 0, 7), (S.difference(), 2, 0, 8)]
    for terms, nin, nout, want in cases:
        assert B.specialization(terms, nin, nout) == want
        # any order of the same terms, and other weights, still match
        shuffled = [(t[0], t[1], t[2], t[3], t[4], t[5], 0.5 * t[6] + 1.0) for t in reversed(terms)]
        assert B.specialization(shuffled, nin, nout) == want
    # a different structure or grid count falls back to the generic kernel
    assert B.specialization(S.heat7(0.125)[:-1], 2, 1) == -1
    assert B.specialization(S.heat7(0.125), 3, 1) == -1
    assert B.specialization(S.fig1b()[:3] + [(2, 0, 0, 0, B.NONE, 0, 1.0)], 1, 1) == -1
    monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    assert B.specialization(S.heat7(0.125), 2, 1) == -1


def test_ordered_recurrences_map_to_compiled_shapes(monkeypatch):
    """gscl_ordered_specialization on host-only handles: the five compiled
    recurrences in every order and storage dtype, the interpreted paths
    otherwise."""
    from gpu_common import ordered_shape_terms
    monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    n, h = (16, 8, 8), (1, 1, 1)
    for dtype in ("f64", "f32", "bf16"):
        g = [FakeGrid(n, h, dtype) for _ in range(3)]
        interp = -2 if dtype == "bf16" else -1
        for order in (B.J_INC, B.J_DEC, B.K_INC, B.K_DEC):
            for shape in range(5):
                ins = g[:3] if shape >= 2 else g[:2]
                assert B.ordered_specialization(order, ordered_shape_terms(shape, order), ins, g[:1]) == shape
            # the returned value in the loop, and a second output: interpreted
            prev = (0, 0, -1) if order == B.K_INC else (0, 0, 1) if order == B.K_DEC else \
                (0, -1, 0) if order == B.J_INC else (0, 1, 0)
            via_value = [(*prev, 0, B.NONE, B.VALUE, 1.0), (0, 0, 0, 1, B.NONE, B.VALUE, 1.0),
                         (0, 0, 0, B.VALUE, B.NONE, 0, 1.0)]
            assert B.ordered_specialization(order, via_value, g[:2], g[:1]) == interp
            two_out = ordered_shape_terms(0, order) + [(0, 0, 0, 1, B.NONE, 1, 1.0)]
            assert B.ordered_specialization(order, two_out, g[:2], [g[0], g[2]]) == interp
        # more than 8 distinct loads per element: loads per term
        many = [(dx, dy, 0, 1, B.NONE, 0, 1.0) for dx in (-1, 0, 1) for dy in (-1, 0, 1)]
        assert B.ordered_specialization(B.K_INC, many, g[:2], g[:1]) == -2
        # rows along x: staged in shared memory (up to 8 loads per element),
        # the same compiled shapes, the interpreted loop reported as -3
        for order in (B.I_INC, B.I_DEC):
            for shape in range(5):
                ins = g[:3] if shape >= 2 else g[:2]
                assert B.ordered_specialization(order, ordered_shape_terms(shape, order), ins, g[:1]) == shape
            assert B.ordered_specialization(order,
                                            [(-1 if order == B.I_INC else 1, 0, 0, 0, B.NONE, B.VALUE, 1.0),
                                             (0, 0, 0, 1, B.NONE, B.VALUE, 1.0), (0, 0, 0, B.VALUE, B.NONE, 0, 1.0)],
                                            g[:2], g[:1]) == -3
        with pytest.raises(B.GsclError) as e:
            B.ordered_specialization(B.I_INC, many, g[:2], g[:1])
        assert e.value.status == 10
        monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
        assert B.ordered_specialization(B.K_INC, ordered_shape_terms(2, B.K_INC), g, g[:1]) == interp
        monkeypatch.delenv("GSCL_GENERIC_ONLY")
        # alias rules apply as in gscl_do_ordered
        with pytest.raises(B.GsclError):
            B.ordered_specialization(B.K_DEC, ordered_shape_terms(0, B.K_INC), g[:2], g[:1])


def colored_status(terms, ins, outs, color=0, half_sweeps=1):
    st = B.Stencil(terms)
    return B.lib().gscl_do_colored(ctypes.byref(st.c), B._handles(ins), len(ins), B._handles(outs), len(outs), None,
                                   color, half_sweeps, None)


def test_colored_validation_errors():
    """Red-black colouring: in place only through the same grid, and then
    read only at offset 0 or at odd offsets (the other colour)."""
    u, f = FakeGrid((16, 8, 8), (1, 1, 1)), FakeGrid((16, 8, 8), (1, 1, 1))
    gs = [(dx, dy, dz, 0, B.NONE, 0, 1.0 / 6) for dx, dy, dz in
          ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))] + [(0, 0, 0, 1, B.NONE, 0, 1.0 / 6)]
    assert colored_status([(1, 1, 0, 0, B.NONE, 0, 1.0)], [u], [u]) == 3     # same colour
    assert colored_status([(2, 0, 0, 0, B.NONE, 0, 1.0)], [u], [u]) == 2     # beyond the halo
    assert colored_status(gs, [u, f], [u], color=2) == 1
    assert colored_status(gs, [u, f], [u], color=-1) == 1
    assert colored_status(gs, [u, f], [u], half_sweeps=0) == 1
    assert colored_status(gs, [u, f], []) == 1
    # ordinary do_all still refuses the in-place Gauss-Seidel operator
    assert do_all_status(gs, [u, f], [u]) == 3


def diamond_status(terms, ins, outs, rng=None):
    st = B.Stencil(terms)
    return B.lib().gscl_do_diamond(ctypes.byref(st.c), B._handles(ins), len(ins), B._handles(outs), len(outs),
                                   B._range(rng), None)


def test_diamond_validation_errors():
    """do_diamond: an output read in place only in its own plane, at offsets
    whose dx and dy have one sign (elements processed before or after)."""
    x, f = FakeGrid((16, 8, 4), (1, 1, 1)), FakeGrid((16, 8, 4), (1, 1, 1))
    assert diamond_status([(1, -1, 0, 0, B.NONE, 0, 1.0)], [x], [x]) == 3      # mixed signs
    assert diamond_status([(-1, 1, 0, 0, B.NONE, 0, 1.0)], [x], [x]) == 3
    assert diamond_status([(0, 0, 1, 0, B.NONE, 0, 1.0)], [x], [x]) == 3       # another plane
    assert diamond_status([(2, 0, 0, 0, B.NONE, 0, 1.0)], [x], [x]) == 2       # beyond the halo
    assert diamond_status([(0, 0, 0, 0, B.NONE, 0, 1.0)], [x], []) == 1
    # allowed in place (an empty range enqueues nothing, so no GPU is needed)
    empty = ((0, 0, 2), (16, 8, 2))
    ok = [(-1, 0, 0, 0, B.NONE, 0, 1.0), (0, -1, 0, 0, B.NONE, 0, 1.0), (-1, -1, 0, 0, B.NONE, 0, -1.0),
          (1, 1, 0, 0, B.NONE, 0, 0.5), (0, 0, 0, 1, B.NONE, 0, 1.0), (1, -1, 1, 1, B.NONE, 0, 1.0)]
    assert diamond_status(ok, [x, f], [x], rng=empty) == 0


def test_program_compiles_on_the_host_and_reports_errors():
    """NVRTC compiles run-time operators without a GPU; a body that does not
    compile is GSCL_ERR_INVALID with the compiler's message; arguments are
    checked before compiling."""
    p = B.Program("out0 = 0.5 * (in0(1,0,0) + in0(-1,0,0)) + sin(in1(0,0,0)) + (real)i;", 2, 1, "f64")
    assert p.handle
    for dt in ("f32", "bf16"):
        assert B.Program("out0 = in0(0,0,0) * in0(0,0,0); out1 = (real)(i + j + k);", 1, 2, dt, (0, 0, 0)).handle
    with pytest.raises(B.GsclError) as e:
        B.Program("out0 = in0(0,0,0) +;", 1, 1)
    assert e.value.status == 1 and b"did not compile" in B.lib().gscl_last_error()
    with pytest.raises(B.GsclError) as e:
        B.Program("out0 = in1(0,0,0);", 1, 1)          # only in0 exists
    assert e.value.status == 1
    with pytest.raises(B.GsclError) as e:
        B.Program("out0 = 1;", 9, 1)
    assert e.value.status == 10
    with pytest.raises(B.GsclError) as e:
        B.Program("out0 = 1;", 1, 1, reach=(-1, 0, 0))
    assert e.value.status == 1
    L = B.lib()
    assert L.gscl_program_destroy(p.handle) == 0
    assert L.gscl_program_destroy(p.handle) == 8
    p.handle = 0


def test_program_binding_rules():
    """A program runs under do_all's range, halo and alias rules for its
    declared reach; no GPU work happens for an empty range."""
    u, v = FakeGrid((16, 8, 8), (1, 1, 1)), FakeGrid((16, 8, 8), (1, 1, 1))
    fa, fb = FakeGrid((16, 8, 8), (1, 1, 1), "f32"), FakeGrid((16, 8, 8), (1, 1, 1), "f32")
    p = B.Program("out0 = in0(1,0,0);", 1, 1, "f64", (1, 1, 1))
    L = B.lib()

    def run(prog, ins, outs, rng=None, sweeps=1):
        return L.gscl_do_all_program(prog.handle, B._handles(ins), len(ins), B._handles(outs), len(outs),
                                     B._range(rng), sweeps, None)

    assert run(p, [u], [u]) == 3                         # in place needs reach 0
    assert run(p, [u, v], [v]) == 1                      # compiled for one input
    assert run(p, [fa], [fb]) == 4                       # compiled for FP64 grids
    wide = B.Program("out0 = in0(0,0,0);", 1, 1, "f64", (2, 0, 0))
    assert run(wide, [u], [v]) == 2                      # reach beyond the halo
    assert run(p, [u], [v], sweeps=0) == 1
    assert run(p, [u], [v], rng=((0, 0, 3), (16, 8, 3))) == 0


def test_program_reduce_validation():
    u = FakeGrid((16, 8, 8), (1, 1, 1))
    p = B.Program("value = in0(0,0,0);", 1, 0, "f64", (0, 0, 0))
    L = B.lib()
    res = ctypes.c_double()
    ws = ctypes.c_void_p(1 << 30)

    def red(op, result=True, outs=()):
        return L.gscl_do_reduce_program(p.handle, op, B._handles([u]), 1, B._handles(list(outs)), len(outs), None,
                                        ctypes.byref(res) if result else None, 1, ws, 1 << 22, None)

    assert red(7) == 1                    # unknown reduce op
    assert red(0, result=False) == 1      # no result pointer
    assert red(0, outs=[u]) == 1          # compiled for no outputs
    assert L.gscl_do_all_program(p.handle, B._handles([u]), 1, None, 0, None, 1, None) == 1   # do_all needs an output
