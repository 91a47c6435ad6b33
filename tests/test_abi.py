"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every function include/fwi.h declares; the
leapfrog stability limit it reports matches an independent computation."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from paper_2110_03345_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fwi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.EXPORTS)


def test_library_is_built_for_sm_103a():
    # the fatbin of an sm_103a build carries the architecture name
    data = open(build.build(), "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_last_error_empty_and_cfl_limits():
    lib = binding.load()
    assert isinstance(lib.fwi_last_error(), bytes)
    # lambda_max of the exact central weights (Fornberg) -> 2/sqrt(d lambda)
    for order, w in ((8, [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315),
                          Fraction(-1, 560)]),
                     (10, [Fraction(-5269, 1800), Fraction(5, 3), Fraction(-5, 21),
                           Fraction(5, 126), Fraction(-5, 1008), Fraction(1, 3150)])):
        lam = abs(w[0] + 2 * sum((-1) ** j * w[j] for j in range(1, len(w))))
        for d in (2, 3):
            assert binding.cfl_limit(d, order) == pytest.approx(2 / np.sqrt(d * float(lam)), rel=1e-14)
    assert binding.cfl_limit(4, 8) < 0 and binding.cfl_limit(2, 6) < 0


def test_paper_homogeneous_setup_is_within_the_limit():
    """Sec. 3.1 runs the homogeneous case at c = 1500 m/s, 0.250 mm and 0.060 us
    (the paper's CFL 0.36, see tests/golden/paper_sec31_setup.txt); that CFL
    is stable for this leapfrog in 2D and 3D at both orders."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "paper_sec31_setup.txt"))
            if l.strip() and not l.startswith("#")]
    for c, dx, dt, cfl in ((float(a), float(b), float(c_), float(d)) for a, b, c_, d in rows):
        assert c * dt / dx == pytest.approx(cfl, abs=5e-3)
        for d in (2, 3):
            for order in (8, 10):
                assert cfl < binding.cfl_limit(d, order)


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the no-GPU path")
def test_no_cpu_fallback_without_a_gpu():
    """Without a GPU the solver calls raise: there is no CPU path to fall back to."""
    with pytest.raises(Exception):
        binding.Plan((64, 64), 1e-3, 20, 1e-7)
    lib = binding.load()
    plan = ctypes.c_void_p()
    g = binding.make_grid((64, 64), 1e-3, 8, 8, 1500.0)
    status = lib.fwi_plan_create(ctypes.byref(plan), ctypes.byref(g), 20, 1e-7, 0, None)
    assert status == 4   # FWI_ERR_CUDA: no device
    assert len(lib.fwi_last_error()) > 0


def test_inversion_entry_points_validate_on_the_host():
    """fwi_lowpass and fwi_vp_update reject bad arguments before any device
    work (so these calls need no GPU), and an empty request is a no-op."""
    lib = binding.load()
    P = ctypes.POINTER(ctypes.c_int)
    ids = (ctypes.c_int * 2)(0, 3)
    fake_in, fake_out = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x90000)
    lp = lib.fwi_lowpass
    assert lp(fake_in, 2, 1, 100, ids, 0, 1e-7, 1e6, 8, fake_out, None) == 0      # no ids
    assert lp(fake_in, 2, 1, 100, ids, -1, 1e-7, 1e6, 8, fake_out, None) == 1
    assert lp(None, 2, 1, 100, ids, 1, 1e-7, 1e6, 8, fake_out, None) == 1
    assert lp(fake_in, 2, 1, 100, ids, 2, 1e-7, 1e6, 8, fake_out, None) == 1       # id 3 >= n_in
    assert b"outside" in lib.fwi_last_error()
    assert lp(fake_in, 4, 1, 100, ids, 2, 1e-7, 1e6, 2049, fake_out, None) == 1    # half-width
    assert lp(fake_in, 4, 1, 100, ids, 2, 0.0, 1e6, 8, fake_out, None) == 1        # dt
    assert lp(fake_in, 4, 1, 100, ids, 2, 1e-7, 1e6, 8, fake_in, None) == 1        # overlap
    assert lp(fake_in, 4, 70000, 100, ids, 2, 1e-7, 1e6, 8, fake_out, None) == 1   # rows
    up = lib.fwi_vp_update
    assert up(fake_in, fake_in, None, 0, 1.0, 1.0, 2.0, fake_out, None) == 0       # n = 0
    assert up(fake_in, fake_in, None, -5, 1.0, 1.0, 2.0, fake_out, None) == 1
    assert up(None, fake_in, None, 5, 1.0, 1.0, 2.0, fake_out, None) == 1
    assert up(fake_in, fake_in, None, 5, -1.0, 1.0, 2.0, fake_out, None) == 1      # step < 0
    assert up(fake_in, fake_in, None, 5, 1.0, 2.0, 1.0, fake_out, None) == 1       # bounds
    assert up(fake_in, fake_in, None, 5, float("nan"), 1.0, 2.0, fake_out, None) == 1


def test_grids_beyond_32_bit_field_offsets_are_rejected_on_the_host():
    """A padded field must hold fewer than 2^31 floats (in-field offsets are
    32-bit) and the second-fastest axis at most 524280 points (grid.y); larger
    grids fail with FWI_ERR_INVALID_ARG before any device call."""
    lib = binding.load()
    for shape in [(1300, 1300, 1300), (1 << 20, 4096), (40000, 60000),
                  (600000, 20), (20, 600000, 20)]:                   # grid.y beyond 65535 CTAs
        plan = ctypes.c_void_p()
        g = binding.make_grid(shape, 1e-3, 8, 8, 1500.0)
        assert lib.fwi_plan_create(ctypes.byref(plan), ctypes.byref(g), 20, 1e-7, 0, None) == 1
        assert b"2^31" in lib.fwi_last_error() or b"524280" in lib.fwi_last_error()
    for shape in [(1200, 1200, 1200), (20000, 20000)]:              # below the limit
        plan = ctypes.c_void_p()
        g = binding.make_grid(shape, 1e-3, 8, 8, 1500.0)
        st = lib.fwi_plan_create(ctypes.byref(plan), ctypes.byref(g), 20, 1e-7, 0, None)
        assert st != 1, lib.fwi_last_error()
        if st == 0:
            lib.fwi_plan_destroy(plan)


@pytest.mark.parametrize("shape,spacing", [((40, 44), (0.5e-3, 0.4e-3)),
                                           ((20, 22, 24), (0.5e-3, 0.5e-3, 0.45e-3))])
def test_point_weights_match_the_oracle(shape, spacing):
    """fwi_point_weights (host only): the solver's bi-/tri-linear corners and
    the Kaiser-windowed sinc weights equal the oracle's (oracle.point_weights,
    oracle.sinc, each pinned), node for node."""
    import oracle
    from oracle import sinc
    g = oracle.Grid(shape, spacing, dt=1e-7, nt=2)
    rng = np.random.default_rng(5)
    for _ in range(6):
        p = np.array([rng.uniform(4, n - 5) * h for n, h in zip(shape, spacing)])
        for interp, ref in ((binding.INTERP_LINEAR, oracle.point_weights),
                            (binding.INTERP_SINC, sinc.hicks())):
            nodes, w = binding.point_weights(shape, spacing, p, interp)
            idx_ref, w_ref = ref(g, p)
            flat = np.ravel_multi_index(nodes.T, shape)
            order, order_ref = np.argsort(flat), np.argsort(idx_ref)
            np.testing.assert_array_equal(flat[order], np.asarray(idx_ref)[order_ref])
            np.testing.assert_allclose(w[order], np.asarray(w_ref)[order_ref], rtol=0, atol=1e-13)
    lib = binding.load()
    gc = binding.make_grid(shape, spacing, 8, 0, 0.0)
    cnt = ctypes.c_int(0)
    edge = (ctypes.c_double * len(shape))(*([1.5 * spacing[0]] + [10 * h for h in spacing[1:]]))
    assert lib.fwi_point_weights(ctypes.byref(gc), edge, binding.INTERP_SINC, None, None, 0,
                                 ctypes.byref(cnt)) == 1            # too close to a face
    nodes, w = binding.point_weights(shape, spacing, [1.5 * spacing[0]] + [10 * h for h in spacing[1:]])
    assert len(w) == 2 ** len(shape) and abs(w.sum() - 1.0) < 1e-14   # bilinear works there
