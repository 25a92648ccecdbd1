"""The pipelined co-processing cost model (PL, Sec. 4, Eq. 1-5) and its exhaustive
ratio search, as host arithmetic (no GPU).  Expected values are worked out by hand
from the printed equations."""
import itertools

import pytest

from paper_1307_1955_gb300 import build as B


@pytest.fixture(scope="module")
def hjm():
    B.build()
    from paper_1307_1955_gb300 import hj

    hj.load_library()
    return hj


def test_equal_ratios_have_no_delay(hjm):
    # DD (one ratio for every step): T_XPU is the plain sum of Eq. 2-3 per processor
    x, c, g = [100.0, 50.0, 200.0], [2.0, 1.0, 0.5], [1.0, 3.0, 0.25]
    for r in (0.0, 0.3, 1.0):
        t, tc, tg = hjm.hj_coproc_time(x, c, g, [r] * 3, xfer_s=7.0)
        assert tc == pytest.approx(r * (200 + 50 + 100))
        assert tg == pytest.approx((1 - r) * (100 + 150 + 50))
        assert t == max(tc, tg)


def test_eq4_cpu_waits_for_the_gpu(hjm):
    # r = (0.1, 0.9): step 0 CPU 0.1*0.1*100 = 1, GPU 10*0.9*100 = 900; step 1 CPU
    # 2*0.9*100 = 180, GPU 0.1*0.1*100 = 1.  Eq. 4: D = (900 - 900 * 0.1/0.9) - (1 + 180)
    # = 619, so T_CPU = 1 + 180 + 619 = 800 (the GPU's end of the pipelined area in
    # step 0) and T_GPU = 901.
    t, tc, tg = hjm.hj_coproc_time([100, 100], [0.1, 2.0], [10.0, 0.1], [0.1, 0.9])
    assert tc == pytest.approx(800.0) and tg == pytest.approx(901.0) and t == pytest.approx(901.0)


def test_eq5_gpu_waits_for_the_cpu(hjm):
    # r = (0.9, 0.1): step 0 CPU 10*0.9*100 = 900, GPU 0.1*0.1*100 = 1; step 1 CPU
    # 1*0.1*100 = 10, GPU 1*0.9*100 = 90.  Eq. 5: D = 900 - ((1 + 90) - 90 * 0.1/0.9)
    # = 819, so T_GPU = 1 + 90 + 819 = 910 and T_CPU = 910.
    t, tc, tg = hjm.hj_coproc_time([100, 100], [10.0, 1.0], [0.1, 1.0], [0.9, 0.1])
    assert tg == pytest.approx(910.0) and tc == pytest.approx(910.0) and t == pytest.approx(910.0)


def test_negative_delays_are_clamped(hjm):
    # r = (0.2, 0.6), unit costs: Eq. 4 gives (80 - 80 * 0.4/0.8) - (20 + 60) = -40 -> 0
    t, tc, tg = hjm.hj_coproc_time([100, 100], [1.0, 1.0], [1.0, 1.0], [0.2, 0.6])
    assert tc == pytest.approx(80.0) and tg == pytest.approx(120.0) and t == pytest.approx(120.0)


def test_intermediate_results_cost_the_receiver(hjm):
    # 0.4 * 100 items move from the GPU to the CPU between the steps, 0.5 s each
    base = hjm.hj_coproc_time([100, 100], [1.0, 1.0], [1.0, 1.0], [0.2, 0.6])
    moved = hjm.hj_coproc_time([100, 100], [1.0, 1.0], [1.0, 1.0], [0.2, 0.6], xfer_s=0.5)
    assert moved[1] == pytest.approx(base[1] + 0.4 * 100 * 0.5) and moved[2] == pytest.approx(base[2])


def test_search_splits_a_step_between_equal_processors(hjm):
    r, t = hjm.hj_coproc_ratios([1000.0], [1.0], [1.0])
    assert r == [pytest.approx(0.5)] and t == pytest.approx(500.0)


def test_search_is_the_minimum_over_its_grid(hjm):
    # brute force over every ratio vector of a 3-step series at delta = 0.1
    x, c, g = [300.0, 100.0, 200.0], [1.0, 4.0, 0.5], [2.0, 0.5, 1.5]
    grid = [round(0.1 * k, 10) for k in range(11)]
    best = min(hjm.hj_coproc_time(x, c, g, list(rv), xfer_s=0.2)[0] for rv in itertools.product(grid, repeat=3))
    r, t = hjm.hj_coproc_ratios(x, c, g, xfer_s=0.2, delta=0.1)
    assert t == pytest.approx(best)
    assert hjm.hj_coproc_time(x, c, g, r, xfer_s=0.2)[0] == pytest.approx(t)


def test_a_much_slower_cpu_gets_nothing(hjm):
    # the GB300 situation: the oracle's single core is ~3000x slower per tuple than
    # the GPU, so every step stays on the GPU (OL with all ratios 0)
    x = [2.85e8, 2.85e8, 2.85e8]
    g = [0.36e-3 / 2.85e8, 1.50e-3 / 2.85e8, 1.04e-3 / 2.85e8]
    c = [1.0 / 3.1e7] * 3
    r, t = hjm.hj_coproc_ratios(x, c, g)
    assert r == [0.0, 0.0, 0.0]
    assert t == pytest.approx(sum(gi * xi for gi, xi in zip(g, x)))


def test_invalid_arguments(hjm):
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_coproc_ratios([1.0], [1.0], [1.0], delta=0.0)
    assert e.value.status == hjm.HJ_E_INVALID
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_coproc_time([-1.0], [1.0], [1.0], [0.5])
    assert e.value.status == hjm.HJ_E_INVALID
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_coproc_time([1.0], [1.0], [1.0], [1.5])
    assert e.value.status == hjm.HJ_E_INVALID
    with pytest.raises(hjm.HJError) as e:  # 51^8 ratio vectors
        hjm.hj_coproc_ratios([1.0] * 8, [1.0] * 8, [1.0] * 8)
    assert e.value.status == hjm.HJ_E_UNSUPPORTED


def test_tiny_delta_is_refused_before_the_grid_is_built(hjm):
    # 1 / delta = 1e12 grid points per ratio: refused at once, without building the
    # grid (or converting 1e12 to an int)
    for d in (1e-12, 1e-9):
        with pytest.raises(hjm.HJError) as e:
            hjm.hj_coproc_ratios([1.0], [1.0], [1.0], delta=d)
        assert e.value.status == hjm.HJ_E_UNSUPPORTED
