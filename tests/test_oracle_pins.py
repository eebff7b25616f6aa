"""The oracle against its pins (CPU only)."""

import pytest

import oracle
import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.Oracle())


def test_star_margin_report():
    """Records the objlim margin of the FWHM-2 star (script form below 1, article form above)."""
    rs, _ = oracle_pins.star_margin(oracle.Oracle(), 0)
    ra, _ = oracle_pins.star_margin(oracle.Oracle(), 1)
    print(f"star R max: script form {rs:.3f}, article form {ra:.3f} (objlim 1.0)")
    assert rs < 1.0 < ra


def test_oracle_result_does_not_depend_on_the_thread_count():
    """Rows are independent in every stage, so the oracle gives the same bytes on 1 and on many threads
    (its timed CPU baseline runs on all cores, its tests on fewer)."""
    import numpy as np

    import synth
    img = synth.frame(211, 157, seed=5, sky=100.0, nstars=10, ncr=80)
    P = oracle.Params()
    outs = []
    orig = oracle.max_threads()
    try:
        for n in (1, 4):
            oracle.set_threads(n)
            for prec in ("f64", "f32"):
                r = oracle.clean(img, P, 4, precision=prec, fragile=(prec == "f64"))
                outs.append((n, prec, r))
    finally:
        oracle.set_threads(orig)
    for prec in ("f64", "f32"):
        a, b = [r for n, p, r in outs if p == prec]
        assert np.array_equal(a.clean, b.clean) and np.array_equal(a.mask, b.mask)
        assert a.n_new == b.n_new and a.n_none_left == b.n_none_left
        if prec == "f64":
            assert np.array_equal(a.fragile, b.fragile)
