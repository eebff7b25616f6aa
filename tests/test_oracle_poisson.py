"""The POISSON work function oracle (Sec. 6.3.2) against what mathematics fixes (the pins of
``poisson_pins``), and planted mistakes in copies of it, each of which a pin must catch."""

from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import poisson_pins as pp

GAMMA = 0x9E3779B97F4A7C15
M64 = 2**64 - 1
SRC = os.path.join(os.path.dirname(oracle.__file__), "poisson.cpp")


@pytest.fixture(scope="module")
def lib():
    return pp.PoissonLib(oracle.build_poisson())


def test_exp_neg_matches_libm(lib):
    pp.pin_exp_neg(lib)


def test_algorithm_q_hand_cases(lib):
    pp.pin_algorithm_q_hand_cases(lib)


@pytest.mark.parametrize("mu,shape", [(24.3, (750, 750)), (0.7, (300, 300)), (300.0, (200, 200))])
def test_deviates_follow_the_poisson_law(lib, mu, shape):
    pp.pin_poisson_law(lib, mu, shape)


def test_seeds_and_edge_values(lib):
    pp.pin_seeds_and_edges(lib)


def test_stream_published_outputs(lib):
    pp.pin_stream_published_outputs(lib)


def test_stream_value_arithmetic(lib):
    """The C stream's 64-bit arithmetic against Python integers (a cross-check of the build, not a pin)."""
    def mix13(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    for s, j in [(0, 0), (0, 1), (1, 0), (M64, 5), (123456789, 2**40), (0xDEADBEEF, 3)]:
        assert lib.stream_value(s, j) == mix13((s + (j + 1) * GAMMA) & M64)


def test_uniforms_are_uniform(lib):
    from scipy import stats
    v = np.array([lib.stream_value(7, j) >> 11 for j in range(200_000)], dtype=np.float64) * 2.0**-53
    assert v.min() >= 0.0 and v.max() < 1.0
    assert stats.kstest(v, "uniform").pvalue > 1e-6
    assert abs(np.corrcoef(v[:-1], v[1:])[0, 1]) < 0.01  # successive draws: no linear correlation


MUTANTS = {
    "off_by_one": ("  return k;\n}", "  return k + 1;\n}"),
    "strict_comparison": ("while (q >= L && k < kQMax)", "while (q > L && k < kQMax)"),
    "exp_sign": ("const double x = -mu;", "const double x = mu;"),
    "exp_short_polynomial": ("double p = c[13];\n  for (int i = 12; i >= 0; --i)", "double p = c[5];\n  for (int i = 4; i >= 0; --i)"),
    "exp_no_scaling": ("return std::ldexp(p, int(n));", "return p;"),
    "uniform_scale": ("double(v >> 11) * 0x1.0p-53", "double(v >> 11) * 0x1.0p-52"),
    "mean_cap": ("constexpr double kMuMax = 700.0;", "constexpr double kMuMax = 70.0;"),
    "seed_ignored": ("const uint64_t key = stream_value(seed, uint64_t(p));",
                     "const uint64_t key = stream_value(0, uint64_t(p));"),
    "first_factor_skipped": ("double q = u(0);", "double q = 1.0;"),
    "mix_shift": ("z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;", "z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ULL;"),
    "mix_constant": ("z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;", "z = (z ^ (z >> 27)) * 0x94d049bb133111ecULL;"),
    "gamma": ("constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;", "constexpr uint64_t kGamma = 0x9e3779b97f4a7c17ULL;"),
    "counter_offset": ("return mix13(s + (j + 1) * kGamma);", "return mix13(s + j * kGamma);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    with open(SRC) as f:
        source = f.read()
    find, repl = MUTANTS[name]
    assert source.count(find) == 1, f"mutation site of {name} not found"
    src = tmp_path / "poisson_mut.cpp"
    src.write_text(source.replace(find, repl, 1))
    path = oracle.build(force=True, src=str(src), out=str(tmp_path / "libpoisson_mut.so"))
    mut = pp.PoissonLib(path)
    caught = None
    for pin in pp.ALL_PINS:
        try:
            pin(mut)
        except Exception as e:  # noqa: BLE001 - a crash also counts as caught
            caught = f"{pin.__name__}: {type(e).__name__}"
            break
    assert caught, f"mutant {name} passed every pin"
