"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each mutant is a textual change of ``oracle/lacosmic.cpp`` (a dropped term, a
wrong sign, index, radius or neighbour, a transposed operand, a wrong
threshold). The copy is compiled into a temporary library and the pins of
``oracle_pins`` run against it; if a mutant passes every pin, the pins would
not catch that mistake in the oracle.
"""

import os

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "lacosmic.cpp")

MUTANTS = {
    "lplus_sign": ("std::max(zero, dn + dw)", "std::max(zero, dn - dw)"),
    "lplus_dropped_term": ("acc = acc + std::max(zero, ds + de);", ""),
    "lplus_no_clip": ("acc = acc + std::max(zero, ds + dw);", "acc = acc + (ds + dw);"),
    "lplus_scale": ("out.v[size_t(y) * J.w + x] = quarter * acc;", "out.v[size_t(y) * J.w + x] = acc;"),
    "lplus_wrong_neighbour": ("const T dw = c - J.clamped(x - 1, y);", "const T dw = c - J.clamped(x, y - 1);"),
    "lplus_transposed": ("const T ds = c - J.clamped(x, y + 1);", "const T ds = c - J.clamped(y + 1, x);"),
    "median_rank": ("out.v[size_t(y) * in.w + x] = win[size_t(n / 2)];",
                    "out.v[size_t(y) * in.w + x] = win[size_t(n / 2 + 1)];"),
    "median_index": ("win[size_t(k++)] = in.clamped(x + dx, y + dy);",
                     "win[size_t(k++)] = in.clamped(x + dx, y + dx);"),
    "edge_rule": ("x = std::min(std::max(x, 0), w - 1);", "x = std::min(std::abs(x), w - 1);"),
    "noise_rn": ("const T rn2 = rn * rn;", "const T rn2 = rn;"),
    "noise_gain": ("std::sqrt(gain * m5.v[i] + rn2) / gain;", "std::sqrt(gain * m5.v[i] + rn2);"),
    "s_factor2": ("s.v[i] = lp.v[i] / (T(2) * noise.v[i]);", "s.v[i] = lp.v[i] / noise.v[i];"),
    "sprime_dropped": ("sp.v[i] = s.v[i] - s_med.v[i];", "sp.v[i] = s.v[i];"),
    "med7_radius": ("Map<T> m37 = median_filter(m3, 3);", "Map<T> m37 = median_filter(m3, 2);"),
    "med3_radius": ("Map<T> m3 = median_filter(J, 1);", "Map<T> m3 = median_filter(J, 2);"),
    "f_floor": ("std::max(f.v[i] / noise.v[i], T(0.01));", "std::max(f.v[i] / noise.v[i], T(0.1));"),
    "objlim_form": ("r.v[i] = (p.objlim_form == 1) ? (T(2) * s.v[i]) / fn : sp.v[i] / fn;",
                    "r.v[i] = (T(2) * s.v[i]) / fn;"),
    "objlim_sense": ("(sp.v[i] > sigclip && r.v[i] > objlim)", "(sp.v[i] > sigclip && r.v[i] < objlim)"),
    "grow2_threshold": ("g2.v[i] = (g2.v[i] && sp.v[i] > sigcliplow)", "g2.v[i] = (g2.v[i] && sp.v[i] > sigclip)"),
    "grow1_skipped": ("Map<uint8_t> g1 = dilate3(cand);", "Map<uint8_t> g1 = cand;"),
    "grow2_skipped": ("Map<uint8_t> g2 = dilate3(g1);", "Map<uint8_t> g2 = g1;"),
    "not_cumulative": ("Mk.v[i] = prev | g2.v[i];", "Mk.v[i] = g2.v[i];"),
    "upper_median": ("const size_t k = (n + 1) / 2 - 1;", "const size_t k = n / 2;"),
    "replace_uses_flagged": ("if (!Mk.clamped(x + dx, y + dy)) vals.push_back",
                             "if (true) vals.push_back"),
    "replace_window3": ("for (int dy = -2; dy <= 2; ++dy)\n        for (int dx = -2; dx <= 2; ++dx)\n          if (!Mk",
                        "for (int dy = -1; dy <= 1; ++dy)\n        for (int dx = -1; dx <= 1; ++dx)\n          if (!Mk"),
    "m5_floor_missing": ("if (v <= T(0)) v = T(0.0001);\n  Map<T> noise", "if (v < T(-1e30)) v = T(0.0001);\n  Map<T> noise"),
    "m5_floor_value": ("if (v <= T(0)) v = T(0.0001);", "if (v <= T(0)) v = T(0.01);"),
    "noise_median_radius": ("Map<T> m5 = median_filter(J, 2);", "Map<T> m5 = median_filter(J, 1);"),
    "sprime_median_radius": ("Map<T> s_med = median_filter(s, 2);", "Map<T> s_med = median_filter(s, 1);"),
    "med7_of_image": ("Map<T> m37 = median_filter(m3, 3);", "Map<T> m37 = median_filter(J, 3);"),
    "f_sign": ("f.v[i] = m3.v[i] - m37.v[i];", "f.v[i] = m37.v[i] - m3.v[i];"),
    "r_uses_s": ("sp.v[i] / fn;", "s.v[i] / fn;"),
    "sigfrac_added": ("const T sigcliplow = sigfrac * sigclip;", "const T sigcliplow = sigfrac + sigclip;"),
    "dilate_radius2": ("for (int dy = -1; dy <= 1; ++dy)\n        for (int dx = -1; dx <= 1; ++dx) any |= in.clamped",
                       "for (int dy = -2; dy <= 2; ++dy)\n        for (int dx = -2; dx <= 2; ++dx) any |= in.clamped"),
    # strictness of each of the four threshold comparisons
    "cand_sigclip_nonstrict": ("(sp.v[i] > sigclip && r.v[i] > objlim)", "(sp.v[i] >= sigclip && r.v[i] > objlim)"),
    "cand_objlim_nonstrict": ("(sp.v[i] > sigclip && r.v[i] > objlim)", "(sp.v[i] > sigclip && r.v[i] >= objlim)"),
    "grow1_nonstrict": ("g1.v[i] = (g1.v[i] && sp.v[i] > sigclip)", "g1.v[i] = (g1.v[i] && sp.v[i] >= sigclip)"),
    "grow2_nonstrict": ("g2.v[i] = (g2.v[i] && sp.v[i] > sigcliplow)", "g2.v[i] = (g2.v[i] && sp.v[i] >= sigcliplow)"),
    "none_left_keeps_pixel": ("out.v[i] = m5.v[i];\n        ++none_left;", "out.v[i] = J.v[i];\n        ++none_left;"),
    "new_count_includes_old": ("o.n_new += (g2.v[i] && !prev) ? 1 : 0;", "o.n_new += g2.v[i] ? 1 : 0;"),
    "clamp_y_to_width": ("y = std::min(std::max(y, 0), h - 1);", "y = std::min(std::max(y, 0), w - 1);"),
    "f_floor_unnormalised": ("std::max(f.v[i] / noise.v[i], T(0.01));", "std::max(f.v[i], T(0.01));"),
    "dilate_without_centre": ("for (int dx = -1; dx <= 1; ++dx) any |= in.clamped(x + dx, y + dy);",
                              "for (int dx = -1; dx <= 1; ++dx) if (dx || dy) any |= in.clamped(x + dx, y + dy);"),
    "grow2_from_candidates": ("Map<uint8_t> g2 = dilate3(g1);", "Map<uint8_t> g2 = dilate3(cand);"),
    "article_form_factor": ("r.v[i] = (p.objlim_form == 1) ? (T(2) * s.v[i]) / fn : sp.v[i] / fn;",
                            "r.v[i] = (p.objlim_form == 1) ? s.v[i] / fn : sp.v[i] / fn;"),
    "sprime_median_of_lplus": ("Map<T> s_med = median_filter(s, 2);", "Map<T> s_med = median_filter(lp, 2);"),
    "noise_from_pixel": ("std::sqrt(gain * m5.v[i] + rn2) / gain;", "std::sqrt(gain * J.v[i] + rn2) / gain;"),
    "replace_reads_output": ("if (!Mk.clamped(x + dx, y + dy)) vals.push_back(J.clamped(x + dx, y + dy));",
                             "if (!Mk.clamped(x + dx, y + dy)) vals.push_back(out.clamped(x + dx, y + dy));"),
    "clean_forgets_flags": ("iterate<T>(J.data(), M.data(), w, h, *p, o, false, fragile_any != nullptr);",
                            "iterate<T>(J.data(), nullptr, w, h, *p, o, false, fragile_any != nullptr);"),
    # the fragile map: its tolerance, its cone, and each of its three threshold conditions
    "fragile_tol": ("const double tol = 1e-4;", "const double tol = 10;"),
    "fragile_tol_loose": ("const double tol = 1e-4;", "const double tol = 2e-4;"),
    "fragile_cone_1x1": ("for (int dy = -2; dy <= 2; ++dy)\n          for (int dx = -2; dx <= 2; ++dx) any |= near",
                         "for (int dy = 0; dy <= 0; ++dy)\n          for (int dx = 0; dx <= 0; ++dx) any |= near"),
    "fragile_cone_3x3": ("for (int dy = -2; dy <= 2; ++dy)\n          for (int dx = -2; dx <= 2; ++dx) any |= near",
                         "for (int dy = -1; dy <= 1; ++dy)\n          for (int dx = -1; dx <= 1; ++dx) any |= near"),
    "fragile_no_sigclip": ("const bool a = std::fabs(spv - c) <= tol * c;", "const bool a = false;"),
    "fragile_no_sigfrac": ("const bool b = std::fabs(spv - c2) <= tol * c2;", "const bool b = false;"),
    "fragile_no_objlim": ("const bool d = spv > c * (1.0 - tol) && std::fabs(rv - ol) <= tol * ol;",
                          "const bool d = false;"),
    "fragile_objlim_ungated": ("const bool d = spv > c * (1.0 - tol) && std::fabs(rv - ol) <= tol * ol;",
                               "const bool d = std::fabs(rv - ol) <= tol * ol;"),
    "fragile_objlim_gated_low": ("const bool d = spv > c * (1.0 - tol) && std::fabs(rv - ol) <= tol * ol;",
                                 "const bool d = spv > c2 * (1.0 - tol) && std::fabs(rv - ol) <= tol * ol;"),
    "fragile_union_last": ("fragile_any[i] |= o.fragile[i];", "fragile_any[i] = o.fragile[i];"),
}


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, tmp_path):
    find, repl = MUTANTS[name]
    assert source.count(find) >= 1, f"mutation site of {name} not found"
    src = tmp_path / "lacosmic_mut.cpp"
    src.write_text(source.replace(find, repl, 1))
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / "libmut.so"))
    orc = oracle.Oracle(lib)
    orc.lib.oracle_set_threads(2)
    caught = None
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except Exception as e:  # noqa: BLE001 - a crash also counts as caught
            caught = f"{pin.__name__}: {type(e).__name__}"
            break
    assert caught, f"mutant {name} passed every pin"
