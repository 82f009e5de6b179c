"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle package to a temporary directory, plants one
mistake in the C source (a wrong sign, a dropped term, an off-by-one index,
a wrong permutation), compiles it and runs a compact set of pin checks.  Every
planted mistake must make at least one check fail, and the unmodified copy
must pass them all.  Nothing here touches the real oracle build.
"""
import importlib.util
import os
import shutil
import sys

import numpy as np
import pytest

import qft_inputs

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTANTS = {
    "cp_sign": ("const double theta = sign * ORACLE_TWO_PI / ldexp(1.0, m);",
                "const double theta = -sign * ORACLE_TWO_PI / ldexp(1.0, m);"),
    "cp_order_off_by_one": ("apply_cp(psi, n, t - d, t, d + 1, sign)",
                            "apply_cp(psi, n, t - d, t, d + 2, sign)"),
    "cp_dropped_last_distance": ("for (int d = 1; d <= kk && d <= t; d++) apply_cp",
                                 "for (int d = 1; d < kk && d <= t; d++) apply_cp"),
    "cp_wrong_control": ("apply_cp(psi, n, t - d, t, d + 1, sign)",
                         "apply_cp(psi, n, (t + d) % n, t, d + 1, sign)"),
    "h_wrong_wire": ("        apply_h(psi, n, t);", "        apply_h(psi, n, n - 1 - t);"),
    "h_butterfly_sign": ("psi[2 * i1 + 1] = (ai - bi) * r;", "psi[2 * i1 + 1] = (bi - ai) * r;"),
    "h_unnormalised": ("const double r = 1.0 / sqrt(2.0);", "const double r = 1.0;"),
    "swap_wrong_partner": ("bk = (int64_t)1 << (n - 1 - j);", "bk = (int64_t)1 << (n - 2 - j);"),
    "dft_sign": ("const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);\n            const double c = cos(th), s = sin(th);\n            sr += x[2 * j] * c - x[2 * j + 1] * s;\n            si += x[2 * j] * s + x[2 * j + 1] * c;\n        }\n        X[2 * y]",
                 "const double th = -sign * ORACLE_TWO_PI * ldexp((double)p, -n);\n            const double c = cos(th), s = sin(th);\n            sr += x[2 * j] * c - x[2 * j + 1] * s;\n            si += x[2 * j] * s + x[2 * j + 1] * c;\n        }\n        X[2 * y]"),
    "closed_form_window": ("int jlo = n - 1 - kk - i;", "int jlo = n - kk - i;"),
    "encode_norm_squared": ("const double scale_in = sqrt(s);", "const double scale_in = s;"),
    "decode_unnorm_scale": ("else if (mode == 2) f = scale_in * rootN;", "else if (mode == 2) f = scale_in * rootN * rootN;"),
    "counts_off_by_one": ("for (int d = 1; d <= kk && d <= t; d++) cp++;",
                          "for (int d = 0; d <= kk && d <= t; d++) cp++;"),
    "mc_weight_not_divided_by_p": ("const double f = (double)T / (double)q;", "const double f = 1.0;"),
    "mc_phase_sign": ("const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);\n            const double c = cos(th), s = sin(th);\n            const double zr",
                      "const double th = -sign * ORACLE_TWO_PI * ldexp((double)p, -n);\n            const double c = cos(th), s = sin(th);\n            const double zr"),
    "mc_power_biased": ("(sr * sr + si * si - sq) / (M * (M - 1.0))", "(sr * sr + si * si) / (M * M)"),
    "mc_proposal_uniform": ("return (sh < 64 ? sig >> sh : 0) + 1;", "return (uint64_t)1 << 20;"),
    "mc_proposal_real_part_only": ("    return a > b ? a : b;\n}\n\n/* q_j", "    return a | 1;\n}\n\n/* q_j"),
}


def _load_copy(tmp_path, name, mutation):
    dst = tmp_path / name
    shutil.copytree(ORACLE_DIR, dst, ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    src = dst / "qft_oracle.c"
    text = src.read_text()
    if mutation is not None:
        old, new = mutation
        assert text.count(old) == 1, f"mutation anchor not unique: {name}"
        text = text.replace(old, new)
        src.write_text(text)
    modname = f"oracle_copy_{name}"
    spec = importlib.util.spec_from_file_location(modname, dst / "__init__.py",
                                                  submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[modname] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _pin_failures(o):
    """Compact pin suite; returns the names of the checks that fail."""
    from scipy.linalg import hadamard

    bad = []
    n = 5
    N = 1 << n
    x = qft_inputs.gaussian(n, seed=77, normalise=False)
    for sign, ref in ((-1, np.fft.fft(x)), (+1, np.fft.ifft(x) * N)):
        out, _ = o.qft(x, k=-1, sign=sign, mode=o.SCALE_UNNORM)
        if _rel(out, ref) > 1e-12:
            bad.append(f"qft_vs_numpy_{sign}")
        if _rel(o.dft(x, sign), ref) > 1e-12:
            bad.append(f"dft_vs_numpy_{sign}")
    xn = x / np.linalg.norm(x)
    for k in range(n):
        if _rel(o.circuit(xn, k=k), o.aqft_direct(xn, k=k)) > 1e-12:
            bad.append(f"aqft_closed_form_k{k}")
    rev = np.array([int(format(i, f"0{n}b")[::-1], 2) for i in range(N)])
    if _rel(o.circuit(xn, k=0), (hadamard(N) @ xn / np.sqrt(N))[rev]) > 1e-12:
        bad.append("k0_walsh_hadamard")
    if o.gate_counts(22, 16)[1] != 216 or o.gate_counts(22, 4)[1] != 78:
        bad.append("table2")
    _, s = o.encode(x)
    if abs(s - np.linalg.norm(x)) > 1e-12 * np.linalg.norm(x):
        bad.append("encode_norm")
    # Monte Carlo backend (Sec. 6): a tone on its own bin is exact; over many
    # runs the mean and the power estimate are unbiased; the draw frequencies
    # follow |x_j|
    nt, k0 = 6, 16  # bin N/4: x_j = i^j, uniform proposal
    tone = np.exp(2j * np.pi * k0 * np.arange(1 << nt) / (1 << nt))
    rng = np.random.default_rng(1)
    idx, w, _ = o.mc_sample(tone, rng.integers(0, 2 ** 53, 64).astype(np.float64) / 2.0 ** 53)
    amp, _, _ = o.mc_bins(idx, w, nt, [k0], -1, -1)
    if abs(amp[0] - np.sqrt(1 << nt)) > 1e-9:
        bad.append("mc_tone_exact")
    xg = qft_inputs.gaussian(nt, seed=5, normalise=False)
    ys = np.array([0, 3, 40])
    ref = o.aqft_bins(xg, ys, -1, -1)
    amps, pows = [], []
    for _ in range(300):
        idx, w, _ = o.mc_sample(xg, rng.integers(0, 2 ** 53, 32).astype(np.float64) / 2.0 ** 53)
        a, p, _ = o.mc_bins(idx, w, nt, ys, -1, -1)
        amps.append(a)
        pows.append(p)
    amps, pows = np.array(amps), np.array(pows)
    if np.any(np.abs(amps.mean(0) - ref) > 5 * amps.std(0) / np.sqrt(300)):
        bad.append("mc_unbiased_mean")
    if np.any(np.abs(pows.mean(0) - np.abs(ref) ** 2) > 5 * pows.std(0) / np.sqrt(300)):
        bad.append("mc_unbiased_power")
    K = 1 << 14
    idx, _, _ = o.mc_sample(xg, np.arange(K) / K)
    freq = np.bincount(idx, minlength=1 << nt) / K
    mag = np.maximum(np.abs(xg.real), np.abs(xg.imag))
    if np.max(np.abs(freq - mag / mag.sum())) > 1e-3:
        bad.append("mc_draw_law")
    return bad


def test_unmodified_copy_passes(tmp_path):
    o = _load_copy(tmp_path, "clean", None)
    assert _pin_failures(o) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    o = _load_copy(tmp_path, name, MUTANTS[name])
    assert _pin_failures(o), f"planted mistake {name} was not caught by any pin"
