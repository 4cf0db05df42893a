"""The oracle's pins have teeth: plausible mistakes planted in a copy of the
oracle (a dropped term, a wrong modulus, sign, index or operand) must each
make tests/test_oracle_pins.py fail.  Everything runs on the CPU; the planted
copies are compiled into a temporary directory and never used elsewhere."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "9a_wrong_modulus": ("s = or_mulmod(a, s, p);", "s = or_mulmod(a, s, n);"),
    "9b_dropped_m": ("m = (uint64_t)(((u128)m + s) % n);", "m = (uint64_t)(((u128)s) % n);"),
    "9b_wrong_sign": ("m = (uint64_t)(((u128)m + s) % n);",
                      "m = (uint64_t)(((u128)m + n - s % n) % n);"),
    "9c_transposed": ("uint64_t c = or_powmod(m, e, n);", "uint64_t c = or_powmod(s, e, n);"),
    "9d_dropped_plus1": ("return (double)(c + 1) / (double)(n + 1);",
                         "return (double)(c) / (double)(n + 1);"),
    "9d_wrong_denominator": ("return (double)(c + 1) / (double)(n + 1);",
                             "return (double)(c + 1) / (double)(n);"),
    "powmod_wrong_square": ("base = or_mulmod(base, base, n);",
                            "base = or_mulmod(base, result, n);"),
    "mulmod_off_by_one": ("return (x * y) % n;", "return (x * y + 1) % n;"),
    "skip_dropped_cycle_term": ("st[0] = (uint64_t)(((u128)m + add + sum % n) % n);",
                                "st[0] = (uint64_t)(((u128)m + sum % n) % n);"),
    "skip_wrong_cycle_length": ("uint64_t q = k / (p - 1), r = k % (p - 1);",
                                "uint64_t q = k / p, r = k % p;"),
    "state_at_wrap_index": ("+ or_pref(p, a, table, stride, hi - (p - 1));",
                            "+ or_pref(p, a, table, stride, hi - p);"),
    "state_at_s_index": ("st_out[1] = or_powmod(a, L0 + r, p);",
                         "st_out[1] = or_powmod(a, L0 + r + 1, p);"),
    "table_entry": ("if (i % stride == 0) table[j++] = sum;",
                    "if (i % stride == 0) table[j++] = sum - x;"),
    "pref_tail_index": ("for (uint64_t i = j * stride + 1; i <= t; ++i) {",
                        "for (uint64_t i = j * stride + 1; i < t; ++i) {"),
    "stats_square": ("Y += v * v;", "Y += v * (v - 1);"),
    "stats_hist_scale": ("int b = (int)(R * 256.0);", "int b = (int)(R * 255.0);"),
    "stats_var_N": ("u128 num = (u128)N * Y - X * X;", "u128 num = (u128)(N - 1) * Y - X * X;"),
    "corr_transposed": ("Z += ((u128)ca[k] + 1) * ((u128)cb[k] + 1);",
                        "Z += ((u128)ca[k] + 1) * ((u128)ca[k] + 1);"),
    "serial_overlapping_tuples": ("double R = or_real(c[t * (uint64_t)D + (uint64_t)d], n);",
                                  "double R = or_real(c[t + (uint64_t)d], n);"),
    "serial_scale_order": ("scale *= B;", "scale *= B - 1;"),
    "serial_bin_scale": ("uint64_t b = (uint64_t)(R * (double)B);",
                         "uint64_t b = (uint64_t)(R * (double)(B - 1));"),
    "serial_exact_integer_bin": (
        "double R = or_real(c[t * (uint64_t)D + (uint64_t)d], n);\n            uint64_t b = (uint64_t)(R * (double)B);",
        "double R = or_real(c[t * (uint64_t)D + (uint64_t)d], n);\n"
        "            uint64_t b = (uint64_t)(((u128)B * (c[t * (uint64_t)D + (uint64_t)d] + 1)) / ((u128)n + 1));"
        " (void)R;"),
    "interstream_exact_integer_bin": (
        "double R = or_real(c[a * L + j], nmod[a]);\n            uint64_t b = (uint64_t)(R * (double)B);",
        "double R = or_real(c[a * L + j], nmod[a]);\n"
        "            uint64_t b = (uint64_t)(((u128)B * (c[a * L + j] + 1)) / ((u128)nmod[a] + 1)); (void)R;"),
    "collision_exact_integer_bin": (
        "uint64_t b = (uint64_t)(or_real(c[k], n) * (double)B);\n            if (b >= B) b = B - 1;\n"
        "            if (seen[b]) ++C;",
        "uint64_t b = (uint64_t)(((u128)B * (c[k] + 1)) / ((u128)n + 1));\n            if (b >= B) b = B - 1;\n"
        "            if (seen[b]) ++C;"),
    "interstream_transposed": ("double R = or_real(c[a * L + j], nmod[a]);",
                               "double R = or_real(c[(j * Np + a) % (Np * L)], nmod[a]);"),
    "interstream_wrong_modulus": ("double R = or_real(c[a * L + j], nmod[a]);",
                                  "double R = or_real(c[a * L + j], nmod[0]);"),
    "poker_full_house": ("else if (threes && pairs) cat = 4;", "else if (threes) cat = 4;"),
    "poker_denominations": ("int d = (int)(or_real(c[t * 5 + (uint64_t)k], n) * 10.0);",
                            "int d = (int)(or_real(c[t * 5 + (uint64_t)k], n) * 9.0);"),
    "runs_threshold": ("int b = or_real(c[k], n) > 0.5;", "int b = or_real(c[k], n) >= 0.5;"),
    "runs_length_reset": ("        len = 1;\n    }", "        len = 0;\n    }"),
    "pattern_skip_modulus": ("                t = or_mulmod(a, t, p);", "                t = or_mulmod(a, t, n);"),
    "pattern_encrypts_not_decrypts": ("uint64_t m = or_powmod(c0, d, n);", "uint64_t m = or_powmod(c0, e, n);"),
    "collision_counts_distinct": ("            if (seen[b]) ++C;", "            if (!seen[b]) ++C;"),
    "collision_no_reset": ("            seen[b] = 0;\n", "            seen[b] = 1;\n"),
    "pattern_const_offset": ("uint64_t mj = (uint64_t)(((u128)m + (u128)j * (b % n)) % n);",
                             "uint64_t mj = (uint64_t)(((u128)m + (u128)(j + 1) * (b % n)) % n);"),
    "pattern_region_drops_last_skip": (
        "uint64_t d = or_inverse_exponent(n, e);\n    for (uint64_t c0 = c_lo; c0 < c_lo + L0; ++c0) {\n"
        "        uint64_t m = or_powmod(c0, d, n);\n        for (uint64_t s = 1; s < p; ++s) {",
        "uint64_t d = or_inverse_exponent(n, e);\n    for (uint64_t c0 = c_lo; c0 < c_lo + L0; ++c0) {\n"
        "        uint64_t m = or_powmod(c0, d, n);\n        for (uint64_t s = 1; s + 1 < p; ++s) {"),
    "pattern_const_region_encrypts": (
        "uint64_t m = or_powmod(c0, d, n), idx = 0, scale = 1;\n        int inside = 1;",
        "uint64_t m = or_powmod(c0, e, n), idx = 0, scale = 1;\n        int inside = 1;"),
    "dlog_index": ("L_out[q] = (i * M + val[h]) % order;", "L_out[q] = (i * M + val[h] + 1) % order;"),
}


def _run_pins(so_path):
    env = dict(os.environ, PHPRNG_ORACLE_SO=so_path)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not slow and not gpu",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, "mutation anchor missing: " + old
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    c_path.write_text(mutated)
    so = oracle.build(force=True, src=str(c_path), out=str(tmp_path / "mutant.so"))
    rc, out = _run_pins(so)
    assert rc != 0, "pins did not catch mutant %s:\n%s" % (name, out)


def test_unmutated_copy_passes(tmp_path):
    so = oracle.build(force=True, src=oracle._SRC, out=str(tmp_path / "clean.so"))
    rc, out = _run_pins(so)
    assert rc == 0, out


# Mistakes planted in the Python part of the oracle (the Fourier test): the
# function is re-made from its own source with one change and the pins run
# against it in this process.
PY_MUTANTS = {
    "fourier_negative_exponent": ("fourier_coefficients", "X = np.fft.ifft(x, axis=1) * M",
                                  "X = np.fft.fft(x, axis=1)"),
    "fourier_dropped_offset": ("fourier_coefficients", "reshape(seqs, M) - 0.5", "reshape(seqs, M)"),
    "fourier_scale": ("fourier_coefficients", "/ np.sqrt(M)", "/ M"),
    "fourier_bin_width": ("fourier_bin", "(nbins / (2.0 * w))", "(nbins / w)"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_planted_python_mistake_is_caught(monkeypatch, name):
    import inspect
    import textwrap
    import test_oracle_pins as pins
    fn_name, old, new = PY_MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fn_name)))
    assert src.count(old) == 1, "mutation anchor missing: " + old
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    monkeypatch.setattr(oracle, fn_name, ns[fn_name])
    failed = False
    for test in (pins.test_fourier_pure_tone_and_parseval, pins.test_fourier_direct_sum_and_bin_edges,
                 pins.test_fourier_variance_one_over_24):
        try:
            test(oracle._default())
        except AssertionError:
            failed = True
    assert failed, "pins did not catch mutant " + name
