"""The CPU oracle against its pins, and the pins against planted mistakes."""
import os
import re

import numpy as np
import pytest

import oracle
import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    pin(oracle.default())


def test_pair_and_full_agree_with_triangle():
    rng = np.random.default_rng(3)
    volt = rng.integers(0, 256, (17, 3, 6), dtype=np.uint8)
    tri = oracle.xmac(volt)
    full = oracle.xmac_full(volt)
    for f in range(3):
        for i in range(6):
            for j in range(6):
                assert oracle.xmac_pair(volt, f, i, j) == tuple(int(v) for v in full[f, i, j])
                if j <= i:
                    assert tuple(full[f, i, j]) == tuple(tri[f, _pins.tri_index(i, j)])


def test_to_int32_checks_range():
    ok = np.array([[[2**31 - 1, -2**31]]], np.int64)
    assert oracle.to_int32(ok).dtype == np.int32
    with pytest.raises(OverflowError):
        oracle.to_int32(np.array([[[2**31, 0]]], np.int64))


def test_empty_time_gives_zero():
    volt = np.zeros((0, 2, 3), np.uint8)
    assert np.array_equal(oracle.xmac(volt), np.zeros((2, 6, 2), np.int64))


# Plausible mistakes, each planted in a copy of the oracle source on the CPU;
# every one must make at least one pin fail.
MUTANTS = {
    "dropped_imag_imag_term": (
        r"sre \+= \(int64_t\)ri\[t\] \* rj\[t\] \+ \(int64_t\)mi\[t\] \* mj\[t\];",
        "sre += (int64_t)ri[t] * rj[t];"),
    "imag_sign_flipped": (
        r"sim \+= \(int64_t\)mi\[t\] \* rj\[t\] - \(int64_t\)ri\[t\] \* mj\[t\];",
        "sim += (int64_t)ri[t] * mj[t] - (int64_t)mi[t] * rj[t];"),
    "nibbles_swapped": (
        r"unsigned hi = \(b >> 4\) & 0xFu, lo = b & 0xFu;",
        "unsigned lo = (b >> 4) & 0xFu, hi = b & 0xFu;"),
    "offset_binary_not_twos_complement": (
        r"return code >= 8u \? \(int\)code - 16 : \(int\)code;",
        "return (int)code - 8;"),
    "triangle_index_transposed": (
        r"int64_t p = \(int64_t\)i \* \(i \+ 1\) / 2 \+ j;\n                vf",
        "int64_t p = (int64_t)j * (j + 1) / 2 + i; if (p >= P) p = P - 1;\n                vf"),
    "real_imag_planes_of_row_swapped": (
        r"const int32_t \*ri = xr \+ \(int64_t\)i \* T, \*mi = xi \+ \(int64_t\)i \* T;",
        "const int32_t *mi = xr + (int64_t)i * T, *ri = xi + (int64_t)i * T;"),
    "conjugate_on_wrong_operand": (
        r"sim \+= \(int64_t\)mi\[t\] \* rj\[t\] - \(int64_t\)ri\[t\] \* mj\[t\];",
        "sim += (int64_t)mj[t] * ri[t] - (int64_t)rj[t] * mi[t];"),
    "last_sample_dropped": (
        r"for \(int t = 0; t < T; \+\+t\) \{\n                    sre",
        "for (int t = 0; t < T - 1; ++t) {\n                    sre"),
    "invalid_flag_ignored": (
        r"if \(zero_invalid && \(hi == 8u \|\| lo == 8u\)\)",
        "if (0)"),
    "beam_drops_imaginary_power": (
        r"p \+= \(int64_t\)r \* r \+ \(int64_t\)m \* m;",
        "p += (int64_t)r * r;"),
    "beam_window_off_by_one": (
        r"for \(int t = k \* n_avg; t < \(k \+ 1\) \* n_avg; \+\+t\)",
        "for (int t = k * n_avg; t <= (k + 1) * n_avg && t < T; ++t)"),
    "remap_conjugate_not_applied": (
        r"im -= vf\[2 \* k \+ 1\];",
        "im += vf[2 * k + 1];"),
    "remap_uses_permutation_not_inverse": (
        r"const int i = pos\[2 \* s1 \+ p1\], j = pos\[2 \* s2 \+ p2\];",
        "const int i = nat_of_pfb[2 * s1 + p1], j = nat_of_pfb[2 * s2 + p2];"),
    "remap_pols_swapped": (
        r"\(\(int64_t\)g \* Q \+ \(int64_t\)s1 \* \(s1 \+ 1\) / 2 \+ s2\) \* 4 \+ p1 \* 2 \+ p2\)",
        "((int64_t)g * Q + (int64_t)s1 * (s1 + 1) / 2 + s2) * 4 + p2 * 2 + p1)"),
    "ingest_channel_and_input_swapped": (
        r"= b\[6 \+ 64 \* f2 \+ k\];",
        "= b[6 + 4 * k + f2 % 4 + 0 * f2];"),
    "ingest_group_stride": (
        r"const int cgroup = 32 \* chan \+ 4 \* mgt \+ grp;",
        "const int cgroup = 32 * chan + 4 * mgt + 2 * grp;"),
    "ingest_checksum_bytes_swapped": (
        r"if \(xhi != b\[262\] \|\| xlo != b\[263\]\)",
        "if (xhi != b[263] || xlo != b[262])"),
    "ingest_missing_not_marked": (
        r"volt\[\(\(int64_t\)frame \* PKT_CHANNELS \+ 4 \* cgroup \+ f2\) \* PKT_INPUTS \+ 64 \* pfb \+ k\] = 0x88;",
        "(void)0;"),
    "ingest_frame_five_bits": (
        r"const int frame = \(int\)\(w3 & 511u\);",
        "const int frame = (int)(w3 & 31u);"),
    "fpfb_exponent_sign_flipped": (
        r"yr \+= ur\[n\] \* cs\[r\] \+ um\[n\] \* sn\[r\];\n                        ym \+= um\[n\] \* cs\[r\] - ur\[n\] \* sn\[r\];",
        "yr += ur[n] * cs[r] - um[n] * sn[r];\n                        ym += um[n] * cs[r] + ur[n] * sn[r];"),
    "fpfb_channels_not_centred": (
        r"const int c = \(k \+ L / 2\) % L;",
        "const int c = k;"),
    "fpfb_taps_reversed": (
        r"ar \+= h\[p \* L \+ n\] \* xi\[2 \* s\];\n                        am \+= h\[p \* L \+ n\] \* xi\[2 \* s \+ 1\];",
        "ar += h[(n_taps - 1 - p) * L + n] * xi[2 * s];\n                        am += h[(n_taps - 1 - p) * L + n] * xi[2 * s + 1];"),
    "fpfb_block_time_reversed": (
        r"const int64_t s = \(m \+ p\) \* L \+ n;",
        "const int64_t s = (m + p) * L + (L - 1 - n);"),
    "fpfb_round_half_away": (
        r"double r = rint\(v\);",
        "double r = round(v);"),
    "fpfb_saturates_at_minus_8": (
        r"if \(r < -7\.0\)\n        r = -7\.0;",
        "if (r < -8.0)\n        r = -8.0;"),
    "fpfb_nibbles_swapped": (
        r"\(\(fpfb_q4\(scale \* yr\) & 15\) << 4\) \| \(fpfb_q4\(scale \* ym\) & 15\)",
        "((fpfb_q4(scale * ym) & 15) << 4) | (fpfb_q4(scale * yr) & 15)"),
    "accumulate_overwrites": (
        r"vf\[2 \* p\] \+= sre;\n                vf\[2 \* p \+ 1\] \+= sim;",
        "vf[2 * p] = sre;\n                vf[2 * p + 1] = sim;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(name, tmp_path):
    pattern, repl = MUTANTS[name]
    with open(oracle.SOURCE) as f:
        src = f.read()
    mutated, n = re.subn(pattern, repl, src)
    assert n >= 1, f"mutant {name} did not apply"
    src_path = tmp_path / "mutant.c"
    src_path.write_text(mutated)
    lib = oracle.OracleLib(oracle.build(force=True, src=str(src_path), out=str(tmp_path / "libmut.so")))
    failures = []
    for pin in _pins.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, f"no pin caught the planted mistake {name}"
