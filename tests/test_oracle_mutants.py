"""Planted mistakes in copies of the oracle must each fail a pin (CPU only).

Each mutant is the oracle source with one plausible slip (a comparator, an
off-by-one, a dropped term, a sign or signedness error). It is compiled into
a temporary library and the pin suite of tests/pins.py runs against it in a
child process (a mutant may crash or loop; a crash or a timeout also counts
as caught). The unmodified source runs through the same harness as control.

A change of the RAM end-of-data rule ("at most w bytes left") is not listed:
every variant that still returns len there is equivalent, because the scan
past the window then meets the end of the data and returns len as well.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "ram_geq_to_gt": ("if (B[j] >= M) return j + 1;", "if (B[j] > M) return j + 1;"),
    "ram_window_one_long": ("for (uint64_t i = s; i < s + w; i++)", "for (uint64_t i = s; i <= s + w; i++)"),
    "ram_min_off_by_one": ("umax(s + w, s + mn - 1)", "umax(s + w, s + mn)"),
    "ram_min_dropped": ("umax(s + w, s + mn - 1)", "(s + w)"),
    "ram_window_starts_late": ("for (uint64_t i = s; i < s + w; i++)", "for (uint64_t i = s + 1; i < s + w; i++)"),
    "ram_max_off_by_one": ("    uint64_t limit = umin(len, s + mx);\n    for (uint64_t j",
                           "    uint64_t limit = umin(len, s + mx + 1);\n    for (uint64_t j"),
    "ae_gt_to_geq": ("dir > 0 ? (B[i] > B[p])", "dir > 0 ? (B[i] >= B[p])"),
    "ae_window_strict": ("i - p >= w && i + 1 - s >= mn", "i - p > w && i + 1 - s >= mn"),
    "ae_min_dropped": ("i - p >= w && i + 1 - s >= mn", "i - p >= w"),
    "ae_cut_position": ("            return i + 1;                           /* window after p is clear */",
                        "            return i;"),
    "ae_min_direction": (": (B[i] < B[p]);", ": (B[i] > B[p]);"),
    "ae_transposed": ("dir > 0 ? (B[i] > B[p])", "dir > 0 ? (B[p] > B[i])"),
    "maxp_left_tie": ("if (B[i - k] >= B[i]) return 0;", "if (B[i - k] > B[i]) return 0;"),
    "maxp_right_tie": ("if (B[i + k] >= B[i]) return 0;", "if (B[i + k] > B[i]) return 0;"),
    "maxp_right_window_dropped": ("        if (B[i + k] >= B[i]) return 0;\n", ""),
    "maxp_window_fit": ("if (i < w || i + w >= len) return 0;", "if (i < w || i + w > len) return 0;"),
    "maxp_cut_position": ("if (oracle_maxp_is_target(B, len, c, w)) return c + 1;",
                          "if (oracle_maxp_is_target(B, len, c, w)) return c + 2;"),
    "maxp_min_off_by_one": ("for (uint64_t c = s + mn - 1; c < limit; c++)",
                            "for (uint64_t c = s + mn; c < limit; c++)"),
    "signed_bytes": None,  # handled below
}

RUNNER = r"""
import sys
sys.path[:0] = [{root!r}, {here!r}]
import oracle, pins
orc = oracle.Oracle({lib!r})
failed = []
for f in pins.ALL_PINS + (pins.check_uniform_statistics,):
    try:
        f(orc)
    except AssertionError as e:
        failed.append(f.__name__)
print("FAILED:" + ",".join(failed))
sys.exit(1 if failed else 0)
"""


def _mutate(name):
    src = open(SRC).read()
    if name is None:
        return src
    if name == "signed_bytes":
        assert src.count("const uint8_t* B") >= 4
        out = src.replace("const uint8_t* B", "const int8_t* B").replace("uint8_t M = 0;", "int8_t M = -128;")
        return out
    old, new = MUTANTS[name]
    assert src.count(old) == 1, (name, src.count(old))
    return src.replace(old, new)


def _run(tmp_path, name):
    import oracle
    csrc = tmp_path / ("m_%s.c" % (name or "control"))
    csrc.write_text(_mutate(name))
    lib = oracle.build(str(csrc), str(tmp_path / ("m_%s.so" % (name or "control"))), force=True)
    code = RUNNER.format(root=ROOT, here=HERE, lib=lib)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    except subprocess.TimeoutExpired:
        return "timeout", ""
    return r.returncode, r.stdout + r.stderr


def test_control_passes(tmp_path):
    rc, out = _run(tmp_path, None)
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    rc, out = _run(tmp_path, name)
    assert rc != 0, "mutant %s survived every pin:\n%s" % (name, out)
