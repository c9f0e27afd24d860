"""The oracle's pins catch planted mistakes.

Each case copies oracle.c, plants one plausible mistake (a dropped term, a wrong
sign or index, transposed axes, the h^2/v misreading, a missing push, a
missing upwind max, G summed in reverse axis order, c rounded as
fl(h^2)/fl(v^2)), builds
the copy with the oracle's own flags and runs the cheap pins of
tests/oracle_pins.py against it in a child process.  The pins must fail (or the
child must not finish) for every mutant, and must all pass for the real oracle.
"""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "dropped_term": ("        g = g + m * m;\n", "        if (k == 0) g = g + m * m;\n"),
    "wrong_axis_index": ("        double m = tau - a[k];\n", "        double m = tau - a[0];\n"),
    "wrong_sign_in_difference": ("        double m = tau - a[k];\n",
                                 "        double m = tau + a[k] - 2.0 * a[0];\n"),
    "h2_over_v_reading": ("        c[i] = r[i] * r[i];\n", "        c[i] = h * h / v[i];\n"),
    "neighbour_stride": ("        double hi = (coord + 1 < g->n[k]) ? t[idx + g->s[k]] : ORC_INF;\n",
                         "        double hi = (coord + 1 < g->n[k]) ? t[idx + g->s[0]] : ORC_INF;\n"),
    "transposed_axes": ("        g->n[k] = dims[ndim - 1 - k];\n", "        g->n[k] = dims[k];\n"),
    "no_push_on_decrease": ("                    if (heap_push(&hp, tau, m)) goto fail;\n",
                            "                    if (k > 0 && heap_push(&hp, tau, m)) goto fail;\n"),
    "dtilde_sign": ("    double disc = s * s - 2.0 * (q - c);\n", "    double disc = s * s - 2.0 * (q + c);\n"),
    # G summed in the reverse axis order (z, y, x) instead of x, y, z
    "reversed_G_term_order": ("    for (int k = 0; k < D; ++k) {\n        double m = tau - a[k];\n",
                              "    for (int k = D - 1; k >= 0; --k) {\n        double m = tau - a[k];\n"),
    # c rounded as fl(h^2) / fl(v^2) in the grid solvers (consistently in the
    # residual too) instead of fl(fl(h/v)^2)
    "c_from_squares": ("        c[i] = r[i] * r[i];\n", "        c[i] = (h * h) / (v[i] * v[i]);\n"),
    "missing_upwind_max": ("        if (!(m > 0.0)) m = 0.0;     /* max(., 0); a_k = +inf gives -inf -> 0 */\n",
                           "        if (!(m > -1e300)) m = 0.0;\n"),
}

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import oracle
    oracle._lib = None
    oracle.build = lambda force=False: {lib!r}
    from tests.oracle_pins import run_pin_suite
    print("FAILED:" + ",".join(run_pin_suite(oracle)))
""")


def _run_child(lib_path, timeout=120):
    code = CHILD.format(root=ROOT, lib=lib_path)
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             timeout=timeout)
    except subprocess.TimeoutExpired:
        return None
    for line in out.stdout.splitlines():
        if line.startswith("FAILED:"):
            return [x for x in line[len("FAILED:"):].split(",") if x]
    return ["crashed"]


def test_real_oracle_passes_every_pin():
    assert _run_child(oracle.build()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new, 1)
    if name == "c_from_squares":    # the residual's own constant, consistently
        old2 = "        double r = h / v[i];\n        double c = r * r;\n"
        assert mutated.count(old2) == 1
        mutated = mutated.replace(old2, "        double r = h / v[i];\n        double c = (h * h) / (v[i] * v[i]);\n")
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(lib), str(csrc), "-lm"])
    failed = _run_child(str(lib), timeout=6)
    assert failed is None or len(failed) >= 1, f"mutant {name} passed every pin"
