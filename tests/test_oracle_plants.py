"""Plant plausible mistakes in a copy of the oracle (on the CPU) and show that at
least one pin fails for each: a dropped term, a wrong sign, a transposed operand,
a wrong tie-break order, a wrong hull rule, a wrong adjacency index, a wrong
canonical rotation.  The unmodified copy must pass every pin (control)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dt_oracle.c")

PLANTS = {
    "control": None,
    "sos_row_b_sign": ("cof[1] = -oracle_orient2d(xy, a, c, d);",
                       "cof[1] = oracle_orient2d(xy, a, c, d);"),
    "sos_order_reversed": ("ids[i] < ids[best]", "ids[i] > ids[best]"),
    "incircle_term_dropped": ("i128 det = alift * m_a + blift * m_b + clift * m_c;",
                              "i128 det = alift * m_a + blift * m_b;"),
    "incircle_minor_sign": ("i128 m_b = (i128)cdx * ady - (i128)adx * cdy;",
                            "i128 m_b = (i128)adx * cdy - (i128)cdx * ady;"),
    "lift_drops_y": ("i128 alift = (i128)adx * adx + (i128)ady * ady;",
                     "i128 alift = (i128)adx * adx;"),
    "orient_transposed": ("(px(xy, b) - px(xy, a)) * (py(xy, c) - py(xy, a))",
                          "(px(xy, b) - px(xy, a)) * (py(xy, a) - py(xy, c))"),
    "ghost_collinear_dropped": ("    return strictly_between(xy, u, v, q);\n}",
                                "    return 0;\n}"),
    "ghost_side_reversed": ("        return o > 0;", "        return o < 0;"),
    "canonical_rotation": ("if (v[1] < v[r]) r = 1;", "if (v[1] > v[r]) r = 1;"),
    "cavity_link_index": ("s->tn[3 * (int64_t)N + 0] = M;", "s->tn[3 * (int64_t)N + 1] = M;"),
}


@pytest.mark.parametrize("name", list(PLANTS))
def test_plant_is_caught(name, tmp_path):
    src = open(SRC).read()
    if PLANTS[name] is not None:
        old, new = PLANTS[name]
        assert src.count(old) == 1, "plant site not found: %s" % name
        src = src.replace(old, new)
    c = tmp_path / "plant.c"
    c.write_text(src)
    so = tmp_path / "libplant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-w", "-o", str(so), str(c)])
    r = subprocess.run([sys.executable, "-m", "tests._pin_suite", str(so)], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    if name == "control":
        assert r.returncode == 0, r.stdout + r.stderr
    else:
        assert r.returncode != 0, "planted mistake %s passed every pin" % name
