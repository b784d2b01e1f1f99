"""The oracle's pins catch planted mistakes.

Each case copies the committed oracle source, plants one plausible mistake
(a dropped term, a wrong rounding, a flipped comparison, a wrong tap), builds
it with gcc into a temporary library and runs the pins that cover that part
of the method against it (oracle/ref.py loads the library named by
CDEF_REF_LIB).  The run must fail: a mistake the pins cannot see would make
them worthless for that part.  CPU only; nothing here touches the CUDA
library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cdef_ref.c")

# (what the mistake is, committed text, planted text, pins that should see it)
MUTANTS = [
    ("eq. 7: the printed ceiling kept in the d < 0 branch (reading R7)",
     "return -min64(-diff, max64(0, strength - (-diff) / scale));",
     "return -min64(-diff, max64(0, strength - (-diff + scale - 1) / scale));",
     "constrain"),
    ("eq. 8: negative ties rounded toward zero (reading R10)",
     "return -((-sum + 8) / 16);",
     "return -((-sum + 7) / 16);",
     "round16"),
    ("eq. 13: the rounding term dropped",
     "return (int)((strength * (4 + i) + 8) / 16);",
     "return (int)((strength * (4 + i)) / 16);",
     "adjust_strength_rounds"),
    ("eq. 9-12: the clip dropped",
     "    return min64(ymax, max64(ymin, y));\n}",
     "    return y;\n}",
     "clip or neighbourhood"),
    ("Algorithm 1: ties go to the last direction",
     "if (s[d] > s[best])",
     "if (s[d] >= s[best])",
     "constant_block or directional"),
    ("eq. 5: the line weights 840 / N dropped",
     "s[d] += partial[L] * partial[L] * (840 / count[L]);",
     "s[d] += partial[L] * partial[L];",
     "e2_identity or argmin"),
    ("eq. 14: C1 dropped",
     "const double c1 = 6.25 *",
     "const double c1 = 0.0 *",
     "eq14_term"),
    ("section 3.1: the secondary cross taken at d + 4 instead of d - 2",
     "int dd = c == 0 ? (d + 2) % 8 : (d + 6) % 8;",
     "int dd = c == 0 ? (d + 2) % 8 : (d + 4) % 8;",
     "tap_geometry or brute_force"),
    ("Fig. 3 (reading R8): one direction's near tap off its line (d = 1 at (-1, 1))",
     "    {{0, 1}, {-1, 2}},\n",
     "    {{-1, 1}, {-1, 2}},\n",
     "dihedral"),
    ("Fig. 4 (reading R9): the secondary weights summing to less (1, 1 instead of 2, 1)",
     "static const int sec_weight[2] = {2, 1};",
     "static const int sec_weight[2] = {1, 1};",
     "exceed_unity"),
    ("eq. 15: greedy ties go to the highest preset index (reading R16)",
     "            if (best_t < 0 || tot < best_total) {\n                best_t = t;\n                best_total = tot;\n            }\n        }\n        presets[n - 1] = best_t;",
     "            if (best_t < 0 || tot <= best_total) {\n                best_t = t;\n                best_total = tot;\n            }\n        }\n        presets[n - 1] = best_t;",
     "greedy or lambda"),
]


def _build_mutant(tmp_path, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not found once: {old!r}"
    src = tmp_path / "cdef_ref.c"
    src.write_text(text.replace(old, new))
    (tmp_path / "cdef_ref.h").write_text(open(os.path.join(ROOT, "oracle", "cdef_ref.h")).read())
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(lib), str(src), "-lm"])
    return str(lib)


@pytest.mark.parametrize("what,old,new,pins", MUTANTS, ids=[m[0].split(":")[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, what, old, new, pins):
    lib = _build_mutant(tmp_path, old, new)
    env = dict(os.environ, CDEF_REF_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-m", "not gpu", "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
    assert r.returncode != 0, f"the pins ({pins}) did not catch: {what}\n{r.stdout[-1500:]}"
    assert "failed" in r.stdout
