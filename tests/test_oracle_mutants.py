"""The oracle's pins catch plausible mistakes: each case plants one mistake in a
copy of oracle/sclap_oracle.c (on the CPU), builds it, and checks that the pin
suite (tests/test_oracle.py) fails against it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sclap_oracle.c")

MUTANTS = {
    "propose on zero gain": ("if (gain > 0 || overloaded)", "if (gain >= 0 || overloaded)"),
    "tie-break reversed": ("else if (tl != best_tie) better = tl < best_tie;",
                           "else if (tl != best_tie) better = tl > best_tie;"),
    "eligibility off by one": (
        "if (W[L] + vwgt[v] > bound_of(Bv, B, L)) continue; /* not eligible */",
        "if (W[L] + vwgt[v] >= bound_of(Bv, B, L)) continue; /* not eligible */"),
    "exclusive prefix at target": ("if (!(p->c == 0 || sum <= cap)) p->keep = 0;",
                                   "if (!(p->c == 0 || sum < cap)) p->keep = 0;"),
    "departure cap inclusive": ("if (departed < excess) departed += ws->props[q].c;",
                                "if (departed <= excess) departed += ws->props[q].c;"),
    "departures by lowest gain": ("if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;\n    return x->v < y->v ? -1 : (x->v > y->v);\n}\n\nstatic int cmp_by_target",
                                  "if (x->gain != y->gain) return x->gain < y->gain ? -1 : 1;\n    return x->v < y->v ? -1 : (x->v > y->v);\n}\n\nstatic int cmp_by_target"),
    "source weight not released": ("W[p->own] -= p->c;", "(void)0;"),
    "intra-cluster edges kept": ("if (cu == cv) continue;                 /* edge inside a cluster */",
                                 "(void)0;"),
    "cut not halved": ("return s / 2;\n}\n\nvoid or_block_weights", "return s;\n}\n\nvoid or_block_weights"),
    "lmax rounded up": ("return (int64_t)floor((1.0 + eps) * (double)avg);",
                        "return (int64_t)ceil((1.0 + eps) * (double)avg);"),
    "colour from low bits": ("return (uint32_t)(node_hash(seed, round, v) >> 32) % (uint32_t)S;",
                             "return (uint32_t)(node_hash(seed, round, v) >> 31) % (uint32_t)S;"),
    "isolated packing to U": ("int64_t Up = U - cmax + 1;", "int64_t Up = U;"),
    "LPT ties to last block": ("if (bw[b] < bw[bb]) bb = b;", "if (bw[b] <= bw[bb]) bb = b;"),
    "mix64 constant": ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;",
                       "z = (z ^ (z >> 27)) * 0x94D049BB133111EFULL;"),
    "coarse weight overwritten": ("for (int64_t v = 0; v < n; v++) cvwgt[f2c[v]] += vwgt[v];",
                                  "for (int64_t v = 0; v < n; v++) cvwgt[f2c[v]] = vwgt[v];"),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mutated = tmp_path / "sclap_oracle.c"
    mutated.write_text(src.replace(old, new))
    (tmp_path / "sclap_oracle.h").write_text(open(SRC.replace(".c", ".h")).read())
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", str(so),
                           str(mutated), "-lm"])
    env = dict(os.environ, SCLAP_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant '{name}'\n{r.stdout[-2000:]}"
