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
    "batched run keyed by its union node id": ("lv = v - rm->off[r];", "lv = v;"),
    "batched ties on union block ids": ("uint32_t tl = or_tie(sv, round, lv, L - lb);",
                                        "uint32_t tl = or_tie(sv, round, lv, L);"),
    "batched runs share one seed": ("sv = rm->seed[r];", "sv = rm->seed[0];"),
    "coarse weight overwritten": ("for (int64_t v = 0; v < n; v++) cvwgt[f2c[v]] += vwgt[v];",
                                  "for (int64_t v = 0; v < n; v++) cvwgt[f2c[v]] = vwgt[v];"),
}


# mistakes in the learned gate and the V-cycle, caught by their own pin files
MUTANTS_ELSEWHERE = {
    "bf16 ties rounded up": ("u += 0x7FFFu + ((u >> 16) & 1u);", "u += 0x8000u;",
                             "test_oracle_learned.py"),
    "feature 3 drops the own weight": ("f[2] = or_bf16((float)(wb - wo) / (float)wdeg);",
                                       "f[2] = or_bf16((float)wb / (float)wdeg);",
                                       "test_oracle_learned.py"),
    "visit records the own weight as best": ("vis_best[v] = best >= 0 ? acc[best] : 0;",
                                             "vis_best[v] = w_own;", "test_oracle_learned.py"),
    "hidden bias dropped": ("float acc = bf16_bits_to_float(net[OR_MLP_B1 + j]);",
                            "float acc = 0.0f;", "test_oracle_learned.py"),
    "second ReLU dropped": (
        "h1[i], acc);\n        h2[j] = or_bf16(acc > 0.0f ? acc : 0.0f);\n    }\n    float z = bf16",
        "h1[i], acc);\n        h2[j] = or_bf16(acc);\n    }\n    float z = bf16",
        "test_oracle_learned.py"),
    "ReLU gate missing in backprop": ("d2[i] = a2[i] > 0 ? dz * prm[OR_MLP_W3 + i] : 0.0;",
                                      "d2[i] = dz * prm[OR_MLP_W3 + i];",
                                      "test_oracle_learned.py"),
    "bf16 training skips parameter rounding": ("        q[i] = or_bf16(prm[i]);\n        grad[i] = 0.0;",
                                               "        q[i] = prm[i];\n        grad[i] = 0.0;",
                                               "test_oracle_learned.py"),
    "bf16 training skips hidden rounding": ("            h1[j] = or_bf16(acc > 0.0f ? acc : 0.0f);\n        }\n        for (int j = 0; j < 32; j++) {\n            float acc = q[OR_MLP_B2 + j];",
                                            "            h1[j] = acc > 0.0f ? acc : 0.0f;\n        }\n        for (int j = 0; j < 32; j++) {\n            float acc = q[OR_MLP_B2 + j];",
                                            "test_oracle_learned.py"),
    "full rounds shifted": (
        "int full = !net || r == 0 || r % full_every == full_every - 1 || r == rounds - 1;",
        "int full = !net || r == 0 || r % full_every == 0 || r == rounds - 1;",
        "test_oracle_learned.py"),
    "gated round ends the run": ("if (full && m == 0) break;", "if (m == 0) break;",
                                 "test_oracle_learned.py"),
    "V-cycle clustering unconstrained": (
        "p->subrounds, level_seed(p->seed, L), cpl[L], p->degree_order != 0,",
        "p->subrounds, level_seed(p->seed, L), NULL, p->degree_order != 0,",
        "test_oracle_vcycle.py"),
    "V-cycle coarse blocks not inherited": ("cpl[L + 1][g->f2c[v]] = cpl[L][v];",
                                            "cpl[L + 1][g->f2c[v]] = 0;", "test_oracle_vcycle.py"),
    "high degree first": ("if (x->deg != y->deg) return x->deg < y->deg ? -1 : 1;",
                          "if (x->deg != y->deg) return x->deg < y->deg ? 1 : -1;",
                          "test_oracle_degree_order.py"),
    "round-robin groups": ("colour_out[k[p].v] = (int32_t)(p * S / n);",
                           "colour_out[k[p].v] = (int32_t)(p % S);",
                           "test_oracle_degree_order.py"),
}


@pytest.mark.parametrize("name", list(MUTANTS_ELSEWHERE))
def test_other_pins_reject_mutant(name, tmp_path):
    old, new, pins = MUTANTS_ELSEWHERE[name]
    _check_mutant(name, old, new, pins, tmp_path)


def _check_mutant(name, old, new, pins, tmp_path):
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
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant '{name}'\n{r.stdout[-2000:]}"


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
