"""Planted mistakes: each mutation of a copy of oracle.c (a wrong sign, a
flipped tie-break, an off-by-one truncation, a dropped neighbour, a broken
staging rule, a wrong merge test, a broken deal, a stall count that counts
the wrong expansions or is never reset) must make at least one pin in
test_oracle_pins.py fail. The mutants are compiled on the CPU into a temporary
directory; the real oracle is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "l2_sign": ("acc += diff * diff;", "acc -= diff * diff;"),
    "tie_break": ("return a->id < b->id;", "return a->id > b->id;"),
    "truncate_off_by_one": ("if (near_tie(S[L - 1].key, S[L].key, p->tie_tol)) st->tie_events++;\n            len = L;",
                            "if (near_tie(S[L - 1].key, S[L].key, p->tie_tol)) st->tie_events++;\n            len = L + 1 < len ? L + 1 : len;"),
    "dropped_neighbour": ("            for (int32_t r = 0; r < R; ++r) {\n                int64_t u = g->adj[(size_t)v * (size_t)R + (size_t)r];\n                if (u < 0) continue;\n                int added = vset_add(vs, u);\n                if (added < 0) { free(S); free(act); return ORC_ERR_OOM; }",
                          "            for (int32_t r = 1; r < R; ++r) {\n                int64_t u = g->adj[(size_t)v * (size_t)R + (size_t)r];\n                if (u < 0) continue;\n                int added = vset_add(vs, u);\n                if (added < 0) { free(S); free(act); return ORC_ERR_OOM; }"),
    "no_doubling": ("int64_t m2 = 2 * (int64_t)M;", "int64_t m2 = (int64_t)M + (M > 2);"),
    "merge_test_strict": ("return sum / (double)cnt >= (double)L * Rr;", "return sum / (double)cnt > (double)L * Rr;"),
    "deal_one_walker": ("int32_t w = dealt % M;", "int32_t w = 0;"),
    "stall_counts_improvements": ("if (upos == L) stall[w]++;", "if (upos < L) stall[w]++;"),
    "stall_not_reset_at_deal": ("lsn[w] = 0; U[w] = 0; stall[w] = 0; active[w] = 0;", "lsn[w] = 0; U[w] = 0; active[w] = 0;"),
    "entry_not_visited": ("    vset_add(vs, g->entry);\n    st->evals++;\n    insert_sorted(S, &len, e0);",
                          "    st->evals++;\n    insert_sorted(S, &len, e0);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = src.replace(old, new, 1)
    c = tmp_path / "oracle_mut.c"
    c.write_text(mut)
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(so), str(c), "-lm", "-lpthread"])
    env = dict(os.environ, ANN_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
