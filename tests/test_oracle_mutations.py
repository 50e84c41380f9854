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


# Planted mistakes in the FP64 block-by-block k-NN of oracle/__init__.py (the
# 10M spot check's reference): each mutant of exact_knn_blocked, rebuilt from
# its own source with one edit, must fail the blocked pins of
# test_oracle_pins.py (integer data with tie runs cut by blocks; float data).
PY_MUTATIONS = {
    "block_cut_drops_ties": ("rows, cols = torch.nonzero(D <= kth[:, None], as_tuple=True)",
                             "rows, cols = torch.nonzero(D < kth[:, None], as_tuple=True)"),
    "query_norm_dropped": ("vals = vals + qn[c:c + qchunk][rows]", "vals = vals + 0.0"),
    "block_offset_dropped": ("cand_i[c + r].append(cols[m].astype(np.int64) + a)",
                             "cand_i[c + r].append(cols[m].astype(np.int64))"),
    "order_by_id_first": ("o = np.lexsort((ci, ck))[:K]", "o = np.lexsort((ck, ci))[:K]"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_blocked_knn_mutant_is_caught(name):
    import inspect
    import types

    import numpy as np

    import oracle
    import test_oracle_pins as pins

    old, new = PY_MUTATIONS[name]
    src = inspect.getsource(oracle.exact_knn_blocked)
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    mut = types.SimpleNamespace(exact_knn=oracle.exact_knn, exact_knn_blocked=ns["exact_knn_blocked"], np=np)
    caught = False
    for check in (lambda: pins.test_exact_knn_blocked_equals_the_plain_sum_on_integer_data(mut, "l2"),
                  lambda: pins.test_exact_knn_blocked_equals_the_plain_sum_on_integer_data(mut, "ip"),
                  lambda: pins.test_exact_knn_blocked_float_data_and_padding(mut)):
        try:
            check()
        except Exception:  # a failed assertion, or a mutant that cannot even fill its output
            caught = True
    assert caught, f"mutant {name} passed every blocked pin"


GEMM_MUTATIONS = {
    "tie_cut_strict": ("cand = np.flatnonzero(D[r] <= kth)", "cand = np.flatnonzero(D[r] < kth)"),
    "query_norm_dropped": ('D = xn[None, :] - 2.0 * dot + np.einsum("ij,ij->i", q, q)[:, None]',
                           "D = xn[None, :] - 2.0 * dot"),
    "order_by_id_first": ("o = np.lexsort((cand, D[r, cand]))[:kk]", "o = np.lexsort((D[r, cand], cand))[:kk]"),
    "dot_sign": ('D = xn[None, :] - 2.0 * dot + np.einsum', 'D = xn[None, :] + 2.0 * dot + np.einsum'),
}


@pytest.mark.parametrize("name", sorted(GEMM_MUTATIONS))
def test_gemm_knn_mutant_is_caught(name):
    """The same for exact_knn_gemm (the 1M-point recall ground truth of the
    full-size tests): each mutant fails one of its pins."""
    import inspect
    import types

    import numpy as np

    import oracle
    import test_oracle_pins as pins

    old, new = GEMM_MUTATIONS[name]
    src = inspect.getsource(oracle.exact_knn_gemm)
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    mut = types.SimpleNamespace(exact_knn=oracle.exact_knn, exact_knn_gemm=ns["exact_knn_gemm"], np=np)
    caught = False
    for check in (lambda: pins.test_exact_knn_gemm_equals_the_plain_sum_on_integer_data(mut, "l2"),
                  lambda: pins.test_exact_knn_gemm_equals_the_plain_sum_on_integer_data(mut, "ip"),
                  lambda: pins.test_exact_knn_gemm_float_data_within_fp64_rounding(mut)):
        try:
            check()
        except Exception:  # a failed assertion, or a mutant that cannot even fill its output
            caught = True
    assert caught, f"mutant {name} passed every GEMM pin"
