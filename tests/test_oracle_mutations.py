"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the oracle's pins catch every one of them.

Each mutation is a one-token change to tl_oracle.c of the kind a slip would
make: a transposed index, a dropped term, a wrong sign, a swapped operand.
The mutated copy is compiled to a temporary library and swapped in for the
duration of the check; the real oracle is never modified."""
import json
import os
import subprocess
import sys

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_ttt as pins_ttt

MUTATIONS = {
    "stride_index_transposed": ("w[pi[r] - 1] = prod;", "w[r] = prod;"),
    "lambda_offset_sign": ("w[r] * (i[r] - (o ? o[r] : 0))", "w[r] * (i[r] + (o ? o[r] : 0))"),
    "view_step_dropped": ("wv[r] = w[r] * t[r];", "wv[r] = w[r];"),
    "ttv_last_term_dropped": (
        "for (int64_t k = 0; k < n[q - 1]; ++k) {\n        iA[q - 1] = k;\n"
        "        acc_add(&s, A[orc_lambda(p, wA, iA, NULL)] * b[k * incb]);",
        "for (int64_t k = 0; k + 1 < n[q - 1]; ++k) {\n        iA[q - 1] = k;\n"
        "        acc_add(&s, A[orc_lambda(p, wA, iA, NULL)] * b[k * incb]);"),
    "ttm_matrix_transposed": ("B[j * ldb_row + k * ldb_col]", "B[k * ldb_row + j * ldb_col]"),
    "ttm_row_index_ignored": ("B, idx[q - 1], ldb_row", "B, 0, ldb_row"),
    "entrywise_sub_sign": ("case ORC_SUB:   return a - b;", "case ORC_SUB:   return b - a;"),
    "entrywise_output_layout": ("C[orc_lambda(p, wC, idx, NULL)] = apply_op",
                                "C[orc_lambda(p, wA, idx, NULL)] = apply_op"),
    "norm_abs_not_square": ("acc_add(&s, a * a);", "acc_add(&s, a < 0 ? -a : a);"),
    "ttv_output_mode_order": ("ext[c++] = n[r];", "ext[p - 2 - c++] = n[r];"),
    "transpose_inverse_permutation": ("ia[tau[r] - 1] = ic[r];", "ia[r] = ic[tau[r] - 1];"),
    "ttt_contraction_pairs_reversed": ("ib[psi[s + k] - 1] = j[k];",
                                       "ib[psi[s + k] - 1] = j[q - 1 - k];"),
    "ttt_b_free_index_from_a_block": ("ib[psi[k] - 1] = ic[r + k];", "ib[psi[k] - 1] = ic[k];"),
    "ttt_last_contracted_term_dropped": ("} while (q > 0 && odometer_next(q, nj, j));",
                                         "} while (q > 0 && odometer_next(q, nj, j) && "
                                         "j[q - 1] + 1 < nj[q - 1]);"),
}

PINS = [getattr(mod, name) for mod in (pins, pins_ttt) for name in dir(mod)
        if name.startswith("test_")]


def _param_sets(fn):
    """Argument sets of a pytest-parametrized pin (one dict per case)."""
    sets = [{}]
    for mark in getattr(fn, "pytestmark", []):
        if mark.name != "parametrize":
            continue
        names = [x.strip() for x in mark.args[0].split(",")]
        vals = [v if len(names) > 1 else (v,) for v in mark.args[1]]
        sets = [dict(base, **dict(zip(names, v))) for base in sets for v in vals]
    return sets


def _run_pins():
    """Runs every pin (a parametrised one over its cases, at most four seeds);
    returns the names of those that failed."""
    failed = []
    for fn in PINS:
        argsets = _param_sets(fn)
        if argsets and set(argsets[0]) == {"seed"}:
            argsets = argsets[:4]
        for kw in argsets:
            try:
                fn(**kw)
            except (AssertionError, ValueError, IndexError):
                failed.append(fn.__name__)
                break
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    with open(oracle._SRC) as fh:
        src = fh.read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new, 1))
    lib_path = oracle.compile_source(str(mutated), str(tmp_path / "libmutant.so"))
    # a mutant may index out of bounds, so it runs in a child process; a crash
    # of the child counts as the mistake being caught
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys, json; sys.path[:0] = [%r, %r]; import oracle, test_oracle_mutations as m; "
            "oracle._load(); oracle._lib = oracle._bind(%r); print(json.dumps(m._run_pins()))"
            % (here, os.path.dirname(here), lib_path))
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        return
    failed = json.loads(res.stdout.strip().splitlines()[-1])
    assert failed, f"no pin caught the planted mistake {name}"


def test_unmutated_oracle_passes_all_pins():
    assert _run_pins() == []
