"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake (a flipped
comparison, a transposed operand, a dropped term, an off-by-one), compiles it
on the CPU and runs the pin suite against it: the suite has to fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "schulze_oracle.c")

MUTANTS = {
    "tally_position_off_by_one": ("for (int32_t q = 0; q < k; ++q) pos[row[q]] = q;",
                                  "for (int32_t q = 0; q < k; ++q) pos[row[q]] = q + 1;"),
    "tally_transposed": ("if (j != i && pos[i] < pos[j]) acc[(int64_t)i * m + j] += 1",
                         "if (j != i && pos[i] < pos[j]) acc[(int64_t)j * m + i] += 1"),
    "tally_unlisted_on_top": ("for (int32_t c = 0; c < m; ++c) pos[c] = k;",
                              "for (int32_t c = 0; c < m; ++c) pos[c] = -1;"),
    "weights_ties_are_edges": ("(i != j && a > b) ? a : 0", "(i != j && a >= b) ? a : 0"),
    "pregel_no_width_merge": ("else if (s[u] == bs) bw = imax(bw, cw);", "else if (s[u] == bs) bw = bw;"),
    "pregel_no_incoming_rule": ("if (s[c] != s[v] || t[c] != t[v]) {", "if (0) {"),
    "iterated_not_restricted": ("if (level[c] == 0) idx[r++] = c;", "idx[r++] = c;"),
    "iterated_level_off_by_one": ("if (win[a]) level[idx[a]] = t, ++placed;",
                                  "if (win[a]) level[idx[a]] = t + 1, ++placed;"),
    "positions_ties_counted": ("if (row[i] < row[j]) acc[(int64_t)i * m + j] += 1;",
                               "if (i != j && row[i] <= row[j]) acc[(int64_t)i * m + j] += 1;"),
    "positions_transposed": ("if (row[i] < row[j]) acc[(int64_t)i * m + j] += 1;",
                             "if (row[i] < row[j]) acc[(int64_t)j * m + i] += 1;"),
    "closure_max_instead_of_min": ("pi[j] = imax(pi[j], imin(pik, pk[j]));",
                                   "pi[j] = imax(pi[j], imax(pik, pk[j]));"),
    "closure_no_accumulate": ("pi[j] = imax(pi[j], imin(pik, pk[j]));", "pi[j] = imin(pik, pk[j]);"),
    "closure_transposed_operand": ("const int32_t pik = pi[k];",
                                   "const int32_t pik = p[(int64_t)k * m + i];"),
    "closure_last_pivot_dropped": ("for (int32_t k = 0; k < m; ++k) {\n    const int32_t* pk",
                                   "for (int32_t k = 0; k + 1 < m; ++k) {\n    const int32_t* pk"),
    "winners_strict": ("if (j != i && p[(int64_t)i * m + j] < p[(int64_t)j * m + i]) ok = 0;",
                       "if (j != i && p[(int64_t)i * m + j] <= p[(int64_t)j * m + i]) ok = 0;"),
    "beaten_by_reversed": ("if (j != i && p[(int64_t)j * m + i] > p[(int64_t)i * m + j]) ++c;",
                           "if (j != i && p[(int64_t)j * m + i] < p[(int64_t)i * m + j]) ++c;"),
    "ranking_tiebreak_reversed": ("order[t - 1] > i))", "order[t - 1] < i))"),
    "tally_entry_ties_counted": ("if (pi < pj) cnt += 1;", "if (pi <= pj) cnt += 1;"),
    "tally_entry_unlisted_first": ("int32_t pi = k, pj = k;", "int32_t pi = 0, pj = 0;"),
    "dijkstra_max_instead_of_min": ("int64_t cand = best[u] < (int64_t)e ? best[u] : (int64_t)e;",
                                    "int64_t cand = best[u] > (int64_t)e ? best[u] : (int64_t)e;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(mutated), "-o", str(lib)], check=True)
    env = dict(os.environ, SCHULZE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
