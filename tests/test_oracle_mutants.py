"""The oracle's pins are sensitive: each planted mistake fails at least one pin.

Every mutant below is a plausible slip in the oracle (a comparison relaxed, a
sign flipped, an index transposed, a share or a rank reordered, a term
dropped).  The mutated C file is compiled on the CPU into a temporary library
and the pin suites (test_oracle_lap.py, test_oracle_rlt2.py, test_oracle_f64.py) are run against
it; each must fail.

Not listed: putting the rows of a tile in descending order.  The reduced
costs the Hungarian method leaves do not depend on the order of rows or
columns (only the assignment does, which the hand traces pin), so that slip
changes no state of the dual ascent.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rlt2_oracle.c")

MUTANTS = {
    "tie_to_largest_column": ("if (dist[j] < delta) { delta = dist[j]; next = j; }",
                              "if (dist[j] <= delta) { delta = dist[j]; next = j; }"),
    "label_on_equal": ("if (red < dist[j]) { dist[j] = red; pred[j] = col; }",
                       "if (red <= dist[j]) { dist[j] = red; pred[j] = col; }"),
    "column_potential_sign": ("v[j] -= delta;", "v[j] += delta;"),
    "share_remainder_to_last_rows": ("return x / m + (t < x % m ? 1 : 0);",
                                     "return x / m + (t >= m - x % m ? 1 : 0);"),
    "spread_into_meaningless_column": ("if (q == j || q == n) continue;\n                            if (up)",
                                       "if (q == j) continue;\n                            if (up)"),
    "complementary_D_rank_swap": ("ix6(N, k, n, i, j, p, q), ix6(N, k, n, p, q, i, j)",
                                  "ix6(N, k, n, p, q, i, j), ix6(N, k, n, i, j, p, q)"),
    "complementary_C_odd_unit_to_second": (
        "st->c[ix4(N, i, j, k, n)] = T / 2 + T % 2;\n                    st->c[ix4(N, k, n, i, j)] = T / 2;",
        "st->c[ix4(N, i, j, k, n)] = T / 2;\n                    st->c[ix4(N, k, n, i, j)] = T / 2 + T % 2;"),
    "residual_column_sign": ("M[r * m + s] - u[r] - v[s];\n                }\n            }\n    free(M)",
                             "M[r * m + s] - u[r] + v[s];\n                }\n            }\n    free(M)"),
    "concentration_drops_a_unit": ("st->c[ix4(N, i, j, k, n)] += S;",
                                   "st->c[ix4(N, i, j, k, n)] += S - (S > 0);"),
    "subproblem_distance_transposed": ("Dist[ix2(N, fl[y], loc[t])] +", "Dist[ix2(N, loc[t], fl[y])] +"),
    "init_flow_transposed": ("(int64_t)F[ix2(N, i, k)] * (int64_t)Dist[ix2(N, j, n)]",
                             "(int64_t)F[ix2(N, k, i)] * (int64_t)Dist[ix2(N, j, n)]"),
    # FP64 form (reading R14)
    "f64_B_share_divisor": ("b[ix2(N, i, j)] / (double)(N - 1)", "b[ix2(N, i, j)] / (double)(N - 2)"),
    "f64_spread_into_meaningless_column": ("if (q != j && q != n) st->d[ix6(N, i, j, k, n, p, q)] += sh;",
                                           "if (q != j) st->d[ix6(N, i, j, k, n, p, q)] += sh;"),
    "f64_class_divisor": ("d[mem[t]] = T / 6.0;", "d[mem[t]] = T / 5.0;"),
    "f64_column_potential_sign": ("double red = M[(size_t)i0 * n + j] - u[i0] - v[j];",
                                  "double red = M[(size_t)i0 * n + j] - u[i0] + v[j];"),
    "f64_tie_to_largest_column": (
        "double red = M[(size_t)i0 * n + j] - u[i0] - v[j];\n"
        "                if (red < dist[j]) { dist[j] = red; pred[j] = col; }\n"
        "                if (dist[j] < delta)",
        "double red = M[(size_t)i0 * n + j] - u[i0] - v[j];\n"
        "                if (red < dist[j]) { dist[j] = red; pred[j] = col; }\n"
        "                if (dist[j] <= delta)"),
    "f64_residual_transposed": (
        "const double S = orf_lap(m, M, u, v, NULL, NULL, st);\n"
        "                    st->c[ix4(N, i, j, k, n)] += S;\n"
        "                    for (r = 0; r < m; r++)\n"
        "                        for (s = 0; s < m; s++)\n"
        "                            st->d[ix6(N, i, j, k, n, rows[r], cols[s])] = M[r * m + s] - u[r] - v[s];",
        "const double S = orf_lap(m, M, u, v, NULL, NULL, st);\n"
        "                    st->c[ix4(N, i, j, k, n)] += S;\n"
        "                    for (r = 0; r < m; r++)\n"
        "                        for (s = 0; s < m; s++)\n"
        "                            st->d[ix6(N, i, j, k, n, rows[r], cols[s])] = M[r * m + s] - u[s] - v[r];"),
    "f64_complementary_C_one_side": ("st->c[ix4(N, k, n, i, j)] = T / 2.0;",
                                     "st->c[ix4(N, k, n, i, j)] = st->c[ix4(N, k, n, i, j)];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    a, b = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(a) >= 1, "mutation site vanished: " + name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(a, b, 1))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", str(lib), str(mut)])
    env = dict(os.environ, RLT2_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_lap.py", "tests/test_oracle_rlt2.py",
                        "tests/test_oracle_f64.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutant %s survived the pins:\n%s" % (name, r.stdout[-2000:])
