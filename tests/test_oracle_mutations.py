"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one (a mutation test of the oracle; nothing here touches a GPU).

Each mutant is compiled from a patched copy of ``oracle/oracle.c`` in a
temporary directory and run through ``tests/pin_battery.py`` in a child
process with a time limit: a failing pin or a refine that no longer ends
(dropping eps, for instance, can stall a price war) both count as caught.
"""

import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")
BATTERY = os.path.join(HERE, "pin_battery.py")

# (name, original text, planted mistake)
MUTANTS = [
    ("no-scaling", "const int64_t np1 = (int64_t)n + 1;\n    int32_t cmin",
     "const int64_t np1 = 1;\n    int32_t cmin"),
    ("price-sign", "const int64_t cp = np1 * (int64_t)row[y] - p[y];   /* c'_p(x,y) */",
     "const int64_t cp = np1 * (int64_t)row[y] + p[y];   /* c'_p(x,y) */"),
    ("transposed-scan", "const int64_t cp = np1 * (int64_t)row[y] - p[y];   /* c'_p(x,y) */",
     "const int64_t cp = np1 * (int64_t)C[(int64_t)y * n + x] - p[y];"),
    ("no-eps-in-bid", "p[w] -= (second - best) + eps;", "p[w] -= (second - best) + 0;"),
    ("no-second-update", "else if (cp < second) second = cp;", ";"),
    ("skip-final-phase", "} while (eps > final_eps);", "} while (eps / alpha > final_eps);"),
    ("displaced-not-requeued", "queue[tail % n] = old;\n                tail++;", ";"),
    ("hungarian-dual-sign", "int64_t red = (int64_t)row[j] - u[i] - v[j];",
     "int64_t red = (int64_t)row[j] - u[i] + v[j];"),
    ("hungarian-no-dual-update", "if (intree[j]) { u[owner[j]] += delta; v[j] -= delta; }",
     "if (intree[j]) { u[owner[j]] += delta; }"),
    ("hungarian-transposed", "const int32_t *row = C + (int64_t)i * n;\n            int64_t delta",
     "const int32_t *row = C + (int64_t)i;\n            int64_t delta"),
    ("brute-force-skips-perms", "while (i < n) {", "while (i < n - 1) {"),
    ("sparse-ssp-dual-sign", "const int64_t red = dmin + (int64_t)costs[k] - u[x] - v[j];",
     "const int64_t red = dmin + (int64_t)costs[k] - u[x] + v[j];"),
    ("sparse-ssp-no-row-dual", "            u[owner[j]] += d;\n", ""),
    ("sparse-ssp-root-dual-kept", "        u[r] += dfree;\n", ""),
    ("sparse-parallel-arc-max", "if (cols[k] == y && costs[k] < best) best = costs[k];",
     "if (cols[k] == y && (best == OR_INF || costs[k] > best)) best = costs[k];"),
    ("dinic-backward-residual-sign", "res[stack_a[i]] -= d; res[stack_a[i] ^ 1] += d;",
     "res[stack_a[i]] -= d; res[stack_a[i] ^ 1] -= d;"),
    ("dinic-arcs-undirected", "res[2 * a + 1] = 0;   to[2 * a + 1] = tail[a];",
     "res[2 * a + 1] = cap[a];   to[2 * a + 1] = tail[a];"),
    ("min-cut-brute-allows-t-inside", "if (!(mask >> s & 1u) || (mask >> t & 1u)) continue;",
     "if (!(mask >> s & 1u)) continue;"),
    ("certify-arc-reversed", "const int64_t from = d[match[x]] - (int64_t)row[match[x]];",
     "const int64_t from = d[match[x]] + (int64_t)row[match[x]];"),
    ("certify-one-sweep", "for (int32_t sweep = 0; changed && sweep <= n; ++sweep) {",
     "for (int32_t sweep = 0; changed && sweep < 1; ++sweep) {"),
    ("certify-dual-from-own-row", "if (u_out) u_out[x] = (int64_t)C[(int64_t)x * n + match[x]] - d[match[x]];",
     "if (u_out) u_out[x] = (int64_t)C[(int64_t)x * n + x] - d[match[x]];"),
    ("arcfix-threshold-zero", "if (cp > 2 * (int64_t)n * eps) { dead[y] = 1; deleted++; }",
     "if (cp > 0) { dead[y] = 1; deleted++; }"),
    ("arcfix-threshold-eps", "if (cp > 2 * (int64_t)n * eps) { dead[y] = 1; deleted++; }",
     "if (cp > eps) { dead[y] = 1; deleted++; }"),
    ("arcfix-next-phase-eps", "if (cp > 2 * (int64_t)n * eps) { dead[y] = 1; deleted++; }",
     "if (cp > 2 * (int64_t)n * (eps / alpha)) { dead[y] = 1; deleted++; }"),
    ("arcfix-no-row-price", "const int64_t cp = np1 * (int64_t)row[y] + px - p[y];   /* c_p(x,y) */",
     "const int64_t cp = np1 * (int64_t)row[y] - p[y];"),
    ("arcfix-row-price-sign", "const int64_t px = -(mn + eps);", "const int64_t px = (mn + eps);"),
    ("sparse-brute-force-ignores-arcs", "s = w[x][perm[x]] >= OR_INF ? OR_INF : s + w[x][perm[x]];",
     "s = w[x][perm[x]] >= OR_INF ? s : s + w[x][perm[x]];"),
]


def _run_battery(src, tmp_path, timeout=120):
    env = dict(os.environ, PYTHONPATH=ROOT)
    try:
        r = subprocess.run([sys.executable, BATTERY, src], cwd=str(tmp_path), env=env,
                           capture_output=True, timeout=timeout)
        return r.returncode
    except subprocess.TimeoutExpired:
        return "timeout"


def test_battery_passes_on_real_oracle(tmp_path):
    assert _run_battery(SRC, tmp_path) == 0


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    if name == "hungarian-transposed":
        # the transposed row walks down column i: stride n instead of 1
        text = text.replace("int64_t red = (int64_t)row[j] - u[i] - v[j];",
                            "int64_t red = (int64_t)row[(int64_t)j * n] - u[i] - v[j];")
    mutant = tmp_path / "oracle.c"
    mutant.write_text(text.replace(old, new, 1))
    rc = _run_battery(str(mutant), tmp_path, timeout=30)
    assert rc != 0, f"planted mistake {name} was not caught"
