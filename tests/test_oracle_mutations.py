"""The oracle's pins catch plausible slips.

Each case plants one mistake in a copy of oracle.c (on the CPU), builds it
into a temporary library and runs the pin suites against it through
ORACLE_LIB; the suites must fail.  The committed oracle is untouched.
"""
import os
import subprocess
import sys

import pytest

from oracle import oracle as orc_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "derivative_sign": ("q[m + 1][i + 1] += -2.0 * g * c;", "q[m + 1][i + 1] += 2.0 * g * c;"),
    "power_rule": ("q[m + 1][i - 1] += (double)i * c;", "q[m + 1][i - 1] += (double)(i + 1) * c;"),
    "laplacian_term": ("o[4 * na + k] = d[4 * na + k] + d[5 * na + k] + d[6 * na + k];",
                       "o[4 * na + k] = d[4 * na + k] + d[5 * na + k];"),
    "ao_factor": ("const double w = b->ao_factor[ao0 + j] * cf * e;", "const double w = cf * e;"),
    "cartesian_order": ("for (int bb = l - aa; bb >= 0; --bb) {",
                        "for (int bb = 0; bb <= l - aa; ++bb) {"),
    "threshold_bits": ("return (double)(bits - 1) * log(2.0);", "return (double)(bits) * log(2.0);"),
    "radial_power": ("const double e = exp(-g * r2);", "const double e = exp(-g * sqrt(r2));"),
    "dot2_error_term": ("acc->s += q + r;", "acc->s += q;"),
    "two_product_dropped": ("double r = fma(x, y, -h);", "double r = 0.0;"),
    "mo_transpose": ("dot2_add(&acc, ci[k], a[k]);",
                     "dot2_add(&acc, C[(size_t)k * mo_num + i], a[k]);"),
    "adjoint_sign": ("dot2_add(&accR[3 * A + j], -abar[(size_t)c * na + k], g[c]);",
                     "dot2_add(&accR[3 * A + j], abar[(size_t)c * na + k], g[c]);"),
    "adjoint_hessian_index": ("g[1] = DV(1 + e[0], e[1], e[2], k);",
                              "g[1] = DV(e[0], 1 + e[1], e[2], k);"),
    "shell_factor": ("const double cf = b->shell_factor[s] * b->coefficient[k] * b->prim_factor[k];",
                     "const double cf = b->coefficient[k] * b->prim_factor[k];"),
    "screen_count_radius": ("if (b->exponent[k] * r2 < T) ++np;",
                            "if (b->exponent[k] * sqrt(r2) < T) ++np;"),
    "screen_count_cartesians": ("counts[2] += (l + 1) * (l + 2) / 2;",
                                "counts[2] += 2 * l + 1;"),
    "screen_count_nucleus": ("const double* R = b->nucl_coord + 3 * b->shell_nucleus[s];\n"
                             "      const double dx",
                             "const double* R = b->nucl_coord;\n      const double dx"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_fail_on_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(orc_mod.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    msrc = tmp_path / "oracle_mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = orc_mod.build(force=True, src=str(msrc), out=str(tmp_path / "liboracle_mutant.so"))
    env = dict(os.environ, ORACLE_LIB=lib)
    suites = [os.path.join(ROOT, "tests", "test_oracle_pins.py"),
              os.path.join(ROOT, "tests", "test_oracle_adjoint.py")]
    if name.startswith("adjoint"):
        suites.reverse()          # the same suites; the adjoint pins first (-x stops early)
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *suites],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
