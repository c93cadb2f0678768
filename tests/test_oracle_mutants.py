"""The oracle's pins must catch plausible mistakes.

Each case copies oracle/tgp_oracle.c to a temporary directory, plants one
mistake (a swapped operand, a dropped term, a wrong index, ...), builds the
copy and runs tests/test_oracle.py against it in a subprocess.  The pin suite
must fail for every mutant.  Nothing here runs on a GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tgp_oracle.c")

MUTANTS = {
    "sub_operands_swapped": ("case O_SUB: return a - b;", "case O_SUB: return b - a;"),
    "div_protection_value": ("if (b == 0.0) return 0.0;", "if (b == 0.0) return 1.0;"),
    "trig_not_pi_scaled": ("double pf = ORACLE_PI * f, v;", "double pf = f, v;"),
    "sin_cos_swapped": ("case O_SIN: return rad ? sin(a) : oracle_sinpi(a);\n    case O_COS: return rad ? cos(a) : oracle_cospi(a);",
                        "case O_SIN: return rad ? sin(a) : oracle_cospi(a);\n    case O_COS: return rad ? cos(a) : oracle_sinpi(a);"),
    "radian_sin_pi_scaled": ("case O_SIN: return rad ? sin(a)", "case O_SIN: return rad ? sin(ORACLE_PI * a)"),
    "radian_cos_is_sin": ("case O_COS: return rad ? cos(a)", "case O_COS: return rad ? sin(a)"),
    "radian_tan_pi_scaled": ("case O_TAN: return rad ? tan(a)", "case O_TAN: return rad ? tan(ORACLE_PI * a)"),
    "bound_radian_no_propagation": ("const double k = rad ? 1.0 : ORACLE_PI;", "const double k = rad ? 0.0 : ORACLE_PI;"),
    "pagie_wrong_index": ("y4 / (1.0 + y4)", "x4 / (1.0 + y4)"),
    "pagie_dropped_term": ("return x4 / (1.0 + x4) + y4 / (1.0 + y4);", "return x4 / (1.0 + x4);"),
    "linspace_off_by_one": ("float step = (hi - lo) / (float)(n - 1);", "float step = (hi - lo) / (float)n;"),
    "rmse_divides_by_n_minus_1": ("double r64 = sqrt(s64 / (double)N);", "double r64 = sqrt(s64 / (double)(N - 1));"),
    "postfix_operands_transposed": ("for (int c = ar - 1; c >= 0; c--) nodes[me].kid[c] = stack[--sp];",
                                    "for (int c = 0; c < ar; c++) nodes[me].kid[c] = stack[--sp];"),
    "grid_row_col_swapped": ("int64_t row = p / W, col = p % W;", "int64_t col = p / W, row = p % W;"),
    "min_is_max": ("case O_MIN: return fmin(a, b);", "case O_MIN: return fmax(a, b);"),
    "fp32_mode_not_rounded_per_node": ("*v32 = (float)apply64(n->op, (double)a32, (double)b32, (double)c32, pt->rad);",
                                       "*v32 = (float)apply64(n->op, a64, b64, c64, pt->rad);"),
    "near_singular_threshold": ("#define NEAR_SINGULAR 1e-6", "#define NEAR_SINGULAR 1e-9"),
    "nan_fitness_not_inf": ("rmse64[t] = isfinite(r64) ? r64 : INFINITY;", "rmse64[t] = r64;"),
    "abs_dropped": ("case O_ABS: return fabs(a);", "case O_ABS: return a;"),
    "bound_mul_drops_term": ("prop = fabs(b) * ea + fabs(a) * eb + ea * eb;", "prop = fabs(b) * ea + ea * eb;"),
    "bound_div_drops_term": ("prop = (ea + fabs(a / b) * eb) / (fabs(b) - eb);", "prop = ea / (fabs(b) - eb);"),
    "bound_trig_not_pi": ("const double k = rad ? 1.0 : ORACLE_PI;", "const double k = 1.0;"),
    "bound_add_no_rounding": ("e = prop + rnd32(v, prop, 1);", "e = prop;"),
    "log_protection_value": ("if (a < 0.0) return -1.0;", "if (a < 0.0) return 0.0;"),
    "pow_zero_zero_is_one": ("if (a == 0.0 && b == 0.0) return 0.0;", "if (a == 0.0 && b == 0.0) return 1.0;"),
    "sqrt_of_abs": ("if (a < 0.0) return 0.0;\n    return sqrt(a);", "return sqrt(fabs(a));"),
    "mod_truncated": ("if (r != 0.0 && ((r < 0.0) != (b < 0.0))) r += b;", ""),
    "clip_bounds_swapped": ("case O_CLIP: return fmax(fmin(c, a), b);", "case O_CLIP: return fmax(fmin(b, a), c);"),
    "if_branches_swapped": ("case O_IF: return a != 0.0 ? b : c;", "case O_IF: return a != 0.0 ? c : b;"),
    "tan_not_pi_scaled": ("case O_TAN: return rad ? tan(a) : oracle_sinpi(a) / oracle_cospi(a);",
                          "case O_TAN: return tan(a);"),
    "frac_truncates": ("case O_FRAC: return a - floor(a);", "case O_FRAC: return a - trunc(a);"),
    "mdist_not_halved": ("case O_MDIST: return (a + b) / 2.0;", "case O_MDIST: return a + b;"),
    "sign_of_zero_is_one": ("if (a == 0.0) return 0.0;\n    return a;", "if (a == 0.0) return 1.0;\n    return a;"),
    "bound_exp_no_propagation": ("prop = fabs(v) * expm1(ea);", "prop = 0.0;"),
    # bounds inflated: the tightness pins (twice the first-order worst case) must catch them
    "bound_rounding_doubled": ("double e = U32 * m;", "double e = 2.0 * U32 * m;"),
    "bound_trig_four_ulps": ("#define TRIG_ULPS 2.0", "#define TRIG_ULPS 4.0"),
    "bound_trig_lipschitz_one": ("prop = fmin(k * ea * slope + 0.5 * (k * ea) * (k * ea), 2.0);",
                                 "prop = fmin(k * ea + 0.5 * (k * ea) * (k * ea), 2.0);"),
    "bound_mul_inflated": ("prop = fabs(b) * ea + fabs(a) * eb + ea * eb;",
                           "prop = 2.0 * (fabs(b) * ea + fabs(a) * eb) + ea * eb;"),
    "bound_div_inflated": ("prop = (ea + fabs(a / b) * eb) / (fabs(b) - eb);",
                           "prop = 2.0 * (ea + fabs(a / b) * eb) / (fabs(b) - eb);"),
    "bound_add_inflated": ("case O_ADD: case O_SUB:\n        prop = ea + eb;",
                           "case O_ADD: case O_SUB:\n        prop = 2.0 * (ea + eb);"),
    "bound_minmax_always_max": ("if (fabs(a - b) > ea + eb) e = (v == a) ? ea : eb;", "if (0) e = ea;"),
    "bound_neg_inflated": ("case O_NEG: case O_ABS:\n        e = ea;", "case O_NEG: case O_ABS:\n        e = 2.0 * ea;"),
    "const_imm_order": ("nodes[me].imm = (double)imm[(*imm_pos)++];\n    }\n    for (int c = 0; c < ar; c++) {",
                        "nodes[me].imm = (double)imm[n_imm - 1 - (*imm_pos)++];\n    }\n    for (int c = 0; c < ar; c++) {"),
}


def _run_mutant(name, workdir):
    """Builds one mutant and runs the pins against it; returns (rc, output)."""
    old, new = MUTANTS[name]
    src = open(SRC).read()
    if src.count(old) < 1:
        return None, f"mutation site for {name} not found"
    c = os.path.join(workdir, f"{name}.c")
    so = os.path.join(workdir, f"lib{name}.so")
    with open(c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                           "-o", so, c, "-lm"])
    env = dict(os.environ, TGP_ORACLE_LIB_OVERRIDE=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """Every mutant's pin run, several at a time (each is its own process)."""
    from concurrent.futures import ThreadPoolExecutor
    workdir = str(tmp_path_factory.mktemp("mutants"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        futs = {n: ex.submit(_run_mutant, n, workdir) for n in sorted(MUTANTS)}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, mutant_results):
    rc, out = mutant_results[name]
    assert rc is not None, out
    assert rc != 0, f"mutant {name} survived the oracle pins:\n{out}"
