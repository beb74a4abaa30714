"""Plants plausible mistakes in copies of the oracle (on the CPU) and checks that the pins
catch each one: a dropped term, a wrong sign or index, a transposed operand, a wrong
boundary or tie rule. A mutant the pins do not reject would mean a blind spot in the pins.
"""

import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "zncc_oracle.c")

# (name, original text, mutated text): each original must occur exactly once
MUTANTS = [
    ("disparity_sign", "(pix(R, W, H, x - d + i, y + j) - mR)",
     "(pix(R, W, H, x + d + i, y + j) - mR)"),
    ("target_stats_centre", "int t = x - d + (D - 1);", "int t = x + (D - 1);"),
    ("swapped_operands", "(pix(L, W, H, x + i, y + j) - mL) * (pix(R, W, H, x - d + i, y + j) - mR)",
     "(pix(R, W, H, x + i, y + j) - mL) * (pix(L, W, H, x - d + i, y + j) - mR)"),
    ("mean_divisor", "double m = s / n;", "double m = s / (n - 1);"),
    ("sigma_no_sqrt", "*sigma = sqrt(ss);", "*sigma = ss;"),
    ("zero_variance_cost", "if (sL == 0.0 || sR == 0.0) return 0.0;",
     "if (sL == 0.0 || sR == 0.0) return 1.0;"),
    ("integral_corner_dropped", "S[(long)y * nx + xi] = B1[a] + B1[b] - B1[c] - B1[e];",
     "S[(long)y * nx + xi] = B1[a] - B1[c] - B1[e];"),
    ("weight_sigma_r_inverted", "return K * exp(-fabs(gdiff) / sigma_r);",
     "return K * exp(-fabs(gdiff) * sigma_r);"),
    ("weight_R_wrong_neighbour", "dt_weight(g - guide[i + 1] / 255.0",
     "dt_weight(g - guide[i - (x > 0)] / 255.0"),
    ("boundary_unscaled", "c[k] = x == 0 ? j->s * c[k] :", "c[k] = x == 0 ? c[k] :"),
    ("scale_factor", "double s = scaled ? 1.0 - exp(-1.0 / sigma_s) : 1.0;",
     "double s = scaled ? exp(-1.0 / sigma_s) : 1.0;"),
    ("pass_order", "parallel_for(H, nthreads, pass_l2r, &jl);\n        parallel_for(H, nthreads, pass_r2l, &jr);",
     "parallel_for(H, nthreads, pass_r2l, &jr);\n        parallel_for(H, nthreads, pass_l2r, &jl);"),
    ("vertical_neighbour", "c[k] = y == 0 ? j->s * c[k] : j->s * c[k] + c[k - row] * wgt;",
     "c[k] = y == 0 ? j->s * c[k] : j->s * c[k] + c[k - j->nd] * wgt;"),
    ("wta_tie_largest", "if (1.0 - c[d] < bcost) { bcost = 1.0 - c[d]; bd = d; }",
     "if (1.0 - c[d] <= bcost) { bcost = 1.0 - c[d]; bd = d; }"),
    ("fastdt_zero_encoded", "if (value >= 0) return 0;", "if (value > 0) return 0;"),
    ("fastdt_flag_swapped", "if (mid4 != 0xF) return (uint8_t)((((v >> 5) & 0x3F) << 2) | 2u);",
     "if (mid4 != 0xF) return (uint8_t)((((v >> 5) & 0x3F) << 2) | 1u);"),
    ("fastdt_fill_short", "for (int b = low + 6; b < 16; ++b) v |= 1u << b;",
     "for (int b = low + 7; b < 16; ++b) v |= 1u << b;"),
    ("fastdt_store_after_last_pair", "if (pair < 2 * iters) rc = oracle_fastdt_store(C, ones, W, H, nd, d_arb, T);",
     "if (pair <= 2 * iters) rc = oracle_fastdt_store(C, ones, W, H, nd, d_arb, T);"),
    # the store divides by A_hat of the previous pair (all ones before the first)
    ("fastdt_ahat_one_pair_behind",
     "if (pair < 2 * iters) rc = oracle_fastdt_store(C, ones, W, H, nd, d_arb, T);",
     "{ static double lag[1 << 16]; if (pair == 1) for (size_t i = 0; i < n; ++i) lag[i] = 1.0;\n"
     "          if (pair < 2 * iters) rc = oracle_fastdt_store(C, lag, W, H, nd, d_arb, T);\n"
     "          for (size_t i = 0; i < n; ++i) lag[i] = ones[i]; }"),
    ("fastdt_d_arb_one", "const double ref = c[d_arb], a = ahat[p];",
     "const double ref = c[d_arb + (nd > 1)], a = ahat[p];"),
    ("fastdt_reference_sign", "double e = rint(T * (ref - c[d]) / a);", "double e = rint(T * (c[d] - ref) / a);"),
]

RUNNER = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, oracle_pins
lib = oracle.load({lib!r})
failed = []
for pin in oracle_pins.ALL_PINS:
    try:
        pin(lib)
    except Exception as e:
        failed.append(pin.__name__)
print("CAUGHT_BY", ",".join(failed))
sys.exit(1 if failed else 0)
"""


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, orig, mut, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found exactly once"
    msrc = tmp_path / f"oracle_{name}.c"
    msrc.write_text(src.replace(orig, mut))
    lib = str(tmp_path / f"lib_{name}.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", str(msrc), "-o",
                    lib, "-lm"], check=True)
    proc = subprocess.run([sys.executable, "-c", RUNNER.format(
        root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)], capture_output=True,
        text=True, timeout=300)
    assert proc.returncode != 0, f"mutant {name} survived every pin:\n{proc.stdout}{proc.stderr}"


def test_unmutated_oracle_passes_runner(tmp_path):
    """The runner itself reports success on the real oracle (so a caught mutant means a pin
    failure, not a broken harness)."""
    proc = subprocess.run([sys.executable, "-c", RUNNER.format(
        root=ROOT, tests=os.path.join(ROOT, "tests"), lib=oracle.build())],
        capture_output=True, text=True, timeout=300)
    assert proc.returncode == 0, proc.stdout + proc.stderr
