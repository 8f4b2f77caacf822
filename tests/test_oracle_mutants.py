"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that the pin suite rejects every one of them: a dropped term, a wrong sign,
a wrong index or offset, a transposed operand.

Dropping the CA's neighbour-membership check is not listed: the step requires
its input to be 0 off the gasket, so on every valid input that check changes
nothing (an equivalent mutant)."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "sg_oracle.c")

# (name, text in sg_oracle.c, planted replacement)
MUTANTS = [
    ("recursion-offset", "bm[(y + h) * n + x] = 1;", "bm[(y + h) * n + x + h] = 1;"),
    ("beta-axis-swap",
     "wx * (uint64_t)((mu + 1) % 2) + wy * (uint64_t)(mu % 2)",
     "wx * (uint64_t)(mu % 2) + wy * (uint64_t)((mu + 1) % 2)"),
    ("beta-divisor-off-by-one", "ipow3((mu + 1) / 2 - 1)", "ipow3((mu + 1) / 2)"),
    ("delta-transposed", "uint64_t dx = beta / 2;", "uint64_t dx = beta - beta / 2;"),
    ("tau-offset", "dx * ((uint64_t)1 << (mu - 1))", "dx * ((uint64_t)1 << mu)"),
    ("mirror-dropped", "*by = (((uint64_t)1 << rb) - 1) - ly;", "*by = ly;"),
    ("hash-shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;",
     "z = (z ^ (z >> 29)) * 0x94D049BB133111EBULL;"),
    ("linear31-transposed", "return (uint8_t)((x * 31 + y) & 0xFF);",
     "return (uint8_t)((y * 31 + x) & 0xFF);"),
    ("ca-self-counted", "if (dx == 0 && dy == 0) continue;", ";"),
    ("ca-birth-on-2", "next = (uint8_t)((count == 3 || (alive && count == 2)) ? 1 : 0);",
     "next = (uint8_t)((count == 2 || (alive && count == 3)) ? 1 : 0);"),
    ("diffusion-sign", "next = u + alpha * (sum - (double)deg * u);",
     "next = u + alpha * (sum + (double)deg * u);"),
    ("diffusion-deg-ignores-border",
     "if (!in_grid(nx, n) || !in_grid(ny, n)) continue;\n                    if (!or_member((uint64_t)nx, (uint64_t)ny)) continue;\n                    ++deg;",
     "if (!or_member((uint64_t)nx, (uint64_t)ny)) continue;\n                    ++deg;\n                    if (!in_grid(nx, n) || !in_grid(ny, n)) continue;"),
    ("launch-bbox-count", "                        ++l;\n", "                        l += 2;\n"),
    ("compact-scan-by-columns",
     "if (or_member(tx, ty)) { ltx[m] = tx; lty[m] = ty; ++m; }",
     "if (or_member(tx, ty)) { ltx[m] = ty; lty[m] = tx; ++m; }"),
    ("compact-tile-transposed", "xs[q * per_tile + e] = bx * rho + ltx[e];",
     "xs[q * per_tile + e] = by * rho + ltx[e];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                    "-ffp-contract=off", "-o", str(lib), str(mutated)], check=True)
    env = dict(os.environ, SG_ORACLE_LIB=str(lib))
    res = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
         os.path.join(ROOT, "tests", "test_oracle_pins.py"),
         "-k", "not level16"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"pins accepted the planted mistake {name}"
