"""Each planted mistake in the oracle (compiled in only with -DORC_MUTANT=k) must
make at least one pin of tests/test_oracle_pins.py fail: the pins are sharp
enough to catch a wrong sign, a misplaced coefficient, a dropped term, an
uncompensated sum, transposed axes, lost NaNs, an ignored fused value, the
wrong norm or an absolute stencil (the tolerance scale) missing a |.|.
Each mutant runs in its own process."""
import json
import os
import subprocess
import sys

import pytest

from oracle import oracle as O

MUTANTS = {
    1: "x offset read with the wrong sign",
    2: "coefficient grid read off the core element",
    3: "last term of the operator dropped",
    4: "plain recursive sum instead of the compensated one",
    5: "x and y axes exchanged in the layout",
    6: "NaN ignored by max-abs",
    7: "the operator's value read as zero by fused terms",
    8: "1-norm instead of 2-norm",
    9: "red-black colour taken from i + j only",
    10: "do_diamond rows visited in reverse",
    11: "absolute stencil without |C| on the coefficient",
    12: "absolute stencil without |X| on the value read",
}

RUNNER = r"""
import inspect, json, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[2])
from oracle import oracle as O
O.use_library(sys.argv[3] if sys.argv[3] != "-" else None)
import test_oracle_pins as P
failed, passed = [], []
for name, fn in inspect.getmembers(P, inspect.isfunction):
    if not name.startswith("test_"):
        continue
    params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    cases = [{}]
    if params:
        names = [a.strip() for a in params[0].args[0].split(",")]
        cases = [dict(zip(names, v if len(names) > 1 else (v,))) for v in params[0].args[1]]
    for kw in cases:
        try:
            fn(**kw)
            passed.append(name)
        except (AssertionError, ValueError):
            failed.append(name)
print(json.dumps({"failed": failed, "passed": len(passed)}))
"""

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_pins(lib_path):
    out = subprocess.run([sys.executable, "-c", RUNNER, ROOT, HERE, lib_path or "-"],
                         capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        return {"crashed": out.returncode, "stderr": out.stderr[-2000:]}
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_detect_planted_mistake(mutant):
    res = run_pins(O.build(mutant=mutant))
    assert "crashed" not in res, res
    assert res["failed"], f"no pin caught mutant {mutant}: {MUTANTS[mutant]}"


def test_unmutated_oracle_passes_every_pin():
    res = run_pins(None)
    assert res.get("failed") == [], res
