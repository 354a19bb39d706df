"""The oracle's pins are strong enough to catch plausible mistakes.  Each
mutant of tests/oracle_mutants.py plants one mistake in the oracle on the CPU:

- a dropped term;
- a transposed operand;
- a wrong sign, factor or branch;
- a wrong pair order or normalisation.

The pin file named for it is then run in a fresh interpreter, which must end
with a failing test (pytest exit status 1).  Without a mutant the same files
pass: they are part of this suite."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from tests.oracle_mutants import MUTANTS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(name):
    files = MUTANTS[name][1]
    code = ("import sys; sys.path.insert(0, %r); import tests.oracle_mutants as M; "
            "M.apply(%r); import pytest; "
            "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu', %s]))"
            % (ROOT, name, ", ".join(repr(f) for f in files)))
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=600, env=env)
    return r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


@pytest.fixture(scope="module")
def results():
    with cf.ThreadPoolExecutor(4) as ex:
        return dict(zip(MUTANTS, ex.map(_run, MUTANTS)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_mutant(results, name):
    rc, tail = results[name]
    assert rc == 1, f"mutant {name} survived its pins (pytest status {rc}):\n{tail}"
