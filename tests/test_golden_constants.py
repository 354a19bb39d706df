"""The solver constants that the paper prints (tests/golden/solver_constants.txt,
each line with its passage) against the oracle's defaults, the workloads'
tolerances and the C header's documented defaults."""
import inspect
import os
import re

from oracle import fullspace, lbfgs, reduced
from workloads import CONFIGS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden():
    out = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "solver_constants.txt")):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, rest = line.split("=", 1)
        value, cite = rest.split("|", 1)
        assert cite.strip(), key                     # every value carries its passage
        vals = [float(v) for v in value.split()]
        out[key.strip()] = vals[0] if len(vals) == 1 else vals
    return out


def _default(fn, name):
    return inspect.signature(fn).parameters[name].default


def test_oracle_caps_are_the_papers():
    g = _golden()
    for fn, it_name in ((reduced.newton_solve, "max_newton"), (fullspace.newton_solve, "max_newton"),
                        (lbfgs.lbfgs_minimize, "max_iters"), (lbfgs.lbfgs_solve, "max_iters"),
                        (reduced.ReducedSimulator.__init__, "max_newton")):
        assert _default(fn, it_name) == g["max_iters"], fn
        assert _default(fn, "max_ls") == g["max_ls"], fn
    assert _default(reduced.ReducedSimulator.__init__, "eps") == g["eps_inf"]


def test_workload_tolerances_and_caps():
    """The full-size workloads use the paper's eps; the small parity cases are
    tighter (1e-6 to 1e-8) so that parity is checked below it."""
    g = _golden()
    for name in ("bar_twist_dyn_14976", "block_twist_960k", "block_twist_207k",
                 "torus_drop_200k"):
        c = CONFIGS[name]
        assert c.eps == g["eps_inf"], name
        assert c.max_newton == g["max_iters"] and c.max_ls == g["max_ls"], name
    for name in ("tiny_quasistatic", "tiny_dyn", "small_dyn_full"):
        assert CONFIGS[name].eps <= min(g["eps_sweep"]), name


def test_header_and_context_use_the_same_defaults():
    """The header's documented defaults and the context's initial values."""
    g = _golden()
    src = open(os.path.join(ROOT, "include", "lsn.h")).read()
    m = re.search(r"Defaults of a new context: tol_inf = ([0-9.e+-]+), max_newton = (\d+),"
                  r"\s*\*?\s*max_ls = (\d+)", src)
    assert m, "lsn.h states the solver defaults"
    assert float(m.group(1)) == g["eps_inf"]
    assert int(m.group(2)) == g["max_iters"] and int(m.group(3)) == g["max_ls"]
    api = open(os.path.join(ROOT, "paper_2409_03807_gb300", "csrc", "api.cu")).read()
    assert re.search(r"double tol = ([0-9.e+-]+)", api).group(1) == "1e-5"
    assert re.search(r"int max_newton = (\d+), max_ls = (\d+);", api).groups() == ("1024", "128")
