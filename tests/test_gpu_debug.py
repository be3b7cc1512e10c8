"""Debug mode (BTE_DEBUG): guard words after every device buffer, checked
after each solve, and the index tables checked at plan creation.

The library reads BTE_DEBUG once, when it first allocates, so each case runs
in a child process with the variable set.  The overwritten guard is written
by the host into the allocation (a legal write just past the buffer's end);
nothing here faults the GPU."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    import bte_inputs as bi
    import paper_2503_23657_gb300 as bte
    from paper_2503_23657_gb300.binding import BTEError
    cases = [bi.tiny(2, n=(9, 7, 1), B=2, masked=True, diffuse=(2, 3), source=True),
             bi.tiny(3, n=(6, 5, 4), B=2, masked=True, diffuse=(0, 3, 5), two_regions=True),
             bi.tiny(2, n=(8, 6, 1), B=2, specular=(2, 3))]
    for p in cases:
        plan = bte.Plan(p)                       # index tables checked here
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=1, tol=1e-8, max_iter=100000, check=False)
        print("solve", rc)
        g = np.zeros(p.n_cells)
        g[np.flatnonzero(p.mask)[:3]] = 1.0
        rc = plan.adjoint(g, tol=1e-8, check=False)[0]
        print("adjoint", rc)
    plan = bte.Plan(cases[0])
    T = np.zeros(cases[0].n_cells)
    plan.solve(T, precision=0, tol=0.0, max_iter=3)
    plan.debug_overwrite_guard()
    rc, st = plan.solve(T, precision=0, tol=0.0, max_iter=3, check=False)
    print("corrupt", rc, plan.error())
""")


def _run(env_value):
    env = dict(os.environ)
    if env_value is None:
        env.pop("BTE_DEBUG", None)
    else:
        env["BTE_DEBUG"] = env_value
    return subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True,
                          text=True, timeout=600)


def test_guards_hold_and_an_overwritten_guard_is_reported():
    r = _run("1")
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    assert [l for l in lines if l.startswith("solve")] == ["solve 0"] * 3
    assert [l for l in lines if l.startswith("adjoint")] == ["adjoint 0"] * 3
    corrupt = [l for l in lines if l.startswith("corrupt")][0]
    assert corrupt.startswith("corrupt -8") and "guard" in corrupt


def test_guard_hook_needs_debug_mode():
    r = _run(None)
    assert r.returncode != 0 and "ESTATE" in r.stderr
