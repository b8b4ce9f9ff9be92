"""The checked build (-DESPNMF_CHECKED: device-side bounds checks of every
data-dependent index, see espnmf_checked_flags) on the paths the tests
exercise: no check fails, and the results are bitwise those of the regular
library.  The checked library runs in a child process (the binding loads one
library per process, chosen by ESPNMF_CHECKED)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_1510_05237_gb300 as E

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs the workloads, reads the check flags after each, prints JSON.
SCRIPT = r'''
import json, sys
import numpy as np, torch
import paper_1510_05237_gb300 as E
from gen import planted_50k_100k, small_zipf, uniform_init, zipf_corpus
checked = E.library_path().endswith("_checked.so")
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
out = {"checked": checked, "runs": {}}

def flags():
    if not checked:
        return 0
    return E.espnmf_checked_flags()

def run(name, A, k, t_u, t_v, mode, comp, sweeps, U0):
    vals = A.val if comp == E.F64 else A.val.astype(np.float32)
    u0 = U0 if comp == E.F64 else U0.astype(np.float32)
    ctx = E.espnmf_init(dev(A.rowptr), dev(A.colidx), dev(vals), A.n, A.m, k, t_u, t_v, mode,
                        comp, dev(u0))
    R, Es = E.espnmf_iterate(ctx, sweeps)
    Uf = E.espnmf_get_factor(ctx, E.U)
    E.espnmf_destroy(ctx)
    out["runs"][name] = {"E": [float(e) for e in Es], "Usum": float(np.abs(Uf).sum()),
                         "flags": flags()}

flags()
A1 = planted_50k_100k(seed=2, scale=0.4)
run("planted_fp32_column_split", A1, 50, 300, 400, E.TOPT_COLUMN, E.F32, 4,
    uniform_init(A1.n, 50, 2))
A2 = small_zipf(seed=3)
run("zipf_fp64_column", A2, 10, 100, 100, E.TOPT_COLUMN, E.F64, 3, uniform_init(A2.n, 10, 3))
run("zipf_fp32_matrix", A2, 10, 700, 500, E.TOPT_MATRIX, E.F32, 3, uniform_init(A2.n, 10, 4))
A3 = planted_50k_100k(seed=5, scale=0.05)
run("planted_fp32_k72", A3, 72, 150, 200, E.TOPT_COLUMN, E.F32, 3, uniform_init(A3.n, 72, 5))
A4 = zipf_corpus(60000, 40000, 60.0, 1.05, 7, sigma=0.7)
run("zipf_fp32_k100_two_tier_frequent", A4, 100, 1200, 400, E.TOPT_COLUMN, E.F32, 3,
    uniform_init(A4.n, 100, 7))
U, V = E.espnmf_sequential(dev(A2.rowptr), dev(A2.colidx), dev(A2.val.astype(np.float32)),
                           A2.n, A2.m, 4, 100, 80, 2, dev(uniform_init(A2.n, 2, 6).astype(np.float32)),
                           E.F32, k2=2)
out["runs"]["sequential_k2"] = {"Usum": float(U.abs().sum()), "Vsum": float(V.abs().sum()),
                                "flags": flags()}
print(json.dumps(out))
'''


def _run(checked: bool):
    env = dict(os.environ)
    env.pop("ESPNMF_CHECKED", None)
    if checked:
        env["ESPNMF_CHECKED"] = "1"
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_passes_every_check_and_matches_the_regular_build():
    from paper_1510_05237_gb300 import build as B
    if not os.path.exists(B.LIB_CHECKED):
        pytest.fail("the checked build is missing: __graft_entry__.build() makes it")
    chk = _run(True)
    reg = _run(False)
    assert chk["checked"] and not reg["checked"]
    for name, r in chk["runs"].items():
        assert r["flags"] == 0, f"{name}: bounds checks failed (flags {r['flags']:#x})"
        g = reg["runs"][name]
        for key in r:
            if key != "flags":
                assert r[key] == g[key], (name, key, r[key], g[key])
