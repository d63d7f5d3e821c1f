"""The README's C example, compiled against include/varlingam_gb300.h and
linked with the shared library (by __graft_entry__.build()), run as its own
process, and compared with the Python binding on the same seeded series."""
import os
import subprocess

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EXE = os.path.join(ROOT, "paper_2409_05500_gb300", "_build", "readme_example")


def lcg_series(m, n, seed):
    """The C program's series: the same 64-bit LCG and recursion."""
    mask = (1 << 64) - 1
    s = seed
    X = np.zeros((m, n))
    for t in range(n):
        carry = 0.0
        for i in range(m):
            s = (s * 6364136223846793005 + 1442695040888963407) & mask
            e = 2.0 * ((s >> 11) * (1.0 / 9007199254740992.0)) - 1.0
            prev = X[i, t - 1] if t else 0.0
            X[i, t] = 0.3 * prev + e + 0.5 * carry
            carry = e
    return X


def test_lcg_series_is_deterministic():
    a = lcg_series(3, 5, 7)
    assert np.array_equal(a, lcg_series(3, 5, 7)) and np.all(np.abs(a) < 4)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_readme_c_example_matches_the_binding(vl, prec):
    assert os.path.exists(EXE), "built by __graft_entry__.build()"
    m, n, seed = 12, 800, 2409
    env = dict(os.environ)
    lib_dir = os.path.join(ROOT, "paper_2409_05500_gb300")
    env["LD_LIBRARY_PATH"] = lib_dir + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    r = subprocess.run([EXE, str(m), str(n), str(seed), str(prec)], capture_output=True,
                       text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    order_c = [int(v) for v in lines["order"].split()]
    B0_c = np.array([float(v) for v in lines["B0"].split()]).reshape(m, m)
    h = vl.Handle(0)
    X = torch.from_numpy(lcg_series(m, n, seed)).cuda()
    out = vl.fit(h, X, 1, prec="mixed" if prec else "fp64")
    h.close()
    assert order_c == [int(c) for c in out["order"].cpu().numpy()]
    assert np.abs(B0_c - out["B0"].cpu().numpy()).max() <= 1e-12
