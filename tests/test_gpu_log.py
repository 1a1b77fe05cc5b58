"""BTAS_LOG=1 reports each entry point's execution choices on stderr (read
once per process, so each case runs in a fresh interpreter)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import torch
import gen
import paper_1701_04733_gb300 as btas
W = torch.from_numpy(gen.random_graph(1, 1, {n}, {p}, 1, 100)).cuda()
btas.apsp(W)
A = torch.from_numpy(gen.uniform_int(1, 2, (300, 200), 0, 100)).cuda()
btas.gemm(A, A.t().contiguous(), 0)
btas.gemm(A, A.t().contiguous(), 0, packed=True)
torch.cuda.synchronize()
"""


@pytest.mark.parametrize("n,p,regime", [(48, 0.1, "one-block kernel"), (300, 0.1, "cooperative kernel"),
                                        (2000, 0.1, "cooperative kernel"), (2816, 0.02, "cooperative kernel"),
                                        (2816, 0.5, "tiled kernels"), (4608, 0.02, "tiled kernels")])
def test_log_reports_regime_and_kernel_choice(n, p, regime):
    """Above n = 1792 the cooperative kernel keeps a graph only if every row
    fits its edge lists (up to 256 edges): p = 0.1 at n = 2000 and p = 0.02 at
    2816 stay, p = 0.5 at 2816 is declined after the domain check and solved
    on the tiled kernels, and n = 4608 is above the cooperative kernel's
    range."""
    env = dict(os.environ, BTAS_LOG="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, n=n, p=p)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stderr.splitlines() if x.startswith("[btas]")]
    assert any(f"apsp n={n}: {regime}" in x for x in lines), lines
    if p == 0.5:
        assert any(f"apsp n={n}: too dense for the cooperative kernel's edge lists" in x for x in lines), lines
    assert any("product 300x300x200 int32 min-plus: variant" in x for x in lines), lines
    assert any("packed path requested" in x for x in lines), lines
    quiet = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, n=n, p=p)],
                           env=dict(os.environ, BTAS_LOG="0"), capture_output=True, text=True, timeout=300)
    assert quiet.returncode == 0 and "[btas]" not in quiet.stderr
