"""Bounds checking in place of a memory checker: the library rebuilt with
-DHISQ_BOUNDS_CHECK range-checks every neighbour and site index in its kernels;
the Dslash on lattices that exercise every wrap-around (L = 4 aliasing, ragged
half-volumes, several tiles), the single and batched solves, the eigensolver and
the network layer all run without an out-of-range index, and give the normal
build's results."""
import os
import subprocess
import sys
import textwrap

import pytest

from paper_2502_00152_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import numpy as np, torch, sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    from paper_2502_00152_gb300 import hisq as H, inputs as I
    from gpu_common import make, rel, dslash_ref
    for dims in [(4, 4, 4, 4), (4, 6, 4, 10), (8, 4, 6, 6), (6, 6, 6, 8)]:
        for recon in (18, 12, 8):
            ctx, o = make(dims, recon=recon, mass=0.05)
            src = I.gaussian_field(dims, 18)
            for par in (0, 1):
                ref = dslash_ref(o, dims, src, par)
                assert rel(H.hisq_apply_dslash(ctx, par, 64, src, link_precision=64), ref) <= 1e-13
                assert rel(H.hisq_apply_dslash(ctx, par, 16, src, link_precision=32), ref) <= 5e-3
            eta = I.gaussian_source(dims, 3, 0)
            psi, st, s = H.hisq_solve(ctx, eta, H.hisq_default_solve_params(precision_sloppy=16))
            assert s == H.HISQ_OK and o.full_residual(0.05, psi, eta) <= 1e-10
            etas = np.stack([I.gaussian_source(dims, 3, j) for j in range(5)])
            psi, st, s = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(precision_sloppy=16, batch=1))
            assert s == H.HISQ_OK
            assert H.hisq_bounds_violations(ctx) == 0, (dims, recon)
            ctx.close()
    dims = (6, 6, 6, 6)
    ctx, o = make(dims, mass=0.01)
    H.hisq_eigensolve(ctx, H.hisq_default_eig_params(n_ev=8, n_kr=32, cheby_degree=8, a_min=-2.0, block_size=4))
    x = torch.from_numpy(np.stack([I.gaussian_field(dims, 5 + a) for a in range(3)]).astype(np.complex64)).cuda()
    w = torch.ones((4, 3, 9), dtype=torch.complex64, device="cuda")
    out = torch.empty((4,) + tuple(x.shape[1:]), dtype=torch.complex64, device="cuda")
    H.hisq_net_layer(ctx, w, x, out)
    torch.cuda.synchronize()
    assert H.hisq_bounds_violations(ctx) == 0
    ctx.close()
    print("bounds ok")
""")


def test_bounds_checking_build_finds_no_out_of_range_index():
    lib = B.build(bounds_check=True)
    env = dict(os.environ, HISQ_LIBRARY=lib)
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "bounds ok" in r.stdout


def test_normal_build_reports_unchecked():
    from gpu_common import make
    from paper_2502_00152_gb300 import hisq as H

    ctx, o = make((4, 4, 4, 4))
    try:
        with pytest.raises(H.HisqError) as e:
            H.hisq_bounds_violations(ctx)
        assert e.value.status == H.HISQ_ERR_STATE
    finally:
        ctx.close()
