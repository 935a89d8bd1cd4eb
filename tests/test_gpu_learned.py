"""Learned initial guess on the GPU: the parallel-transport layer kernels
(forward, adjoint, weight gradient) against the FP64 network oracle, the
torch.autograd wrapper against finite differences, and a trained network that
starts CG closer to the solution while the solve still meets the 1e-10 FP64
true residual."""
import numpy as np
import pytest
import torch

from gpu_common import make, rel
from oracle.oracle import net_layer, net_wgrad, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I
from paper_2502_00152_gb300.learned import GuessNet, PTLayer

pytestmark = pytest.mark.gpu


def _rng_c(shape, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal(shape) + 1j * r.standard_normal(shape)) / np.sqrt(9 * shape[1])


def _ctx_on_torch_stream(dims, seed=3, eps=0.4, mass=None):
    fat, lng = I.hisq_links(dims, seed, eps)
    ctx = H.hisq_create(dims, True, 0, torch.cuda.current_stream().cuda_stream)
    H.hisq_load_links(ctx, fat, lng)
    if mass is not None:
        H.hisq_set_mass(ctx, mass)
    return ctx, fat, lng


@pytest.mark.parametrize("cin,cout,bf16", [(1, 1, False), (3, 16, False), (16, 16, False), (16, 3, True)])
def test_layer_forward_adjoint_wgrad(cin, cout, bf16):
    dims = (6, 4, 6, 8)
    ctx, fat, _ = _ctx_on_torch_stream(dims)
    try:
        w = _rng_c((cout, cin, 9), cin * 100 + cout)
        ins = np.stack([I.gaussian_field(dims, 20 + a) for a in range(cin)])
        wd = torch.from_numpy(w.astype(np.complex64)).cuda()
        xd = torch.from_numpy(ins.astype(np.complex64)).cuda()
        out = torch.empty((cout,) + xd.shape[1:], dtype=torch.complex64, device="cuda")
        H.hisq_net_layer(ctx, wd, xd, out, w_bf16=bf16)
        wq = w
        if bf16:  # the kernel rounds each weight to BF16
            wq = torch.view_as_complex(torch.view_as_real(wd).to(torch.bfloat16).float()).cpu().numpy().astype(np.complex128)
        ref = net_layer(dims, fat, wq.astype(np.complex64).astype(np.complex128), ins.astype(np.complex64).astype(np.complex128))
        assert rel(out.cpu().numpy(), ref) <= 2e-6
        # adjoint: <u, L v> = <L^dag u, v>
        u = np.stack([I.gaussian_field(dims, 60 + b) for b in range(cout)])
        ud = torch.from_numpy(u.astype(np.complex64)).cuda()
        lu = torch.empty_like(xd)
        H.hisq_net_layer(ctx, wd, ud, lu, w_bf16=bf16, adjoint=True)
        lhs = np.vdot(u.astype(np.complex64).astype(np.complex128), out.cpu().numpy().astype(np.complex128))
        rhs = np.vdot(lu.cpu().numpy().astype(np.complex128), ins.astype(np.complex64).astype(np.complex128))
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
        # weight gradient
        gw = torch.empty_like(wd)
        H.hisq_net_wgrad(ctx, xd, ud, gw)
        gref = net_wgrad(dims, fat, ins.astype(np.complex64).astype(np.complex128), u.astype(np.complex64).astype(np.complex128))
        assert rel(gw.cpu().numpy(), gref) <= 1e-5
    finally:
        ctx.close()


def test_autograd_matches_finite_differences():
    dims = (4, 4, 6, 6)
    ctx, fat, _ = _ctx_on_torch_stream(dims)
    try:
        w1 = torch.from_numpy(_rng_c((4, 2, 9), 1).astype(np.complex64)).cuda().requires_grad_(True)
        w2 = torch.from_numpy(_rng_c((2, 4, 9), 2).astype(np.complex64)).cuda().requires_grad_(True)
        x = torch.from_numpy(np.stack([I.gaussian_field(dims, 3), I.gaussian_field(dims, 4)]).astype(np.complex64)).cuda()
        t = torch.from_numpy(np.stack([I.gaussian_field(dims, 5), I.gaussian_field(dims, 6)]).astype(np.complex64)).cuda()

        def loss(a, b):
            out = PTLayer.apply(PTLayer.apply(x, a, ctx, False), b, ctx, False)
            return ((out - t).abs() ** 2).sum()

        L = loss(w1, w2)
        L.backward()
        for (b_, a_, h_) in [(0, 0, 0), (3, 1, 4), (1, 0, 8)]:
            for comp in (1.0, 1j):
                d = 1e-2
                with torch.no_grad():
                    wp = w1.detach().clone()
                    wm = w1.detach().clone()
                    wp[b_, a_, h_] += d * comp
                    wm[b_, a_, h_] -= d * comp
                    fd = (loss(wp, w2.detach()) - loss(wm, w2.detach())).item() / (2 * d)
                g = w1.grad[b_, a_, h_]
                got = g.real.item() if comp == 1.0 else g.imag.item()
                assert abs(got - fd) <= 2e-3 * max(1.0, abs(fd)) + 1e-3 * abs(L.item()) / 1e3
    finally:
        ctx.close()


def test_learned_guess_saves_iterations():
    """Train briefly on (eta, psi) pairs from the deflated solver; a solve that
    starts from deflation + the network's guess needs fewer iterations than the
    deflated-only solve and still meets 1e-10 under the oracle operator."""
    dims = (8, 8, 8, 8)
    m = 0.01
    fat, lng = I.hisq_links(dims, 3, 0.3)
    from oracle.oracle import Oracle

    o = Oracle(dims, fat, lng)
    ctx = H.hisq_create(dims, True, 0, torch.cuda.current_stream().cuda_stream)
    H.hisq_load_links(ctx, fat, lng)
    H.hisq_set_mass(ctx, m)
    try:
        eps, nconv = H.hisq_eigensolve(ctx, H.hisq_default_eig_params(n_ev=24, n_kr=64, tol=1e-6, max_restarts=100))
        prm = H.hisq_default_solve_params(deflate=1, batch=0)
        par = torch.from_numpy((np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)).cuda()
        even = (par == 0).to(torch.complex64)[None, :, None]
        # training pairs: 3 sources per sample, target = solution - deflated guess (even sites)
        def pair(seed0):
            etas = np.stack([I.gaussian_source(dims, 3, seed0 + q) for q in range(3)])
            psi, st, s = H.hisq_solve(ctx, etas, prm)
            tgt = np.stack([project_parity(dims, psi[q], 0) - H.hisq_deflate(ctx, o.prepare_source(m, etas[q]))
                            for q in range(3)])
            return (torch.from_numpy(etas.astype(np.complex64)).cuda(), torch.from_numpy(tgt.astype(np.complex64)).cuda())
        data = [pair(3 * k) for k in range(12)]
        net = GuessNet(ctx, seed=1, bf16=True)
        losses = []
        for epoch in range(60):
            for x, t in data:
                losses.append(net.train_step(x, t, even, lr=3e-3))
        assert np.mean(losses[-12:]) < 0.9 * np.mean(losses[:12])
        # held-out sources
        etas = np.stack([I.gaussian_source(dims, 3, 900 + q) for q in range(3)])
        with torch.no_grad():
            guess = net(torch.from_numpy(etas.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
        psi0, st0, s0 = H.hisq_solve(ctx, etas, prm)
        psi1, st1, s1 = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(deflate=1, batch=0, guess=1), guess=guess)
        assert s0 == H.HISQ_OK and s1 == H.HISQ_OK
        for q in range(3):
            assert o.full_residual(m, psi1[q], etas[q]) <= 1e-10
        assert sum(s["iterations"] for s in st1) < sum(s["iterations"] for s in st0)
    finally:
        ctx.close()

