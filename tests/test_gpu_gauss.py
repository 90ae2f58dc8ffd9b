"""Differentiable CUR apply on Gaussian-kernel blocks (fixed pivots): forward,
hand-written backward (x, sampled entries, length scale) and the autograd
Function, against the FP64 oracle and finite differences."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ELL = 0.3


def blocks(nb=3, size=1024, k=32, nrhs=16, seed=0):
    X, Y, ell = li.gaussian_blocks(nblk=nb, size=size, ell=ELL, seed=seed)
    I = np.zeros((nb, k), np.int32); J = np.zeros((nb, k), np.int32)
    for b in range(nb):
        p = li.Problem(li.SRC_GAUSSIAN, size, size, X=X[b], Y=Y[b], ell=ELL)
        o = oracle.ca_run(p, k, 3, li.initial_rows(size, k, 10 + b))
        I[b], J[b] = o["I"], o["J"]
    g = np.random.default_rng(seed + 7)
    x = g.standard_normal((nb, size, nrhs)).astype(np.float32)
    dy = g.standard_normal((nb, size, nrhs)).astype(np.float32)
    return X, Y, I, J, x, dy


def dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def assert_close(g, o, tol, what):
    """Element-wise |g - o| <= tol * max|o| (one block's output; the max-norm of the
    oracle's values scales the tolerance, so one wrong entry of ordinary size fails)."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    assert g.shape == o.shape, (what, g.shape, o.shape)
    scale = np.abs(o).max()
    err = np.abs(g - o).max()
    assert err <= tol * scale, f"{what}: max |g - o| = {err:.3e} = {err / scale:.3e} of max|o| > {tol:.1e}"


# Tolerances (element-wise, relative to each output's max-norm).  The device
# evaluates C and R in FP32: an entry exp(-a) with a = |x - y|^2 / (2 l^2) <= 50 on
# these blocks carries a relative error of about a * 2^-24 <= 3e-6, and R x sums
# 1024 such FP32 products.  y = C (U (R x)) and dx = R^T (U^T (C^T dy)) map the
# error of R x back through C U, which undoes U's amplification: TOL_Y.  The
# entry gradients dC = dy t2^T, dR = s2 x^T and dG = -s2 t2^T see t2 = U (R x) or
# s2 = U^T (C^T dy) directly, and U amplifies the FP32 error of R x by up to
# cond(G) ~ 5e3 in some directions: TOL_ENTRY.  dl is one sum over all entries.
TOL_Y = 2e-5
TOL_ENTRY = 5e-4
TOL_DL = 1e-4


@pytest.mark.parametrize("nrhs", [1, 16, 64])
def test_forward_backward_match_oracle(nrhs):
    import paper_1710_07946_gb300 as lra
    X, Y, I, J, x, dy = blocks(nrhs=nrhs)
    Xd, Yd, Id, Jd, xd, dyd = dev(X, Y, I, J, x, dy)
    y, ctx = lra.lra_gauss_cur_forward(Xd, Yd, Id, Jd, ELL, xd)
    g = lra.lra_gauss_cur_backward(Xd, Yd, Id, Jd, ELL, xd, dyd, ctx, entry_grads=True)
    torch.cuda.synchronize()
    for b in range(len(X)):
        yo = oracle.gauss_cur_apply(X[b], Y[b], I[b], J[b], ELL, x[b].astype(np.float64))[0]
        assert_close(y[b].cpu().numpy(), yo, TOL_Y, f"y[{b}]")
        bo = oracle.gauss_cur_backward(X[b], Y[b], I[b], J[b], ELL, x[b].astype(np.float64),
                                       dy[b].astype(np.float64))
        assert_close(g["dx"][b].cpu().numpy(), bo["dx"], TOL_Y, f"dx[{b}]")
        assert abs(g["dell"][b].item() - bo["dell"]) <= TOL_DL * abs(bo["dell"])
        for key in ("dC", "dR", "dG"):
            assert_close(g[key][b].cpu().numpy(), bo[key], TOL_ENTRY, f"{key}[{b}]")


def test_autograd_function_and_finite_differences():
    import paper_1710_07946_gb300 as lra
    X, Y, I, J, x, dy = blocks(nb=2, nrhs=4, seed=3)
    Xd, Yd, Id, Jd, xd, dyd = dev(X, Y, I, J, x, dy)
    xd.requires_grad_(True)
    ell = torch.tensor(ELL, dtype=torch.float64, device="cuda", requires_grad=True)
    y = lra.gauss_cur_apply(xd, ell, Xd, Yd, Id, Jd)
    (y * dyd).sum().backward()
    dl_o = sum(oracle.gauss_cur_backward(X[b], Y[b], I[b], J[b], ELL, x[b].astype(np.float64),
                                         dy[b].astype(np.float64))["dell"] for b in range(2))
    assert abs(ell.grad.item() - dl_o) <= TOL_DL * abs(dl_o)
    dx_o = oracle.gauss_cur_backward(X[0], Y[0], I[0], J[0], ELL, x[0].astype(np.float64),
                                     dy[0].astype(np.float64))["dx"]
    assert_close(xd.grad[0].cpu().numpy(), dx_o, TOL_Y, "dx (autograd)")
    # central difference of the GPU forward in the length scale
    h = 1e-4
    with torch.no_grad():
        Lp = (lra.gauss_cur_apply(xd, ELL + h, Xd, Yd, Id, Jd).double() * dyd.double()).sum().item()
        Lm = (lra.gauss_cur_apply(xd, ELL - h, Xd, Yd, Id, Jd).double() * dyd.double()).sum().item()
    assert abs((Lp - Lm) / (2 * h) - ell.grad.item()) <= 2e-3 * abs(ell.grad.item())


def test_register_tiled_loops_equal_the_scalar_ones_bit_for_bit():
    """With nrhs a multiple of 4 the apply takes four right-hand sides per thread
    (vector loads, the same per-output fmaf chains), so column c of y and of dx
    equals, bit for bit, the nrhs = 1 run on column c alone.  Odd sizes: 999
    points per block (a ragged last tile of 39) and rank 31; also against the
    oracle."""
    import paper_1710_07946_gb300 as lra
    X, Y, I, J, x, dy = blocks(nb=2, size=999, k=31, nrhs=8, seed=5)
    Xd, Yd, Id, Jd, xd, dyd = dev(X, Y, I, J, x, dy)
    y8, ctx8 = lra.lra_gauss_cur_forward(Xd, Yd, Id, Jd, ELL, xd)
    g8 = lra.lra_gauss_cur_backward(Xd, Yd, Id, Jd, ELL, xd, dyd, ctx8, entry_grads=True)
    torch.cuda.synchronize()
    for c in range(8):
        xc, dyc = xd[:, :, c:c + 1].contiguous(), dyd[:, :, c:c + 1].contiguous()
        y1, ctx1 = lra.lra_gauss_cur_forward(Xd, Yd, Id, Jd, ELL, xc)
        g1 = lra.lra_gauss_cur_backward(Xd, Yd, Id, Jd, ELL, xc, dyc, ctx1)
        torch.cuda.synchronize()
        assert torch.equal(y8[:, :, c], y1[:, :, 0]), c
        assert torch.equal(g8["dx"][:, :, c], g1["dx"][:, :, 0]), c
    for b in range(2):
        yo = oracle.gauss_cur_apply(X[b], Y[b], I[b], J[b], ELL, x[b].astype(np.float64))[0]
        assert_close(y8[b].cpu().numpy(), yo, TOL_Y, f"y[{b}]")
        bo = oracle.gauss_cur_backward(X[b], Y[b], I[b], J[b], ELL, x[b].astype(np.float64),
                                       dy[b].astype(np.float64))
        assert_close(g8["dx"][b].cpu().numpy(), bo["dx"], TOL_Y, f"dx[{b}]")
        assert abs(g8["dell"][b].item() - bo["dell"]) <= TOL_DL * abs(bo["dell"])
        for key in ("dC", "dR", "dG"):
            assert_close(g8[key][b].cpu().numpy(), bo[key], TOL_ENTRY, f"{key}[{b}]")
