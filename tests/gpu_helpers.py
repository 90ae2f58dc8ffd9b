"""Shared helpers of the GPU tests: move a seeded input to the device and run
the library through its C ABI binding; compare with the oracle."""
import numpy as np
import torch

import lra_inputs as li


def to_device(p: li.Problem):
    import paper_1710_07946_gb300 as lra
    dev = torch.device("cuda:0")
    if p.src == li.SRC_DENSE:
        prob = lra.Problem.dense(torch.from_numpy(np.ascontiguousarray(p.W)).to(dev))
    else:
        kind = "laplace" if p.src == li.SRC_LAPLACE else "gaussian"
        prob = lra.Problem.kernel(kind, torch.from_numpy(p.X).to(dev), torch.from_numpy(p.Y).to(dev), p.ell,
                                  entries=p.entries)
    mult = None
    side = "left" if p.mside else "right"
    order = p.m if p.mside else p.n
    if p.mkind == li.MULT_ARHT:
        mult = lra.lra_precondition("arht", order, p.depth, p.perm, p.dsign, side=side)
    elif p.mkind == li.MULT_SPARSE:
        mult = lra.lra_precondition("sparse", order, p.nnz, p.srow, p.ssign, side=side)
    elif p.mkind == li.MULT_BIDIAG:
        mult = lra.lra_precondition("bidiag", order, p.depth, p.perm, p.dsign, side=side)
    elif p.mkind == li.MULT_ARFT:
        mult = lra.lra_precondition_fourier(p.n, p.depth, p.perm, p.dcplx)
    return prob, mult


def gpu_ca(p: li.Problem, k, sweeps, I0, **kw):
    import paper_1710_07946_gb300 as lra
    prob, mult = to_device(p)
    I0d = torch.from_numpy(np.ascontiguousarray(I0, dtype=np.int32)).cuda()
    out = lra.lra_ca_run(prob, I0d, k, sweeps, multiplier=mult, **kw)
    torch.cuda.synchronize()
    res = {key: v.cpu().numpy() for key, v in out.items() if not key.startswith("_")}
    info = res.pop("info")
    res.update(rank=int(info[0]), swaps=int(info[1]), loops=int(info[2]), status=int(info[3]),
               fp32_steps=int(info[4]), fp64_steps=int(info[5]))
    return res


def assert_parity(o, g, *, factor_rtol=1e-10, exact_factors=False):
    """Index sets bit-exact; C and R (gathered entries) identical; U within
    factor_rtol relative (max-norm); counters and status equal."""
    assert g["status"] == o["status"], (g["status"], o["status"])
    assert g["loops"] == o["loops"] and g["swaps"] == o["swaps"], (g["loops"], o["loops"], g["swaps"], o["swaps"])
    np.testing.assert_array_equal(g["I"], o["I"])
    np.testing.assert_array_equal(g["J"], o["J"])
    np.testing.assert_array_equal(g["C"], o["C"])
    np.testing.assert_array_equal(g["R"], o["R"])
    assert g["rank"] == o["rank"]
    scale = max(np.abs(o["U"]).max(), 1e-300)
    if exact_factors:
        np.testing.assert_array_equal(g["U"], o["U"])
    else:
        assert np.abs(g["U"] - o["U"]).max() <= factor_rtol * scale
    lo, lg = o["logvol"], g["logvol"]
    assert np.array_equal(np.isnan(lo), np.isnan(lg))
    fin = np.isfinite(lo)
    np.testing.assert_allclose(lg[fin], lo[fin], rtol=1e-12, atol=1e-12)
