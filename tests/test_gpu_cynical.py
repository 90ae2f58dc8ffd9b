"""Cynical CUR (the tests' Tests 3 and Tests 4) on a batch of blocks, one CTA
per block, against the FP64 oracle run block by block: sketch sets, generators
and gathered factors bit-exact, the nucleus within 1e-10."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402


def stacked(nb, n, r, seed):
    """nb independent n x n inputs W_b = G1 G2 + 1e-10 G3 stacked as blocks of one (nb n) x n matrix."""
    Ws = [li.factor_gaussian(n, r, 1e-10, seed + b).W for b in range(nb)]
    W = np.ascontiguousarray(np.concatenate(Ws, axis=0))
    blocks = np.array([[b * n, n, 0, n] for b in range(nb)], dtype=np.int64)
    return li.Problem(li.SRC_DENSE, nb * n, n, W=W), blocks


def sketch_sets(blocks, r, q, seed):
    g = np.random.default_rng(seed)
    K = np.stack([g.choice(int(b[1]), q, replace=False) for b in blocks]).astype(np.int32)
    L = np.stack([g.choice(int(b[3]), q, replace=False) for b in blocks]).astype(np.int32)
    I0s = np.stack([g.choice(q, r, replace=False) for _ in blocks]).astype(np.int32)
    return K, L, I0s


def run_and_check(p, blocks, kind, r, q, sweeps, rank_tol, seed=0):
    import paper_1710_07946_gb300 as lra
    prob, _ = to_device(p)
    K, L, I0s = sketch_sets(blocks, r, q, seed)
    bt = lra.Batch(prob, blocks, r, sweeps, I0s, rank_tol=rank_tol)
    Kd, Ld, Id = (torch.from_numpy(a).cuda() for a in (K, L, I0s))
    lra.lra_cynical_run_batched(bt, kind, q, Kd, Ld, Id)
    torch.cuda.synchronize()
    Kg, Lg = Kd.cpu().numpy(), Ld.cpu().numpy()
    for b, (r0, nr, c0, nc) in enumerate(blocks):
        if p.src == li.SRC_DENSE:
            sub = li.Problem(li.SRC_DENSE, int(nr), int(nc), W=np.ascontiguousarray(p.W[r0:r0 + nr, c0:c0 + nc]))
        else:
            sub = li.Problem(p.src, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc], ell=p.ell)
        o = oracle.cynical(sub, kind, r, q, K[b] if kind == 0 else None, L[b], I0s[b], sweeps=sweeps,
                           rank_tol=rank_tol)
        g = bt.block(b)
        assert g["status"] == o["status"] and g["swaps"] == o["swaps"] and g["loops"] == o["loops"], b
        np.testing.assert_array_equal(Kg[b], o["K"])
        np.testing.assert_array_equal(Lg[b], o["L"])
        np.testing.assert_array_equal(g["I"], o["I"])
        np.testing.assert_array_equal(g["J"], o["J"])
        np.testing.assert_array_equal(g["C"], o["C"])
        np.testing.assert_array_equal(g["R"], o["R"])
        assert g["rank"] == o["rank"]
        assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * np.abs(o["U"]).max()
    return bt


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("r", [8, 16])
def test_factor_gaussian_blocks(kind, r):
    p, blocks = stacked(12, 256, r, 30 + r)
    run_and_check(p, blocks, kind, r, 4 * r, 5, 1e-13, seed=kind)


@pytest.mark.parametrize("kind", [0, 1])
def test_laplace_fmm_blocks(kind):
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=48, seed=6)
    run_and_check(p, blocks, kind, 16, 64, 3, 1e-6, seed=3)


def test_invalid_blocks_are_isolated():
    import paper_1710_07946_gb300 as lra
    p, blocks = stacked(3, 128, 4, 5)
    blocks = blocks.copy()
    blocks[1, 1] = 12                       # fewer rows than the sketch (q = 16)
    prob, _ = to_device(p)
    K, L, I0s = sketch_sets(np.array([[0, 128, 0, 128]] * 3), 4, 16, 1)
    K[2, 3] = K[2, 4]                       # repeated sketch row
    bt = lra.Batch(prob, blocks, 4, 3, I0s)
    lra.lra_cynical_run_batched(bt, 0, 16, *(torch.from_numpy(a).cuda() for a in (K, L, I0s)))
    st = bt.out["info"][:, 3].cpu().numpy()
    assert st[1] == lra.LRA_ERR_INVALID_ARG and st[2] == lra.LRA_ERR_INVALID_ARG and st[0] in (0, 16)
