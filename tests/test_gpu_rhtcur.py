"""CUR LRA with Gaussian sampling (Algorithm algrhtcur) through the C ABI
against the FP64 oracle: the sketch, both selections and the gathered factors
bit-exact, U within 1e-10, counters and statuses equal; dense FP64 / FP32 and
kernel inputs, ragged sizes, and the 8192^2 FP32 benchmark input in full."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402


def run_both(p, k, seed, h=1.01):
    import paper_1710_07946_gb300 as lra
    H = li.gaussian_sketch(p.n, k, seed)
    o = oracle.rhtcur(p, H, h=h)
    prob, _ = to_device(p)
    out = lra.lra_rhtcur_run(prob, torch.from_numpy(H).cuda(), h=h)
    torch.cuda.synchronize()
    g = {key: v.cpu().numpy() for key, v in out.items() if not key.startswith("_")}
    info = g.pop("info")
    assert (int(info[0]), int(info[1]), int(info[2]), int(info[3])) == (o["rank"], o["swaps"], o["loops"], o["status"])
    assert int(info[6]) == k and int(info[7]) == k
    np.testing.assert_array_equal(g["I"], o["I"])
    np.testing.assert_array_equal(g["J"], o["J"])
    np.testing.assert_array_equal(g["C"], o["C"])
    np.testing.assert_array_equal(g["R"], o["R"])
    assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * max(np.abs(o["U"]).max(), 1e-300)
    np.testing.assert_allclose(g["logvol"], o["logvol"], rtol=1e-12, atol=1e-12)
    return o, g


@pytest.mark.parametrize("m,n,k", [(700, 500, 8), (513, 301, 16), (64, 2000, 12), (2001, 33, 20), (300, 280, 64),
                                   (90, 400, 33)])
def test_dense_f64(m, n, k):
    p = li.dense_lowrank(m, n, r=min(m, n, 24), noise=1e-7, seed=m)
    run_both(p, k, m + n)


def test_exact_low_rank_and_dense_f32():
    o, g = run_both(li.factor_gaussian(400, 10, 0.0, seed=2), 10, 3)
    assert o["status"] == 0
    run_both(li.dense_spiky(1024, r=16, seed=3), 24, 4)


def test_laplace_kernel_entries():
    run_both(li.laplace_clusters(1500, 1200, seed=2), 16, 5, h=1.05)


def test_benchmark_input_in_full():
    """8192 x 8192 FP32 rank-32 + 1% spikes, k = 48 (the dense benchmark input)."""
    run_both(li.dense_spiky(8192, r=32, seed=0), 48, 11)
