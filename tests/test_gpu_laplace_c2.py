"""The Laplace entry-oracle workload between two unit cubes whose centres are 3
apart (65536 targets, 65536 sources, kernel 1/|x - y| evaluated on demand) at
ranks 16, 32 and 64, with FP64 entries and with FP32 entries (FP64 pivots and
nucleus either way): the single-LRA CUDA path against the oracle on the full
problem.  Index sets bit-exact, C and R identical, U within 1e-10.  For FP32
entries the CUR's error against the FP64 matrix is sampled and bounded."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import assert_parity, gpu_ca  # noqa: E402

N = 65536


@pytest.fixture(scope="module")
def points():
    return li.laplace_clusters(N, N, seed=1)


@pytest.mark.parametrize("entries", ["f64", "f32"])
@pytest.mark.parametrize("k", [16, 32, 64])
def test_full_size_parity(points, k, entries):
    p = li.Problem(li.SRC_LAPLACE, N, N, X=points.X, Y=points.Y, entries=entries)
    I0 = li.initial_rows(N, k, 0)
    o = oracle.ca_run(p, k, 3, I0)
    g = gpu_ca(p, k, 3, I0)
    assert_parity(o, g)


@pytest.mark.parametrize("k", [32, 64])
def test_f32_entries_error_against_fp64_matrix(points, k):
    """Sampled relative error of the FP32-entry CUR against the FP64 entries
    (512 x 512 positions), next to the FP64-entry CUR's; both <= 1e-6 at k >= 32.
    The nucleus truncates at 1e-8: at k = 64 the full-rank core's conditioning
    would amplify the entries' rounding to ~1e-6 (rank 45 of 64 gives 1e-8)."""
    p64 = li.Problem(li.SRC_LAPLACE, N, N, X=points.X, Y=points.Y)
    p32 = li.Problem(li.SRC_LAPLACE, N, N, X=points.X, Y=points.Y, entries="f32")
    I0 = li.initial_rows(N, k, 0)
    Q, S = li.sample_positions(N, N, 512, 512, 3)
    errs = {}
    for name, p in (("f64", p64), ("f32", p32)):
        g = gpu_ca(p, k, 3, I0, rank_tol=1e-8)
        st = oracle.residual_sample(p64, g["C"], g["U"], g["R"], Q, S)
        errs[name] = st[4]
    assert errs["f64"] < 1e-6 and errs["f32"] < 1e-6, errs
    assert errs["f32"] <= 1.5 * errs["f64"] + 1.25 * 2.0 ** -23, errs
