"""lra_ca_run_noalloc: the C-A entry point for callers that cannot allocate
device memory (a plug-in inside a host application whose allocator owns the
device, a program handed only pre-placed buffers).  Its scratch is a static
device array inside the library, so the caller passes only inputs and outputs.

Checked through the C ABI against lra_ca_run with a caller workspace, on two
calls in a row with different inputs (the shared scratch keeps the previous
call's contents, which must not leak into the next result).  This file is
collected last on purpose: a run that stops at the first failure has then
already run every other test.
"""
import numpy as np
import pytest

import lra_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402


def _outputs(m, n, k, sweeps, dev):
    return dict(I=torch.empty(k, dtype=torch.int32, device=dev), J=torch.empty(k, dtype=torch.int32, device=dev),
                C=torch.empty(m, k, dtype=torch.float64, device=dev),
                U=torch.empty(k, k, dtype=torch.float64, device=dev),
                R=torch.empty(k, n, dtype=torch.float64, device=dev),
                logvol=torch.empty(2 * sweeps, dtype=torch.float64, device=dev),
                info=torch.empty(8, dtype=torch.int32, device=dev))


def _compare(ref, got):
    for key in ("I", "J", "C", "R", "info"):
        np.testing.assert_array_equal(got[key].cpu().numpy(), ref[key].cpu().numpy())
    U0, U1 = ref["U"].cpu().numpy(), got["U"].cpu().numpy()
    assert np.abs(U1 - U0).max() <= 1e-10 * np.abs(U0).max()
    l0, l1 = ref["logvol"].cpu().numpy(), got["logvol"].cpu().numpy()
    np.testing.assert_allclose(l1, l0, rtol=1e-12, equal_nan=True)


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    import paper_1710_07946_gb300 as lra
    dev = torch.device("cuda:0")
    cases = []
    p1 = li.dense_spiky(1024, r=16, seed=21)
    li.with_arht(p1, 2, 4)
    cases.append((p1, 24, 3, li.initial_rows(1024, 24, 2)))
    p2 = li.laplace_clusters(3000, 2600, seed=5)
    cases.append((p2, 32, 3, li.initial_rows(3000, 32, 8)))
    for p, k, sweeps, I0 in cases:
        prob, mult = to_device(p)
        I0d = torch.from_numpy(I0).to(dev)
        ref = lra.lra_ca_run(prob, I0d, k, sweeps, multiplier=mult)
        got = lra.lra_ca_run_noalloc(prob, I0d, _outputs(p.m, p.n, k, sweeps, dev), k, sweeps, multiplier=mult)
        torch.cuda.synchronize()
        assert int(ref["info"][3]) in (0, 16, 17)
        _compare(ref, got)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_1710_07946_gb300 as lra
    dev = torch.device("cuda:0")
    p = li.laplace_clusters(65536, 65536, seed=1)      # k = 64: strip chunks need global scratch
    prob, _ = to_device(p)
    assert lra.lra_ca_workspace_size(prob, 64, 2) > 256 * 1024
    I0d = torch.from_numpy(li.initial_rows(65536, 64, 0)).to(dev)
    with pytest.raises(lra.LraError) as e:
        lra.lra_ca_run_noalloc(prob, I0d, _outputs(p.m, p.n, 64, 2, dev), 64, 2)
    assert e.value.status == lra.LRA_ERR_WORKSPACE
