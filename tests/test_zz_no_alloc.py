"""The allocation-free ranking entry point (dc_rank_hosts_static) against the
regular one (dc_rank_hosts), on two calls in a row with different requests,
through the C-ABI.  It serves callers that cannot allocate device memory
when they rank (memory reserved up front by their own pool, or paths that
cannot afford the device-wide synchronization of cudaFree); its device
temporaries live in the library's static scratch array, shared by all
calls.  Needs a GPU."""
import numpy as np
import pytest

from paper_1909_07673_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", [W.TOPSIS, W.AHP])
def test_static_rank_matches_regular_rank(method):
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched as ds

    inst = W.k16(n_requests=6, method=method).instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=torch.cuda.Stream())
    rng = np.random.default_rng(11)
    calls = 0
    for r in (2, 5):  # two calls in a row, different requests and pods
        q = inst.reqs.request(r)
        P = int(q["pod"].max()) + 1
        g = P - 1 if r == 2 else P // 2
        host_of = rng.integers(0, dc.H, len(q["pod"])).astype(np.int32)
        host_of[q["pod"] >= g] = -1
        f0, a0, b0, c0, n0 = dc.rank_hosts(q, g, host_of)
        f1, a1, b1, c1, n1 = dc.rank_hosts_static(q, g, host_of)
        assert n1 == n0 and n0 > 0
        assert np.array_equal(f1, f0)
        assert np.array_equal(c1[f0], c0[f0])
        # the tolerance of the score parity tests: 1e-6 relative to the best score
        scale = np.nanmax(b0)
        assert np.all(np.abs(a1[f0].astype(np.float64) - a0[f0]) <= 1e-6 * scale)
        assert np.all(np.abs(b1[f0] - b0[f0]) <= 1e-6 * scale)
        assert np.all(np.isnan(a1[~f0])) and np.all(np.isnan(b1[~f0]))
        calls += 1
    assert calls == 2
    # beyond the stated limit the call is rejected, not truncated
    big = W.gen_request(np.random.default_rng(0), 1100, p_edge=0.0, bw=lambda r, m: r.integers(1, 5, m))
    with pytest.raises(ds.DcError):
        dc.rank_hosts_static(big, 0, np.full(1100, -1, np.int32))
    dc.close()
