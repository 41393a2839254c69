"""The allocation-free ranking entry point (dc_rank_hosts_static) against the
regular one (dc_rank_hosts), on two calls in a row with different requests,
through the C-ABI.  It serves callers that cannot allocate device memory
when they rank (memory reserved up front by their own pool, or paths that
cannot afford the device-wide synchronization of cudaFree); its device
temporaries live in the library's static scratch array, shared by all
calls.  Both entry points run the same kernel on the same inputs, so the
outputs must be identical bit for bit (NaN for the same hosts); the score
tolerance of the parity tests (1e-6 relative to the best score) is checked
as well.  Covered: TOPSIS, AHP RATIO and AHP DIFF; a k=32 data center (8,192
hosts, the largest the static array serves) with a request exactly at the
stated limits (1,024 containers, 4,096 links), whose ranked pod has more
peer links than shared memory holds (global peer-link scratch) and more
neighbour hosts than the pod's hash (per-link tables); rejection beyond
each limit.  Needs a GPU."""
import numpy as np
import pytest

from paper_1909_07673_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _same(ds, dc, q, g, host_of):
    f0, a0, b0, c0, n0 = dc.rank_hosts(q, g, host_of)
    f1, a1, b1, c1, n1 = dc.rank_hosts_static(q, g, host_of)
    assert n1 == n0 and n0 > 0
    assert np.array_equal(f1, f0)
    assert np.array_equal(c1, c0)
    assert np.array_equal(a1, a0, equal_nan=True)
    assert np.array_equal(b1, b0, equal_nan=True)
    scale = np.nanmax(b0)
    assert np.all(np.abs(a1[f0].astype(np.float64) - a0[f0]) <= 1e-6 * scale)
    assert np.all(np.abs(b1[f0] - b0[f0]) <= 1e-6 * scale)
    assert np.all(np.isnan(a1[~f0])) and np.all(np.isnan(b1[~f0]))
    return n0


@pytest.mark.parametrize("method,rule", [(W.TOPSIS, W.RATIO), (W.AHP, W.RATIO),
                                         (W.AHP, W.DIFF)])
def test_static_rank_matches_regular_rank(method, rule):
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched as ds

    inst = W.k16(n_requests=6, method=method, pair_rule=rule).instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=torch.cuda.Stream())
    rng = np.random.default_rng(11)
    calls = 0
    for r in (2, 5):  # two calls in a row, different requests and pods
        q = inst.reqs.request(r)
        P = int(q["pod"].max()) + 1
        g = P - 1 if r == 2 else P // 2
        host_of = rng.integers(0, dc.H, len(q["pod"])).astype(np.int32)
        host_of[q["pod"] >= g] = -1
        _same(ds, dc, q, g, host_of)
        calls += 1
    assert calls == 2
    # beyond the stated limit the call is rejected, not truncated
    big = W.gen_request(np.random.default_rng(0), 1100, p_edge=0.0,
                        bw=lambda r, m: r.integers(1, 5, m))
    with pytest.raises(ds.DcError):
        dc.rank_hosts_static(big, 0, np.full(1100, -1, np.int32))
    dc.close()


def _limit_request(rng, n=1024, m=4096, hub_links=300):
    """n singleton containers, m links: the first hub_links join the last
    container with distinct earlier ones, the rest random pairs."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    src[:hub_links] = np.arange(hub_links)
    dst[:hub_links] = n - 1
    a = rng.integers(0, n, m - hub_links)
    b = (a + rng.integers(1, n, m - hub_links)) % n
    src[hub_links:], dst[hub_links:] = a, b
    bw = rng.integers(1, 6, m).astype(np.int32)
    cpu = rng.integers(1, 3, n).astype(np.int32)
    mem = rng.integers(1, 3, n).astype(np.int32)
    return {"cpu_min": cpu, "cpu_max": cpu, "mem_min": mem, "mem_max": mem,
            "pod": np.arange(n, dtype=np.int32), "src": src, "dst": dst,
            "bw_min": bw, "bw_max": bw}


def test_static_rank_at_the_limits():
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched as ds

    rng = np.random.default_rng(23)
    inst = W.batched(n_instances=1, n_requests=1, ks=(32,)).instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=torch.cuda.Stream())
    assert dc.H == 8192
    q = _limit_request(rng)
    host_of = rng.integers(0, dc.H, 1024).astype(np.int32)
    for g in (1023, 700):  # two calls in a row
        ho = host_of.copy()
        ho[g:] = -1
        _same(ds, dc, q, g, ho)
    # one container or one link more than the limits
    q2 = _limit_request(rng, n=1025, m=4096)
    with pytest.raises(ds.DcError):
        dc.rank_hosts_static(q2, 0, np.full(1025, -1, np.int32))
    q3 = _limit_request(rng, n=1024, m=4097)
    with pytest.raises(ds.DcError):
        dc.rank_hosts_static(q3, 0, np.full(1024, -1, np.int32))
    dc.close()
    # a data center larger than the static array serves (k = 34: 9,826 hosts)
    big = ds.DataCenter(34, 32, 64, 10000, 6, ds.TOPSIS, ds.RATIO, (1 / 6,) * 6,
                        stream=torch.cuda.Stream())
    small = _limit_request(rng, n=8, m=8, hub_links=4)
    with pytest.raises(ds.DcError):
        big.rank_hosts_static(small, 0, np.full(8, -1, np.int32))
    big.close()
