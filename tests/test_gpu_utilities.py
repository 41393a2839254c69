"""Parity of the device utilities (Eqs. 1-2) and fragmentation with the
oracle: per-container and per-link utilities bit-exact, sums in the same
order bit-exact, active server / link counts exact.  Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched

    dcsched.lib()
    return dcsched


@pytest.fixture(scope="module")
def stream():
    import torch

    return torch.cuda.Stream()


def _check(ds, dc, inst, n_req):
    odc = O.OracleDC.from_instance(inst)
    sc = se = 0.0
    nc = ne = 0
    for r in range(n_req):
        q = inst.reqs.request(r)
        ref = odc.schedule(q)
        ouc, oue = O.utilities(q, ref)
        uc, ue = dc.utilities(r)
        assert np.array_equal(uc, ouc), r
        assert np.array_equal(ue, oue), r
        if ref["status"] == O.ACCEPTED:
            s_c = 0.0
            for x in ouc:
                s_c += x
            s_e = 0.0
            for x in oue:
                s_e += x
            sc += s_c
            se += s_e
            nc += len(ouc)
            ne += len(oue)
    summ = dc.utility_summary()
    assert summ == {"sum_u_container": sc, "n_containers": nc, "sum_u_link": se, "n_links": ne}
    assert dc.fragmentation() == odc.fragmentation()
    return odc


@pytest.mark.parametrize("k,method", [(8, W.TOPSIS), (16, W.AHP)])
def test_utilities_interval_requests(ds, stream, k, method):
    inst = W.k16(seed=11, k=k, n_requests=30, method=method, intervals=True).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    _check(ds, dc, inst, inst.reqs.n)


def test_utilities_cluster_shape_and_releases(ds, stream):
    """Same on a data center scheduled by a 4-block cluster, then after
    releasing every accepted request (fragmentation back to the pre-load)."""
    inst = W.k16(seed=12, k=16, n_requests=20, intervals=True).instances[0]
    key = (inst.k, inst.n_criteria, inst.method, inst.pair_rule)
    ds.set_launch(*key, 256, 4)
    try:
        dc = ds.load_instance(inst, stream=stream)
        ds.schedule([dc])
        odc = _check(ds, dc, inst, inst.reqs.n)
        for r in range(inst.reqs.n):
            if dc.status(r)[0] == ds.ACCEPTED:
                dc.release(r)
                q = inst.reqs.request(r)
        ds.schedule([dc])
        pre_h = int(np.sum((inst.pre_cpu > 0) | (inst.pre_mem > 0)))
        pre_l = int(np.sum(inst.pre_link > 0))
        a, b, fs, fl = dc.fragmentation()
        assert (a, b) == (pre_h, pre_l)
        assert fs == pre_h / inst.hosts and fl == pre_l / (3 * inst.hosts)
    finally:
        ds.set_launch(*key, 0, 1)


def test_utilities_pending_request_is_busy(ds, stream):
    inst = W.small().instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=stream)
    dc.submit(inst.reqs.request(0))
    with pytest.raises(ds.DcError):
        dc.utilities(0)
    ds.schedule([dc])
    uc, ue = dc.utilities(0)
    assert len(uc) == len(inst.reqs.request(0)["pod"])
