"""Parity of the best-fit / worst-fit comparators run by the fused kernel with
the oracle: placements, allocations, paths, pod scores and the state
bit-exact, one block and clusters.  Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W
from parity_util import check_instance

pytestmark = pytest.mark.gpu

FITS = [W.BF, W.WF]


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


@pytest.mark.parametrize("method", FITS)
def test_fit_small(ds, stream, method):
    inst = W.small(method=method).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="small fit %d" % method)


@pytest.mark.parametrize("method", FITS)
@pytest.mark.parametrize("k", [8, 16])
def test_fit_preloaded(ds, stream, method, k):
    inst = W.k16(k=k, n_requests=60, method=method).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="k%d fit %d" % (k, method))


@pytest.mark.parametrize("method", FITS)
def test_fit_pods_intervals(ds, stream, method):
    rng = np.random.Generator(np.random.PCG64(90))
    reqs = [W.gen_request(rng, int(rng.integers(2, 12)), p_edge=0.5,
                          bw=lambda r, m: r.integers(10, 400, m), max_pod=3, intervals=True,
                          intra_pod_links=True) for _ in range(40)]
    inst = W.Instance(4, 16, 32, 1000, 6, method, W.RATIO, W.WEIGHTS[6]["flat"],
                      None, None, None, W.pack_requests(reqs))
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="pods fit %d" % method)


@pytest.mark.parametrize("method", FITS)
@pytest.mark.parametrize("k,block,ncta", [(16, 256, 4), (32, 512, 8)])
def test_fit_cluster(ds, stream, method, k, block, ncta):
    if k == 32:
        inst = W.batched(n_instances=1, n_requests=6, ks=(32,), size_hi=48, method=method).instances[0]
    else:
        inst = W.k16(k=k, n_requests=30, method=method).instances[0]
    key = (inst.k, inst.n_criteria, inst.method, inst.pair_rule)
    ds.set_launch(*key, block, ncta)
    try:
        dc = ds.load_instance(inst, stream=stream)
        ds.schedule([dc])
        check_instance(dc, inst, where="cluster fit %d k%d" % (method, k))
    finally:
        ds.set_launch(*key, 0, 1)


@pytest.mark.parametrize("method", FITS)
def test_fit_rank_hosts(ds, stream, method):
    """Per-host viability (capacity only), criteria and the exact key."""
    inst = W.k16(k=8, n_requests=10, method=method).instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=stream)
    odc = O.OracleDC.from_instance(inst)
    q = inst.reqs.request(3)
    ho = np.full(len(q["pod"]), -1, np.int32)
    feas, s32, s64, crit, nv = dc.rank_hosts(q, 0, ho)
    of, oc, osc = odc.rank_pod(q, 0, ho)
    assert np.array_equal(feas, of) and nv == int(of.sum())
    assert np.array_equal(crit, oc.astype(np.int32))
    assert np.array_equal(s64[of], osc[of])
