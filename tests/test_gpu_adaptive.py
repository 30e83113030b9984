"""Adaptive cloning depths (re-estimated between epochs) and the stop rule,
through the C ABI.

* the device update reproduces the oracle's d_k = S^-1(2^-k) on the same
  histogram (the unenhanced ions' histogram is deterministic);
* an adaptive run (captured as one CUDA graph) conserves weight exactly and
  its weighted range distribution and final depths agree with the oracle's
  adaptive run within statistics;
* the stop rule stops handing out primaries once enough tracks finished and
  completes every lineage it started.
"""
import numpy as np
import pytest
from scipy import stats

from paper_0810_4737_gb300.workloads import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_0810_4737_gb300 import build, reed
    build.build()
    return reed


W = dict(sigma=0.076, rot=(0.0, 45.0), energy=2000.0, thresholds=[30.0, 60.0, 90.0, 120.0, 150.0, 180.0],
         n_bins=200, bin_w=2.0)


def test_first_update_matches_oracle(R, O):
    w = workload("b1kev_si_0k_zbl", **W)
    with R.Reed(w) as ctx:
        ctx.run(n_ions=450, seed=4, adaptive=True, n_initial=50, epoch_size=200)
        hist_rows = ctx.thresholds()
    assert hist_rows.shape[0] == 2
    # the same 50 unenhanced primaries alone
    with R.Reed(dict(w, thresholds=[])) as ctx0:
        ctx0.run(n_ions=50, seed=4)
        bins, extra = ctx0.profile()
    full = np.concatenate([bins, extra])
    expect = O.update_thresholds(full, w["bin_w"], 6)
    got = hist_rows[0, :6]
    fin = np.isfinite(expect)
    assert np.array_equal(np.isfinite(got), fin)
    np.testing.assert_allclose(got[fin], expect[fin], rtol=1e-12)


def test_adaptive_run_matches_oracle_statistically(R, O):
    w = workload("b1kev_si_0k_zbl", **W)
    n = 2050
    with R.Reed(w) as ctx:
        ctx.run(n_ions=n, seed=6, adaptive=True, n_initial=50, epoch_size=500)
        rec = ctx.records()
        st = ctx.stats()
        th = ctx.thresholds()
    assert th.shape[0] == 4
    wts = np.ldexp(1.0, -rec["level"].astype(int))
    assert np.sum(wts) == n and st["primaries"] == n
    ref = O.run_adaptive(O.params(w), n, 50, 500, seed=6, threads=16)
    assert ref["epochs"] == 4
    tg, to = th[-1, :6], ref["thresholds"][-1]
    both = np.isfinite(tg) & np.isfinite(to)
    assert both.sum() >= 4
    assert np.max(np.abs(tg[both] / to[both] - 1)) < 0.15
    # weighted depth distributions (binned on the common histogram grid)
    sg = rec["status"] == 1
    zg, wg = rec["z"][sg], wts[sg]
    # oracle profile as a weighted histogram
    ho = ref["hist"]
    hg = np.histogram(zg, bins=w["n_bins"], range=(0, w["n_bins"] * w["bin_w"]), weights=wg)[0]
    cg, co = np.cumsum(hg) / hg.sum(), np.cumsum(ho) / ho.sum()
    D = np.max(np.abs(cg - co))
    neff = wg.sum() ** 2 / np.sum(wg ** 2)
    assert stats.kstwo.sf(D, int(neff / 2)) > 0.01, D


def test_stop_rule_completes_started_lineages(R):
    w = workload("b1kev_si_0k_zbl", **W)
    with R.Reed(w) as ctx:
        ctx.run(n_ions=5000, seed=2, target_tracks=300)
        st = ctx.stats()
        rec = ctx.records()
    assert st["tracks"] >= 300
    assert st["primaries"] < 5000
    # every primary handed out was followed with all its clones
    wts = np.ldexp(1.0, -rec["level"].astype(int))
    assert np.sum(wts) == st["primaries"]


def test_sharded_driver_matches_adaptive_run(R):
    # the multi-process driver on one rank: depths re-estimated through
    # reed_update_thresholds between separate runs equal the in-graph epochs
    from paper_0810_4737_gb300 import sharded
    w = workload("b1kev_si_0k_zbl", **W)
    n, epoch, ninit = 1250, 400, 50
    with R.Reed(w) as ctx:
        ctx.run(n_ions=n, seed=9, adaptive=True, n_initial=ninit, epoch_size=epoch)
        ref_bins, ref_extra = ctx.profile()
        ref_th = ctx.thresholds()
        ref_st = ctx.stats()
    with R.Reed(w) as ctx:
        eng = sharded.ReedShard(ctx, seed=9)
        hist = sharded.run_adaptive(eng, n, epoch, ninit, w["thresholds"])
        bins, extra = ctx.profile()
        st = ctx.stats()
    assert np.array_equal(np.array(hist), ref_th[:, :6])
    assert np.array_equal(bins, ref_bins) and np.array_equal(extra, ref_extra)
    assert st["tracks"] == ref_st["tracks"] and st["steps"] == ref_st["steps"]


def test_sharded_driver_over_nccl(R):
    """The multi-process driver with its histogram sum done by a NCCL
    all_reduce on the device (one rank on this GPU): the same depths and
    profile as the in-graph adaptive run."""
    import os
    import socket
    import torch
    import torch.distributed as dist
    from paper_0810_4737_gb300 import sharded
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    w = workload("b1kev_si_0k_zbl", **W)
    n, epoch, ninit = 1250, 400, 50
    with R.Reed(w) as ctx:
        ctx.run(n_ions=n, seed=9, adaptive=True, n_initial=ninit, epoch_size=epoch)
        ref_bins, ref_extra = ctx.profile()
        ref_th = ctx.thresholds()
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, world_size=1, rank=0)
    calls = []

    def allreduce(t):
        assert t.is_cuda and t.dtype == torch.float64
        dist.all_reduce(t)
        calls.append(1)
        return t
    try:
        with R.Reed(w) as ctx:
            eng = sharded.ReedShard(ctx, seed=9)
            hist = sharded.run_adaptive(eng, n, epoch, ninit, w["thresholds"], rank=0, world=1,
                                        allreduce=allreduce)
            bins, extra = ctx.profile()
    finally:
        dist.destroy_process_group()
    assert len(calls) == len(hist) > 1
    assert np.array_equal(np.array(hist), ref_th[:, :6])
    assert np.array_equal(bins, ref_bins) and np.array_equal(extra, ref_extra)
