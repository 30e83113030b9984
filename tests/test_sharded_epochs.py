"""Host logic of the multi-process adaptive run (no GPU).

The driver in paper_0810_4737_gb300.sharded is run over an engine backed by
the oracle:
* the epoch plan and the rank blocks partition the primaries exactly;
* one rank reproduces the oracle's own adaptive run bit for bit (histogram
  and the depths of every epoch);
* two gloo ranks (separate processes, 127.0.0.1) give the same summed
  histogram and the same depths as one rank: the only exchange is the sum of
  the range histograms before each enhanced epoch, exact in FP64.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_0810_4737_gb300 import sharded
from paper_0810_4737_gb300.workloads import workload

N_IONS, EPOCH, N_INIT = 72, 20, 12
DEPTHS0 = [10.0, 25.0, 40.0, 55.0]


def _w():
    return workload("b1kev_si_0k_zbl", sigma=0.076, rot=(0.0, 45.0), thresholds=DEPTHS0, n_bins=100, bin_w=5.0)


class OracleShard:
    """Engine whose tracks are run by the oracle (tests only)."""

    def __init__(self, O, w, seed):
        self.O, self.seed = O, seed
        self.p = O.params(w)
        self.nthr = len(w["thresholds"])
        self.nb, self.bw = int(w["n_bins"]), float(w["bin_w"])
        self.hist = np.zeros(self.nb + 3)
        self.thr = np.array(w["thresholds"], dtype=np.float64)

    def local_profile(self):
        return self.hist.copy()

    def update_depths(self, total):
        try:
            self.thr = self.O.update_thresholds(np.asarray(total), self.bw, self.nthr)
        except ValueError:   # empty histogram: keep the depths
            pass

    def set_depths(self, d):
        self.thr = np.array(d, dtype=np.float64)[:self.nthr]

    def depths(self):
        return self.thr.copy()

    def run(self, first, count, enhanced):
        if count <= 0:
            return
        self.p.nthr = self.nthr if enhanced else 0
        for k in range(self.nthr):
            self.p.thr[k] = self.thr[k]
        r = self.O.run(self.p, count, self.seed, first_id=first, threads=2, records=False)
        self.hist += np.concatenate([r["hist"], [r["under"], r["over"], r["back"]]])


def test_plan_and_blocks():
    for n, e, i in [(72, 20, 12), (5, 10, 0), (100, 7, 200), (0, 3, 2), (33, 33, 1)]:
        plan = sharded.epoch_plan(n, e, i)
        ids = [k for ep in plan for k in range(ep.first, ep.first + ep.count)]
        assert ids == list(range(n))
        assert all(ep.count <= e for ep in plan if ep.enhanced)
        assert [ep.update for ep in plan if ep.enhanced][:1] in ([], [min(i, n) > 0])
        for world in (1, 2, 3, 8):
            for ep in plan:
                got = []
                for r in range(world):
                    lo, c = sharded.rank_block(ep.first, ep.count, r, world)
                    assert c >= 0
                    got += list(range(lo, lo + c))
                assert got == list(range(ep.first, ep.first + ep.count))
    with pytest.raises(ValueError):
        sharded.epoch_plan(10, 0, 0)


def test_one_rank_matches_oracle_adaptive(O):
    w = _w()
    eng = OracleShard(O, w, seed=4)
    hist = sharded.run_adaptive(eng, N_IONS, EPOCH, N_INIT, DEPTHS0)
    ref = O.run_adaptive(O.params(w), N_IONS, N_INIT, EPOCH, 4, threads=2)
    assert np.array_equal(eng.hist[:w["n_bins"]], ref["hist"])
    assert np.array_equal(eng.hist[w["n_bins"]:], [ref["under"], ref["over"], ref["back"]])
    assert np.array_equal(np.array(hist), ref["thresholds"])
    assert len(hist) == ref["epochs"]


def test_one_rank_calls_a_given_allreduce(O):
    # a single-rank process group still sums through its collective (the
    # NCCL path on one GPU); the result is the no-collective run's
    w = _w()
    ref = OracleShard(O, w, seed=4)
    h_ref = sharded.run_adaptive(ref, N_IONS, EPOCH, N_INIT, DEPTHS0)
    calls = []

    def allreduce(a):
        calls.append(1)
        return np.array(a, dtype=np.float64)
    eng = OracleShard(O, w, seed=4)
    hist = sharded.run_adaptive(eng, N_IONS, EPOCH, N_INIT, DEPTHS0, allreduce=allreduce)
    assert len(calls) == len(hist) and np.array_equal(np.array(hist), np.array(h_ref))
    with pytest.raises(ValueError):
        sharded.run_adaptive(OracleShard(O, w, seed=4), N_IONS, EPOCH, N_INIT, DEPTHS0, rank=0, world=2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def allreduce(a):
            t = torch.from_numpy(np.array(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()
        eng = OracleShard(O, _w(), seed=4)
        hist = sharded.run_adaptive(eng, N_IONS, EPOCH, N_INIT, DEPTHS0, rank=rank, world=world,
                                    allreduce=allreduce)
        total = allreduce(eng.local_profile())
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), total=total, depths=np.array(hist),
                 local=eng.local_profile())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one(O, tmp_path):
    w = _w()
    one = OracleShard(O, w, seed=4)
    h1 = sharded.run_adaptive(one, N_IONS, EPOCH, N_INIT, DEPTHS0)
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [np.load(os.path.join(tmp_path, "rank%d.npz" % r)) for r in range(2)]
    for r in res:
        assert np.array_equal(r["total"], one.hist)
        assert np.array_equal(r["depths"], np.array(h1))
    # the ranks did different work
    assert not np.array_equal(res[0]["local"], res[1]["local"])
    assert np.array_equal(res[0]["local"] + res[1]["local"], one.hist)
