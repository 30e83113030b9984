"""Host-side helpers of bench.py: the oracle-parity block (unpaired and
paired against the stored oracle ranges) and the merging of two contexts'
counters.  CPU only."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


REC = np.dtype([("id", "<u8"), ("primary", "<u8"), ("z", "<f8"), ("t", "<f8"), ("steps", "<i8"),
                ("level", "<i4"), ("status", "<i4")])


def test_oracle_parity_pairs_the_same_primaries():
    from paper_0810_4737_gb300.workloads import workload
    b = _bench()
    w = workload("as10kev_si_300k_tersoff")
    G = b._golden()
    ids, z, st, _ = (np.asarray(a) for a in G.read(w["name"]))
    n = 2048
    rng = np.random.default_rng(3)
    perm = rng.permutation(n)              # records arrive in completion order
    rec = np.zeros(n, dtype=REC)
    rec["id"] = perm
    rec["status"] = st[perm]
    rec["z"] = 1.01 * z[perm] + rng.normal(0.0, 0.5, n)
    out = b.oracle_parity(w, {"mixed": rec})
    p = out["mixed"]["paired"]
    assert p["primaries"] == int(np.sum(st[:n] == 1))
    # a 1 % longer range on every primary: the paired mean sees it to a
    # fraction of its error bar, and the pairs stay correlated
    assert abs(p["mean_rel_err"] - 0.01) < 3 * p["mean_rel_se"] + 1e-4
    assert p["mean_rel_se"] < 0.001 and p["correlation"] > 0.99
    # the unpaired figures compare the distributions
    assert abs(out["mixed"]["mean_rel_err"] - 0.01) < 3 * out["mixed"]["mean_rel_se"]


def test_merge_stats_adds_counters():
    b = _bench()
    a = {"steps": 10, "pair_evals": 5, "phase_cycles": [1, 2], "threads_per_track": 256, "kernel_ms": 3.0,
         "w_stopped": 1.5}
    c = {"steps": 7, "pair_evals": 1, "phase_cycles": [3, 4], "threads_per_track": 256, "kernel_ms": 9.0,
         "w_stopped": 0.5}
    m = b._merge_stats(a, c)
    assert m["steps"] == 17 and m["pair_evals"] == 6 and m["phase_cycles"] == [4, 6]
    assert m["threads_per_track"] == 256 and m["kernel_ms"] == 3.0 and m["w_stopped"] == 2.0
