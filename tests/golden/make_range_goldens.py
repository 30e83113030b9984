"""Write the oracle's range records for fixed sets of primaries.

The files this script writes hold the expected values of the range-profile
parity tests (``tests/test_gpu_range_parity.py``): one row per primary, the
projected range (or, in a bulk target, the distance from the starting site)
at which the FP64 CPU oracle stopped it (Sec. 2, the range density).  It calls
only ``oracle/`` and reads its inputs from the workload definitions; nothing
here comes from the CUDA path.

    python tests/golden/make_range_goldens.py --workload as10kev_si_300k_tersoff --n 8192
    python tests/golden/make_range_goldens.py --workload ar30kev_ceo2_300k_buck --n 2048
    python tests/golden/make_range_goldens.py --workload kr85mev_uo2_300k_recoil --n 256

Rows are appended chunk by chunk, so an interrupted run resumes where it
stopped, and a larger --n extends a file.  Cloning depths are switched off:
every primary is one unweighted track.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_0810_4737_gb300.workloads import workload  # noqa: E402

SEED = 0


def path_for(name: str) -> str:
    return os.path.join(HERE, f"ranges_{name}.txt")


def read(name: str):
    """(ids, z, status, steps) of a golden file, as lists."""
    ids, z, st, steps = [], [], [], []
    with open(path_for(name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a = line.split()
            ids.append(int(a[0]))
            z.append(float(a[1]))
            st.append(int(a[2]))
            steps.append(int(a[3]))
    return ids, z, st, steps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True)
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--chunk", type=int, default=64)
    a = ap.parse_args()
    w = workload(a.workload, thresholds=[])
    p = O.params(w)
    out = path_for(a.workload)
    header = [f"# oracle range records of {a.workload}, primaries 0..{a.n - 1}, seed {SEED}, no cloning\n",
              f"# written by: python tests/golden/make_range_goldens.py --workload {a.workload} --n {a.n}\n",
              "# id  depth_A  status(1 stopped, 2 backscattered, 3 truncated)  steps\n"]
    done = 0
    if os.path.exists(out):
        done = len(read(a.workload)[0])
        # (more primaries than the file holds: the rows stay, the header names the new count)
        with open(out) as f:
            rows = [line for line in f if not line.startswith("#")]
        with open(out, "w") as f:
            f.writelines(header + rows)
    else:
        with open(out, "w") as f:
            f.writelines(header)
    t0 = time.time()
    while done < a.n:
        m = min(a.chunk, a.n - done)
        r = O.run(p, m, seed=SEED, first_id=done, threads=a.threads)
        rec = r["records"]
        rec = rec[rec["id"].argsort(kind="stable")]
        with open(out, "a") as f:
            for row in rec:
                f.write(f"{int(row['id'])} {float(row['z']):.17g} {int(row['status'])} {int(row['steps'])}\n")
        done += m
        print(f"{a.workload}: {done}/{a.n} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
