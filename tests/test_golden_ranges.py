"""The stored oracle range records (tests/golden/ranges_*.txt) are well formed:
primaries 0, 1, ... in order with no gap, no more rows than the header
announces, a valid status per row, finite depths and positive step counts,
and stopped tracks inside the target or just above its surface."""
import os
import re
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_range_goldens as G  # noqa: E402

NAMES = sorted(re.match(r"ranges_(.+)\.txt$", f).group(1)
               for f in os.listdir(os.path.join(HERE, "golden")) if re.match(r"ranges_.+\.txt$", f))


@pytest.mark.parametrize("name", NAMES)
def test_range_golden_is_well_formed(name):
    ids, z, st, steps = (np.asarray(a) for a in G.read(name))
    with open(G.path_for(name)) as f:
        head = f.readline()
    m = re.search(r"primaries 0\.\.(\d+), seed (\d+)", head)
    assert m, head
    assert len(ids) > 0 and len(ids) <= int(m.group(1)) + 1
    assert np.array_equal(ids, np.arange(len(ids)))
    assert set(np.unique(st)) <= {1, 2, 3}
    assert np.all(np.isfinite(z)) and np.all(steps > 0)
    # stopped tracks come to rest in the target or within the interaction
    # range above its surface (an ion on its way out can stop there before
    # it passes the backscatter plane at z = -r_c; a distance from the start
    # site in a bulk target)
    from paper_0810_4737_gb300.workloads import workload
    assert np.all(z[st == 1] > -workload(name)["rc"])
    assert np.mean(z[st == 1] >= 0.0) > 0.99
    assert np.mean(st == 1) > 0.5
