"""Failure detection without a GPU fault: the one device-side wait (a CTA
out of work polling the shared clone pool) is given a tiny poll limit so it
runs out while other CTAs still run tracks; the run reports
REED_E_TIMEOUT through the status word, no track is lost (nothing was
donated), and the context stays usable."""
import pytest

from paper_0810_4737_gb300.workloads import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_0810_4737_gb300 import build, reed
    build.build()
    return reed


def test_idle_wait_runs_out_and_reports(R):
    # one cloning depth that no track reaches: the pool is on, nobody donates
    w = workload("b1kev_si_0k_zbl", sigma=0.076, rot=(0.0, 45.0), thresholds=[1e9])
    with R.Reed(w) as ctx:
        with pytest.raises(R.ReedError) as e:
            ctx.run(n_ions=64, seed=1, pool_poll_limit=8)
        assert e.value.code == R.E_TIMEOUT
        st = ctx.stats()
        assert st["tracks"] == 64 and st["clones"] == 0
        # the context stays usable; with the default limit the run is clean
        assert ctx.run(n_ions=64, seed=1, first_id=64) == R.OK
        assert ctx.stats()["tracks"] == 128
