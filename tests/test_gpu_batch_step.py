"""sisph_batch_step: every case of a batch handle advances together and the
call reports the PPE sweeps each case took, equal to the case's own run."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sisph():
    import paper_1908_01762_gb300 as pkg
    pkg.build()
    from paper_1908_01762_gb300 import sisph as mod
    mod.load_library()
    return mod


def test_batch_step_reports_sweeps_per_case(sisph):
    cases = [workloads.taylor_green(24, perturb=0.05, seed=7, tol=1e-4),
             workloads.lid_driven_cavity(20),
             workloads.dam_break_2d(dx=0.05)]
    batch = sisph.Simulation(cases, precision=sisph.MIXED)
    t0 = np.array([s.total_iters for s in batch.stats()])
    rc, its = sisph.sisph_batch_step(batch.h, 4, len(cases))
    t1 = np.array([s.total_iters for s in batch.stats()])
    assert np.array_equal(its, t1 - t0)
    assert np.all(its >= 4 * 2)            # at least min_iter sweeps per step
    for k, c in enumerate(cases):
        solo = sisph.Simulation(c, precision=sisph.MIXED)
        rc1, its1 = sisph.sisph_batch_step(solo.h, 4, 1)
        assert its1[0] == its[k]
        solo.close()
    batch.close()
