"""The Sec. 4.2 study set-ups (2D half-wheel, 3D simply supported beam) on
the GPU against the oracle, at sizes the oracle finishes in seconds: the
AARMR run and the MGCG-only reference run of the study runner take the
oracle's branches with its compliances, and the runner's Eq. 35 / 36
figures are formed from them."""

import pytest

from oracle import aarmr
from workloads import study_beam, study_halfwheel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["halfwheel", "beam"])
def test_study_runs_match_the_oracle(case):
    from paper_2205_00385_gb300.driver import TopoSolver
    from paper_2205_00385_gb300.studies import run_pair
    p = (study_halfwheel(64, 32, 0.05, n_iter=30) if case == "halfwheel"
         else study_beam(24, 8, 16, 0.05, n_iter=30))
    for q, mode in ((p, "aarmr"), (p.with_(n_on=10 ** 9), "mgcg")):
        ref = aarmr.run(q, mode=mode)
        s = TopoSolver(q, precision="fp64")
        try:
            hist = s.run(q.n_iter)
        finally:
            s.close()
        assert [h.branch for h in hist] == [h.branch for h in ref.history], mode
        for hg, hr in zip(hist, ref.history):
            assert abs(hg.compliance - hr.compliance) <= 1e-6 * hr.compliance, (mode, hg.k)
    r = run_pair(p)
    assert r["speedup"] > 0.0 and r["mgcg"]["mgcg_evaluations"] == p.n_iter
    assert r["aarmr"]["mgcg_evaluations"] + r["aarmr"]["carm_accepted"] == p.n_iter
    assert abs(r["diff_percent"]) < 5.0
