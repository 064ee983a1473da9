"""The preconditioner / Laplacian / step-size study (paper_2303_14495_gb300.study)
on the 256 x 256 synthetic image: every configuration reaches a stable DICE score,
the smallest step size needs more outer steps than the infinite one (the
shape of Table 5), and the iterates converge to u*."""

import pytest

pytestmark = pytest.mark.gpu


def test_study_shape(cuda_lib):
    from paper_2303_14495_gb300 import study
    res = study.study(size=256, max_outer=3000, verbose=False, noise=0.15)
    runs = res["runs"]
    assert all(r["steps"] is not None for r in runs), runs
    for pc in ("perturbed", "Richardson"):
        t5 = {r["step"]: r["steps"] for r in runs if r["table"] == "5" and r["precond"] == pc}
        assert t5[0.01] > t5["inf"], (pc, t5)
    assert res["rate"]["loglog_slope"] < 0
