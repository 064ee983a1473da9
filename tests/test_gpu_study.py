"""The preconditioner / Laplacian / step-size study (paper_2303_14495_gb300.study)
on a small synthetic image: every configuration reaches the target DICE, and
the step-size tables keep the paper's shape (small step sizes need at least
as many outer steps as large ones, the largest no fewer than the infinite
one's, and the iterates converge to u*)."""

import pytest

pytestmark = pytest.mark.gpu


def test_study_shape(cuda_lib):
    from paper_2303_14495_gb300 import study
    res = study.study(size=64, max_outer=1500, verbose=False)
    runs = res["runs"]
    assert all(r["steps"] is not None for r in runs), runs
    for pc in ("perturbed", "Richardson"):
        t5 = {r["step"]: r["steps"] for r in runs if r["table"] == "5" and r["precond"] == pc}
        ks = [0.01, 0.05, 0.1, 1.0, 5.0]
        for a, b in zip(ks, ks[1:]):
            assert t5[a] >= t5[b], (pc, t5)
        assert t5[5.0] >= t5["inf"], (pc, t5)
    assert res["rate"]["loglog_slope"] < 0
