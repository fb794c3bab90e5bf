"""The autotuner: timed plan choices per step shape, cached per device.

hotrg_autotune / HOTRG_OPT_AUTOTUNE time the plans of a step that compute the same
contraction (closing direction; tensor-core pipeline with the same products) and keep the
fastest. These tests check that the cache is filled once per step shape and then used (step
records and counters), that a tuned run gives the planner's ln Z/V to the mixed-mode bar
(a different closing direction changes only the rounding order), that two runs on the same
cached plans are bit-identical, and that an explicit hotrg_autotune call leaves the run
where it was.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(sched, prec, autotune, beta=1 / 6.65):
    from paper_1911_12954_gb300 import HOTRG
    g = HOTRG(batch=1, dcut_max=6, precision=prec, schedule=sched, autotune=autotune)
    g.init_tensor(beta, 0.0)
    lnz = []
    for mu, dc in sched:
        g.step(mu, dc)
        lnz.append(float(g.lnZ()[0]))
    return g, lnz


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3", "fp64"])
def test_autotuned_runs_use_the_cache_and_agree(prec):
    # 8 steps at D_cut = 6: three transient shapes, then (6,6,6,6) along t, x, y, z, t (the
    # last repeats step 4's shape); 7 distinct step shapes
    sched = [(i % 4, 6) for i in range(8)]
    _, ref = _run(sched, prec, autotune=False)
    g1, lnz1 = _run(sched, prec, autotune=True)
    st1 = g1.tune_stats()
    assert st1["timed"] + st1["hits"] == 8 and st1["timed"] <= 7
    opts = {"fp16x3": (0, 3), "tf32x3": (0, 1), "fp64": (-1,)}[prec]
    for k in range(1, 9):
        info = g1.step_info(k)
        assert info["closing"] in {0, 1, 2, 3} - {info["mu"]}
        assert info["gemm_option"] in opts
    g2, lnz2 = _run(sched, prec, autotune=True)
    st2 = g2.tune_stats()
    assert st2 == {"timed": 0, "hits": 8}                    # every plan from the cache
    assert all(g2.step_info(k)["tuned"] for k in range(1, 9))
    assert lnz2 == lnz1                                      # same plans: bit-identical
    tol = 1e-10 if prec == "fp64" else 1e-6
    assert np.allclose(lnz1, ref, rtol=0, atol=tol)


def test_explicit_autotune_does_not_advance_the_run():
    from paper_1911_12954_gb300 import HOTRG
    sched = [(i % 4, 5) for i in range(5)]
    g = HOTRG(batch=1, dcut_max=5, precision="fp16x3", schedule=sched)
    g.init_tensor(1 / 6.7, 0.0)
    for mu, dc in sched[:4]:
        g.step(mu, dc)
    before = (g.lnZ()[0], g.state(), g.tensor().copy())
    g.autotune(0, 5)
    after = (g.lnZ()[0], g.state(), g.tensor())
    assert before[0] == after[0] and before[1] == after[1] and np.array_equal(before[2], after[2])
    assert g.tune_stats() == {"timed": 1, "hits": 0}
    from paper_1911_12954_gb300 import OPT_AUTOTUNE
    g.set_option(OPT_AUTOTUNE, 1)
    g.step(0, 5)
    assert g.tune_stats() == {"timed": 1, "hits": 1} and g.step_info(5)["tuned"]
