"""Planned shell sums (sf_plan_*): one persistent launch for a batch of irregular vertices, plain
runs and CUDA-graph replays, autotuned tilings.

* with the default tiling a plan's run is bitwise equal to sf_vertex_amplitude over the same range
  (same schedule, same fixed-order reductions), in both precisions;
* graph replays equal plain runs bitwise, and pick up boosters uploaded after the capture;
* an autotuned tiling changes only the summation grouping: within 1e-13 of the default;
* the batched FP64 result equals the oracle on small vertices;
* argument errors are reported, not run.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import vertex as ov
from paper_2107_13952_gb300 import inputs

pytestmark = pytest.mark.gpu

SHELL_END = 729


@pytest.fixture(scope="module")
def batch(lib):
    bt = inputs.random_batch(48, seed=5)
    verts = [sf.vertex(b["two_j"], b["gamma"], b["dl"]) for b in bt]
    t = sf.sf_6j_table(verts)
    bss = [ob.random_boosters(b["two_j"], b["dl"], 500 + i) for i, b in enumerate(bt)]
    for i, bs in enumerate(bss):
        for e in (2, 3, 4, 5):
            sf.sf_boosters_upload(t, i, e, bs[e]["B"])
    return bt, t, bss


@pytest.mark.parametrize("prec", [sf.SF_FP64, sf.SF_MIXED, sf.SF_MIXED_FF, sf.SF_MIXED_TC, sf.SF_MIXED_PX])
def test_plan_run_equals_plain_call(batch, prec):
    bt, t, _ = batch
    plan = sf.Plan(t, prec, 0, SHELL_END)
    outs = plan.run()
    plan.sync()
    ref = sf.sf_vertex_amplitude(t, precision=prec, shell_end=SHELL_END)
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)


def test_graph_replay(batch):
    bt, t, bss = batch
    plan = sf.Plan(t, sf.SF_FP64, 0, SHELL_END)
    first = [o.clone() for o in plan.run()]
    n0 = sf.kernel_launches()
    for _ in range(3):
        for o in plan.outputs:
            o.fill_(float("nan"))
        plan.graph_launch()
        plan.sync()
        for a, b in zip(plan.outputs, first):
            assert torch.equal(a, b)
    assert sf.kernel_launches() - n0 == 3 * 2
    # boosters replaced after the capture: the replay reads the new values
    e, i = 3, 0
    B2 = bss[i][e]["B"] * 2.0
    sf.sf_boosters_upload(t, i, e, B2)
    try:
        plan.graph_launch()
        plan.sync()
        ref = sf.sf_vertex_amplitude(t, shell_end=SHELL_END)
        for a, b in zip(plan.outputs, ref):
            assert torch.equal(a, b)
        assert torch.allclose(plan.outputs[i], 2.0 * first[i], rtol=1e-13, atol=0)
    finally:
        sf.sf_boosters_upload(t, i, e, bss[i][e]["B"])


def test_autotune(batch):
    bt, t, _ = batch
    plan = sf.Plan(t, sf.SF_FP64, 0, SHELL_END)
    base = [o.clone() for o in plan.run()]
    xc, ips, nt, split = plan.autotune(sample_shells=64)
    info = plan.info()
    assert 1 <= xc <= 16 and ips in (4, 8, 16) and nt in (256, 512) and split in (1, 2)
    assert (info["x_chunk"], info["items_per_sm"], info["threads"], info["i3_split"]) == (xc, ips, nt, split)
    assert info["grid"] >= 1 and info["n_items"] >= len(bt)
    outs = plan.graph_launch()
    plan.sync()
    for a, b in zip(outs, base):
        n = float(b.norm())
        assert float((a - b).norm()) <= 1e-13 * max(n, 1e-300)


@pytest.mark.parametrize("tiling", [(1, 1), (4, 32), (16, 256), (6, 8, 512, 1), (3, 8, 256, 1), (5, 4, 256, 2),
                                    (16, 16, 256, 2)])
def test_explicit_tilings(batch, tiling):
    bt, t, _ = batch
    base = sf.sf_vertex_amplitude(t, shell_end=SHELL_END)
    plan = sf.Plan(t, sf.SF_FP64, 0, SHELL_END, tiling=tiling)
    info = plan.info()
    if len(tiling) == 4:
        assert (info["threads"], info["i3_split"]) == tiling[2:]
    outs = plan.run()
    plan.sync()
    for a, b in zip(outs, base):
        assert float((a - b).norm()) <= 1e-13 * max(float(b.norm()), 1e-300)
    for prec in (sf.SF_MIXED, sf.SF_MIXED_FF, sf.SF_MIXED_TC, sf.SF_MIXED_PX):
        mixed = sf.Plan(t, prec, 0, SHELL_END, tiling=tiling)
        outm = mixed.run()
        mixed.sync()
        for a, b in zip(outm, base):
            assert float((a - b).norm()) <= 1e-6 * max(float(b.norm()), 1e-300)


def test_batched_plan_against_oracle(batch):
    bt, t, bss = batch
    plan = sf.Plan(t, sf.SF_FP64, 0, SHELL_END)
    outs = plan.graph_launch()
    plan.sync()
    small = [i for i, b in enumerate(bt) if b["dl"] <= 1][:4]
    assert small
    for i in small:
        ref = ov.vertex_amplitude(bt[i]["two_j"], bt[i]["dl"], bss[i])
        got = outs[i].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_plan_errors(batch):
    bt, t, _ = batch
    with pytest.raises(sf.SfError) as ei:
        sf.Plan(t, sf.SF_FP64, 0, SHELL_END, tiling=(17, 0))
    assert ei.value.code == sf.SF_ERR_ARG
    for bad in ((0, 0, 384, 0), (0, 0, 128, 1), (0, 0, 0, 3), (0, -1), (17, 0), (0, 0, 1024, 0)):
        with pytest.raises(sf.SfError) as ei:
            sf.Plan(t, sf.SF_FP64, 0, SHELL_END, tiling=bad)
        assert ei.value.code == sf.SF_ERR_ARG
    with pytest.raises(sf.SfError) as ei:
        sf.Plan(t, sf.SF_FP64, -1, SHELL_END)
    assert ei.value.code == sf.SF_ERR_ARG
    plan = sf.Plan(t, sf.SF_FP64, 0, SHELL_END)
    with pytest.raises(sf.SfError) as ei:
        plan.autotune(0)
    assert ei.value.code == sf.SF_ERR_ARG
