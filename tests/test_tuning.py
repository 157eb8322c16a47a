"""Autotuner and learned cost model: host logic on the CPU, tuning, training,
installation and the measured gain on the GPU."""
import math

import numpy as np
import pytest

import paper_1604_05872_gb300 as fea
from paper_1604_05872_gb300 import build as fbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    fbuild.build()
    return fea.load()


def test_candidates_and_features():
    from paper_1604_05872_gb300 import tuning
    for form in range(4):
        for p in range(1, 5):
            cands = tuning.candidates(form, p)
            assert cands, (form, p)
            variants = {v for v, _ in cands}
            assert fea.VARIANT_SE in variants
            assert (fea.VARIANT_PRE in variants) == (form != fea.NEOHOOKEAN)
            for v, t in cands:
                x = tuning.features(form, p, v, t)
                assert len(x) == tuning.D_IN and all(math.isfinite(z) for z in x)
                assert max(abs(z) for z in x) <= 4


def test_tune_set_changes_auto_plan_and_clear_restores():
    base = fea.plan(fea.HELMHOLTZ, 2)
    fea.tune_set(fea.HELMHOLTZ, 2, variant=fea.VARIANT_SE, tile=8)
    try:
        pl = fea.plan(fea.HELMHOLTZ, 2)
        assert pl["variant"] == fea.VARIANT_SE and pl["tile"] == 8
    finally:
        fea.tune_clear()
    again = fea.plan(fea.HELMHOLTZ, 2)
    assert again["variant"] == base["variant"] and again["tile"] == base["tile"]
    with pytest.raises(fea.FeaError):
        fea.tune_set(fea.NEOHOOKEAN, 2, variant=fea.VARIANT_PRE)


def test_over_budget_candidate_is_in_the_set():
    """Elasticity P4 in FP64: Algorithm 3 drops pre-evaluation because its
    tables exceed T_H (Constraint 2), but the tuner still offers it."""
    from paper_1604_05872_gb300 import tuning
    mask, _ = fea.algorithm3(fea.ELASTICITY, 4, fea.PREC_FP64)
    assert mask == 0
    assert tuning.flop_choice(fea.ELASTICITY, 4, fea.PREC_FP64)[0] == fea.VARIANT_SE
    assert tuning.over_budget(fea.ELASTICITY, 4, fea.VARIANT_PRE, fea.PREC_FP64) > 1.4
    cands = tuning.candidates(fea.ELASTICITY, 4, fea.PREC_FP64)
    assert any(v == fea.VARIANT_PRE for v, _ in cands)
    x_pre = tuning.features(fea.ELASTICITY, 4, fea.VARIANT_PRE, 1, fea.PREC_FP64)
    x_se = tuning.features(fea.ELASTICITY, 4, fea.VARIANT_SE, 1, fea.PREC_FP64)
    assert x_pre[-1] > 0.5 and x_se[-1] == 0.0 and x_pre[-3] == 1.0
    # in FP32 the same tables fit T_H and Algorithm 3 pre-evaluates
    assert tuning.over_budget(fea.ELASTICITY, 4, fea.VARIANT_PRE, fea.PREC_FP32) < 1.0
    assert tuning.flop_choice(fea.ELASTICITY, 4)[0] == fea.VARIANT_PRE


GAIN_CONFIGS = [(0, 2), (0, 3), (1, 2), (1, 3), (1, 4), (2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3),
                (1, 4, fea.PREC_FP64), (2, 3, fea.PREC_FP64), (2, 4, fea.PREC_FP64)]


@pytest.mark.gpu
def test_tuned_choice_is_correct_and_mlp_gains(fea, orc, tmp_path, capsys):
    import torch
    from paper_1604_05872_gb300 import inputs, tuning
    records = tuning.autotune(GAIN_CONFIGS, reps=3)
    assert len(records) >= 3 * len(GAIN_CONFIGS)
    # the learned choice, trained without the configuration it is asked about,
    # against the paper's flop-count choice, measured
    rows = tuning.leave_one_out(records, GAIN_CONFIGS, epochs=800)
    gains = np.array([r["gain"] for r in rows])
    regrets = np.array([r["regret"] for r in rows])
    with capsys.disabled():
        print()
        for r in rows:
            print(tuning.format_row(r))
        print("geomean gain of the learned choice over the flop-count choice: %.4f" % np.exp(np.log(gains).mean()))
    assert np.exp(np.mean(np.log(gains))) >= 1.0
    assert np.exp(np.mean(np.log(regrets))) < 1.3
    # the paper's over-budget case: pre-evaluation with tables over T_H beats
    # Algorithm 3's sharing elimination by a wide margin
    pre_best = min(r["sec_per_elem"] for r in records
                   if tuning.record_config(r) == (2, 4, fea.PREC_FP64) and r["variant"] == fea.VARIANT_PRE)
    row = [r for r in rows if (r["form"], r["p"], r["prec"]) == (2, 4, fea.PREC_FP64)][0]
    assert row["flop"][0] == fea.VARIANT_SE and row["flop"][2] > 2 * pre_best
    # install a model's choice and check the assembled result
    model = tuning.train(records, epochs=800)
    tuning.save(str(tmp_path / "t.json"), records, model)
    recs2, model2 = tuning.load(str(tmp_path / "t.json"))
    assert len(recs2) == len(records) and len(model2.members) == len(model.members)
    assert all(np.allclose(a, b) for a, b in zip(model2.members, model.members))
    try:
        v, t = tuning.choose(model2, 3, 2)
        pl = fea.plan(3, 2)
        assert (pl["variant"], pl["tile"]) == (v, t)
        coords, coeffs = inputs.workload(3, 2, 64, seed=3)
        c = torch.from_numpy(coords).cuda()
        f = torch.from_numpy(inputs.coeff_array(3, 2, coeffs)).cuda()
        out = fea.assemble(3, 2, c, f)
        fea.sync()
        ref = orc.assemble(3, 2, coords, coeffs)
        assert orc.rel_frobenius(out.cpu().numpy(), ref).max() <= 1e-5
    finally:
        fea.tune_clear()


@pytest.mark.gpu
def test_shipped_model_loads_and_chooses(fea):
    import os
    from paper_1604_05872_gb300 import tuning
    path = os.path.join(os.path.dirname(tuning.__file__), "data", "tuning_gb300.json")
    records, model = tuning.load(path)
    assert model is not None and len(model.members) == tuning.MEMBERS
    assert {tuning.record_config(r)[2] for r in records} == {fea.PREC_FP32, fea.PREC_FP64}
    try:
        for f, p, prec in tuning.ALL_CONFIGS:
            v, t = tuning.choose(model, f, p, prec)
            assert (v, t) in tuning.candidates(f, p, prec)
    finally:
        fea.tune_clear()
