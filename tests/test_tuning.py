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


@pytest.mark.gpu
def test_tuned_choice_is_correct_and_mlp_gains(fea, orc, tmp_path):
    import torch
    from paper_1604_05872_gb300 import inputs, tuning
    configs = [(0, 2), (0, 3), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)]
    records = tuning.autotune(configs, reps=3)
    assert len(records) >= 4 * len(configs)
    gains, regrets = [], []
    for form, p in configs:
        model = tuning.train([r for r in records if (r["form"], r["p"]) != (form, p)], epochs=800)
        v_m, t_m = tuning.choose(model, form, p, install=False)
        v_f, t_f = tuning.flop_choice(form, p)
        times = {(r["variant"], r["tile"]): r["sec_per_elem"] for r in records if (r["form"], r["p"]) == (form, p)}
        gains.append(times[(v_f, t_f)] / times[(v_m, t_m)])
        regrets.append(times[(v_m, t_m)] / min(times.values()))
    # the learned choice, trained without the configuration it is asked about,
    # is never far from the best measured candidate and not worse than the
    # flop-count choice on (geometric) average
    assert np.exp(np.mean(np.log(regrets))) < 1.3
    assert np.exp(np.mean(np.log(gains))) > 0.95
    # install a model's choice and check the assembled result
    model = tuning.train(records, epochs=800)
    tuning.save(str(tmp_path / "t.json"), records, model)
    recs2, model2 = tuning.load(str(tmp_path / "t.json"))
    assert len(recs2) == len(records) and np.allclose(model2.params, model.params)
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
