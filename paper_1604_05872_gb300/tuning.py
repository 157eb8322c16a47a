"""Autotuner and learned cost model for the choice of loop-nest variant and tile.

The paper chooses between sharing elimination and pre-evaluation by operation
count alone (theta, Algorithm 3) and names a better cost model as open work
(Section 8).  Here:

* ``autotune`` times every candidate (variant x tile) of each (form, degree)
  on the GPU through the C ABI and records loop-nest features and the
  measured time per element;
* ``train`` fits the MLP cost model on those records with the library's
  training kernels (``fea_mlp_loss_grad``, ``fea_mlp_adam``) on the device;
* ``choose`` ranks candidates with the inference kernel (``fea_mlp_forward``)
  and installs the pick with ``fea_tune_set``; without a trained model the
  choice stays the paper's flop-count one (Algorithm 3 and the default tile).

Records and weights persist as JSON (``save`` / ``load``).
"""
import json
import math
import time

import numpy as np

import paper_1604_05872_gb300 as fea
from paper_1604_05872_gb300 import inputs

D_IN = 12
HIDDEN = 32


def candidates(form, p, precision=fea.PREC_FP32):
    """(variant, tile) pairs that plan successfully for (form, p)."""
    out = []
    variants = [fea.VARIANT_SE] + ([fea.VARIANT_PRE] if form != fea.NEOHOOKEAN else [])
    for v in variants:
        t0 = fea.plan(form, p, precision=precision, variant=v)["tile"]
        tiles = sorted({max(1, t0 // 4), max(1, t0 // 2), t0, t0 * 2, t0 * 4})
        for t in tiles:
            try:
                fea.plan(form, p, precision=precision, variant=v, tile=t)
            except fea.FeaError:
                continue
            out.append((v, t))
    return out


HBM_GBS = 6753.8           # GB300 copy bandwidth, STREAM-style measurement (a fixed feature scale)
FP32_TFLOPS = 80.5         # 152 SMs x 128 lanes x 2 x 2.07 GHz
FP64_TFLOPS = 1.26         # 152 SMs x 2 lanes x 2 x 2.07 GHz


def features(form, p, variant, tile, precision=fea.PREC_FP32):
    """Loop-nest features of one candidate (fixed scaling, D_IN values): the
    roofline times its operation and byte counts predict, the tile and the
    occupancy its shared memory allows, and what the loop nest is."""
    pl = fea.plan(form, p, precision=precision, variant=variant, tile=tile)
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    fp64 = 30 + (70 * pl["quad_points"] if form == fea.NEOHOOKEAN else 0)
    t_mem = pl["bytes"] / (HBM_GBS * 1e9)
    t_f32 = pl["flops_run"] / (FP32_TFLOPS * 1e12)
    t_f64 = fp64 / (FP64_TFLOPS * 1e12)
    ctas = max(1, min(8, 232448 // max(pl["smem_bytes"], 1)))
    return [ns / 35.0,
            math.log2(pl["quad_points"]) / 9.0,
            1.0 if form in (fea.ELASTICITY, fea.NEOHOOKEAN) else 0.0,
            1.0 if variant == fea.VARIANT_PRE else 0.0,
            math.log2(tile) / 8.0,
            (math.log2(t_mem) + 30.0) / 10.0,
            (math.log2(max(t_f32, 1e-15)) + 30.0) / 10.0,
            (math.log2(t_f64) + 30.0) / 10.0,
            ctas / 8.0,
            math.log2(max(t_mem, t_f32, t_f64) * 1e9) / 10.0,
            1.0 if form == fea.NEOHOOKEAN else 0.0,
            1.0 if form == fea.MASS else 0.0]


def _inputs(form, p, E, seed):
    import torch
    coords, coeffs = inputs.workload(form, p, E, seed=seed)
    c = torch.from_numpy(coords).cuda()
    f = None if form == fea.MASS else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return c, f


def elements_for(form, p, target_bytes=256 << 20, cap=400_000):
    """Batch size of a timing run: about 256 MB of output, at least a few tiles."""
    n = fea.local_dim(form, p)
    return int(max(2048, min(cap, target_bytes // (8 * n * n))))


def measure(form, p, variant, tile, E=None, reps=5, data=None):
    """Seconds per element of one candidate (CUDA events, after warm-up)."""
    import torch
    E = E or elements_for(form, p)
    c, f = data if data is not None else _inputs(form, p, E, seed=7)
    out = fea.empty_out(form, p, c.shape[0])
    for _ in range(2):
        fea.assemble(form, p, c, f, out=out, variant=variant, tile=tile)
    fea.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        fea.assemble(form, p, c, f, out=out, variant=variant, tile=tile)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) * 1e-3 / reps / c.shape[0]


def autotune(configs, precision=fea.PREC_FP32, reps=5, log=None):
    """Time every candidate of each (form, degree); returns the records."""
    records = []
    for form, p in configs:
        E = elements_for(form, p)
        data = _inputs(form, p, E, seed=7)
        for v, t in candidates(form, p, precision):
            s = measure(form, p, v, t, E=E, reps=reps, data=data)
            records.append({"form": form, "p": p, "variant": v, "tile": t, "sec_per_elem": s,
                            "x": features(form, p, v, t, precision)})
            if log:
                log("tune form=%d p=%d variant=%d tile=%d: %.3g s/elem" % (form, p, v, t, s))
    return records


def best_measured(records, form, p):
    rs = [r for r in records if r["form"] == form and r["p"] == p]
    return min(rs, key=lambda r: r["sec_per_elem"]) if rs else None


class Model:
    """The MLP cost model: predicts log2(seconds per element)."""

    def __init__(self, params=None, mean=0.0, std=1.0, hidden=HIDDEN):
        self.params, self.mean, self.std, self.hidden = params, mean, std, hidden

    def predict(self, X):
        import torch
        tX = torch.tensor(np.asarray(X, np.float32), device="cuda")
        tp = torch.tensor(np.asarray(self.params, np.float32), device="cuda")
        z = fea.mlp_forward(tp, tX, self.hidden).cpu().numpy().astype(np.float64)
        return z * self.std + self.mean

    def to_json(self):
        return {"params": [float(x) for x in self.params], "mean": self.mean, "std": self.std, "hidden": self.hidden}

    @staticmethod
    def from_json(d):
        return Model(np.asarray(d["params"]), d["mean"], d["std"], d["hidden"])


def train(records, epochs=3000, lr=1e-2, hidden=HIDDEN, seed=0):
    """Fit the MLP on log2 time per element with the library's GPU kernels."""
    import torch
    X = np.array([r["x"] for r in records], np.float32)
    t = np.log2(np.array([r["sec_per_elem"] for r in records]))
    mean, std = float(t.mean()), float(t.std() + 1e-9)
    y = ((t - mean) / std).astype(np.float32)
    rng = np.random.default_rng(seed)
    n = fea.mlp_num_params(D_IN, hidden)
    p0 = np.concatenate([rng.normal(0, 1 / np.sqrt(D_IN), hidden * D_IN), np.zeros(hidden),
                         rng.normal(0, 1 / np.sqrt(hidden), hidden * hidden), np.zeros(hidden),
                         rng.normal(0, 1 / np.sqrt(hidden), hidden), [0.0]]).astype(np.float32)
    assert p0.size == n
    tp = torch.tensor(p0, device="cuda")
    tX = torch.tensor(X, device="cuda")
    ty = torch.tensor(y, device="cuda")
    m, v = torch.zeros_like(tp), torch.zeros_like(tp)
    grad = torch.empty_like(tp)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(fea.load().fea_mlp_scratch_floats(X.shape[0], hidden), dtype=torch.float32, device="cuda")
    for step in range(1, epochs + 1):
        fea.mlp_loss_grad(tp, tX, ty, hidden, grad=grad, loss=loss, scratch=scratch)
        fea.mlp_adam(tp, grad, m, v, step, lr=lr)
    torch.cuda.synchronize()
    model = Model(tp.cpu().numpy(), mean, std, hidden)
    model.train_loss = float(loss.item())
    return model


MARGIN = 0.15  # log2 units: switch away from the flop-count choice only for a predicted gain above ~11%


def choose(model, form, p, precision=fea.PREC_FP32, install=True):
    """The candidate the model predicts fastest, installed for AUTO calls.  The
    paper's flop-count choice stays unless the model predicts a clear gain."""
    cands = candidates(form, p, precision)
    pred = model.predict([features(form, p, v, t, precision) for v, t in cands])
    fallback = flop_choice(form, p, precision)
    best = int(np.argmin(pred))
    v, t = cands[best]
    if fallback in cands and pred[cands.index(fallback)] - pred[best] < MARGIN:
        v, t = fallback
    if install:
        fea.tune_set(form, p, variant=v, tile=t, precision=precision)
    return v, t


def flop_choice(form, p, precision=fea.PREC_FP32):
    """The paper's choice: Algorithm 3's variant with the default tile."""
    pl = fea.plan_flop(form, p, precision=precision)
    return pl["variant"], pl["tile"]


def save(path, records=None, model=None):
    with open(path, "w") as f:
        json.dump({"records": records or [], "model": model.to_json() if model else None}, f)


def load(path):
    with open(path) as f:
        d = json.load(f)
    return d["records"], (Model.from_json(d["model"]) if d["model"] else None)


def evaluate(configs, log=print, epochs=3000):
    """Autotune, then for every (form, degree) train the MLP on the OTHER
    configurations' records (leave one out) and compare the measured time of
    its pick with the flop-count choice and with the best measured candidate."""
    t0 = time.time()
    records = autotune(configs, log=None)
    rows = []
    for form, p in configs:
        train_recs = [r for r in records if (r["form"], r["p"]) != (form, p)]
        model = train(train_recs, epochs=epochs)
        v_m, t_m = choose(model, form, p, install=False)
        v_f, t_f = flop_choice(form, p)
        rec = {(r["variant"], r["tile"]): r["sec_per_elem"] for r in records if (r["form"], r["p"]) == (form, p)}
        best = best_measured(records, form, p)
        rows.append({"form": form, "p": p, "mlp": [v_m, t_m, rec[(v_m, t_m)]],
                     "flop": [v_f, t_f, rec.get((v_f, t_f), float("nan"))],
                     "best": [best["variant"], best["tile"], best["sec_per_elem"]]})
        log(json.dumps(rows[-1]))
    full = train(records, epochs=epochs)
    return records, full, rows, time.time() - t0


if __name__ == "__main__":
    import sys
    fea.load()
    cfgs = [(f, p) for f in range(4) for p in range(1, 5)]
    records, model, rows, dt = evaluate(cfgs)
    out = sys.argv[1] if len(sys.argv) > 1 else "tuning.json"
    save(out, records, model)
    gm = np.exp(np.mean([np.log(r["flop"][2] / r["mlp"][2]) for r in rows]))
    print(json.dumps({"configs": len(rows), "geomean_speedup_mlp_over_flop_choice": gm, "seconds": dt}))
