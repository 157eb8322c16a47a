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

The candidate set is not limited by the memory threshold T_H of Constraint 2
(Section 4.1): a pre-evaluated variant whose tables exceed T_H is still timed
(the kernels read the tables through the L2 cache, one column per thread into
registers, so going over T_H costs cache misses, not correctness), and the
features tell the model by how much the tables exceed T_H.  Section 7 reports
exactly this case on the CPU: Algorithm 3 drops pre-evaluation of the
elasticity form because its tables exceed T_H by about 40%, although it would
have won by its five times lower operation count; Section 8 asks for a cost
model that weighs the two.  On the GPU the same case arises in FP64 at P4 (the
elasticity tables take 344 KB against a 227 KB T_H, for 4.3 times fewer
operations).

Records and weights persist as JSON (``save`` / ``load``).
"""
import json
import math
import time

import numpy as np

import paper_1604_05872_gb300 as fea
from paper_1604_05872_gb300 import inputs

D_IN = 15
HIDDEN = 32
MEMBERS = 5          # ensemble size: independently initialised networks, predictions averaged
T_H_DEFAULT = 232448  # the planner's memory threshold without an explicit budget (bytes)


def candidates(form, p, precision=fea.PREC_FP32):
    """(variant, tile) pairs that plan successfully for (form, p), whether or
    not Algorithm 3 would admit the variant's tables under T_H."""
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


def table_bytes(form, p, precision=fea.PREC_FP32):
    """Bytes of the pre-evaluated tables of the whole form (Constraint 2's
    memory, counted as Algorithm 3 counts it); 0 when nothing is pre-evaluable."""
    word = 8 if precision == fea.PREC_FP64 else 4
    return sum(max(w, 0) for _, pre, w in fea.theta(form, p) if pre >= 0) * word


def over_budget(form, p, variant, precision=fea.PREC_FP32, t_h=T_H_DEFAULT):
    """Ratio of the pre-evaluated tables to T_H (0 for sharing elimination)."""
    return table_bytes(form, p, precision) / t_h if variant == fea.VARIANT_PRE else 0.0


def features(form, p, variant, tile, precision=fea.PREC_FP32):
    """Loop-nest features of one candidate (fixed scaling, D_IN values): the
    roofline times its operation and byte counts predict, the tile and the
    occupancy its shared memory allows, what the loop nest is, its precision
    and how far its pre-evaluated tables exceed T_H."""
    pl = fea.plan(form, p, precision=precision, variant=variant, tile=tile)
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    fp64_path = precision == fea.PREC_FP64
    fp64 = 30 + (70 * pl["quad_points"] if form == fea.NEOHOOKEAN else 0)
    f32 = pl["flops_run"]
    if fp64_path:  # the whole contraction runs on the FP64 pipe
        fp64, f32 = fp64 + f32, 0
    t_mem = pl["bytes"] / (HBM_GBS * 1e9)
    t_f32 = f32 / (FP32_TFLOPS * 1e12)
    t_f64 = fp64 / (FP64_TFLOPS * 1e12)
    ctas = max(1, min(8, 232448 // max(pl["smem_bytes"], 1)))
    tb = table_bytes(form, p, precision) if variant == fea.VARIANT_PRE else 0
    over = over_budget(form, p, variant, precision)
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
            1.0 if form == fea.MASS else 0.0,
            1.0 if fp64_path else 0.0,
            math.log2(1.0 + tb / 1024.0) / 10.0,
            math.log2(over) if over > 1.0 else 0.0]


def _inputs(form, p, E, seed):
    import torch
    coords, coeffs = inputs.workload(form, p, E, seed=seed)
    c = torch.from_numpy(coords).cuda()
    f = None if form == fea.MASS else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return c, f


def elements_for(form, p, target_bytes=256 << 20, cap=400_000, precision=fea.PREC_FP32):
    """Batch size of a timing run: about 256 MB of output (64 MB on the slower
    FP64 path), at least a few tiles."""
    n = fea.local_dim(form, p)
    if precision == fea.PREC_FP64:
        target_bytes //= 4
    return int(max(2048, min(cap, target_bytes // (8 * n * n))))


def measure(form, p, variant, tile, E=None, reps=5, data=None, precision=fea.PREC_FP32):
    """Seconds per element of one candidate (CUDA events, after warm-up)."""
    import torch
    E = E or elements_for(form, p, precision=precision)
    c, f = data if data is not None else _inputs(form, p, E, seed=7)
    out = fea.empty_out(form, p, c.shape[0])
    for _ in range(2):
        fea.assemble(form, p, c, f, out=out, variant=variant, tile=tile, precision=precision)
    fea.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        fea.assemble(form, p, c, f, out=out, variant=variant, tile=tile, precision=precision)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) * 1e-3 / reps / c.shape[0]


def _config(c):
    """(form, degree, precision) of a configuration given as (form, degree)
    (FP32) or (form, degree, precision)."""
    return (c[0], c[1], c[2] if len(c) > 2 else fea.PREC_FP32)


def record_config(r):
    return r["form"], r["p"], r.get("prec", fea.PREC_FP32)


def autotune(configs, reps=5, log=None):
    """Time every candidate of each configuration; returns the records."""
    records = []
    for cfg in configs:
        form, p, prec = _config(cfg)
        E = elements_for(form, p, precision=prec)
        data = _inputs(form, p, E, seed=7)
        for v, t in candidates(form, p, prec):
            s = measure(form, p, v, t, E=E, reps=reps, data=data, precision=prec)
            records.append({"form": form, "p": p, "prec": prec, "variant": v, "tile": t, "sec_per_elem": s,
                            "over_budget": over_budget(form, p, v, prec), "x": features(form, p, v, t, prec)})
            if log:
                log("tune form=%d p=%d prec=%d variant=%d tile=%d: %.3g s/elem" % (form, p, prec, v, t, s))
    return records


def best_measured(records, form, p, precision=fea.PREC_FP32):
    rs = [r for r in records if record_config(r) == (form, p, precision)]
    return min(rs, key=lambda r: r["sec_per_elem"]) if rs else None


class Model:
    """The MLP cost model: predicts log2(seconds per element) as the mean of
    an ensemble of independently initialised networks of the same shape."""

    def __init__(self, members=None, mean=0.0, std=1.0, hidden=HIDDEN):
        self.members = [np.asarray(m, np.float32) for m in (members or [])]
        self.mean, self.std, self.hidden = mean, std, hidden

    def predict_members(self, X):
        """[members, rows] predictions of log2 seconds per element."""
        import torch
        tX = torch.tensor(np.asarray(X, np.float32), device="cuda")
        z = []
        for m in self.members:
            tp = torch.tensor(m, device="cuda")
            z.append(fea.mlp_forward(tp, tX, self.hidden).cpu().numpy().astype(np.float64))
        return np.array(z) * self.std + self.mean

    def predict(self, X):
        return self.predict_members(X).mean(axis=0)

    def to_json(self):
        return {"members": [[float(x) for x in m] for m in self.members], "mean": self.mean, "std": self.std,
                "hidden": self.hidden, "d_in": D_IN}

    @staticmethod
    def from_json(d):
        if d.get("d_in", D_IN) != D_IN:
            raise ValueError("weights were trained on %d features, this model has %d" % (d.get("d_in"), D_IN))
        return Model(d["members"], d["mean"], d["std"], d["hidden"])


def _train_one(tX, ty, epochs, lr, hidden, seed):
    import torch
    rng = np.random.default_rng(seed)
    n = fea.mlp_num_params(D_IN, hidden)
    p0 = np.concatenate([rng.normal(0, 1 / np.sqrt(D_IN), hidden * D_IN), np.zeros(hidden),
                         rng.normal(0, 1 / np.sqrt(hidden), hidden * hidden), np.zeros(hidden),
                         rng.normal(0, 1 / np.sqrt(hidden), hidden), [0.0]]).astype(np.float32)
    assert p0.size == n
    tp = torch.tensor(p0, device="cuda")
    m, v = torch.zeros_like(tp), torch.zeros_like(tp)
    grad = torch.empty_like(tp)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(fea.load().fea_mlp_scratch_floats(tX.shape[0], hidden), dtype=torch.float32, device="cuda")
    for step in range(1, epochs + 1):
        fea.mlp_loss_grad(tp, tX, ty, hidden, grad=grad, loss=loss, scratch=scratch)
        fea.mlp_adam(tp, grad, m, v, step, lr=lr)
    torch.cuda.synchronize()
    return tp.cpu().numpy(), float(loss.item())


def train(records, epochs=3000, lr=1e-2, hidden=HIDDEN, seed=0, members=MEMBERS):
    """Fit the MLP ensemble on log2 time per element with the library's GPU
    kernels (features recomputed from the plan, so old records stay usable)."""
    import torch
    X = np.array([features(r["form"], r["p"], r["variant"], r["tile"], r.get("prec", fea.PREC_FP32))
                  for r in records], np.float32)
    t = np.log2(np.array([r["sec_per_elem"] for r in records]))
    mean, std = float(t.mean()), float(t.std() + 1e-9)
    y = ((t - mean) / std).astype(np.float32)
    tX = torch.tensor(X, device="cuda")
    ty = torch.tensor(y, device="cuda")
    params, losses = [], []
    for k in range(members):
        p, l = _train_one(tX, ty, epochs, lr, hidden, seed + k)
        params.append(p)
        losses.append(l)
    model = Model(params, mean, std, hidden)
    model.train_loss = float(np.mean(losses))
    return model


MARGIN = 0.05  # log2 units: every ensemble member must predict a gain above ~3.5%


def choose(model, form, p, precision=fea.PREC_FP32, install=True):
    """The candidate the ensemble predicts fastest on average, installed for
    AUTO calls.  The paper's flop-count choice stays unless every member of the
    ensemble predicts the pick faster than it by MARGIN: where the networks
    disagree, the model does not know enough to overrule the operation count."""
    cands = candidates(form, p, precision)
    pred = model.predict_members([features(form, p, v, t, precision) for v, t in cands])
    fallback = flop_choice(form, p, precision)
    best = int(np.argmin(pred.mean(axis=0)))
    v, t = cands[best]
    if fallback in cands and (pred[:, cands.index(fallback)] - pred[:, best]).min() < MARGIN:
        v, t = fallback
    if install:
        fea.tune_set(form, p, variant=v, tile=t, precision=precision)
    return v, t


def flop_choice(form, p, precision=fea.PREC_FP32):
    """The paper's choice: Algorithm 3's variant (pre-evaluated tables within
    T_H) with the default tile."""
    pl = fea.plan_flop(form, p, precision=precision)
    return pl["variant"], pl["tile"]


def save(path, records=None, model=None):
    with open(path, "w") as f:
        json.dump({"records": records or [], "model": model.to_json() if model else None}, f)


def load(path):
    with open(path) as f:
        d = json.load(f)
    return d["records"], (Model.from_json(d["model"]) if d["model"] else None)


def leave_one_out(records, configs, epochs=800, log=None):
    """For every configuration, train on the OTHER configurations' records and
    compare the measured time of the model's pick with the flop-count choice
    and with the best measured candidate.  Rows: config, picks, times, gain."""
    rows = []
    for cfg in configs:
        form, p, prec = _config(cfg)
        model = train([r for r in records if record_config(r) != (form, p, prec)], epochs=epochs)
        v_m, t_m = choose(model, form, p, prec, install=False)
        v_f, t_f = flop_choice(form, p, prec)
        rec = {(r["variant"], r["tile"]): r["sec_per_elem"] for r in records if record_config(r) == (form, p, prec)}
        best = best_measured(records, form, p, prec)
        row = {"form": form, "p": p, "prec": prec, "mlp": [v_m, t_m, rec[(v_m, t_m)]],
               "flop": [v_f, t_f, rec[(v_f, t_f)]], "best": [best["variant"], best["tile"], best["sec_per_elem"]],
               "gain": rec[(v_f, t_f)] / rec[(v_m, t_m)], "regret": rec[(v_m, t_m)] / best["sec_per_elem"]}
        rows.append(row)
        if log:
            log(format_row(row))
    return rows


def format_row(row):
    name = {fea.VARIANT_SE: "se", fea.VARIANT_PRE: "pre"}
    pick = lambda c: "%s/%d %.3g ns" % (name[c[0]], c[1], c[2] * 1e9)
    return "form=%d p=%d %s  flop-count %-18s learned %-18s best %-18s gain %.3f" % (
        row["form"], row["p"], "fp64" if row["prec"] == fea.PREC_FP64 else "fp32", pick(row["flop"]),
        pick(row["mlp"]), pick(row["best"]), row["gain"])


ALL_CONFIGS = ([(f, p, fea.PREC_FP32) for f in range(4) for p in range(1, 5)]
               + [(f, p, fea.PREC_FP64) for f in range(4) for p in range(2, 5)])


def evaluate(configs=ALL_CONFIGS, log=print, epochs=3000):
    """Autotune, leave-one-out comparison, and the model trained on everything."""
    t0 = time.time()
    records = autotune(configs, log=None)
    rows = leave_one_out(records, configs, epochs=epochs, log=log)
    full = train(records, epochs=epochs)
    return records, full, rows, time.time() - t0


if __name__ == "__main__":
    import sys
    fea.load()
    records, model, rows, dt = evaluate()
    out = sys.argv[1] if len(sys.argv) > 1 else "tuning.json"
    save(out, records, model)
    gm = np.exp(np.mean([np.log(r["gain"]) for r in rows]))
    print(json.dumps({"configs": len(rows), "geomean_speedup_mlp_over_flop_choice": gm, "seconds": dt}))
