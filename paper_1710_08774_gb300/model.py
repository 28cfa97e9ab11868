"""Learned schedule model: corpus collection, training and schedule choice.

The model is the 3-layer MLP of ``csrc/mlp.cu`` (16 plan features -> 64 ->
64 -> 1, ReLU, FP32) predicting the natural log of a schedule's time per
time step.  Everything numeric runs in the library's CUDA kernels:

  * the timings of the corpus come from ``hfav_autotune`` (every valid
    schedule of a plan, CUDA events, L2 flushed between repetitions);
  * the features of a (plan, schedule) pair from ``hfav_plan_features``;
  * training is ``hfav_mlp_train`` (full-batch MSE, Adam) on the GPU;
  * the choice is ``hfav_model_choose`` (forward over every valid schedule,
    argmin installed as the plan's schedule).

This module only lays out the corpus (which workloads of the 2D chain and
Godunov families, at which sizes), the held-out workloads (3D chains, COSMO,
a DAG of rule bodies: families the corpus does not contain) and moves arrays
between them.  The
corpus stores workload descriptors and measured times, not features, so
features are recomputed from the planner when the model is trained.
"""
import csv
import os

import numpy as np

from . import hfav as H
from . import inputs as I

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
CORPUS = os.path.join(DATA, "corpus_gb300.csv")
HIDDEN = 64
# Feature columns the network does not see.  None: the feature set is the
# planner's sixteen columns, fixed before any held-out workload was timed
# with the current kernels and corpus (no selection against held-out data).
DROP = ()
FIELDS = ["family", "dtype", "nx", "ny", "nz", "n_grids", "steps", "schedule", "ms"]


# ---------------------------------------------------------------------------
# workloads of the training families (2D chain, Godunov, batches of Godunov)
# ---------------------------------------------------------------------------
def corpus_workloads():
    w = []
    for dt in ("f64", "f32"):
        for n in (64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 6144, 8192):
            w.append(("chain2d", dt, n, n, 1, 1, 1))
        for nx, ny in ((4096, 256), (256, 4096), (2048, 512)):
            w.append(("chain2d", dt, nx, ny, 1, 1, 1))
    for n in (64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048):
        w.append(("godunov", "f64", n, n, 1, 1, 2))
    for n in (64, 128, 256, 512, 1024, 2048, 4096):
        w.append(("godunov", "f32", n, n, 1, 1, 2))
    for nx, ny in ((128, 2048), (2048, 128), (1000, 300)):
        w.append(("godunov", "f64", nx, ny, 1, 1, 2))
        w.append(("godunov", "f32", nx, ny, 1, 1, 2))
    for seed in (11, 12, 13, 14, 15):
        w.append(("batch", "f32", seed, 0, 1, 8, 2))
    for dt in ("f64", "f32"):
        for n in (5120, 12288):
            w.append(("chain2d", dt, n, n, 1, 1, 1))
    w.append(("godunov", "f64", 3072, 3072, 1, 1, 2))
    w.append(("godunov", "f32", 6144, 6144, 1, 1, 2))
    w.append(("godunov", "f32", 4096, 512, 1, 1, 2))
    return w


# Held-out workloads: families and shapes never in the corpus (3D chains,
# the COSMO diffusion, a DAG of rule bodies on generated kernels), on which
# the trained model's choice is compared with exhaustive tuning.
def heldout_workloads():
    return [("chain3d", "f32", 512, 512, 512, 1, 1), ("chain3d", "f32", 256, 256, 256, 1, 1),
            ("chain3d", "f32", 768, 768, 768, 1, 1), ("chain3d", "f64", 256, 256, 256, 1, 1),
            ("cosmo", "f32", 1024, 1024, 64, 1, 1), ("codegen2d", "f32", 4096, 4096, 1, 1, 1)]


def _dag(family):
    return {"chain2d": H.chain2d_dag, "chain3d": H.chain3d_dag, "codegen2d": H.chain2d_expr_dag,
            "cosmo": H.cosmo_dag}.get(family, H.godunov_dag)()


# array halo per stencil family: the 2D chains' inputs carry a halo of 2 (the
# chain2d input layout), the periodic 3D chain and COSMO grids are stored
# without halo (the bench's layouts; their halo would never be read)
HALO = {"chain2d": 2, "codegen2d": 2, "chain3d": 0, "cosmo": 0}
DEFAULT = {"codegen2d": "full:smem:32x8"}


def plan_for(family, dtype, nx, ny, nz, n_grids, device_arrays=False):
    """Plan of a workload; with device_arrays also the (axioms, goals) tensors."""
    hdt = H.HFAV_F64 if dtype == "f64" else H.HFAV_F32
    if family in HALO:
        halo = HALO[family]
        two = family in ("chain2d", "codegen2d")
        shape = (ny + 2 * halo, nx + 2 * halo) if two else (nz + 2 * halo, ny + 2 * halo, nx + 2 * halo)
        grid = H.Grid.make([nx, ny, nz][:len(shape)], [1] + [int(np.prod(shape[len(shape) - a:])) for a in
                                                              range(1, len(shape))], halo)
        plan = H.Plan(_dag(family), [grid], hdt, H.HFAV_BC_PERIODIC, DEFAULT.get(family, "full:reg:32x4"))
        if not device_arrays:
            return plan, None
        import torch
        npdt = np.float32 if dtype == "f32" else np.float64
        if two:
            u = I.chain2d_input(nx, seed=0, ny=ny).astype(npdt)
        elif family == "chain3d":
            u = I.chain3d_input(nx, seed=4, dtype=npdt, halo=0)
        else:
            u = I.cosmo_input(nx, ny, nz, seed=7, dtype=npdt, halo=0)
        u = torch.from_numpy(u).cuda()
        return plan, ([u], [torch.empty_like(u)])
    if family == "batch":
        sides = I.batch_sides(n_grids, seed=nx, lo=128, hi=1024)
    else:
        sides = [(nx, ny)]
    grids = [H.Grid.make((a, b), (1, a), 0) for a, b in sides]
    plan = H.Plan(H.godunov_dag(), grids, hdt, H.HFAV_BC_PERIODIC, "sweep:reg:32x4")
    if not device_arrays:
        return plan, None
    import torch
    td = torch.float64 if dtype == "f64" else torch.float32
    ins, outs = [], []
    for g, (a, b) in enumerate(sides):
        U = I.sod_state(a, b, seed=1, grid=g)
        t = [torch.from_numpy(U[f].copy()).to(td).cuda() for f in range(4)]
        ins.append(t)
        outs.append([torch.empty_like(x) for x in t])
    return plan, (ins, outs)


def measure(family, dtype, nx, ny, nz, n_grids, steps, reps=2):
    """{schedule: ms per time step} of every valid schedule (hfav_autotune)."""
    import torch
    plan, (ax, go) = plan_for(family, dtype, nx, ny, nz, n_grids, device_arrays=True)
    times = plan.autotune(ax, go, n_steps=steps, reps=reps)
    torch.cuda.synchronize()
    out = {k: v / steps for k, v in times.items() if v > 0}
    plan.free()
    del ax, go
    torch.cuda.empty_cache()
    return out


def collect(path=CORPUS, workloads=None, log=print):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    rows = []
    for wl in workloads or corpus_workloads():
        fam, dt, nx, ny, nz, ng, steps = wl
        t = measure(fam, dt, nx, ny, nz, ng, steps)
        for sch, ms in t.items():
            rows.append(dict(zip(FIELDS, [fam, dt, nx, ny, nz, ng, steps, sch, ms])))
        log(f"{fam} {dt} {nx}x{ny}x{nz} grids={ng}: {len(t)} schedules, best {min(t, key=t.get)} "
            f"{min(t.values()):.4f} ms/step")
    with open(path, "w", newline="") as f:
        wr = csv.DictWriter(f, fieldnames=FIELDS)
        wr.writeheader()
        wr.writerows(rows)
    return rows


def load_corpus(path=CORPUS):
    with open(path) as f:
        return list(csv.DictReader(f))


BASE = 12   # HFAV_FEATURE_BASE: log2(analytic estimate in us) / 16


def base_log(X):
    """ln of the analytic time estimate (microseconds) carried in the features."""
    return X[:, BASE].astype(np.float64) * 16.0 * np.log(2.0)


def features_of(rows):
    """Feature matrix (n x 16) and targets of corpus rows (host planner only).

    The target is ln(measured microseconds per step) minus ln of the planner's
    analytic estimate: the network learns the correction to the cost model."""
    X, y = [], []
    cache = {}
    for r in rows:
        key = (r["family"], r["dtype"], int(r["nx"]), int(r["ny"]), int(r["nz"]), int(r["n_grids"]))
        if key not in cache:
            cache[key] = plan_for(*key)[0]
        X.append(cache[key].features(r["schedule"]))
        y.append(np.log(1e3 * float(r["ms"])))
    X = np.array(X, dtype=np.float32)
    return X, (np.array(y) - base_log(X)).astype(np.float32)


# ---------------------------------------------------------------------------
# training and choice
# ---------------------------------------------------------------------------
class Model:
    """An ensemble of n networks (parameter vectors back to back on the device)."""

    def __init__(self, params, shift, scale, hidden=HIDDEN, losses=None, n_models=1):
        self.params, self.shift, self.scale, self.hidden = params, shift, scale, hidden
        self.losses, self.n_models = losses, n_models

    def predict(self, X, add_base=True):
        """Predicted ln(microseconds per step) of feature rows (network output
        plus the analytic estimate's log when add_base)."""
        import torch
        Xn = torch.from_numpy(((X - self.shift) * self.scale).astype(np.float32)).cuda()
        np_ = H.mlp_n_params(X.shape[1], self.hidden)
        out = np.zeros(X.shape[0])
        for m in range(self.n_models):
            y = torch.empty(Xn.shape[0], dtype=torch.float32, device="cuda")
            H.mlp_forward(self.params[m * np_:(m + 1) * np_], Xn, self.hidden, y)
            torch.cuda.synchronize()
            out += y.cpu().numpy() / self.n_models
        return out + (base_log(X) if add_base else 0.0)

    def choose(self, plan):
        """Install the predicted-fastest schedule on the plan; returns (schedule, {schedule: prediction})."""
        return plan.model_choose(self.params, self.hidden, self.shift, self.scale, self.n_models)

    def save(self, path):
        np.savez(path, params=self.params.cpu().numpy(), shift=self.shift, scale=self.scale, hidden=self.hidden)

    @staticmethod
    def load(path):
        import torch
        z = np.load(path)
        return Model(torch.from_numpy(z["params"]).cuda(), z["shift"], z["scale"], int(z["hidden"]))


def init_params(n_in, hidden, seed=0):
    """He-initialised parameters in the layout of csrc/mlp.cu (seeded)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / n_in), (hidden, n_in))
    W2 = rng.normal(0, np.sqrt(2.0 / hidden), (hidden, hidden))
    w3 = rng.normal(0, np.sqrt(1.0 / hidden), hidden)
    return np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(hidden), w3, [0.0]]).astype(np.float32)


def train(X, y, hidden=HIDDEN, epochs=800, lr=3e-3, seed=0, n_models=1, drop=DROP):
    """Full-batch Adam on the GPU (hfav_mlp_train), one network per seed
    seed .. seed + n_models - 1, on the feature columns not in `drop`.
    Returns a Model (the ensemble)."""
    import torch
    shift = X.mean(axis=0)
    sd = X.std(axis=0)
    scale = np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 1.0).astype(np.float32)
    for c in drop:
        shift[c], scale[c] = 0.0, 0.0
    Xn = torch.from_numpy(((X - shift) * scale).astype(np.float32)).cuda()
    t = torch.from_numpy(y.astype(np.float32)).cuda()
    work = torch.empty(H.mlp_work_floats(X.shape[0], hidden), dtype=torch.float32, device="cuda")
    params, losses = [], []
    for k in range(n_models):
        p = torch.from_numpy(init_params(X.shape[1], hidden, seed + k)).cuda()
        m = torch.zeros_like(p); v = torch.zeros_like(p); g = torch.zeros_like(p)
        lh = torch.empty(epochs, dtype=torch.float32, device="cuda")
        H.mlp_train(p, m, v, Xn, t, hidden, epochs, lr, work, g, lh)
        params.append(p)
        losses.append(lh)
    torch.cuda.synchronize()
    return Model(torch.cat(params), shift.astype(np.float32), scale, hidden,
                 torch.stack(losses).mean(0).cpu().numpy(), n_models)


def evaluate_heldout(mdl, workloads=None, reps=3, log=print):
    """For every held-out workload: the time of every valid schedule
    (hfav_autotune), the model's pick, the analytic estimate's pick and the
    plan's default.  Returns a list of dicts."""
    import torch
    out = []
    for wl in workloads or heldout_workloads():
        fam, dt, nx, ny, nz, ng, steps = wl
        plan, (ax, go) = plan_for(fam, dt, nx, ny, nz, ng, device_arrays=True)
        default = plan.schedule
        times = {k: v for k, v in plan.autotune(ax, go, n_steps=steps, reps=reps).items() if v > 0}
        torch.cuda.synchronize()
        pick, _ = mdl.choose(plan)
        F = np.array([plan.features(k) for k in times], dtype=np.float32)
        base_pick = list(times)[int(np.argmin(base_log(F)))]
        best = min(times.values())
        r = dict(workload=wl, times=times, best=min(times, key=times.get), pick=pick, base_pick=base_pick,
                 default=default, pick_over_best=times[pick] / best, base_over_best=times[base_pick] / best,
                 default_over_best=times[default] / best)
        out.append(r)
        log(f"held-out {fam} {dt} {nx}x{ny}x{nz}: best {r['best']} {best:.4f} ms; model {pick} "
            f"x{r['pick_over_best']:.3f}; analytic {base_pick} x{r['base_over_best']:.3f}; default {default} "
            f"x{r['default_over_best']:.3f}")
        plan.free()
        del ax, go
        torch.cuda.empty_cache()
    return out


def cross_family(rows, X, y, drop=DROP, n_models=3, epochs=800, seed=0):
    """Leave-one-family-out choice quality on the corpus: for each family
    (2D chain; Godunov with its batches) train on the other one and pick the
    predicted-fastest schedule of every workload of the held family.  Returns
    {family: geometric mean of (picked time / best time)}."""
    fam = np.array(["godunov" if r["family"] == "batch" else r["family"] for r in rows])
    ms = np.array([float(r["ms"]) for r in rows])
    groups = {}
    for i, r in enumerate(rows):
        groups.setdefault((r["family"], r["dtype"], r["nx"], r["ny"], r["nz"], r["n_grids"]), []).append(i)
    out = {}
    for held in ("chain2d", "godunov"):
        tr = fam != held
        mdl = train(X[tr], y[tr], epochs=epochs, n_models=n_models, drop=drop, seed=seed)
        logs = []
        for idx in groups.values():
            if fam[idx[0]] != held:
                continue
            k = idx[int(np.argmin(mdl.predict(X[idx])))]
            logs.append(np.log(ms[k] / ms[idx].min()))
        out[held] = float(np.exp(np.mean(logs)))
    return out


if __name__ == "__main__":
    import sys
    import torch
    assert torch.cuda.is_available()
    out = sys.argv[1] if len(sys.argv) > 1 else CORPUS
    collect(out)
