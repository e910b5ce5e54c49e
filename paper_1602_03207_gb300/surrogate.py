"""Delta Z surrogate: dataset generation with the solver, tcgen05 training, evaluation.

Host-side orchestration only: every solve, every Delta Z and every training
step runs in libect.so.  The solver is the data source and the reference
for the surrogate's error:

* dataset: for each seeded deposit (thickness, axial length, conductivity,
  relative permeability, azimuthal coverage, axial centre) the defect matrix
  is re-assembled on a fixed mesh (ect_set_defect), coil 1's sources at all
  probe positions are solved in one batched call that starts from the
  background (vacuum) solutions, and Delta Z_11 at each
  position is reduced by reciprocity against the (shared) vacuum solutions;
  samples are appended to a JSON-lines file keyed by seed, so an interrupted
  run resumes where it stopped;
* model: 6 normalised inputs -> 2 * n_positions outputs (Re, Im of the
  normalised Delta Z_11 signal);
* evaluation: relative L2 error of the surrogate's signal against the solver
  on held-out seeds, and the time of one surrogate batch against one solve.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import ect as E

# parameter ranges of the deposit distribution (thickness, length, sigma, mu_r, coverage, z_c)
LO = np.array([0.0, 2.0e-3, 1.0e4, 1.0, 0.0, -10.0e-3])
HI = np.array([0.5e-3, 20.0e-3, 1.0e6, 5.0, 2.0 * math.pi, 10.0e-3])


def normalise_inputs(params):
    return (2.0 * (np.asarray(params, dtype=np.float64) - LO) / (HI - LO) - 1.0).astype(np.float32)


def load_samples(path):
    out = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                line = line.strip()
                if not line:
                    continue
                try:
                    rec = json.loads(line)
                except json.JSONDecodeError:
                    continue          # a line cut by an interruption
                out[int(rec["seed"])] = rec
    return out


class DatasetGenerator:
    """Solver-generated (deposit parameters -> Delta Z_11 along the probe path) samples."""

    def __init__(self, mesh, background, coil, z_pos, make_defect, options=None, tune=False):
        """mesh/background: an input problem without deposit (its mesh, sigma, nu, physics);
        make_defect(seed) -> (params(6,), sigma_d(T,), nu_d(T,)) on the same mesh.
        tune: pick the solver options (tiles, SpMM variant, Krylov lengths, Gram-Schmidt
        variant, subdomain split) with ect_autotune on the background system first."""
        import torch
        self.torch = torch
        self.p = background
        self.coil = coil
        self.z = np.asarray(z_pos, dtype=np.float64)
        self.make_defect = make_defect
        self.opts = options or E.default_options(tol=1e-8, mode=E.ECT_MODE_MIXED, restart=10, inner_iters=10,
                                                 max_iters=300)
        self.ctx = E.Context()
        self.ctx.load_problem(background)
        n = 4 * background.mesh.n_nodes
        self.n = n
        mask = E.ECT_F64 | E.ECT_F32
        self.ctx.assemble(E.ECT_VACUUM, mask)
        self.ctx.precond_setup(E.ECT_VACUUM, mask, -1)
        k = self.z.size
        self.B = torch.empty(k, n, dtype=torch.complex128, device="cuda")
        self.ctx.coil_rhs(coil, self.z, self.B)
        self.U0 = torch.empty_like(self.B)
        self.Ud = torch.empty_like(self.B)
        if tune:
            self.opts, _ = self.ctx.autotune(E.ECT_VACUUM, self.B, self.U0, k, self.opts)
        self.stats0 = self.ctx.solve(E.ECT_VACUUM, self.B, self.U0, k, self.opts)
        self.current = coil.current
        # the deposit changes the fields near it only: each defect solve starts from the
        # background solutions (positions far from the deposit then converge at once)
        self.opts_warm = E.default_options()
        for f, _ in E.Options._fields_:
            setattr(self.opts_warm, f, getattr(self.opts, f))
        self.opts_warm.x0 = 1

    def sample(self, seed):
        params, sd, nd = self.make_defect(seed)
        mask = E.ECT_F64 | E.ECT_F32
        t0 = time.perf_counter()
        self.ctx.set_defect(sd, nd)
        self.ctx.assemble(E.ECT_DEFECT, mask)
        self.ctx.precond_setup(E.ECT_DEFECT, mask, -1)
        t1 = time.perf_counter()
        self.Ud.copy_(self.U0)
        st = self.ctx.solve(E.ECT_DEFECT, self.B, self.Ud, self.z.size, self.opts_warm)
        t2 = time.perf_counter()
        dz = np.empty(self.z.size, dtype=np.complex128)
        I = [self.current, self.current]
        for q in range(self.z.size):
            u0 = self.U0[q].unsqueeze(0).expand(2, -1).contiguous()
            ud = self.Ud[q].unsqueeze(0).expand(2, -1).contiguous()
            d, _ = self.ctx.delta_z(u0, ud, None, I)
            dz[q] = d[0, 0]
        t3 = time.perf_counter()
        return {"seed": int(seed), "params": [float(v) for v in params], "dz_re": dz.real.tolist(),
                "dz_im": dz.imag.tolist(), "iters": st["iters"], "seconds": t3 - t0,
                "seconds_setup": t1 - t0, "seconds_solve": t2 - t1, "seconds_dz": t3 - t2}

    def run(self, seeds, path, budget_s=None):
        done = load_samples(path)
        t0 = time.time()
        with open(path, "a") as f:
            for s in seeds:
                if int(s) in done:
                    continue
                if budget_s is not None and time.time() - t0 > budget_s:
                    break
                rec = self.sample(s)
                f.write(json.dumps(rec) + "\n")
                f.flush()
                done[int(s)] = rec
        return done


def arrays(samples, seeds):
    X = np.stack([normalise_inputs(samples[s]["params"]) for s in seeds])
    Y = np.stack([np.concatenate([samples[s]["dz_re"], samples[s]["dz_im"]]) for s in seeds])
    return X, Y


class Trainer:
    """Adam training of the tcgen05 MLP on (X, Y) with a global output scale."""

    def __init__(self, n_out=256, batch=256, seed=0):
        import torch
        self.torch = torch
        self.batch = batch
        self.net = E.Surrogate(batch=batch)
        rng = np.random.default_rng(seed)
        layers = []
        for fi, fo in zip(E.MLP_SIZES[:-1], E.MLP_SIZES[1:]):
            layers.append((rng.normal(scale=1.0 / math.sqrt(fi), size=(fo, fi)), np.zeros(fo)))
        self.net.set_params(E.mlp_flatten(layers))
        self.scale = 1.0
        self.n_out = n_out

    def fit(self, X, Y, epochs=200, lr=1e-3, log_every=0):
        torch = self.torch
        assert Y.shape[1] == self.n_out
        self.scale = float(np.std(Y)) or 1.0
        Yn = (Y / self.scale).astype(np.float32)
        n = X.shape[0]
        B = self.batch
        rng = np.random.default_rng(1)
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        Yd = torch.from_numpy(np.ascontiguousarray(Yn)).cuda()
        hist = []
        t0 = time.perf_counter()
        steps = 0
        for ep in range(epochs):
            idx = torch.from_numpy(rng.permutation(n).astype(np.int64)).cuda()
            for b0 in range(0, n - B + 1, B) if n >= B else [0]:
                sel = idx[b0:b0 + B] if n >= B else idx[torch.arange(B, device="cuda") % n]
                xb = Xd[sel].contiguous()
                yb = Yd[sel].contiguous()
                want = log_every and (steps % log_every == 0)
                l = self.net.train_step(xb, yb, lr, want_loss=bool(want))
                if want:
                    hist.append((steps, l))
                steps += 1
        torch.cuda.synchronize()
        return {"steps": steps, "seconds": time.perf_counter() - t0, "history": hist}

    def predict(self, X):
        torch = self.torch
        B = self.batch
        n = X.shape[0]
        out = np.empty((n, self.n_out), dtype=np.float64)
        xb = torch.zeros(B, 6, dtype=torch.float32, device="cuda")
        yb = torch.empty(B, self.n_out, dtype=torch.float32, device="cuda")
        for b0 in range(0, n, B):
            m = min(B, n - b0)
            xb.zero_()
            xb[:m] = torch.from_numpy(np.ascontiguousarray(X[b0:b0 + m], dtype=np.float32)).cuda()
            self.net.forward(xb, yb)
            out[b0:b0 + m] = yb[:m].cpu().numpy()
        return out * self.scale


def relative_errors(pred, ref):
    return np.linalg.norm(pred - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


def deposit_workload(shape=(50, 50, 100), lengths=(20e-3, 20e-3, 40e-3), n_pos=128):
    """The surrogate workload: tube mesh, probe path and a deposit factory (seeded inputs)."""
    import ect_inputs as I
    mesh = I.box_mesh(shape, lengths, (2, 2, 4))
    z = -15.875e-3 + (31.75e-3 / (n_pos - 1)) * np.arange(n_pos) if n_pos > 1 else np.zeros(1)
    background = I.deposit_problem(shape, lengths, I.deposit_params(0), mesh=mesh, z_pos=z)
    background.sigma_d = np.full(mesh.n_tets, np.nan)
    background.nu_d = np.full(mesh.n_tets, np.nan)

    def make_defect(seed):
        q = I.deposit_problem(shape, lengths, I.deposit_params(seed), mesh=mesh, z_pos=z)
        return I.deposit_params(seed), q.sigma_d, q.nu_d

    return background, z, make_defect


def run(out_path, budget_s=600.0, shape=(50, 50, 100), n_pos=128, held_out=0.1, steps=3000, lr=1e-3,
        tol=1e-6, max_seed=2000):
    """Generate (resumable) -> train -> evaluate; returns a report dict.  The last held_out share
    of the seeds is held out (seeds 1800..1999 of the full 2000)."""
    import torch
    background, z, make_defect = deposit_workload(shape, n_pos=n_pos)
    opts = E.default_options(tol=tol, mode=E.ECT_MODE_MIXED, restart=16, inner_iters=12, max_iters=300)
    t0 = time.perf_counter()
    gen = DatasetGenerator(None, background, background.coils[0], z, make_defect, opts, tune=True)
    setup_s = time.perf_counter() - t0
    samples = gen.run(range(max_seed), out_path, budget_s=budget_s)
    seeds = sorted(samples)
    n_test = max(1, int(round(held_out * len(seeds))))
    train, test = seeds[:-n_test], seeds[-n_test:]
    Xtr, Ytr = arrays(samples, train)
    Xte, Yte = arrays(samples, test)
    tr = Trainer(n_out=2 * n_pos)
    epochs = max(1, steps // max(1, len(train) // tr.batch)) if len(train) >= tr.batch else steps
    fit = tr.fit(Xtr, Ytr, epochs=epochs, lr=lr, log_every=200)
    # evaluation: surrogate vs solver on held-out deposits
    t1 = time.perf_counter()
    pred = tr.predict(Xte)
    torch.cuda.synchronize()
    infer_s = (time.perf_counter() - t1) / len(test)
    err = relative_errors(pred, Yte)
    mean_sig = np.broadcast_to(Ytr.mean(axis=0), Yte.shape)                     # predicting the mean signal
    base = relative_errors(mean_sig, Yte)
    agg = float(np.linalg.norm(pred - Yte) / np.linalg.norm(Yte))
    agg_base = float(np.linalg.norm(mean_sig - Yte) / np.linalg.norm(Yte))
    solve_s = float(np.median([samples[s]["seconds"] for s in seeds]))
    return {"samples": len(seeds), "train": len(train), "held_out": len(test), "positions": n_pos,
            "mesh_nodes": int(np.prod(shape)), "solver_tol": tol, "setup_s": setup_s,
            "solver_options": {f: getattr(gen.opts, f) for f in ("restart", "inner_iters", "reorth", "rhs_tile",
                                                                 "spmm_rows")},
            "block_split": gen.ctx.block_split(),
            "solver_s_per_deposit": solve_s, "surrogate_s_per_deposit": infer_s,
            "speedup": solve_s / max(infer_s, 1e-12), "train_steps": fit["steps"], "train_s": fit["seconds"],
            "loss_history": fit["history"][-5:],
            "held_out_rel_l2": {"median": float(np.median(err)), "mean": float(np.mean(err)),
                                "max": float(np.max(err)), "aggregate": agg},
            "mean_signal_rel_l2": {"median": float(np.median(base)), "mean": float(np.mean(base)),
                                   "aggregate": agg_base}}


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="surrogate_samples.jsonl")
    ap.add_argument("--budget", type=float, default=600.0)
    ap.add_argument("--nodes", default="50,50,100")
    ap.add_argument("--positions", type=int, default=128)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--tol", type=float, default=1e-6)
    a = ap.parse_args()
    rep = run(a.out, a.budget, tuple(int(v) for v in a.nodes.split(",")), a.positions, steps=a.steps, tol=a.tol)
    print(json.dumps(rep))
