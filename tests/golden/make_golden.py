"""Write oracle results used as expected values by the parity tests.

Calls only the CPU oracle and the seeded input generator.  Run from the repo
root:  python tests/golden/make_golden.py [c1] [delta] [tsp_mid] [c5_deposit]
(no argument: c1 and delta).  Outputs in tests/golden/:
  c1_oracle.json          config 1: Delta Z of the probe at z = 0 from SuperLU
                          solves of both systems, plus the coil EMF impedances;
  c1_delta_sensitivity.json  config 1 at gauge penalty delta x 0.1, x 1, x 10
                          (SuperLU), the Delta Z sensitivity to the V-gauge
                          penalty of Sec. 4;
  tsp_mid_oracle.json     53 x 53 x 120-node jittered support-plate mesh
                          (337,080 nodes, 1,348,320 complex unknowns), probe at
                          the plate edge; the oracle's FGMRES with its own
                          aggregation multigrid to a relative residual of 1e-11
                          on each of the four systems (SciPy's SuperLU needs
                          2483 s to factorise a 64,000-unknown mesh of this
                          family on 8 cores, so a direct solve is out of reach);
  c5_deposit_oracle.json  config 5's 50 x 50 x 100 mesh with the deposit of
                          seed 0, two probe positions, same iterative oracle.
"""
import dataclasses
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ect_inputs as E  # noqa: E402
from oracle import fem, impedance, rhs, solve  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TSP_MID = dict(shape=(53, 53, 120), lengths=(30e-3, 30e-3, 67.4e-3), block_shape=(2, 2, 4), jitter=0.15,
               seed=0, z_pos=(10e-3,))
C5_DEPOSIT = dict(seed=0, z_pos=(-2.0e-3, 3.0e-3))


def _c(z):
    return [float(np.real(z)), float(np.imag(z))]


def _cm(a):
    return [[_c(a[k, l]) for l in range(2)] for k in range(2)]


def superlu_dz(p, z):
    """Delta Z (reciprocity and EMF forms) of the probe at z from SuperLU solves."""
    M0 = fem.system_matrix(p, "vacuum")
    Md = fem.system_matrix(p, "defect")
    b = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), z), p, "vacuum")
         for c in p.coils]
    _, lu0 = solve.superlu_solve(M0, b[0])
    _, lud = solve.superlu_solve(Md, b[0])
    u0 = [lu0.solve(bk) for bk in b]
    ud = [lud.solve(bk) for bk in b]
    I = [c.current for c in p.coils]
    dz = impedance.delta_z_matrix(M0, Md, u0, ud, I, p.omega)
    dze = impedance.delta_z_emf_matrix(b, u0, ud, I, p.omega)
    z0 = np.array([[impedance.z_emf(b[k], u0[l], I[k], I[l], p.omega) for l in range(2)] for k in range(2)])
    return dz, dze, z0


def c1_golden():
    p = E.make_config("c1")
    t0 = time.time()
    dz, dze, z0 = superlu_dz(p, p.z_pos[0])
    fa, f3 = impedance.signal_modes(dz)
    return {
        "source": "oracle: fem.system_matrix + superlu_solve + impedance.delta_z_matrix (config c1, z=0)",
        "seconds": time.time() - t0,
        "n_nodes": p.mesh.n_nodes,
        "dz": _cm(dz),
        "dz_emf": _cm(dze),
        "z0": _cm(z0),
        "z_fa": _c(fa),
        "z_f3": _c(f3),
    }


def delta_golden():
    p0 = E.make_config("c1")
    out = {"source": "oracle: superlu_solve on config c1 (z=0) with the V-gauge penalty delta scaled",
           "delta_default": p0.delta, "runs": []}
    for f in (0.1, 1.0, 10.0):
        p = dataclasses.replace(p0, delta=p0.delta * f)
        t0 = time.time()
        dz, dze, _ = superlu_dz(p, p.z_pos[0])
        out["runs"].append({"delta": p.delta, "dz": _cm(dz), "dz_emf": _cm(dze), "seconds": time.time() - t0})
    base = np.array([[complex(*v) for v in r] for r in out["runs"][1]["dz"]])
    for r in out["runs"]:
        d = np.array([[complex(*v) for v in row] for row in r["dz"]])
        r["rel_change_vs_default"] = float(np.abs(d - base).max() / np.abs(base).max())
    return out


def iterative_dz(p, z_list, tol=1e-11, log=print):
    """Delta Z of the probe at each z from the oracle's FGMRES(30) with its aggregation
    multigrid on the scaled system of each configuration (true residual <= tol)."""
    I = [c.current for c in p.coils]
    res = {"positions": []}
    mats, sols = {}, {}
    for which in ("vacuum", "defect"):
        t0 = time.time()
        M = fem.system_matrix(p, which)
        t = fem.scaling(M)
        S = fem.scaled(M, t)
        s1, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, which)
        cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s1)
        d, v = fem.fixed_dofs(p.mesh.bc_mask, cond)
        levels = solve.amg_setup(S, solve.near_null_weights(t, np.concatenate([d, v])), p.mesh.block_of_node,
                                 solve.node_graph_from_tets(p.mesh.n_nodes, p.mesh.tets))
        log(f"{which}: assembly + hierarchy {time.time() - t0:.1f} s")
        mats[which] = M
        for iz, z in enumerate(z_list):
            for k, c in enumerate(p.coils):
                b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), z), p, which)
                t1 = time.time()
                y, info = solve.fgmres(S, t * b, lambda r: solve.amg_apply(levels, r), tol=tol, restart=30,
                                       maxiter=5000)
                x = t * y
                rel = np.linalg.norm(t * (b - M @ x)) / np.linalg.norm(t * b)
                log(f"{which} z={z} coil {k}: {info['iters']} iterations, relres {rel:.2e}, "
                    f"{time.time() - t1:.1f} s")
                sols[(which, iz, k)] = (x, b, rel, info["iters"])
    for iz, z in enumerate(z_list):
        u0 = [sols[("vacuum", iz, k)][0] for k in range(2)]
        ud = [sols[("defect", iz, k)][0] for k in range(2)]
        b = [sols[("vacuum", iz, k)][1] for k in range(2)]
        dz = impedance.delta_z_matrix(mats["vacuum"], mats["defect"], u0, ud, I, p.omega)
        dze = impedance.delta_z_emf_matrix(b, u0, ud, I, p.omega)
        res["positions"].append({
            "z": float(z), "dz": _cm(dz), "dz_emf": _cm(dze),
            "emf_vs_reciprocity": float(np.abs(dze - dz).max() / np.abs(dz).max()),
            "relres": [sols[(w, iz, k)][2] for w in ("vacuum", "defect") for k in range(2)],
            "iters": [sols[(w, iz, k)][3] for w in ("vacuum", "defect") for k in range(2)]})
    return res


def tsp_mid_golden():
    g = TSP_MID
    p = E.tsp_problem(g["shape"], g["lengths"], g["block_shape"], g["jitter"], g["seed"], z_pos=g["z_pos"])
    t0 = time.time()
    out = {"source": "oracle: fem.system_matrix + fgmres(amg_apply) to 1e-11 + impedance.delta_z_matrix",
           "problem": "ect_inputs.tsp_problem" + repr((g["shape"], g["lengths"], g["block_shape"], g["jitter"],
                                                        g["seed"])),
           "n_nodes": p.mesh.n_nodes, "tol": 1e-11}
    out.update(iterative_dz(p, g["z_pos"]))
    out["seconds"] = time.time() - t0
    return out


def c5_deposit_golden():
    g = C5_DEPOSIT
    shape, lengths, _ = E.CONFIGS["c5"]
    p = E.deposit_problem(shape, lengths, E.deposit_params(g["seed"]), z_pos=g["z_pos"])
    t0 = time.time()
    out = {"source": "oracle: fem.system_matrix + fgmres(amg_apply) to 1e-11 + impedance.delta_z_matrix",
           "problem": f"ect_inputs.deposit_problem(c5 mesh, deposit_params({g['seed']}))",
           "params": [float(v) for v in E.deposit_params(g["seed"])],
           "n_nodes": p.mesh.n_nodes, "tol": 1e-11}
    out.update(iterative_dz(p, g["z_pos"]))
    out["seconds"] = time.time() - t0
    return out


JOBS = {"c1": ("c1_oracle.json", c1_golden), "delta": ("c1_delta_sensitivity.json", delta_golden),
        "tsp_mid": ("tsp_mid_oracle.json", tsp_mid_golden),
        "c5_deposit": ("c5_deposit_oracle.json", c5_deposit_golden)}


if __name__ == "__main__":
    names = sys.argv[1:] or ["c1", "delta"]
    for n in names:
        fname, fn = JOBS[n]
        rec = fn()
        out = os.path.join(HERE, fname)
        with open(out, "w") as f:
            json.dump(rec, f, indent=1)
        print(out, flush=True)
