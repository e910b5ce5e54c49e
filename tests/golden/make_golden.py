"""Write oracle results used as expected values by the GPU parity tests.

Calls only the CPU oracle and the seeded input generator.  Run from the repo
root:  python tests/golden/make_golden.py
Output: tests/golden/c1_oracle.json (config 1: Delta Z of the probe at z = 0
from SuperLU solves of both systems, plus the coil EMF impedances).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ect_inputs as E  # noqa: E402
from oracle import fem, impedance, rhs, solve  # noqa: E402


def c1_golden():
    p = E.make_config("c1")
    t0 = time.time()
    M0 = fem.system_matrix(p, "vacuum")
    Md = fem.system_matrix(p, "defect")
    b = [fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, c.as_tuple(), p.z_pos[0]), p, "vacuum")
         for c in p.coils]
    u0, ud = [], []
    _, lu0 = solve.superlu_solve(M0, b[0])
    _, lud = solve.superlu_solve(Md, b[0])
    for bk in b:
        u0.append(lu0.solve(bk))
        ud.append(lud.solve(bk))
    I = [c.current for c in p.coils]
    dz = impedance.delta_z_matrix(M0, Md, u0, ud, I, p.omega)
    dze = impedance.delta_z_emf_matrix(b, u0, ud, I, p.omega)
    z0 = np.array([[impedance.z_emf(b[k], u0[l], I[k], I[l], p.omega) for l in range(2)] for k in range(2)])
    fa, f3 = impedance.signal_modes(dz)
    c = lambda z: [float(np.real(z)), float(np.imag(z))]  # noqa: E731
    return {
        "source": "oracle: fem.system_matrix + superlu_solve + impedance.delta_z_matrix (config c1, z=0)",
        "seconds": time.time() - t0,
        "n_nodes": p.mesh.n_nodes,
        "dz": [[c(dz[k, l]) for l in range(2)] for k in range(2)],
        "dz_emf": [[c(dze[k, l]) for l in range(2)] for k in range(2)],
        "z0": [[c(z0[k, l]) for l in range(2)] for k in range(2)],
        "z_fa": c(fa),
        "z_f3": c(f3),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_oracle.json")
    with open(out, "w") as f:
        json.dump(c1_golden(), f, indent=1)
    print(out)
