"""Write sc_coexistence.json: bulk densities of the two-component Shan-Chen
mixture at G = 4 (tau = 1, D3Q19 weights, psi = 1 - exp(-rho)), measured with
the oracle only.

Flat interfaces (Sec. III.A geometry) in a 32 x 1 x 1 periodic box, red 0.7 /
blue 0.04 on one half and swapped on the other, relax for 3000 steps; the
majority and minority densities at the middle of the red half are the bulk
values.  They serve as initial densities of flat-interface runs, which then
need little interdiffusion to reach equilibrium.

    python tests/golden/make_sc_coexistence.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import OracleSystem  # noqa: E402


def main():
    nx, steps = 32, 3000
    w = synth.flat_interface(nx=nx, ny=1, nz=1, prec="fp64", nions=0)
    s = OracleSystem(w.params, w.rho)
    s.run(steps - 100)
    before = s.densities()[:, 0, 0, nx // 4].copy()
    s.run(100)
    rho = s.densities()[:, 0, 0, nx // 4]
    out = {"G": float(w.params.G), "tau": float(w.params.tau), "rho_major": float(rho[0]),
           "rho_minor": float(rho[1]), "change_last_100_steps": float(abs(rho - before).max()),
           "box": [nx, 1, 1], "steps": steps,
           "source": "oracle relaxation of flat interfaces (Sec. III.A geometry), Shan-Chen forces of Sec. II.C"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sc_coexistence.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
