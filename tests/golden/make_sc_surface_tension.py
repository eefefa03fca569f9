"""Write sc_surface_tension.json: the Shan-Chen surface tension of the
two-component model at G = 4 (tau = 1, D3Q19 weights, psi = 1 - exp(-rho)),
measured with the oracle only.

A quasi-2D drop (2 x 48 x 48, radius 12, densities 0.7 / 0.04 swapped inside)
relaxes for 3000 steps, then gamma is averaged over ten samples 100 steps
apart (the drop still breathes slightly); the pressure of the equation of state
p = c_s^2 (rho_a + rho_b) + c_s^2 G psi_a psi_b (Sec. II.C eq. eqofstate) inside
minus outside, times the drop radius, is gamma (two-dimensional Young-Laplace
law dp = gamma / r, Sec. III.B).  The radius is that of the disc with the
area of c = (rho_b - rho_a)/(rho_a + rho_b) > 0.

    python tests/golden/make_sc_surface_tension.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import OracleSystem  # noqa: E402
from oracle.model import psi_of  # noqa: E402


def main():
    n, r, G, relax, samples, every = 48, 12.0, 4.0, 3000, 10, 100
    w = synth.droplet(n=n, r=r, G=G, Ez=0.0, nions=0, tol=1e-8, noise=0.0)
    w.params.nx = 2
    rho = w.rho[:, :, :, n // 2 - 1:n // 2 + 1].copy()
    s = OracleSystem(w.params, rho)
    s.run(relax)
    gam, dps, rds = [], [], []
    for _ in range(samples):
        s.run(every)
        ra, rb = s.densities()
        p = (ra + rb) / 3.0 + G / 3.0 * psi_of(ra) * psi_of(rb)
        c = n // 2
        dp = float(p[c, c, 0] - p[0, 0, 0])
        rd = math.sqrt(float(((rb - ra) > 0)[:, :, 0].sum()) / math.pi)
        gam.append(dp * rd)
        dps.append(dp)
        rds.append(rd)
    steps = relax + samples * every
    out = {"G": G, "tau": 1.0, "gamma": sum(gam) / len(gam), "gamma_min": min(gam), "gamma_max": max(gam),
           "dp": sum(dps) / len(dps), "radius": sum(rds) / len(rds), "box": [2, n, n], "steps": steps,
           "source": "oracle relaxation of a quasi-2D drop; Young-Laplace dp = gamma/r (Sec. III.B) with the "
                     "Shan-Chen equation of state (Sec. II.C)"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sc_surface_tension.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
