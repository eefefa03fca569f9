"""Write the oracle trajectories that the long GPU parity tests compare with.

Both runs use the FP64 oracle only (oracle/ and the seeded inputs of synth/),
with the Poisson solve driven to a relative residual of 1e-10:

* parity_droplet64.npz -- the 128^3 dielectric droplet scaled to a 64^3 copy
  (drop radius 12, seed 1, salt 1e-3, E_z = 1e-3, G = 4): the drop
  deformation every 25 steps for 500 steps, and at step 500 the densities, ion
  concentrations, potential and physical velocity at 2048 seeded sample sites.
* parity_suspension64.npz -- the 256^3 electrophoresis suspension at the same
  colloid number density in a 64^3 box (3 spheres of radius 6, seed 2,
  charges in [-40, -10], salt 1e-3, E_x = 1e-3, moving colloids): colloid
  positions and velocities every 10 steps for `SUSP_STEPS` steps.

    python tests/golden/make_parity_runs.py [droplet|suspension]
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import OracleSystem  # noqa: E402
from oracle import observables  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
DROP_STEPS, DROP_EVERY, NSAMPLE = 500, 25, 2048
SUSP_STEPS, SUSP_EVERY = 1000, 10


def droplet():
    w = synth.droplet(n=64, r=12.0, prec="fp32", seed=1, salt=1e-3, Ez=1e-3)
    w.params.poisson_tol = 1e-10
    w.params.poisson_max_iter = 500
    s = OracleSystem(w.params, w.rho, w.n)
    D = [observables.deformation(s.densities())[0]]
    for t in range(1, DROP_STEPS + 1):
        s.step()
        if t % DROP_EVERY == 0:
            D.append(observables.deformation(s.densities())[0])
            print("droplet step", t, D[-1], flush=True)
    rng = np.random.default_rng(77)
    idx = rng.choice(64 ** 3, size=NSAMPLE, replace=False)
    rho = s.densities().reshape(2, -1)[:, idx]
    n = s.n.reshape(2, -1)[:, idx]
    phi = s.phi.reshape(-1)[idx]
    u = s.last_u.reshape(3, -1)[:, idx]
    np.savez_compressed(os.path.join(HERE, "parity_droplet64.npz"), steps=DROP_STEPS, every=DROP_EVERY,
                        deformation=np.array(D), idx=idx, rho=rho, n=n, phi=phi, u=u,
                        max_rho=s.densities().reshape(2, -1).max(axis=1), max_n=s.n.reshape(2, -1).max(axis=1),
                        max_phi=np.abs(s.phi).max(), max_u=np.abs(s.last_u).max())


def suspension():
    w = synth.suspension(n=64, ncoll=3, r=6.0, prec="fp32", seed=2)
    w.params.poisson_tol = 1e-10
    w.params.poisson_max_iter = 500
    s = OracleSystem(w.params, w.rho, w.n, colloid_x=w.colloid_x, colloid_v=w.colloid_v, colloid_q=w.colloid_q,
                     colloid_r=w.colloid_r)
    xs, vs = [s.cx.copy()], [s.cv.copy()]
    for t in range(1, SUSP_STEPS + 1):
        s.step()
        if t % SUSP_EVERY == 0:
            xs.append(s.cx.copy())
            vs.append(s.cv.copy())
            print("suspension step", t, s.cv[:, 0], flush=True)
            np.savez_compressed(os.path.join(HERE, "parity_suspension64.npz"), steps=t, every=SUSP_EVERY,
                                x=np.array(xs), v=np.array(vs), q=w.colloid_q, r=w.colloid_r)


if __name__ == "__main__":
    what = sys.argv[1:] or ["droplet", "suspension"]
    if "droplet" in what:
        droplet()
    if "suspension" in what:
        suspension()
