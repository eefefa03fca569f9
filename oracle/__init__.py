"""CPU oracle for the coupled electrohydrodynamic lattice step (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the model of Rivas, Frijters, Pagonabarraga and Harting,
"Mesoscopic electrohydrodynamic simulations of binary colloidal suspensions"
(arXiv:1712.08494), Sec. II.  Only the test suite, the smoke check of the
package entry point and the CPU-baseline leg of the benchmark may import it.
The product path (the CUDA library and its Python binding) never imports,
links or runs anything here, and this package imports nothing from the
product path: the two share no code.  The only common module is ``synth``,
which draws seeded inputs and holds none of the method's arithmetic.

Modules
-------
lattice      D3Q19 velocities and weights (Sec. II.A).
geometry     projection of spheres onto the lattice, solid fraction, surface
             nodes and surface charge (Sec. II.E).
poisson      variable-permittivity Poisson solve (Sec. II.D).
model        one coupled timestep: macro fields, forces, ion fluxes,
             Nernst-Planck update, forced BGK collision, streaming and
             halfway bounce-back (Sec. II.A-E).
colloids     colloid forces and motion, node creation/deletion (Sec. II.E).
observables  conserved sums, droplet deformation, colloid drift.

Each function cites the passage (section / equation) it restates.  Readings
where the paper is ambiguous are stated in the docstrings; their list is kept
with the design notes of the repository.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, invariants or brute force; the whole-step composition
of all couplings at once is pinned by a second, site-by-site transcription
on tiny lattices and by physical laws (Young-Laplace, low-zeta mobility,
dielectric drop deformation, flat-interface equilibrium).
"""

from .lattice import C, W, OPP, CS2, Q  # noqa: F401
from .model import OracleSystem  # noqa: F401
