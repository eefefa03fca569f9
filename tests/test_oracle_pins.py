"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every test here compares the oracle with something other than itself: closed
forms (lattice moments, Fourier symbols of the discrete operators, the shear
wave decay rate nu = c_s^2 (tau - 1/2)), exact invariants (mass, ions, charge,
momentum), special cases that reduce to a textbook result (harmonic-mean
displacement of a layered dielectric, the equilibrium of a wall moving with
the fluid), brute force on tiny inputs (geometry, sparse direct Poisson solve).
"""
import math

import numpy as np
import pytest

import synth
from oracle import geometry, poisson
from oracle.lattice import AXES, C, CS2, OPP, Q, W, equilibrium, shift
from oracle.model import (OracleSystem, face_fluxes, friction_force, np_update,
                          virtual_density, electric_field)
from oracle import observables as obs


# ---------------------------------------------------------------- lattice
def test_d3q19_moments_exact():
    assert W.sum() == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    for a in range(3):
        assert abs((W * C[:, a]).sum()) < 1e-15
        for b in range(3):
            assert (W * C[:, a] * C[:, b]).sum() == pytest.approx(d[a, b] * CS2, abs=1e-15)
            for c in range(3):
                assert abs((W * C[:, a] * C[:, b] * C[:, c]).sum()) < 1e-15
                for e in range(3):
                    m4 = (W * C[:, a] * C[:, b] * C[:, c] * C[:, e]).sum()
                    iso = (d[a, b] * d[c, e] + d[a, c] * d[b, e] + d[a, e] * d[b, c]) / 9.0
                    assert m4 == pytest.approx(iso, abs=1e-15)
    for q in range(Q):
        assert OPP[OPP[q]] == q
        assert (C[OPP[q]] == -C[q]).all()


def test_equilibrium_moments_exact():
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.5, 1.5, size=(7,))
    u = rng.uniform(-0.05, 0.05, size=(3, 7))
    feq = equilibrium(rho, u)
    assert np.allclose(feq.sum(axis=0), rho, rtol=1e-14, atol=0)
    for a in range(3):
        assert np.allclose((feq * C[:, a, None]).sum(axis=0), rho * u[a], rtol=1e-13, atol=1e-17)
        for b in range(3):
            pi = (feq * (C[:, a, None] * C[:, b, None])).sum(axis=0)
            ref = rho * CS2 * (a == b) + rho * u[a] * u[b]
            assert np.allclose(pi, ref, rtol=1e-13, atol=1e-17)


# ---------------------------------------------------------------- fluid
def _system(n=8, ncomp=1, G=0.0, rho=None, nions=0, **kw):
    p = synth.Params(nx=n, ny=n, nz=n, ncomp=ncomp, nions=nions, prec="fp64", G=G, **kw)
    if rho is None:
        rho = np.ones((ncomp, n, n, n))
    return OracleSystem(p, rho, **({} if nions == 0 else {"n": np.full((2, n, n, n), 0.01)}))


def test_rest_state_is_a_fixed_point():
    s = _system(n=6, ncomp=2, G=4.0, rho=np.stack([np.full((6, 6, 6), 0.7), np.full((6, 6, 6), 0.04)]))
    f0 = s.f.copy()
    s.run(3)
    # exact up to the rounding of rho = sum_q w_q rho
    assert np.allclose(s.f, f0, rtol=1e-14, atol=0)


def _shear_nu(n, tau, T):
    p = synth.Params(nx=1, ny=1, nz=n, ncomp=1, nions=0, prec="fp64", G=0.0, tau=tau)
    z = np.arange(n)
    k = 2 * math.pi / n
    U = 1e-4
    u = np.zeros((3, n, 1, 1))
    u[0, :, 0, 0] = U * np.sin(k * z)
    s = OracleSystem(p, np.ones((1, n, 1, 1)), u=u)
    s.run(T)
    rho = s.densities()[0]
    ux = sum(C[q, 0] * s.f[0, q] for q in range(Q)) / rho
    amp = 2.0 / n * (ux[:, 0, 0] * np.sin(k * z)).sum()
    return -math.log(amp / U) / (k * k * T)


@pytest.mark.parametrize("tau", [1.0, 0.8, 0.65])
def test_shear_wave_decays_at_lattice_viscosity(tau):
    """u_x(z) = U sin(k z) decays as exp(-nu k^2 t) with the Chapman-Enskog
    viscosity nu = c_s^2 (tau - 1/2) of Sec. II.A.  The lattice dispersion is
    O(k^2): the error falls about fourfold when the wavelength doubles."""
    nu_th = CS2 * (tau - 0.5)
    e32 = _shear_nu(32, tau, 60) / nu_th - 1.0
    e64 = _shear_nu(64, tau, 240) / nu_th - 1.0
    assert abs(e64) < 1e-2
    if abs(e32) > 1e-4:
        assert 3.5 < e32 / e64 < 4.5   # second-order convergence to nu


def test_shan_chen_conserves_mass_and_momentum():
    """Pair antisymmetry of the Shan-Chen force: sum_x (Phi_a + Phi_b) = 0, so
    total momentum is conserved to round-off (Sec. II.C eq. shanChenForce)."""
    rng = np.random.default_rng(1)
    n = 8
    rho = rng.uniform(0.05, 0.8, size=(2, n, n, n))
    s = _system(n=n, ncomp=2, G=4.0, rho=rho)
    c0 = obs.conserved(s)
    s.run(5)
    c1 = obs.conserved(s)
    assert np.allclose(c1["mass"], c0["mass"], rtol=1e-14)
    assert np.abs(np.array(c1["momentum"])).max() < 1e-12


def test_wall_moving_with_fluid_keeps_equilibrium():
    """Halfway bounce-back with the moving-wall term 6 w_q rho c_q.V (Sec. II.E):
    a uniform fluid moving with the colloid's velocity stays exactly at its
    equilibrium on every link."""
    n = 12
    U = np.array([0.02, -0.01, 0.015])
    p = synth.Params(nx=n, ny=n, nz=n, ncomp=1, nions=0, prec="fp64", G=0.0, ncolloid_max=1)
    u = np.broadcast_to(U[:, None, None, None], (3, n, n, n)).copy()
    s = OracleSystem(p, np.ones((1, n, n, n)), u=u, colloid_x=[[5.3, 6.1, 5.7]],
                     colloid_v=[U], colloid_q=[0.0], colloid_r=[3.2])
    s.step()
    feq = equilibrium(np.ones((n, n, n)), u)
    fl = s.fluid
    for q in range(Q):
        assert np.allclose(s.f[0, q][fl], feq[q][fl], rtol=0, atol=1e-15)


def test_virtual_density_brute_force():
    rng = np.random.default_rng(2)
    n = 6
    solid = rng.uniform(size=(n, n, n)) < 0.3
    rho = rng.uniform(0.1, 1.0, size=(2, n, n, n))
    surface = geometry.surface_nodes(solid)
    rv = virtual_density(rho, solid, surface)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                if not solid[z, y, x]:
                    assert np.array_equal(rv[:, z, y, x], rho[:, z, y, x])
                    continue
                vals = []
                for q in range(1, Q):
                    xx, yy, zz = (x + C[q, 0]) % n, (y + C[q, 1]) % n, (z + C[q, 2]) % n
                    if not solid[zz, yy, xx]:
                        vals.append(rho[:, zz, yy, xx])
                if surface[z, y, x]:
                    assert vals
                    assert np.allclose(rv[:, z, y, x], np.mean(vals, axis=0), rtol=1e-14)
                else:
                    assert not vals
                    assert (rv[:, z, y, x] == 0).all()


# ---------------------------------------------------------------- ions
def _mode(shape, k):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return 2 * math.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz)


def test_np_pure_diffusion_fourier_mode_exact():
    """With psi_f = 1, u = 0, E = 0, dmu = 0 the face-flux update is
    n <- n + D Lap_7 n, so a Fourier mode is multiplied exactly by
    1 - D sum_a 2 (1 - cos k_a) (Sec. II.B eq. nernst-planck-disc,
    ionic-fluxes-disc)."""
    shape = (8, 12, 10)
    k = (1, 2, 3)
    th = _mode(shape, k)
    D = 0.05
    n = np.stack([0.01 + 1e-3 * np.cos(th), 0.01 + 2e-3 * np.cos(th)])
    F = face_fluxes(n, np.ones(shape), np.zeros((3,) + shape), np.zeros(shape), D, (0, 0), 1.0)
    n1 = np_update(n, F, np.zeros((3,) + shape), np.ones(shape, dtype=bool))
    g = 1.0 - D * sum(2 * (1 - math.cos(2 * math.pi * k[a] / shape[2 - a])) for a in range(3))
    assert np.allclose(n1[0], 0.01 + g * 1e-3 * np.cos(th), rtol=0, atol=1e-17)
    assert np.allclose(n1[1], 0.01 + g * 2e-3 * np.cos(th), rtol=0, atol=1e-17)


def test_np_drift_symbol_exact():
    """Uniform field E along x: the linear update multiplies exp(i k x) by
    1 + D[2(cos k - 1) - i z E sin k]; cations drift along +E (Sec. II.B eq.
    electric_ion_force with F = q grad phi = -z n E)."""
    shape = (4, 4, 16)
    kx = 2 * math.pi * 3 / 16
    x = np.arange(16)
    D, E = 0.05, 0.2
    base = np.cos(kx * x)[None, None, :] * np.ones(shape)
    n0 = 0.01 + 1e-3 * base
    n = np.stack([n0, n0])
    Ef = np.zeros((3,) + shape)
    Ef[0] = E
    F = face_fluxes(n, np.ones(shape), Ef, np.zeros(shape), D, (0, 0), 1.0)
    n1 = np_update(n, F, np.zeros((3,) + shape), np.ones(shape, dtype=bool))
    for s, z in ((0, 1.0), (1, -1.0)):
        mult = 1 + D * (2 * (math.cos(kx) - 1) - 1j * z * E * math.sin(kx))
        ref = 0.01 + 1e-3 * np.real(mult * np.exp(1j * kx * x))
        assert np.allclose(n1[s][0, 0], ref, rtol=0, atol=1e-17)
    # uniform background carries no divergence
    assert abs(n1[0].mean() - 0.01) < 1e-17


def test_np_solvation_steady_state_and_partition():
    """Steady state of diffusion + solvation (E = 0) across a fixed smooth
    interface of rho_a: on every face the discrete zero-flux relation
    n~_{i+1}/n~_i = (1 + b/2)/(1 - b/2), b = (dmu/drho_a)(rho_a(i+1)-rho_a(i)),
    holds exactly, and the bulk ratio approaches n_b/n_a = exp(-dmu)
    (Sec. III.A initial salt ratio, Sec. II.C eq. solvation_potential)."""
    nx = 64
    shape = (1, 1, nx)
    x = np.arange(nx)
    ra_hi, ra_lo = 0.7, 0.04
    prof = ra_lo + (ra_hi - ra_lo) * 0.5 * (np.tanh((x - 16) / 3.0) - np.tanh((x - 48) / 3.0))
    rho_a = np.broadcast_to(prof, shape).copy()
    drho = ra_hi - ra_lo
    dmu = (2.0, 2.0)
    D = 0.2
    n = np.full((2,) + shape, 0.01)
    zero = np.zeros((3,) + shape)
    one = np.ones(shape)
    fl = np.ones(shape, dtype=bool)
    for _ in range(20000):
        F = face_fluxes(n, one, zero, rho_a, D, dmu, drho)
        n = np_update(n, F, zero, fl)
    F = face_fluxes(n, one, zero, rho_a, D, dmu, drho)
    assert np.abs(F).max() < 1e-14
    b = (dmu[0] / drho) * (np.roll(prof, -1) - prof)
    ratio = np.roll(n[0, 0, 0], -1) / n[0, 0, 0]
    assert np.allclose(ratio, (1 + b / 2) / (1 - b / 2), rtol=1e-9)
    n_a = n[0, 0, 0, 32]   # rho_a high: phase a
    n_b = n[0, 0, 0, 0]    # rho_a low: phase b
    assert n_b / n_a == pytest.approx(math.exp(-dmu[0]), rel=0.03)


def test_np_update_conserves_ions_with_advection_and_solids():
    rng = np.random.default_rng(3)
    shape = (6, 7, 8)
    solid = rng.uniform(size=shape) < 0.2
    fl = ~solid
    psi_f = np.where(fl, rng.uniform(0.3, 1.0, size=shape), 0.0)
    n = rng.uniform(0.0, 0.02, size=(2,) + shape) * fl
    E = rng.normal(0, 0.05, size=(3,) + shape)
    u = rng.normal(0, 0.05, size=(3,) + shape) * fl
    rho_a = rng.uniform(0.04, 0.7, size=shape)
    F = face_fluxes(n, psi_f, E, rho_a, 0.05, (1.5, -0.5), 0.66)
    n1 = np_update(n, F, u, fl)
    for s in range(2):
        assert n1[s].sum() == pytest.approx(n[s].sum(), rel=1e-14)
        assert (n1[s][solid] == 0).all()


def test_friction_total_equals_face_sum():
    """Newton's third law on the faces: sum_i F_fr(i) = -(1/(beta D)) sum_faces j."""
    rng = np.random.default_rng(4)
    shape = (5, 6, 7)
    F = rng.normal(size=(2, 3) + shape)
    D = 0.05
    Ffr = friction_force(F, D)
    for a in range(3):
        assert Ffr[a].sum() == pytest.approx(-F[:, a].sum() / D, rel=1e-12)


# ---------------------------------------------------------------- Poisson
def test_poisson_single_mode_exact():
    """Uniform eps and q = A cos(k.x): phi = q / (eps |lambda_k|) with the
    seven-point symbol lambda_k = -sum_a 2(1 - cos k_a) (Sec. II.D)."""
    shape = (8, 10, 12)
    k = (2, 1, 3)
    th = _mode(shape, k)
    q = 0.3 * np.cos(th)
    eps = np.full(shape, 0.2)
    phi, it, rr = poisson.solve(q, eps, tol=1e-14)
    lam = sum(2 * (1 - math.cos(2 * math.pi * k[a] / shape[2 - a])) for a in range(3))
    assert np.allclose(phi, q / (0.2 * lam), rtol=0, atol=1e-14)


def test_poisson_variable_eps_matches_sparse_direct():
    """Brute force: the oracle's iterative solution equals a sparse direct
    solve of the same seven-point flux-form system with a mean-zero constraint."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(6)
    shape = (4, 5, 6)
    N = int(np.prod(shape))
    eps = rng.uniform(0.1, 0.8, size=shape)
    q = rng.normal(size=shape)
    Eext = (0.01, 0.0, -0.02)
    phi, it, rr = poisson.solve(q, eps, tol=1e-13, max_iter=5000, E_ext=Eext)
    idx = np.arange(N).reshape(shape)
    rows, cols, vals = [], [], []
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                i = idx[z, y, x]
                for a in range(3):
                    for sgn in (1, -1):
                        d = [0, 0, 0]
                        d[a] = sgn
                        xx, yy, zz = (x + d[0]) % shape[2], (y + d[1]) % shape[1], (z + d[2]) % shape[0]
                        e = 0.5 * (eps[z, y, x] + eps[zz, yy, xx])
                        j = idx[zz, yy, xx]
                        rows += [i, i]
                        cols += [j, i]
                        vals += [e, -e]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    b = -(q - q.mean()).ravel()
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                i = idx[z, y, x]
                for a in range(3):
                    if Eext[a] == 0:
                        continue
                    for sgn in (1, -1):
                        d = [0, 0, 0]
                        d[a] = sgn
                        xx, yy, zz = (x + d[0]) % shape[2], (y + d[1]) % shape[1], (z + d[2]) % shape[0]
                        b[i] += 0.5 * (eps[z, y, x] + eps[zz, yy, xx]) * Eext[a] * sgn
    Aaug = sp.vstack([sp.hstack([A, sp.csr_matrix(np.ones((N, 1)))]),
                      sp.csr_matrix(np.concatenate([np.ones(N), [0.0]])[None, :])]).tocsc()
    sol = spla.spsolve(Aaug, np.concatenate([b, [0.0]]))[:N].reshape(shape)
    assert np.allclose(phi, sol, rtol=0, atol=1e-11 * np.abs(sol).max())


def test_poisson_layered_dielectric_harmonic_mean():
    """Ion-free layered dielectric eps(z) in an applied field E along z: the
    displacement eps_face (E - dphi/dz) is uniform and equals E nz / sum(1/eps_face)
    (series capacitors); the field is E_z = D / eps (Sec. II.B, polarised by the
    applied field)."""
    nz = 16
    z = np.arange(nz)
    ez = 0.1 + 0.05 * np.sin(2 * math.pi * z / nz) + 0.02 * (z % 3)
    shape = (nz, 3, 2)
    eps = np.broadcast_to(ez[:, None, None], shape).copy()
    E = 0.01
    phi, it, rr = poisson.solve(np.zeros(shape), eps, tol=1e-14, max_iter=10000, E_ext=(0, 0, E))
    ef = 0.5 * (ez + np.roll(ez, -1))
    Dz = ef * (E - (np.roll(phi[:, 0, 0], -1) - phi[:, 0, 0]))
    assert np.allclose(Dz, E * nz / (1.0 / ef).sum(), rtol=1e-11)


def test_electric_field_central_difference_exact():
    shape = (6, 8, 10)
    th = _mode(shape, (1, 0, 0))
    phi = 0.5 * np.sin(th)
    E = electric_field(phi, (0.0, 1e-3, 0.0))
    k = 2 * math.pi / 10
    assert np.allclose(E[0], -0.5 * np.cos(th) * math.sin(k), atol=1e-15)
    assert np.allclose(E[1], 1e-3, atol=1e-18)


# ---------------------------------------------------------------- geometry
def _brute_project(nx, ny, nz, X, R, h):
    solid = np.zeros((nz, ny, nx), dtype=bool)
    psi = np.zeros((nz, ny, nx))
    offs = [(k + 0.5) / (h + 1) - 0.5 for k in range(h + 1)]
    dims = (nx, ny, nz)

    def d2(p, c):
        s = 0.0
        for a in range(3):
            d = p[a] - c[a]
            if d > 0.5 * dims[a]:
                d -= dims[a]
            elif d < -0.5 * dims[a]:
                d += dims[a]
            s = s + d * d if a else d * d
        return s

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for c, r in zip(X, R):
                    if d2((float(x), float(y), float(z)), c) < r * r:
                        solid[z, y, x] = True
                    cnt = 0
                    for oz in offs:
                        for oy in offs:
                            for ox in offs:
                                if d2((x + ox, y + oy, z + oz), c) < r * r:
                                    cnt += 1
                    psi[z, y, x] += cnt / (h + 1) ** 3
    return solid, np.minimum(psi, 1.0)


def test_boxed_projection_equals_whole_lattice_projection():
    """project_boxed (bounding boxes only) gives the same mask, owners and
    solid fractions bit for bit, with spheres wrapping every face, touching
    and overlapping spheres, and radii with sub-cube samples on the sphere."""
    rng = np.random.default_rng(9)
    nx, ny, nz = 18, 15, 21
    X = np.array([[0.4, 14.7, 10.0], [17.2, 7.5, 0.3], [9.0, 7.5, 20.6], [9.0, 7.5, 12.0], [11.5, 8.0, 12.25]])
    X = np.vstack([X, rng.uniform(0, 1, size=(4, 3)) * [nx, ny, nz]])
    R = np.array([3.2, 2.7, 4.0, 2.5, 2.5, 1.9, 3.375, 2.0, 4.5])
    for h in (1, 3):
        a = geometry.project(nx, ny, nz, X, R, h)
        b = geometry.project_boxed(nx, ny, nz, X, R, h)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)


def test_geometry_matches_brute_force_bit_exact():
    X = np.array([[1.3, 7.9, 4.25], [8.0, 3.0, 9.5]])   # first one wraps in x and y
    R = np.array([3.1, 2.5])
    nx, ny, nz = 12, 11, 13
    solid, owner, psi = geometry.project(nx, ny, nz, X, R, 3)
    s2, p2 = _brute_project(nx, ny, nz, X, R, 3)
    assert np.array_equal(solid, s2)
    assert np.array_equal(psi, p2)
    # every interior solid node is fully covered
    surf = geometry.surface_nodes(solid)
    assert (psi[solid & ~surf] == 1.0).all()
    assert (psi[~solid] < 1.0).all()


def test_solid_fraction_converges_to_sphere_volume():
    X = np.array([[10.2, 10.7, 9.9]])
    R = np.array([5.0])
    vol = 4.0 / 3.0 * math.pi * 125.0
    errs = []
    for h in (1, 3, 7):
        _, _, psi = geometry.project(20, 20, 20, X, R, h)
        errs.append(abs(psi.sum() - vol) / vol)
    assert errs[1] < 0.01 and errs[2] < 0.005
    assert errs[2] <= errs[0]


def test_surface_charge_sums_to_Q_and_links_brute_force():
    X = np.array([[6.0, 6.0, 5.5]])
    R = np.array([3.0])
    solid, owner, psi = geometry.project(12, 12, 12, X, R, 3)
    surf = geometry.surface_nodes(solid)
    qc = geometry.colloid_charge(owner, surf, [-20.0])
    assert qc.sum() == pytest.approx(-20.0, rel=1e-14)
    links = geometry.boundary_links(solid, owner)
    brute = []
    n = 12
    for z in range(n):
        for y in range(n):
            for x in range(n):
                if solid[z, y, x]:
                    continue
                for q in range(1, Q):
                    xx, yy, zz = (x + C[q, 0]) % n, (y + C[q, 1]) % n, (z + C[q, 2]) % n
                    if solid[zz, yy, xx]:
                        brute.append(((z * n + y) * n + x, q, 0))
    assert links == sorted(brute)


# ---------------------------------------------------------------- whole step
def test_coupled_step_conserves_mass_ions_charge_with_fixed_colloid():
    w = synth.two_slab(nx=12, ny=12, nz=12, G=4.0)
    w.colloid_x[:] = [[6.0, 6.0, 5.5]]
    w.colloid_r[:] = [3.0]
    s = OracleSystem(w.params, w.rho, w.n, None, w.colloid_x, w.colloid_v, w.colloid_q, w.colloid_r)
    c0 = obs.conserved(s)
    s.run(4)
    c1 = obs.conserved(s)
    assert np.allclose(c1["mass"], c0["mass"], rtol=1e-14)
    assert np.allclose(c1["ions"], c0["ions"], rtol=1e-14)
    assert abs(c1["charge"]) < 1e-12
    assert s.poisson_relres < w.params.poisson_tol


# ---------------------------------------------------------------- moving colloids
def _moving_system(n=16, V=(0.03, -0.02, 0.01), nions=0, Q=0.0, E=(0.0, 0.0, 0.0), X=(7.45, 8.2, 7.9)):
    p = synth.Params(nx=n, ny=n, nz=n, ncomp=1, nions=nions, prec="fp64", G=0.0, ncolloid_max=1,
                     colloids_move=1, poisson_tol=1e-12, poisson_max_iter=500, E_ext=E, eps_r=(1.0, 1.0))
    kw = {"n": np.full((2, n, n, n), 0.01)} if nions else {}
    return OracleSystem(p, np.ones((1, n, n, n)), colloid_x=[list(X)], colloid_v=[list(V)],
                        colloid_q=[Q], colloid_r=[3.0], **kw)


def _total_momentum(s):
    c = obs.conserved(s)
    return np.array(c["momentum"]) + (s.cmass[:, None] * s.cv).sum(axis=0)


def test_moving_colloid_conserves_total_momentum_across_remaps():
    """Bounce-back exchange, node covering (fluid momentum to the colloid) and
    uncovering (refill momentum from the colloid) with velocity-Verlet keep
    fluid + colloid momentum constant to round-off (Sec. II.E); the colloid
    crosses lattice nodes during the run so both conversions occur."""
    s = _moving_system(V=(0.2, -0.15, 0.1))
    p0 = _total_momentum(s)
    solid0 = s.solid.copy()
    for _ in range(6):
        s.step()
    assert not np.array_equal(solid0, s.solid)   # nodes were created and deleted
    assert np.allclose(_total_momentum(s), p0, rtol=0, atol=1e-12)


def test_moving_colloid_remap_conserves_ions():
    s = _moving_system(V=(0.2, 0.1, -0.1), nions=2)
    n0 = s.n.sum(axis=(1, 2, 3))
    for _ in range(6):
        s.step()
    assert np.allclose(s.n.sum(axis=(1, 2, 3)), n0, rtol=1e-13)
    assert (s.n[:, s.solid] == 0).all()


def test_moving_colloid_is_dragged_by_the_fluid():
    s = _moving_system(V=(0.02, 0.0, 0.0))
    v0 = s.cv[0, 0]
    s.run(10)
    assert 0.0 < s.cv[0, 0] < v0          # decelerates, does not reverse
    assert abs(s.cv[0, 1]) < 1e-3 * v0


def test_negative_colloid_drifts_against_the_field():
    """Electric force sum q_c E on the surface nodes (Sec. II.E): a negatively
    charged colloid at rest in salt accelerates against the applied field."""
    s = _moving_system(V=(0.0, 0.0, 0.0), nions=2, Q=-5.0, E=(1e-3, 0.0, 0.0))
    s.n[0][s.fluid] += 5.0 / s.fluid.sum()   # neutralise with counter-cations
    s.run(3)
    assert s.cv[0, 0] < 0.0
