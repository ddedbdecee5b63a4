"""Pins of the oracle's IBM operators (Sec. 2.2: Eqs. interp, force2, the
quadrature system A eps = 1, Eqs. forceMomentum and corr3.8; Sec. 3.1 marker
dedup) against brute force, exactness properties and identities that do not
depend on the oracle's own code paths."""
import itertools

import numpy as np
import pytest

from paper_2301_09349_gb300 import cases as C


def grid2(n=(16, 12), h=0.25, **kw):
    return C.small_grid(2, n, h=h, **kw)


def grid3(n=(10, 9, 8), h=0.5, **kw):
    return C.small_grid(3, n, h=h, tile=(4, 4, 4), **kw)


def centers(g):
    ax = [g.lo[d] + (np.arange(g.n[d]) + 0.5) * g.h for d in range(g.dim)]
    mesh = np.meshgrid(*ax, indexing="ij")
    # flatten in cell-linear order (x fastest)
    return [m.transpose(tuple(reversed(range(g.dim)))).ravel() for m in mesh]


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_interp_exact_on_multilinear_fields(oracle, g):
    X = C.random_markers(g, 7, seed=11)
    xc = centers(g)
    a = [0.7, -1.3, 2.1]
    f_aff = 0.3 + sum(a[d] * xc[d] for d in range(g.dim))
    f_bil = xc[0] * xc[1] * (xc[2] if g.dim == 3 else 1.0)
    I = oracle.interp(g, X, np.stack([f_aff, f_bil]))
    want_aff = 0.3 + sum(a[d] * X[:, d] for d in range(g.dim))
    want_bil = X[:, 0] * X[:, 1] * (X[:, 2] if g.dim == 3 else 1.0)
    np.testing.assert_allclose(I[:, 0], want_aff, rtol=0, atol=1e-13)
    np.testing.assert_allclose(I[:, 1], want_bil, rtol=0, atol=1e-13)


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_support_paths_match_brute_force(oracle, g):
    rng = np.random.Generator(np.random.PCG64(3))
    X = C.random_markers(g, 5, seed=12)
    f = rng.standard_normal((3, g.ncells))
    np.testing.assert_allclose(oracle.interp(g, X, f), oracle.interp(g, X, f, dense=True),
                               rtol=1e-15, atol=1e-15)
    eps = rng.random(5) + 0.5
    R = rng.standard_normal((5, 2))
    np.testing.assert_allclose(oracle.spread(g, X, eps, R), oracle.spread(g, X, eps, R, dense=True),
                               rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_interp_spread_adjoint(oracle, g):
    # <I u, F>_eps = <u, S F>_{h^d} with eps = h^d eps~
    rng = np.random.Generator(np.random.PCG64(4))
    X = C.random_markers(g, 9, seed=13)
    eps_t = rng.random(9) + 0.5
    u = rng.standard_normal((1, g.ncells))
    F = rng.standard_normal((9, 1))
    hd = g.h ** g.dim
    lhs = np.sum(hd * eps_t * F[:, 0] * oracle.interp(g, X, u)[:, 0])
    rhs = hd * np.sum(u[0] * oracle.spread(g, X, eps_t, F)[0])
    assert abs(lhs - rhs) <= 1e-14 * max(1.0, abs(lhs))


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_spreading_conserves_total(oracle, g):
    # h^d sum_j f_j = sum_k eps_k F_k  (sum_j Phi_k(j) = 1)
    rng = np.random.Generator(np.random.PCG64(5))
    X = C.random_markers(g, 6, seed=14)
    eps_t = rng.random(6) + 0.5
    F = rng.standard_normal((6, 2))
    f = oracle.spread(g, X, eps_t, F)
    np.testing.assert_allclose(f.sum(1), (eps_t[:, None] * F).sum(0), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_quadrature_isolated_marker(oracle, g):
    # one marker: A~ = prod_d sum_i phi^2 = 2^-d, so eps~ = 2^d exactly
    X = C.random_markers(g, 1, seed=15)
    rc, eps, it, res = oracle.quadrature(g, X)
    assert rc == 0
    assert abs(eps[0] - 2.0 ** g.dim) < 1e-13
    A = oracle.assemble_A_dense(g, X)
    assert abs(A[0, 0] - 0.5 ** g.dim) < 1e-15


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_quadrature_partition_of_unity(oracle, g):
    # I(S(1)) = 1 at every marker, computed through the dense operators
    X = C.random_markers(g, 6, seed=16)
    rc, keep = oracle.dedup(g, X)
    X = X[keep]
    rc, eps, it, res = oracle.quadrature(g, X, tol=1e-13)
    assert rc == 0
    ones = np.ones((len(X), 1))
    back = oracle.interp(g, X, oracle.spread(g, X, eps, ones, dense=True), dense=True)
    np.testing.assert_allclose(back[:, 0], 1.0, atol=1e-12)
    A = oracle.assemble_A_dense(g, X)
    np.testing.assert_allclose(A, A.T, atol=1e-16)
    np.testing.assert_allclose(A @ eps, 1.0, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(A) > 0)


def test_quadrature_cylinder_markers_dedup_makes_A_regular(oracle):
    c = C.heated_cylinder()
    A_all = oracle.assemble_A_dense(c.grid, c.X)
    assert np.linalg.eigvalsh(A_all).min() < 1e-10      # 100 markers on 84 support cells
    rc, keep = oracle.dedup(c.grid, c.X)
    assert rc == 0 and len(keep) == 30
    A = oracle.assemble_A_dense(c.grid, c.X[keep])
    assert np.linalg.eigvalsh(A).min() > 1e-4
    rc, eps, it, res = oracle.quadrature(c.grid, c.X[keep])
    assert rc == 0 and res <= 1e-12
    np.testing.assert_allclose(A @ eps, 1.0, atol=1e-11)


def _brute_dedup(g, X):
    best = {}
    for k, x in enumerate(X):
        cell = tuple(int(np.floor((x[d] - g.lo[d]) / g.h)) for d in range(g.dim))
        cen = np.array([g.lo[d] + (cell[d] + 0.5) * g.h for d in range(g.dim)])
        dist = float(np.sum((x - cen) ** 2))
        if cell not in best or dist < best[cell][0]:
            best[cell] = (dist, k)
    return sorted(v[1] for v in best.values())


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_dedup_matches_brute_force(oracle, g):
    X = C.random_markers(g, 400, seed=17)
    rc, keep = oracle.dedup(g, X)
    assert rc == 0
    assert list(keep) == _brute_dedup(g, X)


def test_dedup_tie_keeps_lowest_index(oracle):
    g = grid2()
    c = np.array([g.lo[0] + 5.5 * g.h, g.lo[1] + 5.5 * g.h])
    # exact binary fractions so the two distances tie exactly
    X = np.array([c + [0.0, 0.25 * g.h], c + [-0.25 * g.h, 0.0], c + [0.375 * g.h, 0.0]])
    X = X[[2, 1, 0]]
    rc, keep = oracle.dedup(g, X)
    assert list(keep) == [1]


def test_owner_cell_margin_is_rejected(oracle):
    g = grid2()
    X = np.array([[g.lo[0] + 1.5 * g.h, 0.0]])
    rc, _ = oracle.owner_cells(g, X)
    assert rc != 0
    X = np.array([[g.lo[0] + 2.0 * g.h, 0.0]])
    rc, _ = oracle.owner_cells(g, X)
    assert rc == 0


@pytest.mark.parametrize("g", [grid2(n=(37, 29), tile=(8, 8, 1)), grid3(n=(13, 11, 9))],
                         ids=["2d", "3d"])
def test_binning_matches_brute_force_sort(oracle, g):
    X = C.random_markers(g, 300, seed=18)
    rc, tile_off, perm, keys = oracle.bin_markers(g, X)
    assert rc == 0
    T = list(g.tile[: g.dim]) + [1] * (3 - g.dim)
    nt = [-(-g.n[d] // T[d]) if d < g.dim else 1 for d in range(3)]
    items = []
    for k, x in enumerate(X):
        c = [int(np.floor((x[d] - g.lo[d]) / g.h)) if d < g.dim else 0 for d in range(3)]
        tid = (c[0] // T[0]) + nt[0] * ((c[1] // T[1]) + nt[1] * (c[2] // T[2]))
        cin = (c[0] % T[0]) + T[0] * ((c[1] % T[1]) + T[1] * (c[2] % T[2]))
        items.append((tid, cin, k))
    items.sort()
    assert list(perm) == [k for _, _, k in items]
    counts = np.bincount([t for t, _, _ in items], minlength=nt[0] * nt[1] * nt[2])
    np.testing.assert_array_equal(np.diff(tile_off), counts)
    assert tile_off[0] == 0 and tile_off[-1] == len(X)


def _state(g, rho, u, T):
    """conserved state of a uniform (rho, u, T) gas; p = rho r T"""
    R = 1.0 / (g.gamma * g.Mach ** 2)
    N = g.ncells
    U = np.zeros((g.ncomp, N))
    U[0] = rho
    for d in range(g.dim):
        U[1 + d] = rho * u[d]
    U[-1] = rho * R * T / (g.gamma - 1.0) + 0.5 * rho * float(np.dot(u, u))
    return U


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_zero_forcing_body_at_rest_at_wall_temperature(oracle, g):
    X = C.random_markers(g, 5, seed=19)
    U = _state(g, 1.3, np.zeros(g.dim), 1.7)
    rhoL, G, H = oracle.interp_force(g, X, None, np.full(5, 1.7), U)
    assert np.abs(G).max() <= 1e-14
    assert np.abs(H).max() <= 1e-14 * 20


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_zero_forcing_comoving_body(oracle, g):
    V = np.array([0.4, -0.2, 0.3])[: g.dim]
    X = C.random_markers(g, 5, seed=20)
    U = _state(g, 0.9, V, 1.0)
    rhoL, G, H = oracle.interp_force(g, X, np.tile(V, (5, 1)), np.ones(5), U)
    assert np.abs(G).max() <= 1e-14
    assert np.abs(H).max() <= 1e-13


@pytest.mark.parametrize("g", [grid2(), grid3()], ids=["2d", "3d"])
def test_single_marker_forcing_hits_targets_exactly(oracle, g):
    # with one marker eps~ = 1/sum_j Phi^2, so I(S(.)) is the identity and the
    # interpolated velocity and temperature after the update are U_b and T_w
    rng = np.random.Generator(np.random.PCG64(21))
    X = C.random_markers(g, 1, seed=21)
    U = C.random_state(g, seed=22, amp=0.02).reshape(g.ncomp, -1)
    Ub = rng.standard_normal((1, g.dim)) * 0.1
    Tw = np.array([1.37])
    rc, eps, _, _ = oracle.quadrature(g, X)
    rhoL, G, H = oracle.interp_force(g, X, Ub, Tw, U)
    Un = oracle.spread_apply(g, X, eps, G, H, U)
    N = g.ncells
    ke = 0.5 * sum(Un[1 + d] ** 2 for d in range(g.dim)) / Un[0]
    rho_e = Un[-1] - ke
    I = oracle.interp(g, X, np.stack([Un[0]] + [Un[1 + d] for d in range(g.dim)] + [rho_e]))
    cv = (1.0 / (g.gamma * g.Mach ** 2)) / (g.gamma - 1.0)
    np.testing.assert_allclose(I[0, 1:1 + g.dim] / I[0, 0], Ub[0], atol=1e-13)
    np.testing.assert_allclose(I[0, -1] / I[0, 0] / cv, Tw[0], rtol=1e-13)
    np.testing.assert_array_equal(Un[0], U[0])     # mass is not forced


def test_band_only_update_and_energy_readings(oracle):
    g = grid2()
    X = C.random_markers(g, 3, seed=23)
    U = C.random_state(g, seed=24, amp=0.02).reshape(g.ncomp, -1)
    rc, eps, _, _ = oracle.quadrature(g, X)
    rhoL, G, H = oracle.interp_force(g, X, None, np.full(3, 1.5), U)
    cnt, mask = oracle.band_mask(g, X)
    assert cnt <= 3 * 9 and cnt == mask.sum()
    A = oracle.spread_apply(g, X, eps, G, H, U, energy_reading=0)
    B = oracle.spread_apply(g, X, eps, G, H, U, energy_reading=1)
    out = mask == 0
    np.testing.assert_array_equal(A[:, out], U[:, out])
    np.testing.assert_array_equal(B[:-1], A[:-1])
    # reading 1 adds the spread heat to total energy; reading 0 to internal
    # energy, so the two differ by the kinetic-energy change of the forcing
    ke = lambda V: 0.5 * (V[1] ** 2 + V[2] ** 2) / V[0]
    np.testing.assert_allclose(A[-1] - B[-1], ke(A) - ke(U), atol=1e-12)


def test_body_force_equals_momentum_given_to_fluid(oracle):
    c = C.heated_cylinder()
    g = c.grid
    run = oracle.Run(g, c.X, c.Tw)
    U0 = C.initial_state(g, c.seed).reshape(g.ncomp, -1)
    dt, Us = oracle.predictor(g, U0)
    rhoL, G, H = oracle.interp_force(g, run.X, None, run.Tw, Us)
    Un = oracle.spread_apply(g, run.X, run.eps, G, H, Us)
    f, heat, Cd, Cl, Nu = oracle.forces(g, run.eps, G, H, run.Tw, dt)
    hd = g.h ** 2
    dmom = hd * (Un[1:3] - Us[1:3]).sum(1) / dt
    np.testing.assert_allclose(f[:2], -dmom, rtol=1e-10)
    ke = lambda V: 0.5 * (V[1] ** 2 + V[2] ** 2) / V[0]
    de = hd * ((Un[-1] - ke(Un)) - (Us[-1] - ke(Us))).sum() / dt
    assert abs(heat - de) <= 1e-9 * abs(de)
    assert Cd == pytest.approx(2 * f[0] / g.D)


def test_motion_law(oracle):
    X0 = np.array([[0.5, 0.0], [0.0, 0.5]])
    X, Ub = oracle.motion(X0, 0.2, 0.2, 1, 0.7)
    s = 0.2 * np.sin(2 * np.pi * 0.2 * 0.7)
    np.testing.assert_allclose(X, X0 + [[0, s], [0, s]], atol=1e-15)
    e = 1e-6
    Xp, _ = oracle.motion(X0, 0.2, 0.2, 1, 0.7 + e)
    Xm, _ = oracle.motion(X0, 0.2, 0.2, 1, 0.7 - e)
    np.testing.assert_allclose(Ub, (Xp - Xm) / (2 * e), atol=1e-9)


# ---------------------------------------------------------------------------
# variant: forcing after each SSP-RK2 stage
# ---------------------------------------------------------------------------

def test_per_stage_forcing_single_marker_hits_targets_exactly(oracle):
    """the last stage's forcing with one marker makes I[u] = U_b, I[T] = T_w"""
    import dataclasses
    g = dataclasses.replace(grid2(), forcing_per_stage=1)
    X = C.random_markers(g, 1, seed=31)
    U = C.random_state(g, seed=32, amp=0.02)
    Ub = np.array([[0.05, -0.02]])
    Tw = np.array([1.21])
    rc, eps, _, _ = oracle.quadrature(g, X)
    dt, Un, G, H, rhoL = oracle.step(g, X, Ub, Tw, eps, U)
    Un = Un.reshape(g.ncomp, -1)
    rho_e = Un[-1] - 0.5 * (Un[1] ** 2 + Un[2] ** 2) / Un[0]
    I = oracle.interp(g, X, np.stack([Un[0], Un[1], Un[2], rho_e]))
    cv = (1.0 / (g.gamma * g.Mach ** 2)) / (g.gamma - 1.0)
    np.testing.assert_allclose(I[0, 1:3] / I[0, 0], Ub[0], atol=1e-13)
    np.testing.assert_allclose(I[0, 3] / I[0, 0] / cv, Tw[0], rtol=1e-13)
    # and it differs from the once-per-step variant
    _, Ud, _, _, _ = oracle.step(g, X, Ub, Tw, eps, U)
    g0 = dataclasses.replace(g, forcing_per_stage=0)
    _, U0, _, _, _ = oracle.step(g0, X, Ub, Tw, eps, U)
    assert np.abs(Ud - U0).max() > 1e-8


def test_per_stage_forcing_reported_force_is_the_momentum_given(oracle):
    """With periodic boundaries sum_j L_j = 0, so the momentum the step adds
    is h^d (sum f1 / 2 + sum f2): the body force of the step's sources
    G = G1/2 + G2 must be minus that over dt (conservation, not a retyping)."""
    import dataclasses
    g = dataclasses.replace(grid2(n=(24, 20), h=0.125, bc=(C.BC_PERIODIC,) * 6, Re=50.0),
                            forcing_per_stage=1)
    X = C.circle_markers(12, 0.4, (0.01, 0.02))
    rc, keep = oracle.dedup(g, X)
    X = X[keep]
    Tw = np.full(len(X), 1.3)
    rc, eps, _, _ = oracle.quadrature(g, X)
    U = C.random_state(g, seed=33, amp=0.02)
    dt, Un, G, H, rhoL = oracle.step(g, X, None, Tw, eps, U)
    f, heat, Cd, Cl, Nu = oracle.forces(g, eps, G, H, Tw, dt)
    hd = g.h ** 2
    dmom = hd * (Un.reshape(4, -1)[1:3] - U.reshape(4, -1)[1:3]).sum(1) / dt
    np.testing.assert_allclose(f[:2], -dmom, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_band_is_the_union_of_the_marker_supports(oracle, dim):
    """The forced cells (the oracle's cell-centric band mask: cells with a
    marker whose owner cell is within one cell per axis) are exactly the
    union of the markers' 3^d support cells around their owner cells - the
    marker-centric set the GPU scatters - and every marker reaches 3^d cells
    (the bound that sizes the spreading operator)."""
    n = (40, 36, 28)[:dim]
    g = C.small_grid(dim, n, h=0.1, fp_bytes=8)
    X = C.random_markers(g, 60, seed=71)
    cnt, mask = oracle.band_mask(g, X)
    lo = np.array(g.lo[:dim])
    owner = np.floor((X - lo) / g.h).astype(int)
    ref = np.zeros(tuple(reversed(n)), dtype=np.uint8)
    pairs = 0
    for c in owner:
        for off in np.ndindex(*(3,) * dim):
            cell = c + np.array(off) - 1
            if np.all(cell >= 0) and np.all(cell < np.array(n)):
                ref[tuple(reversed(cell))] = 1
                pairs += 1
    np.testing.assert_array_equal(mask, ref.reshape(-1))
    assert cnt == ref.sum()
    assert pairs == len(X) * 3 ** dim      # markers lie at least two cells inside
