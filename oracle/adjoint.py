"""Discrete adjoint of the IBM step for the oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/ (never by the product path).

The forward map here is the oracle's discrete step (ibm_oracle.c) restated
with plain PyTorch FP64 CPU tensor operations, in the same order:

  ghost fill (boundary maps) -> primitives (rho, u.., p), T = p/(rho r)
  -> face fluxes (MUSCL with the van Leer limiter, Rusanov, central viscous
     stress and heat flux, Sutherland viscosity; Sec. 2.1 and the scheme
     readings) -> L(U) -> SSP-RK2 predictor with a given dt (App. B step 1)
  -> interpolation and direct forcing G = dt F = rho_L U_b - I[rho u],
     H = dt Q = rho_L c_v T_w - I[rho e] (Eqs. interp, forceMomentum,
     corr3.8) -> spreading with the quadrature weights eps~ = A~^{-1} 1
     (Eq. force2, Sec. 2.2) and the forced update of the band cells
     (App. B, Eqs. u_centralF2 and e_centralF2)
  -> after the last step J = dJ_dCd * C_d + dJ_dNu * Nu from the marker sums
     (Eq. Bulk; C_d and Nu as in the oracle's forces).

Reverse-mode automatic differentiation of that map gives the exact discrete
gradient of J with respect to the marker positions X and wall temperatures
T_w, under the conventions the CUDA adjoint states: the step sizes are held
fixed at the values of the forward run, the owner cells (bins) and the set of
kept markers do not move, and the limiter and max/abs kinks take the branch
of the forward evaluation.  The quadrature weights are differentiated
through a dense solve of A~ eps~ = 1.

Pins (tests/test_oracle_adjoint.py): the forward states equal the C
oracle's to round-off, and the gradient equals central finite differences
of the C oracle's J.
"""
from __future__ import annotations

import numpy as np
import torch

from . import oracle as O

_F64 = torch.float64

# largest fraction of a forced cell's internal energy the heat source removes
# in one step (the C oracle's HEAT_SOURCE_CAP)
HEAT_SOURCE_CAP = 0.9


# ---------------------------------------------------------------------------
# grid bookkeeping (integer index maps, no arithmetic of the method)
# ---------------------------------------------------------------------------

def _pad(g):
    return [g.n[d] + 4 if d < g.dim else 1 for d in range(3)]


def _strides(g):
    P = _pad(g)
    return [1, P[0], P[0] * P[1]]


def _map_axis(g, d, idx):
    """interior source of a padded index along axis d: (src, flip, freestream)"""
    n = g.n[d]
    if 0 <= idx < n:
        return idx, 0, 0
    bc = g.bc[2 * d] if idx < 0 else g.bc[2 * d + 1]
    if bc == 0:                       # free stream
        return (0 if idx < 0 else n - 1), 0, 1
    if bc == 1:                       # zero gradient
        return (0 if idx < 0 else n - 1), 0, 0
    if bc == 2:                       # slip wall: mirror, normal velocity flips
        return (-1 - idx if idx < 0 else 2 * n - 1 - idx), 1 << d, 0
    return idx % n, 0, 0              # periodic


class Maps:
    """Ghost-fill gather map of the padded grid and the face index sets."""

    def __init__(self, g):
        self.g = g
        P = _pad(g)
        Np = P[0] * P[1] * P[2]
        nc = g.dim + 2
        src = np.zeros(Np, dtype=np.int64)
        sign = np.ones((nc, Np))
        fs = np.zeros(Np, dtype=bool)
        for q in range(Np):
            pq = (q % P[0], (q // P[0]) % P[1], q // (P[0] * P[1]))
            s = [0, 0, 0]
            flip = 0
            f = 0
            for d in range(g.dim):
                s[d], fl, ff = _map_axis(g, d, pq[d] - 2)
                flip ^= fl
                f |= ff
            src[q] = s[0] + g.n[0] * (s[1] + g.n[1] * s[2])
            fs[q] = bool(f)
            for d in range(g.dim):
                if flip & (1 << d):
                    sign[1 + d, q] = -1.0
        self.src = torch.from_numpy(src)
        self.sign = torch.from_numpy(sign)
        self.fs = torch.from_numpy(fs)
        self.Np = Np
        st = _strides(g)
        self.strides = st
        nz = g.n[2] if g.dim == 3 else 1
        i0, i1, i2 = np.meshgrid(np.arange(g.n[0]), np.arange(g.n[1]), np.arange(nz),
                                 indexing="ij")
        # interior cells in storage order (x fastest)
        i0 = i0.transpose(2, 1, 0).ravel()
        i1 = i1.transpose(2, 1, 0).ravel()
        i2 = i2.transpose(2, 1, 0).ravel()
        a = (i0 + 2) + st[1] * (i1 + 2) + st[2] * ((i2 + 2) if g.dim == 3 else 0)
        self.interior = torch.from_numpy(a.astype(np.int64))


def freestream_state(g):
    p = 1.0 / (g.gamma * g.Mach * g.Mach)
    u = [1.0] + [1.0 if d == 0 else 0.0 for d in range(g.dim)] + [p / (g.gamma - 1.0) + 0.5]
    return torch.tensor(u, dtype=_F64)


def gas_R(g):
    return 1.0 / (g.gamma * g.Mach * g.Mach)


def gas_cv(g):
    return gas_R(g) / (g.gamma - 1.0)


def gas_cp(g):
    return g.gamma * gas_cv(g)


# ---------------------------------------------------------------------------
# fluid operator
# ---------------------------------------------------------------------------

def fill_ghosts(g, U, maps):
    """U: (nc, N) -> padded conserved state (nc, Np)"""
    Uinf = freestream_state(g)
    gathered = U[:, maps.src] * maps.sign
    return torch.where(maps.fs.unsqueeze(0), Uinf.unsqueeze(1).expand_as(gathered), gathered)


def primitives(g, Pd):
    dim = g.dim
    rho = Pd[0]
    vel = [Pd[1 + d] / rho for d in range(dim)]
    ke = sum(v * v for v in vel)
    p = (g.gamma - 1.0) * (Pd[dim + 1] - 0.5 * rho * ke)
    W = torch.stack([rho] + vel + [p])
    T = p / (rho * gas_R(g))
    return W, T


def van_leer(a, b):
    ab = a * b
    pos = ab > 0.0
    den = torch.where(pos, a + b, torch.ones_like(a))
    return torch.where(pos, 2.0 * ab / den, torch.zeros_like(a))


def viscosity(g, T):
    if g.Re <= 0.0:
        return torch.zeros_like(T)
    return (1.0 / g.Re) * T ** 1.5 * (1.0 + g.sutherland_S) / (T + g.sutherland_S)


def face_flux(g, W, T, a, d, st):
    """Fhat (nc, nfaces) through the faces between padded cells a and a + s_d"""
    dim = g.dim
    nw = dim + 2
    s = st[d]
    b = a + s
    wl, wr = [], []
    for m in range(nw):
        wa, wb, wam, wbp = W[m, a], W[m, b], W[m, a - s], W[m, b + s]
        wl.append(wa + 0.5 * van_leer(wa - wam, wb - wa))
        wr.append(wb - 0.5 * van_leer(wb - wa, wbp - wb))

    def euler(w):
        rho, p = w[0], w[dim + 1]
        ke = sum(w[1 + m] * w[1 + m] for m in range(dim))
        E = p / (g.gamma - 1.0) + 0.5 * rho * ke
        un = w[1 + d]
        Uc = [rho] + [rho * w[1 + m] for m in range(dim)] + [E]
        F = [rho * un] + [rho * w[1 + m] * un + (p if m == d else 0.0) for m in range(dim)] + \
            [(E + p) * un]
        return Uc, F

    UL, FL = euler(wl)
    UR, FR = euler(wr)
    cl = torch.sqrt(g.gamma * wl[dim + 1] / wl[0])
    cr = torch.sqrt(g.gamma * wr[dim + 1] / wr[0])
    sl = torch.abs(wl[1 + d]) + cl
    sr = torch.abs(wr[1 + d]) + cr
    smax = torch.where(sl > sr, sl, sr)
    Fh = [0.5 * (FL[m] + FR[m]) - 0.5 * smax * (UR[m] - UL[m]) for m in range(nw)]
    if g.Re <= 0.0:
        return torch.stack(Fh)
    h = g.h
    Tf = 0.5 * (T[a] + T[b])
    mu = viscosity(g, Tf)
    lam = mu * gas_cp(g) / g.Pr
    grad = [[None] * dim for _ in range(dim)]
    for m in range(dim):
        um = W[1 + m]
        for e in range(dim):
            if e == d:
                grad[m][e] = (um[b] - um[a]) / h
            else:
                t = st[e]
                grad[m][e] = (um[a + t] - um[a - t] + um[b + t] - um[b - t]) / (4.0 * h)
    div = sum(grad[m][m] for m in range(dim))
    work = 0.0
    for m in range(dim):
        tau = mu * (grad[d][m] + grad[m][d])
        if m == d:
            tau = tau - (2.0 / 3.0) * mu * div
        uf = 0.5 * (W[1 + m, a] + W[1 + m, b])
        Fh[1 + m] = Fh[1 + m] - tau
        work = work + uf * tau
    Fh[dim + 1] = Fh[dim + 1] - (work + lam * (T[b] - T[a]) / h)
    return torch.stack(Fh)


def rhs(g, U, maps):
    """L(U) = -(1/h) sum_d (Fhat_{i+1/2} - Fhat_{i-1/2}), U and L (nc, N)"""
    Pd = fill_ghosts(g, U, maps)
    W, T = primitives(g, Pd)
    a = maps.interior
    L = 0.0
    for d in range(g.dim):
        s = maps.strides[d]
        Fhi = face_flux(g, W, T, a, d, maps.strides)
        Flo = face_flux(g, W, T, a - s, d, maps.strides)
        L = L - (Fhi - Flo) / g.h
    return L


def predictor(g, U, dt, maps):
    U1 = U + dt * rhs(g, U, maps)
    return 0.5 * U + 0.5 * (U1 + dt * rhs(g, U1, maps))


# ---------------------------------------------------------------------------
# markers
# ---------------------------------------------------------------------------

def phi(r):
    """regularised 3-point delta (Sec. 2.2); the inactive branch's square
    root is kept away from 0 so that its (discarded) derivative stays finite"""
    a = torch.abs(r)
    inner = (1.0 + torch.sqrt(torch.clamp(1.0 - 3.0 * a * a, min=1e-300))) / 3.0
    b = 1.0 - a
    outer = (5.0 - 3.0 * a - torch.sqrt(torch.clamp(1.0 - 3.0 * b * b, min=1e-300))) / 6.0
    return torch.where(a <= 0.5, inner, torch.where(a <= 1.5, outer, torch.zeros_like(a)))


class Support:
    """The 3^d support cells of every marker (owner cell +-1 per axis; the
    owner cells are fixed from the positions given at construction)."""

    def __init__(self, g, X):
        X = np.asarray(X, dtype=np.float64)
        self.g = g
        ns = len(X)
        own = np.floor((X - np.asarray(g.lo[: g.dim])) / g.h).astype(np.int64)
        offs = []
        zr = [-1, 0, 1] if g.dim == 3 else [0]
        for oz in zr:
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    offs.append((ox, oy, oz))
        offs = np.array(offs)[:, : g.dim]
        cells = own[:, None, :] + offs[None, :, :]                   # (ns, S, dim)
        c3 = np.zeros(cells.shape[:2] + (3,), dtype=np.int64)
        c3[..., : g.dim] = cells
        self.lin = torch.from_numpy(c3[..., 0] + g.n[0] * (c3[..., 1] + g.n[1] * c3[..., 2]))
        self.centres = torch.from_numpy(np.asarray(g.lo[: g.dim])[None, None, :] +
                                        (cells + 0.5) * g.h)
        self.ns = ns

    def weights(self, X):
        """Phi_k(j) for every support cell, (ns, S); differentiable in X"""
        r = (self.centres - X[:, None, :]) / self.g.h
        return torch.prod(phi(r), dim=2)


def quadrature(g, sup, Phi):
    """eps~ = A~^{-1} 1 with A~_kl = sum_j Phi_k(j) Phi_l(j) (dense solve)"""
    N = g.ncells
    B = torch.zeros(sup.ns, N, dtype=_F64)
    rows = torch.arange(sup.ns).unsqueeze(1).expand_as(sup.lin)
    B = B.index_put((rows.reshape(-1), sup.lin.reshape(-1)), Phi.reshape(-1), accumulate=True)
    A = B @ B.T
    return torch.linalg.solve(A, torch.ones(sup.ns, dtype=_F64))


def interp_force(g, sup, Phi, Ub, Tw, Us):
    dim = g.dim
    rho = Us[0]
    mom = Us[1: dim + 1]
    ke = (mom * mom).sum(0)
    rhoe = Us[dim + 1] - 0.5 * ke / rho
    fields = torch.cat([rho.unsqueeze(0), mom, rhoe.unsqueeze(0)])      # (dim+2, N)
    I = (Phi.unsqueeze(0) * fields[:, sup.lin]).sum(2)                 # (dim+2, ns)
    rk = I[0]
    G = rk.unsqueeze(1) * Ub - I[1: dim + 1].T                          # (ns, dim)
    H = rk * gas_cv(g) * Tw - I[dim + 1]
    return rk, G, H


def spread_apply(g, sup, Phi, eps, G, H, U, energy_reading=0):
    dim = g.dim
    N = g.ncells
    R = torch.cat([G, H.unsqueeze(1)], dim=1)                           # (ns, dim+1)
    contrib = (R * eps.unsqueeze(1)).unsqueeze(1) * Phi.unsqueeze(2)    # (ns, S, dim+1)
    r = torch.zeros(dim + 1, N, dtype=_F64)
    r = r.index_add(1, sup.lin.reshape(-1), contrib.reshape(-1, dim + 1).T)
    band = torch.zeros(N, dtype=torch.bool)
    band[sup.lin.reshape(-1)] = True
    rho = U[0]
    m0 = U[1: dim + 1]
    m1 = m0 + r[:dim]
    E = U[dim + 1]
    q = r[dim]
    # positivity reading of the forced update: the heat source removes at
    # most HEAT_SOURCE_CAP of the cell's internal energy in one step
    rhoe0 = E - 0.5 * (m0 * m0).sum(0) / rho
    q = torch.maximum(q, -HEAT_SOURCE_CAP * rhoe0)
    if energy_reading == 1:
        En = E + q
    else:
        En = (E - 0.5 * (m0 * m0).sum(0) / rho + q) + 0.5 * (m1 * m1).sum(0) / rho
    mom = torch.where(band.unsqueeze(0), m1, m0)
    En = torch.where(band, En, E)
    return torch.cat([rho.unsqueeze(0), mom, En.unsqueeze(0)])


def coefficients(g, eps, G, H, Tw, dt):
    """C_d, C_l, Nu and the heat rate from the marker sums (oracle forces)"""
    dim = g.dim
    hd = g.h ** dim
    f = [-hd * (eps * G[:, d] / dt).sum() for d in range(dim)]
    heat = hd * (eps * H / dt).sum()
    pi = np.pi
    lref = g.D if dim == 2 else pi * g.D * g.D / 4.0
    As = pi * g.D if dim == 2 else pi * g.D * g.D
    lam_inf = (1.0 / g.Re) * gas_cp(g) / g.Pr
    dT = Tw.mean() - 1.0
    return 2.0 * f[0] / lref, 2.0 * f[1] / lref, heat * g.D / (lam_inf * As * dT), heat


# ---------------------------------------------------------------------------
# the objective and its gradient
# ---------------------------------------------------------------------------

def run(g, X, Tw, U0, dts, Ub=None, energy_reading=0, sup=None, maps=None):
    """len(dts) steps from U0 with the given step sizes; returns the final
    state, the last step's marker forcing and the weights.  X, Tw tensors."""
    maps = maps or Maps(g)
    sup = sup or Support(g, X.detach().numpy())
    U = torch.as_tensor(np.asarray(U0, dtype=np.float64).reshape(g.ncomp, -1))
    Ubt = torch.zeros_like(X) if Ub is None else torch.as_tensor(Ub, dtype=_F64)
    Phi = sup.weights(X)
    eps = quadrature(g, sup, Phi)
    G = H = None
    for dt in dts:
        Us = predictor(g, U, float(dt), maps)
        _, G, H = interp_force(g, sup, Phi, Ubt, Tw, Us)
        U = spread_apply(g, sup, Phi, eps, G, H, Us, energy_reading)
    return U, G, H, eps


def objective(g, X, Tw, U0, dts, dJ_dCd, dJ_dNu, **kw):
    _, G, H, eps = run(g, X, Tw, U0, dts, **kw)
    Cd, _, Nu, _ = coefficients(g, eps, G, H, Tw, float(dts[-1]))
    return dJ_dCd * Cd + dJ_dNu * Nu


def gradient(g, X, Tw, U0, dts, dJ_dCd, dJ_dNu, **kw):
    """(J, dJ/dX (ns, dim), dJ/dTw (ns)) by reverse-mode differentiation"""
    Xt = torch.tensor(np.asarray(X, dtype=np.float64), requires_grad=True)
    Twt = torch.tensor(np.asarray(Tw, dtype=np.float64), requires_grad=True)
    J = objective(g, Xt, Twt, U0, dts, dJ_dCd, dJ_dNu, **kw)
    J.backward()
    return float(J.detach()), Xt.grad.numpy().copy(), Twt.grad.numpy().copy()


def rhs_vjp(g, U, v):
    """v^T dL/dU at U (the flux operator's transpose-Jacobian product)"""
    maps = Maps(g)
    Ut = torch.tensor(np.asarray(U, dtype=np.float64).reshape(g.ncomp, -1), requires_grad=True)
    L = rhs(g, Ut, maps)
    (L * torch.as_tensor(np.asarray(v, dtype=np.float64).reshape(g.ncomp, -1))).sum().backward()
    return Ut.grad.numpy().reshape(np.shape(U))


def objective_c(g, X, Tw, U0, dts, dJ_dCd, dJ_dNu, Ub=None, energy_reading=0):
    """The same J evaluated with the C oracle (FP64 loops): eps~ from a dense
    solve of the oracle's A~, then its steps with the given step sizes."""
    X = np.asarray(X, dtype=np.float64)
    Tw = np.asarray(Tw, dtype=np.float64)
    eps = np.linalg.solve(O.assemble_A_dense(g, X), np.ones(len(X)))
    U = np.asarray(U0, dtype=np.float64)
    G = H = None
    for dt in dts:
        _, U, G, H, _ = O.step(g, X, Ub, Tw, eps, U, dt_fixed=float(dt),
                               energy_reading=energy_reading)
    _, _, Cd, _, Nu = O.forces(g, eps, G, H, Tw, float(dts[-1]))
    return dJ_dCd * Cd + dJ_dNu * Nu
