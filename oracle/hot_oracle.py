"""FP64 CPU oracle for the HOT implicit MPM step.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this module.  The CUDA
library never calls it and shares no code with it.

A plain, slow restatement of Wang et al., "Hierarchical Optimization Time
Integration for CFL-rate MPM Stepping" (HOT), in numpy/scipy float64:

* Sec. 3.1 step sequence: P2G (APIC), grid time step, G2P, strain update,
  advection.
* Eq. 1 incremental potential E(dv), its gradient (the nodal force of
  Sec. 4.1) and its Hessian, projected per particle to PSD (Teran et al.
  2005, as used by Alg. 1 and Alg. 3).
* Sec. 4.1 node-embedding restriction R = (dx^0/dx^1)^T, prolongation
  P = R^T and Galerkin coarsening H^{m+1} = R H^m P (Eq. "buildMultigrid"),
  with the linear embedding kernel of Sec. 4.2.
* Alg. 2 V-cycle: colored symmetric Gauss-Seidel smoothing, coarsest level
  Jacobi-preconditioned CG with the adaptive tolerance of Sec. 5.3.
* Alg. 3 HOT: L-BFGS (window w) with the V-cycle as initial inverse Hessian,
  backtracking line search, node-wise characteristic-norm termination
  (Sec. 5.2, Eq. "nodewiseCN").
* Alg. 1 inexact projected Newton, the paper's comparison solvers: PN-PCG
  (Jacobi-preconditioned CG) and PN-MGPCG (one V-cycle of a hierarchy
  rebuilt every Newton iteration as the preconditioner, Sec. 4.3), both with
  the inexact criterion of Sec. 5.3.

Readings of silent or garbled passages are marked READING and listed in the
design notes; every function says which passage it follows.  Library
primitives used as steps: numpy SVD/eigh/solve, scipy.sparse products.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

LEVI = np.zeros((3, 3, 3))
LEVI[0, 1, 2] = LEVI[1, 2, 0] = LEVI[2, 0, 1] = 1.0
LEVI[0, 2, 1] = LEVI[2, 1, 0] = LEVI[1, 0, 2] = -1.0

# 3^3 stencil offsets in (z, y, x)-major order: offset k = (kx, ky, kz) with
# k = kx + 3 ky + 9 kz.
STENCIL = np.array([(kx, ky, kz) for kz in range(3) for ky in range(3) for kx in range(3)],
                   dtype=np.int64)

WALL_NODES = 3   # nodes within 3 cells of the domain boundary are held (READING)


# --------------------------------------------------------------------------
# Sec. 3.1 / Sec. 6 "Sparse matrix storage": quadratic B-spline kernel
# --------------------------------------------------------------------------
def bspline_N(t):
    """Quadratic B-spline N(t): 3/4 - t^2 for |t| < 1/2,
    (3/2 - |t|)^2 / 2 for 1/2 <= |t| < 3/2, else 0."""
    a = np.abs(t)
    return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def bspline_dN(t):
    """dN/dt of the quadratic B-spline."""
    a = np.abs(t)
    return np.where(a < 0.5, -2.0 * t, np.where(a < 1.5, -np.sign(t) * (1.5 - a), 0.0))


def base_node(x, origin, dx):
    """Lowest node of a particle's 3^3 stencil: floor((x - o)/dx - 1/2), with
    1/dx formed once and each operation rounded separately (no FMA)."""
    inv_dx = 1.0 / dx
    u = (x - origin) * inv_dx
    return np.floor(u - 0.5).astype(np.int64)


def stencil_weights(x, origin, dx):
    """Per particle: stencil node coordinates (N,27,3), w_ip (N,27) and
    grad w_ip (N,27,3) as products of 1-D kernels along each axis."""
    base = base_node(x, origin, dx)
    nodes = base[:, None, :] + STENCIL[None, :, :]
    xi = origin + nodes * dx
    t = (x[:, None, :] - xi) / dx
    n1 = bspline_N(t)
    d1 = bspline_dN(t) / dx
    w = n1[..., 0] * n1[..., 1] * n1[..., 2]
    gw = np.stack([d1[..., 0] * n1[..., 1] * n1[..., 2],
                   n1[..., 0] * d1[..., 1] * n1[..., 2],
                   n1[..., 0] * n1[..., 1] * d1[..., 2]], axis=-1)
    return nodes, w, gw


# --------------------------------------------------------------------------
# Materials (Sec. 6.1: fixed corotated; Neo-Hookean for the stiffness scenes)
# --------------------------------------------------------------------------
def lame(E, nu):
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def cofactor(F):
    """cof(F) = dJ/dF: rows are f1 x f2, f2 x f0, f0 x f1 of the rows f_k."""
    f0, f1, f2 = F[..., 0, :], F[..., 1, :], F[..., 2, :]
    return np.stack([np.cross(f1, f2), np.cross(f2, f0), np.cross(f0, f1)], axis=-2)


def signed_svd(F):
    """F = U diag(s) V^T with det U = det V = +1; the smallest singular value
    carries the sign of det F (the inversion-safe convention)."""
    U, s, Vt = np.linalg.svd(F)
    V = np.swapaxes(Vt, -1, -2).copy()
    s = s.copy()
    U = U.copy()
    du = np.linalg.det(U) < 0
    U[du, :, 2] *= -1.0
    s[du, 2] *= -1.0
    dv = np.linalg.det(V) < 0
    V[dv, :, 2] *= -1.0
    s[dv, 2] *= -1.0
    return U, s, V


def psi(F, mu, lam, model):
    """Energy density per unit reference volume.
    FCR: mu ||F - R||^2 + lam/2 (J - 1)^2 (R from the polar decomposition).
    NH : mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2, +inf for J <= 0."""
    J = np.linalg.det(F)
    out = np.empty(F.shape[0])
    fcr = model == 0
    if np.any(fcr):
        U, s, V = signed_svd(F[fcr])
        R = U @ np.swapaxes(V, -1, -2)
        out[fcr] = mu[fcr] * np.sum((F[fcr] - R) ** 2, axis=(1, 2)) \
            + 0.5 * lam[fcr] * (J[fcr] - 1.0) ** 2
    nh = ~fcr
    if np.any(nh):
        Jn = J[nh]
        good = Jn > 0
        lnJ = np.log(np.where(good, Jn, 1.0))
        val = 0.5 * mu[nh] * (np.sum(F[nh] ** 2, axis=(1, 2)) - 3.0) - mu[nh] * lnJ \
            + 0.5 * lam[nh] * lnJ ** 2
        out[nh] = np.where(good, val, np.inf)
    return out


def first_piola(F, mu, lam, model):
    """P = dpsi/dF.  FCR: 2 mu (F - R) + lam (J - 1) cof F.
    NH: mu F + (lam ln J - mu) F^{-T}."""
    out = np.empty_like(F)
    J = np.linalg.det(F)
    cof = cofactor(F)
    fcr = model == 0
    if np.any(fcr):
        U, s, V = signed_svd(F[fcr])
        R = U @ np.swapaxes(V, -1, -2)
        out[fcr] = 2.0 * mu[fcr, None, None] * (F[fcr] - R) \
            + (lam[fcr] * (J[fcr] - 1.0))[:, None, None] * cof[fcr]
    nh = ~fcr
    if np.any(nh):
        Jn = J[nh]
        FinvT = cof[nh] / Jn[:, None, None]
        out[nh] = mu[nh, None, None] * F[nh] \
            + (lam[nh] * np.log(Jn) - mu[nh])[:, None, None] * FinvT
    return out


def dPdF(F, mu, lam, model):
    """Analytic 9x9 d^2 psi / dF^2 with index (a,b) -> 3a+b; entry
    [(a,b),(c,d)] = dP_ab / dF_cd."""
    n = F.shape[0]
    out = np.zeros((n, 3, 3, 3, 3))
    I3 = np.eye(3)
    J = np.linalg.det(F)
    cof = cofactor(F)
    fcr = model == 0
    if np.any(fcr):
        Ff = F[fcr]
        m = mu[fcr][:, None, None, None, None]
        lm = lam[fcr][:, None, None, None, None]
        U, s, V = signed_svd(Ff)
        # dR along each E_cd: M = U^T E_cd V, W_ij = (M_ij - M_ji)/(s_i + s_j), dR = U W V^T
        M = np.einsum("nci,ndj->ncdij", U, V)          # M[n,c,d,i,j] = U_ci V_dj
        denom = s[:, :, None] + s[:, None, :]
        W = (M - np.swapaxes(M, -1, -2)) / denom[:, None, None, :, :]
        dR = np.einsum("nai,ncdij,nbj->nabcd", U, W, V)
        dcof = np.einsum("acj,bdl,njl->nabcd", LEVI, LEVI, Ff)
        cf = cof[fcr]
        Jm1 = (J[fcr] - 1.0)[:, None, None, None, None]
        out[fcr] = 2.0 * m * (np.einsum("ac,bd->abcd", I3, I3)[None] - dR) \
            + lm * np.einsum("nab,ncd->nabcd", cf, cf) + lm * Jm1 * dcof
    nh = ~fcr
    if np.any(nh):
        Jn = J[nh]
        G = cof[nh] / Jn[:, None, None]                  # F^{-T}
        m = mu[nh][:, None, None, None, None]
        lm = lam[nh][:, None, None, None, None]
        c2 = (mu[nh] - lam[nh] * np.log(Jn))[:, None, None, None, None]
        out[nh] = m * np.einsum("ac,bd->abcd", I3, I3)[None] \
            + c2 * np.einsum("nad,ncb->nabcd", G, G) + lm * np.einsum("nab,ncd->nabcd", G, G)
    return out.reshape(n, 9, 9)


def project_psd(A):
    """Teran et al. 2005 positive-definite fix: clamp the eigenvalues of the
    symmetric 9x9 stiffness at zero (READING: clamp to 0, not to a small
    positive value)."""
    As = 0.5 * (A + np.swapaxes(A, -1, -2))
    lam, Q = np.linalg.eigh(As)
    lam = np.maximum(lam, 0.0)
    return np.einsum("nij,nj,nkj->nik", Q, lam, Q)


def xi_particle(mu, lam):
    """Sec. 5.2: xi_p = ||dP^/dF^|| at the undeformed state.  In the diagonal
    space that 3x3 matrix is 2 mu I + lam 1 1^T for both models (READING:
    Frobenius norm)."""
    return np.sqrt(3.0 * (2.0 * mu + lam) ** 2 + 6.0 * lam ** 2)


# --------------------------------------------------------------------------
# Grid: P2G (Sec. 3.1, APIC) and boundary conditions (Sec. 4.1, projection)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    coords: np.ndarray          # (n,3) int64 node coordinates, (z,y,x)-lexicographic
    m: np.ndarray               # (n,)
    v: np.ndarray               # (n,3) v^n_i (prescribed at held nodes)
    xi: np.ndarray              # (n,)
    fixed: np.ndarray           # (n,) bool, Dirichlet nodes
    pidx: np.ndarray            # (N,27) node index of each particle's stencil node
    w: np.ndarray               # (N,27)
    gw: np.ndarray              # (N,27,3)
    pos: np.ndarray             # (n,3) node positions
    dx: float


def lex_key(c):
    """Scalar key ordering node coordinates (z, y, x)-lexicographically."""
    c = np.asarray(c, np.int64) + (1 << 20)
    return (c[..., 2] << 42) | (c[..., 1] << 21) | c[..., 0]


def material_arrays(sc):
    E = np.array([m.E for m in sc.materials])[sc.mat]
    nu = np.array([m.nu for m in sc.materials])[sc.mat]
    model = np.array([m.model for m in sc.materials])[sc.mat]
    mu, lam = lame(E, nu)
    return mu, lam, model


def p2g(sc) -> Grid:
    """APIC P2G (Jiang et al. 2015, used in Sec. 3.1):
    m_i = sum_p w_ip m_p;  m_i v_i = sum_p w_ip m_p (v_p + C_p (x_i - x_p));
    xi_i = sum_p w_ip m_p xi_p / m_i (Sec. 5.2, mass-weighted).
    Active nodes: the union of the particles' 3^3 stencils."""
    nodes, w, gw = stencil_weights(sc.x, sc.origin, sc.dx)
    dims = sc.grid_dims
    if np.any(nodes < 0) or np.any(nodes > dims[None, None, :]):
        raise ValueError("particle stencil leaves the grid")
    keys = lex_key(nodes).ravel()
    ukeys, inv = np.unique(keys, return_inverse=True)
    pidx = inv.reshape(nodes.shape[:2])
    coords = np.zeros((ukeys.shape[0], 3), np.int64)
    coords[pidx.ravel()] = nodes.reshape(-1, 3)
    n = coords.shape[0]
    pos = sc.origin + coords * sc.dx
    mu, lam, _ = material_arrays(sc)
    xip = xi_particle(mu, lam)
    wm = w * sc.mass[:, None]
    m = np.bincount(pidx.ravel(), wm.ravel(), minlength=n)
    rel = pos[pidx] - sc.x[:, None, :]                       # x_i - x_p
    vel = sc.v[:, None, :] + np.einsum("pab,pkb->pka", sc.C, rel)
    mv = np.stack([np.bincount(pidx.ravel(), (wm[..., None] * vel)[..., a].ravel(), minlength=n)
                   for a in range(3)], axis=1)
    mxi = np.bincount(pidx.ravel(), (wm * xip[:, None]).ravel(), minlength=n)
    pos_m = m > 0
    v = np.zeros((n, 3))
    v[pos_m] = mv[pos_m] / m[pos_m, None]
    xi = np.zeros(n)
    xi[pos_m] = mxi[pos_m] / m[pos_m]
    fixed, vfix = boundary_conditions(sc, coords, pos)
    fixed |= ~pos_m
    v[fixed] = vfix[fixed]
    return Grid(coords=coords, m=m, v=v, xi=xi, fixed=fixed, pidx=pidx, w=w, gw=gw,
                pos=pos, dx=sc.dx)


def boundary_conditions(sc, coords, pos):
    """Dirichlet nodes and their prescribed velocities (READING: nodes within
    three cells of the domain walls are held; boxes are applied in list
    order, a later box overriding an earlier one; a rotating box prescribes
    omega * axis x (x_i - center); a box with radius > 0 holds only its
    nodes within that distance of the rotation axis, a region that the
    rotation it prescribes maps onto itself)."""
    n = coords.shape[0]
    fixed = np.zeros(n, bool)
    vfix = np.zeros((n, 3))
    dims = np.asarray(sc.grid_dims)
    wall = np.any((coords < WALL_NODES) | (coords > dims[None, :] - WALL_NODES), axis=1)
    fixed |= wall
    for bc in sc.bcs:
        lo = np.asarray(bc.lo)
        hi = np.asarray(bc.hi)
        inside = np.all((pos >= lo) & (pos <= hi), axis=1)
        R = getattr(bc, "radius", 0.0)
        if R > 0.0:
            # box intersected with the cylinder of radius R about the line
            # through center along axis (each operation rounded separately)
            a = np.asarray(bc.axis, np.float64)
            r = pos - np.asarray(bc.center, np.float64)[None, :]
            t = r[:, 0] * a[0] + r[:, 1] * a[1] + r[:, 2] * a[2]
            q = r - t[:, None] * a[None, :]
            d2 = q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1] + q[:, 2] * q[:, 2]
            inside &= d2 <= R * R
        fixed |= inside
        if bc.type == 0:
            vfix[inside] = 0.0
        else:
            om = bc.omega * np.asarray(bc.axis, np.float64)
            vfix[inside] = np.cross(om[None, :], pos[inside] - np.asarray(bc.center)[None, :])
    return fixed, vfix


# --------------------------------------------------------------------------
# Eq. 1 incremental potential, gradient and projected Hessian
# --------------------------------------------------------------------------
class Problem:
    """The grid time-step problem of Sec. 3.1 for one step of size dt."""

    def __init__(self, sc, grid: Grid, dt: float):
        self.sc = sc
        self.g = grid
        self.dt = dt
        self.mu, self.lam, self.model = material_arrays(sc)
        self.n = grid.coords.shape[0]
        self.free = ~grid.fixed

    def project(self, u):
        u = u.copy()
        u[self.g.fixed] = 0.0
        return u

    def velocity_gradient(self, u):
        """sum_i u_i grad w_ip^T per particle (3x3)."""
        return np.einsum("pka,pkb->pab", u[self.g.pidx], self.g.gw)

    def deformation(self, dv):
        """F_p(dv) = (I + dt sum_i (v^n_i + dv_i) grad w_ip^T) F^n_p."""
        L = self.velocity_gradient(self.g.v + dv)
        return (np.eye(3)[None] + self.dt * L) @ self.sc.F

    def energy(self, dv):
        """Eq. 1 with gravity inside Phi (READING: Phi includes
        -sum_i m_i g . x_i, which contributes -dt sum_i m_i g . dv_i)."""
        F = self.deformation(dv)
        pe = psi(F, self.mu, self.lam, self.model)
        m = self.g.m
        kin = 0.5 * np.sum(m[:, None] * dv * dv)
        grav = -self.dt * np.sum(m[:, None] * (self.sc.gravity[None, :] * dv))
        return kin + grav + np.sum(self.sc.vol * pe)

    def gradient(self, dv):
        """g_i = m_i dv_i - dt m_i g + dt sum_p V_p P_p F^n_p^T grad w_ip
        (nodal force of Sec. 4.1 with x_i = x^n_i + dt (v^n_i + dv_i)),
        zeroed at held nodes."""
        F = self.deformation(dv)
        P = first_piola(F, self.mu, self.lam, self.model)
        K = self.sc.vol[:, None, None] * (P @ np.swapaxes(self.sc.F, 1, 2))
        contrib = self.dt * np.einsum("pab,pkb->pka", K, self.g.gw)
        g = np.stack([np.bincount(self.g.pidx.ravel(), contrib[..., a].ravel(), minlength=self.n)
                      for a in range(3)], axis=1)
        g += self.g.m[:, None] * (dv - self.dt * self.sc.gravity[None, :])
        return self.project(g)

    def particle_stiffness(self, dv, project=True):
        F = self.deformation(dv)
        A = dPdF(F, self.mu, self.lam, self.model)
        return project_psd(A) if project else A

    def hessian_pattern(self):
        """Block pattern: (i, l) such that some particle has both nodes in its
        stencil, plus the diagonal.  Returns a boolean CSR n x n."""
        pi = self.g.pidx
        rows = np.repeat(pi, 27, axis=1).ravel()
        cols = np.tile(pi, (1, 27)).ravel()
        pat = sp.coo_matrix((np.ones(rows.shape[0]), (rows, cols)), shape=(self.n, self.n)).tocsr()
        pat.data[:] = 1.0
        return pat

    def hessian(self, dv=None, project=True, chunk=2048):
        """H_il = m_i delta_il I + dt^2 sum_p V_p sum_{gd} A_p[(a,g),(b,d)]
        d_ipg d_lpd with d_ip = F^n_p^T grad w_ip and A_p the projected
        d^2 psi/dF^2 at F_p(dv); then the Dirichlet projection (held rows and
        columns zeroed, held diagonal = m_i I, or I when m_i = 0).
        Returned as a 3n x 3n CSR matrix."""
        if dv is None:
            dv = np.zeros((self.n, 3))
        A = self.particle_stiffness(dv, project).reshape(-1, 3, 3, 3, 3)  # [p,a,g,b,d]
        d = np.einsum("pba,pkb->pka", self.sc.F, self.g.gw)                 # F^T grad w
        n3 = 3 * self.n
        H = sp.csr_matrix((n3, n3))
        ar = np.arange(3)
        for s in range(0, self.sc.n, chunk):
            e = min(s + chunk, self.sc.n)
            blk = np.einsum("pagbd,pig,pld->pilab", A[s:e], d[s:e], d[s:e])
            blk *= (self.dt ** 2 * self.sc.vol[s:e])[:, None, None, None, None]
            pi = self.g.pidx[s:e]
            r = (3 * pi[:, :, None, None, None] + ar[None, None, None, :, None])
            c = (3 * pi[:, None, :, None, None] + ar[None, None, None, None, :])
            r = np.broadcast_to(r, blk.shape).ravel()
            c = np.broadcast_to(c, blk.shape).ravel()
            H = H + sp.coo_matrix((blk.ravel(), (r, c)), shape=(n3, n3)).tocsr()
        H = H + sp.diags(np.repeat(self.g.m, 3))
        return self.dirichlet_project(H.tocsr())

    def dirichlet_project(self, H):
        fixed3 = np.repeat(self.g.fixed, 3)
        keep = sp.diags((~fixed3).astype(np.float64))
        H = (keep @ H @ keep).tocsr()
        dia = np.where(self.g.m > 0, self.g.m, 1.0)
        H = H + sp.diags(np.where(fixed3, np.repeat(dia, 3), 0.0))
        return H.tocsr()

    def cn_norm(self, g):
        """Sec. 5.2: g^_i = g_i / (l_i xi_i dt), l_i = 24 dx^2; returns
        (||g^||_2, n_free) (READING: n counts the free active nodes)."""
        scale = 24.0 * self.g.dx ** 2 * self.dt
        f = self.free
        gh = g[f] / (scale * self.g.xi[f, None])
        return float(np.sqrt(np.sum(gh * gh))), int(np.count_nonzero(f))


# --------------------------------------------------------------------------
# Sec. 4: node-embedding multigrid
# --------------------------------------------------------------------------
def embed_weight_1d(d):
    """Linear embedding kernel (Sec. 4.2): 1 at d = 0, 1/2 at |d| = 1."""
    d = np.abs(d)
    return np.where(d == 0, 1.0, np.where(d == 1, 0.5, 0.0))


def coarse_nodes(fine_coords):
    """Coarse nodes A with a non-zero embedding weight to some fine node a,
    i.e. |a - 2A| <= 1 per axis (READING: even fine indices coincide with
    coarse nodes; floor division for odd ones)."""
    cand = []
    for o in STENCIL - 1:
        A2 = fine_coords - o[None, :]
        ok = np.all(A2 % 2 == 0, axis=1)
        cand.append(A2[ok] // 2)
    c = np.concatenate(cand)
    keys = lex_key(c)
    _, first = np.unique(keys, return_index=True)
    return c[first]


def restriction(fine_coords, coarse_coords):
    """R^{m+1}_m = (dx^m / dx^{m+1})^T (Sec. 4.1) with the linear embedding:
    R_{Aa} = prod_axes w(a - 2A), as a scalar n_c x n_f matrix."""
    ck = lex_key(coarse_coords)
    order = np.argsort(ck)
    rows, cols, vals = [], [], []
    for o in STENCIL - 1:
        A2 = fine_coords - o[None, :]
        ok = np.all(A2 % 2 == 0, axis=1)
        A = A2[ok] // 2
        kk = lex_key(A)
        pos = np.searchsorted(ck, kk, sorter=order)
        idx = order[np.minimum(pos, len(order) - 1)]
        found = ck[idx] == kk
        fidx = np.nonzero(ok)[0][found]
        wgt = np.prod(embed_weight_1d(o[None, :].repeat(found.sum(), 0)), axis=1)
        rows.append(idx[found])
        cols.append(fidx)
        vals.append(wgt)
    R = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(coarse_coords.shape[0], fine_coords.shape[0])).tocsr()
    return R


@dataclasses.dataclass
class Level:
    coords: np.ndarray
    H: sp.csr_matrix               # 3n x 3n
    pattern: sp.csr_matrix         # n x n block pattern
    R: Optional[sp.csr_matrix]     # scalar restriction to the next level (n_next x n)
    colors: List[np.ndarray]       # node indices per color 0..26
    Dblk: np.ndarray               # (n,3,3) diagonal blocks
    row_slices: Optional[dict] = None   # cache: color -> rows of H (no arithmetic)


def node_colors(coords):
    """READING: 27-coloring c = (x mod 3) + 3 (y mod 3) + 9 (z mod 3); blocks
    couple only nodes within offset 2 per axis, so a color's nodes are
    mutually uncoupled."""
    c = coords % 3
    col = c[:, 0] + 3 * c[:, 1] + 9 * c[:, 2]
    return [np.nonzero(col == k)[0] for k in range(27)]


def diag_blocks(H, n):
    """The 3x3 diagonal blocks H_ii."""
    D = np.zeros((n, 3, 3))
    Hc = H.tocsr()
    for a in range(3):
        for b in range(3):
            D[:, a, b] = np.asarray(Hc[3 * np.arange(n) + a, 3 * np.arange(n) + b]).ravel()
    return D


def build_hierarchy(coords0, H0, pattern0, levels):
    """buildMultigrid (Eq. 'buildMultigrid'): H^{m+1} = R H^m R^T with
    R (x) I_3; the block pattern of level m+1 is the symbolic product."""
    out = []
    coords, H, pat = coords0, H0, pattern0
    for m in range(levels):
        n = coords.shape[0]
        if m < levels - 1:
            cc = coarse_nodes(coords)
            R = restriction(coords, cc)
        else:
            cc, R = None, None
        out.append(Level(coords=coords, H=H, pattern=pat, R=R, colors=node_colors(coords),
                         Dblk=diag_blocks(H, n)))
        if R is None:
            break
        R3 = sp.kron(R, sp.eye(3)).tocsr()
        H = (R3 @ H @ R3.T).tocsr()
        Rp = R.copy()
        Rp.data[:] = 1.0
        pat = (Rp @ pat @ Rp.T).tocsr()
        pat.data[:] = 1.0
        coords = cc
    return out


def sgs(level: Level, u, b, forward=True):
    """One Gauss-Seidel sweep over the 27 colors (0..26 forward, 26..0
    backward); each node solves its 3x3 diagonal block exactly:
    u_i <- H_ii^{-1} (b_i - sum_{j != i} H_ij u_j)."""
    H = level.H
    order = range(27) if forward else range(26, -1, -1)
    u = u.copy()
    for c in order:
        rows = level.colors[c]
        if rows.size == 0:
            continue
        if level.row_slices is None:
            level.row_slices = {}
        if c not in level.row_slices:
            r3 = (3 * rows[:, None] + np.arange(3)[None, :]).ravel()
            level.row_slices[c] = H[r3]
        Hu = (level.row_slices[c] @ u.ravel()).reshape(-1, 3)
        D = level.Dblk[rows]
        rhs = b[rows] - Hu + np.einsum("nab,nb->na", D, u[rows])
        u[rows] = np.linalg.solve(D, rhs[..., None])[..., 0]
    return u


def symmetric_gauss_seidel(level, u, b):
    u = sgs(level, u, b, True)
    return sgs(level, u, b, False)


def coarse_pcg(H, b, tau, max_iter, forced_iters=None):
    """Coarsest-level Jacobi PCG (Alg. 2, Sec. 5.3).  READING of the garbled
    tolerance: k = min(0.5, sqrt(max(sqrt(b^T D^-1 b), tau))); stop when
    sqrt(r^T D^-1 r) <= k sqrt(b^T D^-1 b); D = diag(H) (scalar Jacobi).
    Returns (u, iterations)."""
    d = H.diagonal()
    bf = b.ravel()
    x = np.zeros_like(bf)
    r = bf.copy()
    z = r / d
    p = z.copy()
    rz = float(r @ z)
    bn = np.sqrt(max(rz, 0.0))
    k = min(0.5, np.sqrt(max(bn, tau)))
    it = 0
    while True:
        if forced_iters is not None:
            if it >= forced_iters:
                break
        elif np.sqrt(max(rz, 0.0)) <= k * bn or it >= max_iter:
            break
        Ap = H @ p
        pAp = float(p @ Ap)
        if pAp <= 0:
            break
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * Ap
        z = r / d
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        it += 1
    return x.reshape(b.shape), it


class VCycle:
    """Alg. 2 applied to a 3n-vector b (n x 3 array)."""

    def __init__(self, levels: List[Level], fixed, tau, max_coarse, exact_coarse=False):
        self.exact_coarse = exact_coarse
        self.L = levels
        self.fixed = fixed
        self.tau = tau
        self.max_coarse = max_coarse
        self.cg_counts: List[int] = []
        self.forced: Optional[List[int]] = None

    def __call__(self, b0):
        L = self.L
        M = len(L)
        b = [None] * M
        u = [None] * M
        b[0] = b0.copy()
        b[0][self.fixed] = 0.0
        for m in range(M - 1):
            u[m] = np.zeros_like(b[m])
            u[m] = symmetric_gauss_seidel(L[m], u[m], b[m])
            r = b[m] - (L[m].H @ u[m].ravel()).reshape(-1, 3)
            b[m + 1] = L[m].R @ r
        forced = None
        if self.forced is not None:
            forced = self.forced.pop(0)
        cap = self.max_coarse if self.max_coarse > 0 else 3 * L[-1].coords.shape[0]
        if self.exact_coarse:
            u[M - 1] = np.linalg.solve(L[-1].H.toarray(), b[M - 1].ravel()).reshape(-1, 3)
            its = 0
        else:
            u[M - 1], its = coarse_pcg(L[-1].H, b[M - 1], self.tau, cap, forced)
        self.cg_counts.append(its)
        for m in range(M - 2, -1, -1):
            u[m] = u[m] + L[m].R.T @ u[m + 1]
            u[m] = symmetric_gauss_seidel(L[m], u[m], b[m])
        out = u[0]
        out[self.fixed] = 0.0
        return out


# --------------------------------------------------------------------------
# Alg. 3: HOT
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Trace:
    iters: int = 0
    alphas: List[float] = dataclasses.field(default_factory=list)
    ls_trials: List[int] = dataclasses.field(default_factory=list)
    cg_counts: List[int] = dataclasses.field(default_factory=list)
    skipped: List[int] = dataclasses.field(default_factory=list)
    fallback: List[int] = dataclasses.field(default_factory=list)
    norms: List[float] = dataclasses.field(default_factory=list)
    energies: List[float] = dataclasses.field(default_factory=list)
    inner: List[int] = dataclasses.field(default_factory=list)   # CG counts after a fallback to PN-MGPCG
    status: str = "ok"


def line_search(prob: Problem, dv, p, E0, max_ls, forced_alpha=None):
    """Backtracking from alpha = 1, halving until E(dv + alpha p) <= E(dv)
    (READING of 'ensure energy decrease').  Returns (alpha, E, trials)."""
    if forced_alpha is not None:
        return forced_alpha, prob.energy(dv + forced_alpha * p), None
    alpha = 1.0
    for t in range(1, max_ls + 1):
        E1 = prob.energy(dv + alpha * p)
        if E1 <= E0:
            return alpha, E1, t
        alpha *= 0.5
    return None, E0, max_ls


def two_loop(hist, q, apply_h0):
    """Alg. 3's two-loop recursion: returns H q, where H is the L-BFGS inverse
    Hessian built from the initial inverse H_0 (``apply_h0``, the V-cycle in
    HOT) by the BFGS inverse updates of the stored pairs (s, y, rho = 1/y^T s),
    oldest first.  First loop from the newest pair back: a_j = rho_j s_j^T q,
    q <- q - a_j y_j; then r = H_0 q; second loop from the oldest pair on:
    b_j = rho_j y_j^T r, r <- r + (a_j - b_j) s_j."""
    alph = []
    for (s, y, rho) in reversed(hist):
        a = rho * float(np.sum(s * q))
        q = q - a * y
        alph.append(a)
    r = apply_h0(q)
    for (s, y, rho), a in zip(hist, reversed(alph)):
        beta = rho * float(np.sum(y * r))
        r = r + (a - beta) * s
    return r


def hot_solve(prob: Problem, opts, replay: Optional[Trace] = None, levels=None):
    """Alg. 3.  Returns (dv, trace).  With ``replay`` the decisions recorded
    by another implementation (iteration count, step lengths, coarse CG
    iteration counts, skipped pairs, fallbacks) are imposed instead of taken."""
    n = prob.n
    dv = np.zeros((n, 3))
    g = prob.gradient(dv)
    H0 = prob.hessian(dv)
    if levels is None:
        levels = build_hierarchy(prob.g.coords, H0, prob.hessian_pattern(), opts.levels)
    vc = VCycle(levels, prob.g.fixed, opts.eps, opts.max_coarse_cg)
    if replay is not None:
        vc.forced = list(replay.cg_counts)
    tr = Trace()
    hist = []   # (s, y, rho)
    g1n = float(np.sqrt(np.sum(g * g)))
    E = prob.energy(dv)
    tr.energies.append(E)
    it = 0
    while True:
        if opts.cn_mode == 0:
            nrm, nfree = prob.cn_norm(g)
            done = nrm <= opts.eps * np.sqrt(nfree)
        else:
            nrm = float(np.sqrt(np.sum(g * g)))
            done = nrm <= opts.eps * g1n
        tr.norms.append(nrm)
        if replay is not None:
            done = it >= replay.iters
        if done:
            break
        if it >= opts.max_iters:
            tr.status = "not_converged"
            break
        fb_after = getattr(opts, "fallback_after", 0)
        if fb_after > 0 and it >= fb_after:
            # Extension, not in Alg. 3: a step that has not converged after
            # fallback_after L-BFGS iterations is finished by PN-MGPCG (Alg. 1)
            # from the current iterate.
            rp = None
            if replay is not None:
                rp = PNTrace(iters=replay.iters, alphas=replay.alphas, ls_trials=replay.ls_trials,
                             cg_iters=replay.inner)
            dv, ptr = pn_solve(prob, opts, "mg", replay=rp, dv0=dv, it0=it, g1n=g1n, vc_forced=vc.forced)
            tr.alphas.extend(ptr.alphas)
            tr.ls_trials.extend(ptr.ls_trials)
            tr.inner = list(ptr.cg_iters)
            tr.energies.extend(ptr.energies[1:])
            tr.norms.extend(ptr.norms[1:])
            tr.status = ptr.status
            tr.iters = ptr.iters
            tr.cg_counts = list(vc.cg_counts) + list(ptr.vc_cg_counts)
            return dv, tr
        refresh = getattr(opts, "refresh_every", 0)
        if refresh > 0 and it > 0 and it % refresh == 0:
            # Extension, not in Alg. 3 (which builds the hierarchy once per
            # step): rebuild the projected Hessian and its hierarchy at the
            # current iterate and restart the history.
            H = prob.hessian(dv)
            levels = build_hierarchy(prob.g.coords, H, prob.hessian_pattern(), opts.levels)
            vc_new = VCycle(levels, prob.g.fixed, opts.eps, opts.max_coarse_cg)
            vc_new.cg_counts = vc.cg_counts
            vc_new.forced = vc.forced
            vc = vc_new
            hist = []
        p = two_loop(hist, -g, vc)
        fb = 0
        if replay is not None:
            fb = replay.fallback[it]
        elif not float(np.sum(p * g)) < 0.0:
            fb = 1
        if fb:
            # READING: a non-descent direction restarts from the V-cycle alone,
            # and from steepest descent if that is not a descent direction
            hist = []
            p = vc(-g)
            if replay is None and not float(np.sum(p * g)) < 0.0:
                fb = 2
            if fb == 2:
                p = -g
        tr.fallback.append(fb)
        forced = replay.alphas[it] if replay is not None else None
        alpha, E1, trials = line_search(prob, dv, p, E, opts.max_ls, forced)
        if alpha is None:
            tr.status = "linesearch"
            break
        tr.alphas.append(alpha)
        tr.ls_trials.append(trials if trials is not None else replay.ls_trials[it])
        dv_new = dv + alpha * p
        g_new = prob.gradient(dv_new)
        s = dv_new - dv
        y = g_new - g
        ys = float(np.sum(y * s))
        if replay is not None:
            skip = replay.skipped[it]
        else:
            # READING: keep a pair only with positive curvature
            skip = int(not (ys > 1e-14 * np.sqrt(np.sum(y * y) * np.sum(s * s))))
        tr.skipped.append(skip)
        if not skip:
            hist.append((s, y, 1.0 / ys))
            if len(hist) > opts.lbfgs_m:
                hist.pop(0)
        dv, g, E = dv_new, g_new, E1
        tr.energies.append(E)
        it += 1
    tr.iters = it
    tr.cg_counts = list(vc.cg_counts)
    return dv, tr


# --------------------------------------------------------------------------
# Alg. 1: inexact projected Newton (PN-PCG, PN-MGPCG)
# --------------------------------------------------------------------------
def pn_pcg(H, b, precond, tau, max_iter, forced_iters=None):
    """CG on H x = b from x = 0 with preconditioner z = precond(r), stopped by
    the inexact criterion of Sec. 5.3: k = min(0.5, sqrt(max(sqrt(r0^T P r0),
    tau))) and stop when sqrt(r^T P r) <= k sqrt(r0^T P r0), P the
    preconditioner (r^T P r = r^T z).  READING: the run is capped at
    max_iter iterations (the paper states no cap).  Returns (x, iterations)."""
    bf = b.ravel()
    x = np.zeros_like(bf)
    r = bf.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    bn = np.sqrt(max(rz, 0.0))
    k = min(0.5, np.sqrt(max(bn, tau)))
    it = 0
    while True:
        if forced_iters is not None:
            if it >= forced_iters:
                break
        elif np.sqrt(max(rz, 0.0)) <= k * bn or it >= max_iter:
            break
        Ap = H @ p
        pAp = float(p @ Ap)
        if pAp <= 0:
            break
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * Ap
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        it += 1
    return x.reshape(b.shape), it


@dataclasses.dataclass
class PNTrace:
    iters: int = 0
    alphas: List[float] = dataclasses.field(default_factory=list)
    ls_trials: List[int] = dataclasses.field(default_factory=list)
    cg_iters: List[int] = dataclasses.field(default_factory=list)      # per Newton iteration
    vc_cg_counts: List[int] = dataclasses.field(default_factory=list)  # coarsest PCG, per V-cycle (PN-MGPCG)
    energies: List[float] = dataclasses.field(default_factory=list)
    norms: List[float] = dataclasses.field(default_factory=list)
    status: str = "ok"


def pn_solve(prob: Problem, opts, precond: str = "jacobi", max_cg: int = 10000,
             replay: Optional[PNTrace] = None, dv0=None, it0: int = 0, g1n: Optional[float] = None,
             vc_forced: Optional[list] = None):
    """Alg. 1: Newton iterations on E(dv), each solving the projected Hessian
    system H p = -g at the current dv (Teran projection, Dirichlet projection)
    inexactly by PCG (pn_pcg), then the backtracking line search from alpha =
    1 and the same termination test as Alg. 3.  precond "jacobi": the scalar
    diagonal of H (PN-PCG); "mg": one V-cycle (Alg. 2, same coarsest solve)
    of the Galerkin hierarchy built from that H (PN-MGPCG).  With ``replay``
    the CG iteration counts (and coarsest-PCG counts) and step lengths of
    another implementation are imposed.  dv0, it0, g1n: continue another
    solver's iterations from its iterate (iteration numbers, and the replayed
    step lengths, continue from it0; replay.cg_iters counts from it0);
    vc_forced: a coarsest-PCG count list shared with that solver.
    Returns (dv, trace)."""
    n = prob.n
    dv = np.zeros((n, 3)) if dv0 is None else dv0.copy()
    g = prob.gradient(dv)
    if g1n is None:
        g1n = float(np.sqrt(np.sum(g * g)))
    E = prob.energy(dv)
    tr = PNTrace()
    tr.energies.append(E)
    pattern = prob.hessian_pattern() if precond == "mg" else None
    if vc_forced is None and replay is not None:
        vc_forced = list(replay.vc_cg_counts)
    it = it0
    while True:
        if opts.cn_mode == 0:
            nrm, nfree = prob.cn_norm(g)
            done = nrm <= opts.eps * np.sqrt(nfree)
        else:
            nrm = float(np.sqrt(np.sum(g * g)))
            done = nrm <= opts.eps * g1n
        tr.norms.append(nrm)
        if replay is not None:
            done = it >= replay.iters
        if done:
            break
        if it >= opts.max_iters:
            tr.status = "not_converged"
            break
        H = prob.hessian(dv)
        if precond == "jacobi":
            d = H.diagonal()
            M = lambda r: r / d  # noqa: E731
        else:
            levels = build_hierarchy(prob.g.coords, H, pattern, opts.levels)
            vc = VCycle(levels, prob.g.fixed, opts.eps, opts.max_coarse_cg)
            if vc_forced is not None:
                vc.forced = vc_forced           # shared: consumed across Newton iterations
            M = lambda r: vc(r.reshape(-1, 3)).ravel()  # noqa: E731
        forced = replay.cg_iters[it - it0] if replay is not None else None
        p, its = pn_pcg(H, -g, M, opts.eps, max_cg, forced)
        tr.cg_iters.append(its)
        if precond == "mg":
            tr.vc_cg_counts.extend(vc.cg_counts)
        fa = replay.alphas[it] if replay is not None else None
        alpha, E1, trials = line_search(prob, dv, p, E, opts.max_ls, fa)
        if alpha is None:
            tr.status = "linesearch"
            break
        tr.alphas.append(alpha)
        tr.ls_trials.append(trials if trials is not None else replay.ls_trials[it])
        dv = dv + alpha * p
        g = prob.gradient(dv)
        E = E1
        tr.energies.append(E)
        it += 1
    tr.iters = it
    return dv, tr


# --------------------------------------------------------------------------
# Sec. 3.1: step driver and G2P
# --------------------------------------------------------------------------
def step_dt(sc, opts):
    """Sec. 6.1: dt = min(1/FPS, CFL dx / v_max) unless a fixed dt is given."""
    if opts.dt > 0:
        return float(opts.dt)
    vmax = float(np.max(np.sqrt(np.sum(sc.v * sc.v, axis=1)))) if sc.n else 0.0
    if vmax <= 0.0:
        return 1.0 / opts.fps
    return min(1.0 / opts.fps, opts.cfl * sc.dx / vmax)


def plasticity(F, mu, plastic, yield_stress):
    """Lagged plastic projection of the deformation gradient, once per step
    after the F update (the paper lags plasticity to keep the step a
    minimisation; it prints no formulas, READING):
      1 von Mises: principal Hencky strains e = ln s, deviatoric part
        d = e - tr(e)/3; if 2 mu |d| > tau_Y, d is scaled onto the yield
        surface 2 mu |d| = tau_Y (tr e, hence det F, unchanged);
      2 snow: singular values clamped into [0.99, 1.001] (Table 2).
    F = U diag(s) V^T with the inversion-safe SVD; other rows unchanged."""
    out = F.copy()
    vm = plastic == 1
    if np.any(vm):
        U, s, V = signed_svd(F[vm])
        e = np.log(np.maximum(s, 1e-300))
        dev = e - e.mean(axis=1, keepdims=True)
        nd = np.sqrt(np.sum(dev * dev, axis=1))
        ty = yield_stress[vm]
        m = mu[vm]
        yielding = 2.0 * m * nd > ty
        scale = np.where(yielding, ty / np.maximum(2.0 * m * nd, 1e-300), 1.0)
        e_new = e.mean(axis=1, keepdims=True) + dev * scale[:, None]
        rebuilt = np.einsum("nij,nj,nkj->nik", U, np.exp(e_new), V)
        idx = np.nonzero(vm)[0]
        out[idx[yielding]] = rebuilt[yielding]
    sn = plastic == 2
    if np.any(sn):
        U, s, V = signed_svd(F[sn])
        s_new = np.clip(s, 0.99, 1.001)
        changed = np.any(s_new != s, axis=1)
        rebuilt = np.einsum("nij,nj,nkj->nik", U, s_new, V)
        idx = np.nonzero(sn)[0]
        out[idx[changed]] = rebuilt[changed]
    return out


def g2p(sc, grid: Grid, v_new, dt):
    """APIC G2P: v_p = sum_i w_ip v_i; C_p = 4/dx^2 sum_i w_ip v_i (x_i - x_p)^T;
    F_p <- (I + dt sum_i v_i grad w_ip^T) F_p, then the lagged plastic
    projection; x_p <- x_p + dt v_p."""
    vi = v_new[grid.pidx]                                   # (N,27,3)
    vp = np.einsum("pk,pka->pa", grid.w, vi)
    rel = grid.pos[grid.pidx] - sc.x[:, None, :]
    Cp = (4.0 / grid.dx ** 2) * np.einsum("pk,pka,pkb->pab", grid.w, vi, rel)
    L = np.einsum("pka,pkb->pab", vi, grid.gw)
    F = (np.eye(3)[None] + dt * L) @ sc.F
    plastic = np.array([m.plasticity for m in sc.materials])[sc.mat]
    if np.any(plastic):
        mu, _, _ = material_arrays(sc)
        ty = np.array([m.yield_stress for m in sc.materials])[sc.mat]
        F = plasticity(F, mu, plastic, ty)
    out = sc.copy()
    out.v = vp
    out.C = Cp
    out.F = F
    out.x = sc.x + dt * vp
    return out


def hot_step(sc, opts, replay: Optional[Trace] = None):
    """One implicit MPM step: dt, P2G, HOT solve (Alg. 3), G2P.
    Returns (new scene, dict with dv, v_new, grid, trace, dt)."""
    dt = step_dt(sc, opts)
    grid = p2g(sc)
    prob = Problem(sc, grid, dt)
    dv, tr = hot_solve(prob, opts, replay)
    v_new = grid.v + dv
    out = g2p(sc, grid, v_new, dt)
    return out, {"dv": dv, "v_new": v_new, "grid": grid, "trace": tr, "dt": dt, "problem": prob}
