"""Pins for the FP64 oracle: each checks it against something other than
itself -- closed forms, invariants, finite differences, brute-force dense
algebra and the paper's stated settings -- so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one of them."""
import copy
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hot_oracle as O
from paper_1911_07913_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_F(rng, n, amp=0.3):
    return np.eye(3)[None] + amp * rng.uniform(-1, 1, size=(n, 3, 3))


def rand_rot(rng, n):
    Q, _ = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    Q[np.linalg.det(Q) < 0, :, 0] *= -1
    return Q


def mats(n, model, E=1e5, nu=0.3):
    mu, lam = O.lame(np.full(n, E), np.full(n, nu))
    return mu, lam, np.full(n, model)


# ---------------------------------------------------------------- kernel
def test_bspline_golden_values():
    rows = np.loadtxt(os.path.join(GOLD, "bspline_values.txt"))
    np.testing.assert_allclose(O.bspline_N(rows[:, 0]), rows[:, 1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.bspline_dN(rows[:, 0]), rows[:, 2], rtol=0, atol=1e-15)


def test_kernel_moments():
    """sum_i w_ip = 1, sum_i w_ip (x_i - x_p) = 0,
    sum_i w_ip (x_i - x_p)(x_i - x_p)^T = dx^2/4 I, sum_i grad w_ip = 0,
    sum_i (x_i - x_p) grad w_ip^T = I."""
    rng = np.random.default_rng(1)
    dx = 1.0 / 16
    x = rng.uniform(0.3, 0.7, size=(500, 3))
    nodes, w, gw = O.stencil_weights(x, np.zeros(3), dx)
    rel = nodes * dx - x[:, None, :]
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.einsum("pk,pka->pa", w, rel), 0.0, atol=1e-15)
    M2 = np.einsum("pk,pka,pkb->pab", w, rel, rel)
    np.testing.assert_allclose(M2, np.broadcast_to(dx * dx / 4 * np.eye(3), M2.shape), atol=1e-15)
    np.testing.assert_allclose(gw.sum(1), 0.0, atol=1e-11)
    G = np.einsum("pka,pkb->pab", rel, gw)
    np.testing.assert_allclose(G, np.broadcast_to(np.eye(3), G.shape), atol=1e-12)


def test_kernel_gradient_finite_difference():
    rng = np.random.default_rng(2)
    dx = 1.0 / 8
    x = rng.uniform(0.3, 0.7, size=(50, 3))
    nodes, w, gw = O.stencil_weights(x, np.zeros(3), dx)
    h = 1e-7
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        # weights of the same nodes at shifted positions
        t_p = ((x[:, None, :] + e) - nodes * dx) / dx
        t_m = ((x[:, None, :] - e) - nodes * dx) / dx
        wp = np.prod(O.bspline_N(t_p), axis=-1)
        wm = np.prod(O.bspline_N(t_m), axis=-1)
        np.testing.assert_allclose((wp - wm) / (2 * h), gw[..., a], atol=1e-5 / dx)


def test_base_node_cell_center_gives_zero_weight():
    """A particle at a cell centre has fx = 1/2: node base+2 gets weight 0."""
    dx = 1.0 / 32
    x = np.array([[10.5 * dx, 7.5 * dx, 3.5 * dx]])
    base = O.base_node(x, np.zeros(3), dx)
    assert base.tolist() == [[10, 7, 3]]
    nodes, w, gw = O.stencil_weights(x, np.zeros(3), dx)
    far = nodes[0, :, 0] == 12
    assert np.all(w[0, far] == 0.0)


# ---------------------------------------------------------------- materials
@pytest.mark.parametrize("model", [0, 1])
def test_zero_stress_at_identity(model):
    F = np.tile(np.eye(3), (4, 1, 1))
    mu, lam, md = mats(4, model)
    np.testing.assert_allclose(O.first_piola(F, mu, lam, md), 0.0, atol=1e-9)
    np.testing.assert_allclose(O.psi(F, mu, lam, md), 0.0, atol=1e-9)


@pytest.mark.parametrize("model", [0, 1])
def test_rotation_invariance(model):
    rng = np.random.default_rng(3)
    F = rand_F(rng, 20)
    Q = rand_rot(rng, 20)
    mu, lam, md = mats(20, model)
    np.testing.assert_allclose(O.psi(Q @ F, mu, lam, md), O.psi(F, mu, lam, md), rtol=1e-11)
    np.testing.assert_allclose(O.first_piola(Q @ F, mu, lam, md), Q @ O.first_piola(F, mu, lam, md),
                               rtol=1e-9, atol=1e-6)


@pytest.mark.parametrize("model", [0, 1])
def test_stress_finite_difference(model):
    rng = np.random.default_rng(4)
    F = rand_F(rng, 10)
    mu, lam, md = mats(10, model)
    P = O.first_piola(F, mu, lam, md)
    h = 1e-6
    for a in range(3):
        for b in range(3):
            E = np.zeros((3, 3))
            E[a, b] = h
            fd = (O.psi(F + E, mu, lam, md) - O.psi(F - E, mu, lam, md)) / (2 * h)
            np.testing.assert_allclose(fd, P[:, a, b], rtol=1e-6, atol=1e-6 * np.abs(P).max())


@pytest.mark.parametrize("model", [0, 1])
def test_stiffness_finite_difference(model):
    rng = np.random.default_rng(5)
    F = rand_F(rng, 10)
    if model == 0:
        F[0] = np.diag([1.2, 0.9, -0.8])        # inverted element, FCR is defined there
    mu, lam, md = mats(10, model)
    A = O.dPdF(F, mu, lam, md)
    h = 1e-6
    for c in range(3):
        for d in range(3):
            E = np.zeros((3, 3))
            E[c, d] = h
            fd = (O.first_piola(F + E, mu, lam, md) - O.first_piola(F - E, mu, lam, md)) / (2 * h)
            np.testing.assert_allclose(fd.reshape(-1, 9), A[:, :, 3 * c + d], rtol=1e-6,
                                       atol=1e-6 * np.abs(A).max())


@pytest.mark.parametrize("model", [0, 1])
def test_stiffness_closed_form_at_identity(model):
    """dP/dF at F = I: mu (d_ac d_bd + d_ad d_bc) + lam d_ab d_cd for both models."""
    mu, lam, md = mats(1, model, E=3e5, nu=0.35)
    A = O.dPdF(np.eye(3)[None], mu, lam, md).reshape(3, 3, 3, 3)
    I = np.eye(3)
    ref = mu[0] * (np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) \
        + lam[0] * np.einsum("ab,cd->abcd", I, I)
    np.testing.assert_allclose(A, ref, rtol=1e-12, atol=1e-12 * mu[0])


def test_xi_particle_is_diagonal_space_stiffness_norm():
    mu, lam, md = mats(1, 0, E=2e6, nu=0.4)
    A = O.dPdF(np.eye(3)[None], mu, lam, md)[0]
    idx = [0, 4, 8]
    sub = A[np.ix_(idx, idx)]
    np.testing.assert_allclose(np.linalg.norm(sub), O.xi_particle(mu, lam)[0], rtol=1e-13)


def teran_projected(F, mu, lam, model):
    """Independent restatement of the SVD-space eigen-system of an isotropic
    stiffness (Teran et al. 2005): a 3x3 block in the singular values plus
    twist/flip pairs, each eigenvalue clamped at zero."""
    U, s, V = O.signed_svd(F[None])
    U, s, V = U[0], s[0], V[0]
    J = s.prod()
    if model == 0:
        g = 2 * mu * (s - 1) + lam * (J - 1) * J / s
        Hs = 2 * mu * np.eye(3) + lam * np.outer(J / s, J / s)
        for i in range(3):
            for j in range(3):
                if i != j:
                    k = 3 - i - j
                    Hs[i, j] += lam * (J - 1) * s[k]
    else:
        lnJ = np.log(J)
        g = mu * s + (lam * lnJ - mu) / s
        Hs = np.diag(mu + (mu - lam * lnJ) / s ** 2) + lam * np.outer(1 / s, 1 / s)
    ev, Q = np.linalg.eigh(Hs)
    modes = [(max(ev[k], 0.0), U @ np.diag(Q[:, k]) @ V.T) for k in range(3)]
    for i, j in [(0, 1), (0, 2), (1, 2)]:
        flip = (g[i] - g[j]) / (s[i] - s[j])
        twist = (g[i] + g[j]) / (s[i] + s[j])
        Eij = np.zeros((3, 3))
        Eij[i, j] = 1
        modes.append((max(flip, 0.0), U @ ((Eij + Eij.T) / np.sqrt(2)) @ V.T))
        modes.append((max(twist, 0.0), U @ ((Eij - Eij.T) / np.sqrt(2)) @ V.T))
    A = np.zeros((9, 9))
    for lam_k, D in modes:
        A += lam_k * np.outer(D.ravel(), D.ravel())
    return A


@pytest.mark.parametrize("model", [0, 1])
def test_projection_matches_teran_block_form(model):
    rng = np.random.default_rng(6)
    F = rand_F(rng, 12, amp=0.45)
    F = F[np.linalg.det(F) > 0.2]
    mu, lam, md = mats(F.shape[0], model)
    Ad = O.project_psd(O.dPdF(F, mu, lam, md))
    for k in range(F.shape[0]):
        At = teran_projected(F[k], mu[k], lam[k], model)
        np.testing.assert_allclose(Ad[k], At, rtol=1e-9, atol=1e-9 * np.abs(At).max())


@pytest.mark.parametrize("model", [0, 1])
def test_projection_is_identity_at_rotations(model):
    rng = np.random.default_rng(7)
    Q = rand_rot(rng, 6)
    mu, lam, md = mats(6, model)
    A = O.dPdF(Q, mu, lam, md)
    As = 0.5 * (A + np.swapaxes(A, 1, 2))
    np.testing.assert_allclose(O.project_psd(A), As, atol=1e-9 * np.abs(A).max())
    ev = np.linalg.eigvalsh(O.project_psd(O.dPdF(rand_F(rng, 6, 0.6), mu, lam, md)))
    assert ev.min() >= -1e-9 * np.abs(ev).max()


# ---------------------------------------------------------------- transfers
def free_scene(seed=0, model=0, **kw):
    sc = scenes.tiny_scene(seed=seed, res=16, cells=(3, 3, 3), lo=(6, 6, 6), ppc_axis=2,
                           model=model, **kw)
    sc.bcs = []
    return sc


def test_p2g_conserves_mass_and_momenta():
    sc = free_scene(1)
    g = O.p2g(sc)
    assert not g.fixed.any()
    np.testing.assert_allclose(g.m.sum(), sc.mass.sum(), rtol=1e-14)
    P_grid = (g.m[:, None] * g.v).sum(0)
    P_part = (sc.mass[:, None] * sc.v).sum(0)
    np.testing.assert_allclose(P_grid, P_part, rtol=1e-12, atol=1e-15)
    # APIC angular momentum: sum_i x_i x m_i v_i =
    #   sum_p m_p [x_p x v_p + dx^2/4 eps_abc C_cb]
    L_grid = np.cross(g.pos, g.m[:, None] * g.v).sum(0)
    aff = np.einsum("abc,pcb->pa", O.LEVI, sc.C) * sc.dx ** 2 / 4
    L_part = (sc.mass[:, None] * (np.cross(sc.x, sc.v) + aff)).sum(0)
    np.testing.assert_allclose(L_grid, L_part, rtol=1e-11, atol=1e-15)


def test_affine_field_round_trips():
    """An affine particle field (v_p = u + M x_p, C_p = M) maps to the grid
    field u + M x_i and back unchanged (APIC is exact for affine fields)."""
    sc = free_scene(2)
    rng = np.random.default_rng(9)
    u = rng.normal(size=3)
    M = rng.normal(size=(3, 3))
    sc.v = u[None] + sc.x @ M.T
    sc.C = np.tile(M, (sc.n, 1, 1))
    g = O.p2g(sc)
    np.testing.assert_allclose(g.v, u[None] + g.pos @ M.T, rtol=1e-12, atol=1e-12)
    out = O.g2p(sc, g, g.v, 0.0)
    np.testing.assert_allclose(out.v, sc.v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out.C, sc.C, rtol=1e-10, atol=1e-10)


def test_boundary_conditions_rotation_box():
    sc = free_scene(3)
    bc = scenes.BoundaryBox(scenes.BC_ROTATE, (0, 0, 0), (1, 1, 0.43), (0, 0, 1), (0.5, 0.5, 0), 2.0)
    sc.bcs = [bc]
    g = O.p2g(sc)
    held = g.pos[:, 2] <= 0.43
    assert np.array_equal(g.fixed, held)
    r = g.pos[held] - np.array([0.5, 0.5, 0.0])
    np.testing.assert_allclose(g.v[held][:, 0], -2.0 * r[:, 1], atol=1e-15)
    np.testing.assert_allclose(g.v[held][:, 1], 2.0 * r[:, 0], atol=1e-15)
    np.testing.assert_allclose(g.v[held][:, 2], 0.0, atol=1e-15)


def test_boundary_conditions_rotation_cylinder():
    """A box with radius > 0 holds exactly its nodes whose distance from the
    rotation axis (|axis x (x_i - c)|, an independent formula) is at most the
    radius; the held velocity is the rigid rotation."""
    sc = free_scene(3)
    ax = np.array([0.0, 0.0, 1.0])
    c = np.array([0.47, 0.52, 0.0])
    bc = scenes.BoundaryBox(scenes.BC_ROTATE, (0, 0, 0), (1, 1, 0.43), tuple(ax), tuple(c), -1.5, 0.09)
    sc.bcs = [bc]
    g = O.p2g(sc)
    dist = np.linalg.norm(np.cross(ax[None, :], g.pos - c[None, :]), axis=1)
    held = (g.pos[:, 2] <= 0.43) & (dist <= 0.09)
    assert held.any() and (~held).any()
    assert np.array_equal(g.fixed, held)
    r = g.pos[held] - c
    np.testing.assert_allclose(g.v[held][:, 0], 1.5 * r[:, 1], atol=1e-15)
    np.testing.assert_allclose(g.v[held][:, 1], -1.5 * r[:, 0], atol=1e-15)


# ---------------------------------------------------------------- E, grad E, hess E
@pytest.mark.parametrize("model", [0, 1])
def test_energy_gradient_hessian_finite_difference(model):
    sc = free_scene(4, model=model, E=1e3, F_jitter=0.1)
    g = O.p2g(sc)
    prob = O.Problem(sc, g, 1e-2)
    rng = np.random.default_rng(10)
    dv = 0.05 * rng.normal(size=(prob.n, 3))
    gr = prob.gradient(dv)
    h = 1e-6
    idx = rng.choice(prob.n * 3, 25, replace=False)
    for k in idx:
        e = np.zeros(prob.n * 3)
        e[k] = h
        e = e.reshape(-1, 3)
        fd = (prob.energy(dv + e) - prob.energy(dv - e)) / (2 * h)
        assert abs(fd - gr.ravel()[k]) <= 1e-6 * np.abs(gr).max() + 1e-9
    H = prob.hessian(dv, project=False).toarray()
    np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    for k in idx[:10]:
        e = np.zeros(prob.n * 3)
        e[k] = h
        e = e.reshape(-1, 3)
        fd = ((prob.gradient(dv + e) - prob.gradient(dv - e)) / (2 * h)).ravel()
        np.testing.assert_allclose(fd, H[:, k], atol=1e-6 * np.abs(H).max())


def test_projected_hessian_is_psd_and_pattern_exact():
    sc = free_scene(5, F_jitter=0.4)
    g = O.p2g(sc)
    prob = O.Problem(sc, g, 5e-2)
    H = prob.hessian().toarray()
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev.min() >= -1e-12 * np.abs(ev).max()
    # block pattern: brute force over particles
    pat = prob.hessian_pattern().toarray() > 0
    brute = np.zeros_like(pat)
    for p in range(sc.n):
        for i in g.pidx[p]:
            brute[i, g.pidx[p]] = True
    assert np.array_equal(pat, brute)
    Hb = np.abs(H).reshape(prob.n, 3, prob.n, 3).sum(axis=(1, 3)) > 0
    assert not np.any(Hb & ~pat)


def test_dirichlet_projection():
    sc = scenes.cube_scene(seed=1, res=16, cube_lo=(5, 3, 5), side=3)
    g = O.p2g(sc)
    assert g.fixed.any() and (~g.fixed).any()
    prob = O.Problem(sc, g, 1e-3)
    H = prob.hessian().toarray()
    f3 = np.repeat(g.fixed, 3)
    off = H[np.ix_(f3, ~f3)]
    assert np.all(off == 0)
    np.testing.assert_allclose(np.diag(H)[f3], np.repeat(g.m[g.fixed], 3))
    gr = prob.gradient(np.zeros((prob.n, 3)))
    assert np.all(gr[g.fixed] == 0)


# ---------------------------------------------------------------- multigrid
def hierarchy_for(sc, levels=3, dt=2e-2):
    g = O.p2g(sc)
    prob = O.Problem(sc, g, dt)
    H0 = prob.hessian()
    L = O.build_hierarchy(g.coords, H0, prob.hessian_pattern(), levels)
    return g, prob, L


def test_prolongation_reproduces_linear_fields():
    sc = free_scene(6)
    g, prob, L = hierarchy_for(sc)
    for m in range(len(L) - 1):
        R = L[m].R
        np.testing.assert_allclose(R.T @ np.ones(R.shape[0]), 1.0, atol=1e-15)
        c = np.array([0.3, -1.1, 2.0])
        uc = (2 * L[m + 1].coords) @ c
        np.testing.assert_allclose(R.T @ uc, L[m].coords @ c, atol=1e-12)
        # interior coarse columns sum to 8 (R = (dx^0/dx^1)^T, Sec. 4.1)
        assert np.isclose((R @ np.ones(R.shape[1])).max(), 8.0)


def test_rap_matches_dense_triple_product_and_full_rank():
    sc = free_scene(7, F_jitter=0.2)
    g, prob, L = hierarchy_for(sc)
    for m in range(len(L) - 1):
        R3 = np.kron(L[m].R.toarray(), np.eye(3))
        dense = R3 @ L[m].H.toarray() @ R3.T
        np.testing.assert_allclose(L[m + 1].H.toarray(), dense, rtol=1e-12,
                                   atol=1e-13 * np.abs(dense).max())
        np.linalg.cholesky(0.5 * (dense + dense.T))
        # the block pattern covers every non-zero block of the coarse matrix
        nb = L[m + 1].coords.shape[0]
        Hb = np.abs(dense).reshape(nb, 3, nb, 3).sum(axis=(1, 3)) > 0
        assert not np.any(Hb & ~(L[m + 1].pattern.toarray() > 0))
        # coarse couplings stay within offset 2 per axis
        i, j = L[m + 1].pattern.nonzero()
        off = L[m + 1].coords[i] - L[m + 1].coords[j]
        assert np.abs(off).max() <= 2


def test_colors_uncoupled_and_zero_start_forward_sweep_uses_earlier_colors_only():
    """The 27-coloring: no block couples two nodes of one color (couplings
    reach offset 2, colors repeat every 3), so the blocks of earlier-colored
    neighbours are exactly half of the off-diagonal blocks of the symmetric
    pattern.  From u = 0, a forward sweep equals the substitution that uses
    only those blocks: the later-colored neighbours are still zero when a
    row is updated."""
    sc = free_scene(9, F_jitter=0.2)
    g, prob, L = hierarchy_for(sc)
    rng = np.random.default_rng(9)
    for lev in L:
        n = lev.coords.shape[0]
        col = np.zeros(n, int)
        for c, rows in enumerate(lev.colors):
            col[rows] = c
        P = lev.pattern.tocoo()
        off = P.row != P.col
        assert np.all(col[P.row[off]] != col[P.col[off]])
        assert (lev.pattern != lev.pattern.T).nnz == 0
        nnz, earlier = P.nnz, int(np.sum(col[P.col] < col[P.row]))
        assert 2 * earlier == nnz - n
        b = rng.normal(size=(n, 3))
        u_sweep = O.sgs(lev, np.zeros((n, 3)), b, forward=True)
        H = lev.H.toarray().reshape(n, 3, n, 3)
        u = np.zeros((n, 3))
        for c in range(27):
            for i in lev.colors[c]:
                js = np.nonzero(col < c)[0]
                # H[i, :, js, :] has shape (len(js), 3, 3): the index array's axis comes first
                rhs = b[i] - np.einsum("jab,jb->a", H[i, :, js, :], u[js]) if js.size else b[i].copy()
                u[i] = np.linalg.solve(lev.Dblk[i], rhs)
        np.testing.assert_allclose(u, u_sweep, rtol=1e-12, atol=1e-12 * np.abs(u_sweep).max())


def test_galerkin_force_identity():
    """R f^0 equals the force computed with the embedded weight gradients
    sum_i R_ji grad w_ip (Sec. 4.2)."""
    sc = free_scene(8, F_jitter=0.2)
    g, prob, L = hierarchy_for(sc, levels=2)
    mu, lam, md = O.material_arrays(sc)
    P = O.first_piola(sc.F, mu, lam, md)
    K = sc.vol[:, None, None] * (P @ np.swapaxes(sc.F, 1, 2))
    f0 = np.zeros((prob.n, 3))
    np.add.at(f0, g.pidx.ravel(), -np.einsum("pab,pkb->pka", K, g.gw).reshape(-1, 3))
    R = L[0].R.toarray()
    # embedded gradient per particle and coarse node: sum_i R_ji grad w_ip
    Rp = R[:, g.pidx]                                   # (nc, N, 27)
    gw_c = np.einsum("jpk,pkb->pjb", Rp, g.gw)          # (N, nc, 3)
    f1 = -np.einsum("pab,pjb->ja", K, gw_c)
    np.testing.assert_allclose(R @ f0, f1, rtol=1e-11, atol=1e-12 * np.abs(f1).max())


def test_vcycle_symmetric_positive_with_exact_coarse_solve():
    sc = free_scene(9, F_jitter=0.2)
    g, prob, L = hierarchy_for(sc)
    vc = O.VCycle(L, g.fixed, 1e-7, 0, exact_coarse=True)
    rng = np.random.default_rng(11)
    x = rng.normal(size=(prob.n, 3))
    y = rng.normal(size=(prob.n, 3))
    Vx, Vy = vc(x), vc(y)
    a, b = np.sum(x * Vy), np.sum(Vx * y)
    assert abs(a - b) <= 1e-10 * (abs(a) + abs(b))
    assert np.sum(x * Vx) > 0


def test_vcycle_reduces_residual_and_sgs_solves_small_system():
    sc = free_scene(10, F_jitter=0.2)
    g, prob, L = hierarchy_for(sc)
    rng = np.random.default_rng(12)
    b = rng.normal(size=(prob.n, 3))
    H = L[0].H
    u = np.zeros_like(b)
    for _ in range(200):
        u = O.symmetric_gauss_seidel(L[0], u, b)
    np.testing.assert_allclose((H @ u.ravel()).reshape(-1, 3), b, atol=1e-8 * np.abs(b).max())
    vc = O.VCycle(L, g.fixed, 1e-7, 0)
    x = vc(b)
    r = b.ravel() - H @ x.ravel()
    Hinv = np.linalg.inv(H.toarray())
    assert r @ Hinv @ r < 0.5 * (b.ravel() @ Hinv @ b.ravel())


def test_coarse_pcg_tolerance_rule():
    sc = free_scene(11, F_jitter=0.2)
    g, prob, L = hierarchy_for(sc, levels=1)
    H = L[0].H
    rng = np.random.default_rng(13)
    b = rng.normal(size=(prob.n, 3)) * 1e-3
    x, its = O.coarse_pcg(H, b, 1e-7, 10000)
    d = H.diagonal()
    bn = np.sqrt(b.ravel() @ (b.ravel() / d))
    r = b.ravel() - H @ x.ravel()
    k = min(0.5, np.sqrt(max(bn, 1e-7)))
    assert np.sqrt(r @ (r / d)) <= k * bn * (1 + 1e-12)
    assert its > 0
    x0, its0 = O.coarse_pcg(H, np.zeros_like(b), 1e-7, 100)
    assert its0 == 0 and np.all(x0 == 0)


# ---------------------------------------------------------------- solver
def dense_newton(prob, tol=1e-13, iters=60):
    n = prob.n
    dv = np.zeros((n, 3))
    free3 = np.repeat(~prob.g.fixed, 3)
    for _ in range(iters):
        g = prob.gradient(dv).ravel()
        if np.linalg.norm(g) < tol:
            break
        H = prob.hessian(dv, project=False).toarray()
        step = np.zeros(3 * n)
        step[free3] = -np.linalg.solve(H[np.ix_(free3, free3)], g[free3])
        E0 = prob.energy(dv)
        a = 1.0
        while prob.energy(dv + a * step.reshape(-1, 3)) > E0 and a > 1e-12:
            a *= 0.5
        dv = dv + a * step.reshape(-1, 3)
    return dv


@pytest.mark.parametrize("model", [0, 1])
def test_hot_matches_dense_newton_on_tiny_grid(model):
    sc = scenes.tiny_scene(seed=3, res=16, cells=(1, 1, 1), lo=(6, 6, 6), ppc_axis=2,
                           model=model, E=1e4, F_jitter=0.1)
    g = O.p2g(sc)
    assert g.coords.shape[0] <= 64
    prob = O.Problem(sc, g, 2e-2)
    # relative gradient 1e-8: above the FP64 rounding floor of the
    # energy-decrease line search (1e-11 to 4e-9 on this scene)
    opts = scenes.SolverOptions(eps=1e-8, cn_mode=1, levels=2, max_iters=200)
    dv, tr = O.hot_solve(prob, opts)
    assert tr.status == "ok"
    ref = dense_newton(prob)
    np.testing.assert_allclose(dv, ref, rtol=0, atol=1e-6 * np.abs(ref).max())
    # line-search invariant: accepted energies never increase
    assert np.all(np.diff(tr.energies) <= 0)


@pytest.mark.parametrize("model", [0, 1])
def test_minimiser_is_equivariant_under_a_grid_rotation(model):
    """A quarter turn about z through a grid node of the domain's centre maps
    the grid, the stencils and the held wall layers onto themselves.  The
    incremental potential of the rotated scene (x' = c + Q(x - c), v' = Qv,
    F' = QFQ^T, C' = QCQ^T, g' = Qg) is that of the original seen in the
    rotated frame, so its minimiser is the rotated minimiser:
    dv'(c + Q(x_i - c)) = Q dv(x_i).  An axis or index transposed anywhere
    in P2G, the energy or the gradient breaks this."""
    sc = scenes.tiny_scene(seed=21, res=16, cells=(2, 1, 1), lo=(6, 6, 7), ppc_axis=2,
                           model=model, E=1e4, F_jitter=0.1, gravity=(1.0, -9.8, 0.5))
    Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    c = np.full(3, 8 * sc.dx)
    rot = copy.deepcopy(sc)
    rot.x = c + (sc.x - c) @ Q.T
    rot.v = sc.v @ Q.T
    rot.F = Q @ sc.F @ Q.T
    rot.C = Q @ sc.C @ Q.T
    rot.gravity = Q @ sc.gravity
    out = []
    for s_ in (sc, rot):
        g = O.p2g(s_)
        prob = O.Problem(s_, g, 2e-2)
        out.append((g, dense_newton(prob)))
    (g0, dv0), (g1, dv1) = out
    assert g0.coords.shape == g1.coords.shape
    k = np.rint((g0.pos - c) @ Q.T / sc.dx).astype(np.int64) + 8
    index1 = {tuple(t): i for i, t in enumerate(g1.coords.tolist())}
    perm = np.array([index1[tuple(t)] for t in k.tolist()])
    np.testing.assert_array_equal(g1.fixed[perm], g0.fixed)
    np.testing.assert_allclose(g1.m[perm], g0.m, rtol=1e-13)
    # 1e-8: the FCR stress goes through the oracle's polar decomposition, whose
    # rounding leaves Newton's minimiser ~1e-9 relative from exact; a transposed
    # axis or index would show as an O(1) difference
    np.testing.assert_allclose(dv1[perm], dv0 @ Q.T, rtol=0, atol=1e-8 * np.abs(dv0).max())


def test_free_fall_gets_gravity_increment():
    """No stress, no boundary conditions, uniform velocity: the minimiser is
    dv = dt g exactly, so every particle ends at v + dt g."""
    sc = free_scene(12)
    sc.v[:] = np.array([0.1, -0.2, 0.05])
    sc.C[:] = 0.0
    sc.F[:] = np.eye(3)
    opts = scenes.SolverOptions(eps=1e-12, cn_mode=1, dt=1e-2, levels=2)
    out, info = O.hot_step(sc, opts)
    np.testing.assert_allclose(out.v, sc.v + 1e-2 * sc.gravity[None], atol=1e-10)
    np.testing.assert_allclose(out.F, sc.F, atol=1e-10)


def test_replay_reproduces_solve():
    sc = scenes.cube_scene(seed=2, res=16, cube_lo=(5, 4, 5), side=4)
    opts = scenes.SolverOptions(eps=1e-6, cn_mode=1, dt=4e-3, levels=2)
    out, info = O.hot_step(sc, opts)
    out2, info2 = O.hot_step(sc, opts, replay=info["trace"])
    np.testing.assert_array_equal(info2["dv"], info["dv"])
    assert info["trace"].iters >= 1


def test_cn_norm_definition_and_paper_constants():
    gold = json.load(open(os.path.join(GOLD, "paper_settings.json")))
    d = scenes.SolverOptions()
    assert (d.cfl, d.levels, d.lbfgs_m, d.eps, d.fps) == (gold["cfl"], gold["levels"],
                                                          gold["lbfgs_window"], gold["eps"],
                                                          gold["fps"])
    sc = free_scene(13)
    g = O.p2g(sc)
    prob = O.Problem(sc, g, 1e-3)
    gr = np.ones((prob.n, 3))
    nrm, nfree = prob.cn_norm(gr)
    mu, lam, _ = O.material_arrays(sc)
    xi = O.xi_particle(mu[0], lam[0])          # single material: xi_i = xi_p everywhere
    expect = np.sqrt(3 * prob.n) / (gold["cn_area_factor"] * sc.dx ** 2 * 1e-3 * xi)
    np.testing.assert_allclose(nrm, expect, rtol=1e-12)
    assert nfree == prob.n


@pytest.mark.slow
def test_stretched_box_converges_in_tens_of_iterations():
    """Sec. 6.3: HOT converges in 25 iterations on the stretched box; the
    scene here is a synthetic stand-in, so only the order of magnitude is
    checked (parity of the exact count is not claimed)."""
    gold = json.load(open(os.path.join(GOLD, "paper_settings.json")))
    sc = scenes.stretched_box_scene(side=6)
    opts = scenes.SolverOptions(eps=gold["eps"], dt=1.0 / 24, levels=3)
    out, info = O.hot_step(sc, opts)
    tr = info["trace"]
    assert tr.status == "ok"
    assert 2 <= tr.iters <= 10 * gold["stretched_box_hot_iterations"]


# ---------------------------------------------------------------- plasticity
def test_von_mises_return_mapping():
    rng = np.random.default_rng(21)
    F = np.concatenate([rand_F(rng, 20, amp=0.25), rand_F(rng, 20, amp=0.003)])
    F = F[np.linalg.det(F) > 0.3]
    n = F.shape[0]
    mu = np.full(n, 5e4)
    ty = np.full(n, 2e3)
    out = O.plasticity(F, mu, np.ones(n, int), ty)
    # volume (det F) preserved; final state on or inside the yield surface
    np.testing.assert_allclose(np.linalg.det(out), np.linalg.det(F), rtol=1e-12)
    s = np.linalg.svd(out, compute_uv=False)
    e = np.log(s)
    dev = e - e.mean(1, keepdims=True)
    tau = 2 * mu * np.sqrt((dev ** 2).sum(1))
    assert np.all(tau <= ty * (1 + 1e-10))
    s0 = np.linalg.svd(F, compute_uv=False)
    e0 = np.log(s0)
    tau0 = 2 * mu * np.sqrt(((e0 - e0.mean(1, keepdims=True)) ** 2).sum(1))
    yielded = tau0 > ty
    assert yielded.any() and (~yielded).any()
    np.testing.assert_allclose(tau[yielded], ty[yielded], rtol=1e-10)
    assert np.array_equal(out[~yielded], F[~yielded])
    # rotation invariance
    Q = rand_rot(rng, n)
    np.testing.assert_allclose(O.plasticity(Q @ F, mu, np.ones(n, int), ty), Q @ out, atol=1e-12)


def test_snow_clamp():
    rng = np.random.default_rng(22)
    F = rand_F(rng, 30, amp=0.05)
    F = F[np.linalg.det(F) > 0]
    n = F.shape[0]
    out = O.plasticity(F, np.ones(n), np.full(n, 2), np.zeros(n))
    s = np.linalg.svd(out, compute_uv=False)
    assert s.min() >= 0.99 - 1e-14 and s.max() <= 1.001 + 1e-14
    inside = np.eye(3)[None] * np.array([1.0005, 0.995, 1.0])[None, None, :]
    assert np.array_equal(O.plasticity(inside, np.ones(1), np.full(1, 2), np.zeros(1)), inside)
    Q = rand_rot(rng, n)
    np.testing.assert_allclose(O.plasticity(Q @ F, np.ones(n), np.full(n, 2), np.zeros(n)), Q @ out, atol=1e-13)


# ------------------------------------------------- Alg. 1: inexact projected Newton
def test_pn_pcg_is_conjugate_gradients_with_the_inexact_stop():
    """pn_pcg run to n iterations is CG: it solves an SPD system exactly (up
    to rounding), and its own stop is the first iterate whose residual,
    recomputed as b - H x, meets sqrt(r^T P r) <= k sqrt(b^T P b) with
    k = min(0.5, sqrt(max(sqrt(b^T P b), tau))) (Sec. 5.3)."""
    rng = np.random.default_rng(11)
    n = 24
    Q = rng.normal(size=(n, n))
    H = sp.csr_matrix(Q @ Q.T + n * np.diag(rng.uniform(0.5, 4.0, n)))
    b = rng.normal(size=n) * 1e-3
    d = H.diagonal()
    jac = lambda r: r / d  # noqa: E731
    x, its = O.pn_pcg(H, b, jac, 1e-30, 1000, forced_iters=n)
    np.testing.assert_allclose(x, np.linalg.solve(H.toarray(), b), rtol=1e-9, atol=1e-15)
    x, its = O.pn_pcg(H, b, jac, 1e-30, 1000)
    bPb = float(b @ (b / d))
    k = min(0.5, np.sqrt(max(np.sqrt(bPb), 1e-30)))
    def enorm(xx):
        r = b - H @ xx
        return np.sqrt(float(r @ (r / d)))
    assert its >= 1 and enorm(x) <= k * np.sqrt(bPb) * (1 + 1e-9)
    xp, _ = O.pn_pcg(H, b, jac, 1e-30, 1000, forced_iters=its - 1)
    assert enorm(xp) > k * np.sqrt(bPb)


@pytest.mark.parametrize("precond", ["jacobi", "mg"])
def test_pn_solvers_match_dense_newton_on_tiny_grid(precond):
    sc = scenes.tiny_scene(seed=3, res=16, cells=(1, 1, 1), lo=(6, 6, 6), ppc_axis=2,
                           model=1, E=1e4, F_jitter=0.1)
    g = O.p2g(sc)
    prob = O.Problem(sc, g, 2e-2)
    opts = scenes.SolverOptions(eps=1e-8, cn_mode=1, levels=2, max_iters=200)
    dv, tr = O.pn_solve(prob, opts, precond)
    assert tr.status == "ok" and tr.iters >= 1
    ref = dense_newton(prob)
    np.testing.assert_allclose(dv, ref, rtol=0, atol=1e-6 * np.abs(ref).max())
    assert np.all(np.diff(tr.energies) <= 0)
    assert all(c >= 1 for c in tr.cg_iters)
    if precond == "mg":
        assert len(tr.vc_cg_counts) >= sum(tr.cg_iters)   # one V-cycle per CG iteration (+ the initial one)


def test_pn_replay_reproduces_solve_and_agrees_with_hot():
    sc = scenes.cube_scene(seed=2, res=16, cube_lo=(5, 4, 5), side=4)
    opts = scenes.SolverOptions(eps=1e-6, cn_mode=1, dt=4e-3, levels=2)
    grid = O.p2g(sc)
    prob = O.Problem(sc, grid, O.step_dt(sc, opts))
    for pc in ("jacobi", "mg"):
        dv, tr = O.pn_solve(prob, opts, pc)
        dv2, tr2 = O.pn_solve(prob, opts, pc, replay=tr)
        np.testing.assert_array_equal(dv2, dv)
    # all three solvers stop at the same tolerance on the same problem
    dvh, trh = O.hot_solve(prob, opts)
    assert np.abs(dv - dvh).max() <= 1e-4 * np.abs(dvh).max()


def test_hierarchy_refresh_extension_converges_and_replays():
    """The refresh extension (not in Alg. 3): rebuilding the hierarchy at the
    iterate every 2 iterations still minimises E -- it meets the dense
    Newton solution -- and replays exactly."""
    sc = scenes.tiny_scene(seed=3, res=16, cells=(1, 1, 1), lo=(6, 6, 6), ppc_axis=2,
                           model=1, E=1e4, F_jitter=0.1)
    g = O.p2g(sc)
    prob = O.Problem(sc, g, 2e-2)
    opts = scenes.SolverOptions(eps=1e-8, cn_mode=1, levels=2, max_iters=200, refresh_every=2)
    dv, tr = O.hot_solve(prob, opts)
    assert tr.status == "ok" and tr.iters > 2
    ref = dense_newton(prob)
    np.testing.assert_allclose(dv, ref, rtol=0, atol=1e-6 * np.abs(ref).max())
    dv2, _ = O.hot_solve(prob, opts, replay=tr)
    np.testing.assert_array_equal(dv2, dv)


def test_fallback_extension_finishes_with_newton_and_replays():
    """The fallback extension (not in Alg. 3): after 2 L-BFGS iterations the
    step continues as PN-MGPCG from the iterate; it still reaches the dense
    Newton solution and replays exactly."""
    sc = scenes.tiny_scene(seed=3, res=16, cells=(1, 1, 1), lo=(6, 6, 6), ppc_axis=2,
                           model=1, E=1e4, F_jitter=0.1)
    g = O.p2g(sc)
    prob = O.Problem(sc, g, 2e-2)
    opts = scenes.SolverOptions(eps=1e-8, cn_mode=1, levels=2, max_iters=200, fallback_after=2)
    dv, tr = O.hot_solve(prob, opts)
    assert tr.status == "ok" and tr.iters > 2 and len(tr.inner) == tr.iters - 2
    assert len(tr.skipped) == 2 and len(tr.alphas) == tr.iters
    ref = dense_newton(prob)
    np.testing.assert_allclose(dv, ref, rtol=0, atol=1e-6 * np.abs(ref).max())
    assert np.all(np.diff(tr.energies) <= 0)
    dv2, _ = O.hot_solve(prob, opts, replay=tr)
    np.testing.assert_array_equal(dv2, dv)


# ---------------------------------------------------------------- L-BFGS two-loop (Alg. 3)
def _pairs(rng, n, m, A=None):
    """m pairs (s, y, 1/y^T s) with positive curvature; y = A s when A is given."""
    hist = []
    if A is None:
        B = rng.normal(size=(n, n))
        A_ = B @ B.T + n * np.eye(n)
    else:
        A_ = A
    for _ in range(m):
        s = rng.normal(size=n)
        y = A_ @ s if A is not None else A_ @ s + 0.1 * rng.normal(size=n)
        ys = float(y @ s)
        assert ys > 0
        hist.append((s.reshape(-1, 3), y.reshape(-1, 3), 1.0 / ys))
    return hist


def _dense_bfgs_inverse(H0, hist):
    """The inverse-Hessian BFGS update applied pair by pair, oldest first:
    H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T."""
    H = H0.copy()
    n = H.shape[0]
    for s, y, rho in hist:
        s, y = s.ravel(), y.ravel()
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def _spd(rng, n):
    B = rng.normal(size=(n, n))
    return B @ B.T + 0.5 * n * np.eye(n)


@pytest.mark.parametrize("m", [0, 1, 3, 8])
def test_two_loop_equals_dense_bfgs_inverse_updates(m):
    """The two-loop recursion computes H q for the matrix obtained from H_0 by
    the m BFGS inverse updates (Nocedal & Wright, Alg. 7.4 against Eq. 6.17)."""
    rng = np.random.default_rng(40 + m)
    n = 24
    H0 = _spd(rng, n)
    hist = _pairs(rng, n, m)
    q = rng.normal(size=(n // 3, 3))
    got = O.two_loop(hist, q, lambda v: (H0 @ v.ravel()).reshape(v.shape))
    want = (_dense_bfgs_inverse(H0, hist) @ q.ravel()).reshape(q.shape)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_two_loop_secant_condition_and_quadratic_invariance():
    """The newest pair satisfies the secant equation H y = s; on a quadratic
    with y_j = A s_j and H_0 = A^{-1}, every update keeps H = A^{-1}, so the
    first L-BFGS direction is the Newton step."""
    rng = np.random.default_rng(7)
    n = 18
    H0 = _spd(rng, n)
    hist = _pairs(rng, n, 5)
    h0 = lambda v: (H0 @ v.ravel()).reshape(v.shape)  # noqa: E731
    s_new, y_new, _ = hist[-1]
    got = O.two_loop(hist, y_new, h0)
    assert np.abs(got - s_new).max() <= 1e-11 * np.abs(s_new).max()
    A = _spd(rng, n)
    Ainv = np.linalg.inv(A)
    histA = _pairs(rng, n, 6, A=A)
    q = rng.normal(size=(n // 3, 3))
    got = O.two_loop(histA, q, lambda v: (Ainv @ v.ravel()).reshape(v.shape))
    want = (Ainv @ q.ravel()).reshape(q.shape)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_two_loop_pins_catch_planted_mistakes():
    """Each plausible slip in the recursion -- loop order swapped, the a - beta
    update reduced to -beta, rho taken from the neighbouring pair -- breaks
    the dense-update pin above (planted in copies of the recursion)."""
    def swapped(hist, q, h0):
        alph = []
        for (s, y, rho) in hist:                     # oldest first in the first loop
            a = rho * float(np.sum(s * q))
            q = q - a * y
            alph.append(a)
        r = h0(q)
        for (s, y, rho), a in zip(reversed(hist), reversed(alph)):
            r = r + (a - rho * float(np.sum(y * r))) * s
        return r

    def dropped_a(hist, q, h0):
        for (s, y, rho) in reversed(hist):
            q = q - rho * float(np.sum(s * q)) * y
        r = h0(q)
        for (s, y, rho) in hist:
            r = r - rho * float(np.sum(y * r)) * s
        return r

    def wrong_rho(hist, q, h0):
        rhos = [h[2] for h in hist]
        rhos = rhos[1:] + rhos[:1]
        h2 = [(s, y, r) for (s, y, _), r in zip(hist, rhos)]
        return O.two_loop(h2, q, h0)

    rng = np.random.default_rng(11)
    n = 24
    H0 = _spd(rng, n)
    hist = _pairs(rng, n, 4)
    q = rng.normal(size=(n // 3, 3))
    h0 = lambda v: (H0 @ v.ravel()).reshape(v.shape)  # noqa: E731
    want = (_dense_bfgs_inverse(H0, hist) @ q.ravel()).reshape(q.shape)
    assert np.abs(O.two_loop(hist, q, h0) - want).max() <= 1e-12 * np.abs(want).max()
    for bad in (swapped, dropped_a, wrong_rho):
        assert np.abs(bad(hist, q, h0) - want).max() > 1e-6 * np.abs(want).max(), bad.__name__
