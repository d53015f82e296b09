"""FP64 oracle of the optical limit q -> 0 of the RPA dielectric matrix
(Appendix C, Eq. (ol_overlap) and the head and wing formulas after it).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For q -> 0 the G = 0 row and column of Eq. (RPA) carry 1/|q| factors.  First
order perturbation theory in q (Eqs. (V_perturb), (ol_overlap)) gives, for
Bloch eigenstates at the same k,

    rho_t(0) = <c,k+q| e^{iq.r} |v,k>  ->  -(i/m_e) q . <c k|grad|v k> / dE_t,

(the conjugate of Eq. (ol_overlap) with i = v, j = c, and <v|grad|c>^* =
-<c|grad|v>), so |q| cancels against v^{1/2}(q) = sqrt(4 pi)/|q|.  Reading
(the construction used here): the optical-limit matrix is Eq. (RPA) with the
G = 0 column of rho replaced by

    rho~_t = -i (qhat . p_t) / dE_t,    p_t = <c k|grad|v k>   (m_e = 1),

and v^{1/2}(0) replaced by sqrt(4 pi).  This is the q -> 0 limit of Eq. (RPA)
term by term; it reproduces the appendix's eps_0G' and fixes the signs of the
head (the appendix prints "1 +", which would make Im eps_00 negative) and of
eps_G0 (the appendix's "-i" breaks the Hermitian structure that the other two
have); see the pins.

Momentum matrix of the Bloch sums (same k on both sides):

    P_{mu nu}(k) = sum_L e^{ik.L} int chi_mu(r - tau_mu) grad chi_nu(r - tau_nu - L) dr,
    <c k|grad|v k> = sum_{mu nu} conj(C_c[mu]) P_{mu nu}(k) C_v[nu],

with the one-dimensional factors of the Cartesian Gaussians
    d/dx [(x-B)^l e^{-b(x-B)^2}] = l (x-B)^{l-1} e^{..} - 2b (x-B)^{l+1} e^{..}.
"""
from __future__ import annotations

import numpy as np

from . import rpa


def _deriv_1d(la, lb, A, B, a, b):
    """int (x-A)^la e^{-a(x-A)^2} d/dx[(x-B)^lb e^{-b(x-B)^2}] dx (B may be an array)."""
    return lb * rpa._overlap_1d(la, lb - 1, A, B, a, b) - 2.0 * b * rpa._overlap_1d(la, lb + 1, A, B, a, b)


def momentum_matrix(lattice, atoms, shell_atom, shell_l, shell_exp, kpts, cut=rpa.LATTICE_CUT):
    """P[k][x][mu][nu] = sum_L e^{ik.L} int chi_mu(r - tau_mu) d/dr_x chi_nu(r - tau_nu - L) dr,
    the lattice kept as in the overlap (Gaussian-product prefactor >= e^{-cut})."""
    atoms = np.asarray(atoms, float)
    kpts = np.atleast_2d(np.asarray(kpts, float))
    funcs = rpa.basis_functions(shell_atom, shell_l, shell_exp)
    nb = len(funcs)
    out = np.zeros((kpts.shape[0], 3, nb, nb), complex)
    for mu, (_, at_a, ea, la) in enumerate(funcs):
        A = atoms[at_a]
        for nu, (_, at_b, eb, lb) in enumerate(funcs):
            B = atoms[at_b]
            radius = np.sqrt(cut * (ea + eb) / (ea * eb))
            L = rpa.lattice_translations(lattice, A - B, radius)
            Bp = B[None, :] + L
            S1 = [rpa._overlap_1d(la[x], lb[x], A[x], Bp[:, x], ea, eb) for x in range(3)]
            D1 = [_deriv_1d(la[x], lb[x], A[x], Bp[:, x], ea, eb) for x in range(3)]
            norm = rpa.primitive_norm(ea, max(la)) * rpa.primitive_norm(eb, max(lb))
            phase = np.exp(1j * (kpts @ L.T))
            for x in range(3):
                val = norm * (D1[x] * S1[(x + 1) % 3] * S1[(x + 2) % 3])
                out[:, x, mu, nu] = phase @ val
    return out


def momentum_elements(P, Cv, Cc):
    """p[t][x] = <c k|d/dr_x|v k>, t = (k, v, c)."""
    nk, nv, nc = Cv.shape[0], Cv.shape[2], Cc.shape[2]
    p = np.einsum("kmc,kxmn,knv->kvcx", Cc.conj(), P, Cv, optimize=True)
    return p.reshape(nk * nv * nc, 3)


def optical_column(p, dE, qhat):
    """rho~_t = -i (qhat . p_t) / dE_t: rho_t(G = 0)/|q| in the limit q -> 0 along qhat."""
    qhat = np.asarray(qhat, float) / np.linalg.norm(qhat)
    return -1j * (p @ qhat) / dE


def states_joint(problem):
    """Valence and conduction coefficients at the same k orthonormalised together
    (as eigenvectors of one H(k) are): C = L^{-H} Q for [Z_v | Z_c], split by columns.
    Needs q = 0 as the problem's first q."""
    c, b = problem.cell, problem.basis
    S = rpa.overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, problem.kpts)
    C = rpa.orthonormalise(S, np.concatenate([problem.Zk, problem.zkq(0)], axis=2))
    return C[:, :, :problem.nv], C[:, :, problem.nv:]


def solve_optical(problem, qhat, Cv, Cc, w=None):
    """The path at q -> 0 along qhat for the problem's G set (which must hold G = 0):
    pair densities at kappa = G with the G = 0 column replaced by rho~, v^{1/2}(0) =
    sqrt(4 pi), then chi0, eps, eps^{-1} diagonal and losses as at finite q."""
    c, b = problem.cell, problem.basis
    w = problem.w if w is None else np.asarray(w)
    Gc = problem.G_int @ c.recip
    g0 = np.flatnonzero(np.all(problem.G_int == 0, axis=1))
    if g0.size != 1:
        raise ValueError("the G set must hold G = 0 once")
    g0 = int(g0[0])
    rho = rpa.pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp,
                                problem.kpts, Gc, Cv, Cc)
    P = momentum_matrix(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, problem.kpts)
    p = momentum_elements(P, Cv, Cc)
    dE = rpa.transition_energies(problem.Ek, problem.Ekq[0])
    rho[:, g0] = optical_column(p, dE, qhat)
    vs = np.empty(Gc.shape[0])
    nz = np.arange(Gc.shape[0]) != g0
    vs[nz] = np.sqrt(4.0 * np.pi) / np.linalg.norm(Gc[nz], axis=1)
    vs[g0] = np.sqrt(4.0 * np.pi)
    W = rpa.transition_weights(dE, w, problem.eta)
    chi = rpa.chi0(rho, W, problem.nk, c.volume)
    eps = rpa.dielectric_matrix(chi, vs)
    L_lfe, L_nolfe, dinv, d = rpa.loss_functions(eps)
    return {"rho": rho, "p": p, "P": P, "dE": dE, "vs": vs, "g0": g0, "chi0": chi, "eps": eps,
            "L_lfe": L_lfe, "L_nolfe": L_nolfe, "eps_inv_diag": dinv, "eps_diag": d}
