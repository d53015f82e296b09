"""FP64 oracle: pair densities, chi0, dielectric matrix, inverse, loss functions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (Hartree atomic units; 4*pi*alpha of Eq. (RPA) becomes 4*pi):

* Basis: Cartesian primitives chi_mu(r) = N r_x^lx r_y^ly r_z^lz e^{-a r^2},
  l = 0 (s) or 1 (p_x, p_y, p_z), N = (2a/pi)^{3/4} (s) and
  (2a/pi)^{3/4} 2 sqrt(a) (p).  A shell with l=1 gives three functions in
  the order x, y, z.
* Bloch sums phi_{mu k}(r) = N_k^{-1/2} sum_R e^{ik.R} chi_mu(r - tau_mu - R).
  With them, <phi_{mu,k+q}| e^{i kappa.r} |phi_{nu k}> for kappa = q + G
  equals B_{mu nu}(k; kappa) = sum_L e^{ik.L} int chi_mu(r-tau_mu)
  e^{i kappa.r} chi_nu(r - tau_nu - L) dr  (e^{iG.R} = 1 folds the double
  lattice sum into one).
* rho_t(G) = <c,k+q| e^{i(q+G).r} |v,k> = sum_{mu nu} conj(C_kq[mu,c])
  B_{mu nu}(k; q+G) C_k[nu,v],  t = (k, v, c) flattened as (k*nv + v)*nc + c.
* chi0_{GG'} = 2/(N_k V) sum_t W_t rho_t(G)^* rho_t(G'), the numerator
  <ik|e^{-i(q+G)r}|jk'><jk'|e^{i(q+G')r}|ik> of Eq. (RPA);
  W_t(w) = 1/(w - dE_t + i eta) - 1/(w + dE_t + i eta) (retarded, resonant
  plus antiresonant).
* eps_{GG'} = delta_{GG'} - v^{1/2}(q+G) chi0_{GG'} v^{1/2}(q+G'),
  v^{1/2}(k) = sqrt(4 pi)/|k|.
"""
from __future__ import annotations

import numpy as np

SQRT_PI = np.sqrt(np.pi)

# e^{-46} ~ 1e-20: Gaussian-product prefactors below this are dropped.
LATTICE_CUT = 46.0


# --------------------------------------------------------------------------
# basis bookkeeping
# --------------------------------------------------------------------------
def basis_functions(shell_atom, shell_l, shell_exp):
    """List of (shell, atom, exponent, (lx, ly, lz)) in basis order."""
    out = []
    for s, (at, l, e) in enumerate(zip(shell_atom, shell_l, shell_exp)):
        if l == 0:
            out.append((s, int(at), float(e), (0, 0, 0)))
        elif l == 1:
            for d in range(3):
                lv = [0, 0, 0]
                lv[d] = 1
                out.append((s, int(at), float(e), tuple(lv)))
        else:
            raise ValueError("only s and p shells")
    return out


def primitive_norm(a: float, l: int) -> float:
    """Normalisation of r_x^l e^{-a r^2} (l = 0 or 1 along one axis)."""
    n = (2.0 * a / np.pi) ** 0.75
    return n if l == 0 else n * 2.0 * np.sqrt(a)


# --------------------------------------------------------------------------
# closed-form Gaussian-product Fourier integral
# --------------------------------------------------------------------------
def pair_ft(a, A, la, b, Bp, lb, kappa):
    """int chi_a(r - A) e^{i kappa.r} chi_b(r - Bp) dr for normalised
    Cartesian s/p primitives.

    A: [3]; Bp: [nL][3] (centres of the second function); kappa: [nG][3].
    Returns [nL][nG] complex.

    Gaussian product theorem: e^{-a|r-A|^2} e^{-b|r-B|^2} =
    K e^{-p|r-P|^2}, p = a+b, P = (aA+bB)/p, K = e^{-ab/p |A-B|^2}.  With
    u = x - P_x the 1-D moments int u^j e^{i k u} e^{-p u^2} du are
    sqrt(pi/p) e^{-k^2/4p} times 1, ik/2p, 1/2p - k^2/4p^2 for j = 0, 1, 2,
    which gives per axis the factors E(0,0)=1, E(1,0)=PA+ik/2p,
    E(0,1)=PB+ik/2p, E(1,1)=PA PB + (PA+PB) ik/2p + 1/2p - k^2/4p^2.
    """
    A = np.asarray(A, float)
    Bp = np.atleast_2d(np.asarray(Bp, float))
    kappa = np.atleast_2d(np.asarray(kappa, float))
    p = a + b
    P = (a * A[None, :] + b * Bp) / p                               # [nL,3]
    AB2 = np.sum((A[None, :] - Bp) ** 2, axis=1)                     # [nL]
    K = np.exp(-a * b / p * AB2)                                     # [nL]
    k2 = np.sum(kappa ** 2, axis=1)                                  # [nG]
    norm = primitive_norm(a, max(la)) * primitive_norm(b, max(lb))
    base = (norm * (np.pi / p) ** 1.5) * K[:, None] * np.exp(-k2 / (4.0 * p))[None, :] \
        * np.exp(1j * (P @ kappa.T))                                 # [nL,nG]
    for x in range(3):
        if la[x] == 0 and lb[x] == 0:
            continue
        PA = (P[:, x] - A[x])[:, None]
        PB = (P[:, x] - Bp[:, x])[:, None]
        t = (1j * kappa[:, x] / (2.0 * p))[None, :]
        if la[x] == 1 and lb[x] == 0:
            E = PA + t
        elif la[x] == 0 and lb[x] == 1:
            E = PB + t
        else:
            E = PA * PB + (PA + PB) * t + 1.0 / (2.0 * p) - (kappa[:, x] ** 2 / (4.0 * p * p))[None, :]
        base = base * E
    return base


def lattice_translations(lattice, d, radius):
    """All L = n.lattice (integer n) with |d - L| <= radius."""
    lattice = np.asarray(lattice, float)
    recip = np.linalg.inv(lattice).T              # n_i = L . recip_i
    reach = np.linalg.norm(d) + radius
    nmax = [int(np.ceil(reach * np.linalg.norm(recip[i]))) + 1 for i in range(3)]
    r = [np.arange(-m, m + 1) for m in nmax]
    n = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)
    L = n @ lattice
    keep = np.sum((d[None, :] - L) ** 2, axis=1) <= radius * radius
    return L[keep]


def bloch_pair_blocks(lattice, atoms, shell_atom, shell_l, shell_exp, kpts, kappa,
                      cut=LATTICE_CUT):
    """Yield (mu, nu, B_mu_nu[k][G]) for every basis-function pair, where
    B_{mu nu}(k; kappa) = sum_L e^{ik.L} int chi_mu(r - tau_mu) e^{i kappa.r}
    chi_nu(r - tau_nu - L) dr  (the Bloch-sum matrix element of Eq. (RPA)).

    The lattice sum keeps every L whose Gaussian-product prefactor
    e^{-ab/p |tau_mu - tau_nu - L|^2} is at least e^{-cut}.  The integrals do
    not depend on k; the k dependence is the phase sum, done as a matmul.
    """
    atoms = np.asarray(atoms, float)
    kpts = np.atleast_2d(np.asarray(kpts, float))
    kappa = np.atleast_2d(np.asarray(kappa, float))
    funcs = basis_functions(shell_atom, shell_l, shell_exp)
    shells = {}
    for mu, (s, at, e, lv) in enumerate(funcs):
        shells.setdefault(s, []).append(mu)
    for sa, mus in shells.items():
        _, at_a, ea, _ = funcs[mus[0]]
        A = atoms[at_a]
        for sb, nus in shells.items():
            _, at_b, eb, _ = funcs[nus[0]]
            B = atoms[at_b]
            radius = np.sqrt(cut * (ea + eb) / (ea * eb))
            L = lattice_translations(lattice, A - B, radius)
            if L.shape[0] == 0:
                continue
            phase = np.exp(1j * (kpts @ L.T))                       # [nk,nL]
            for mu in mus:
                for nu in nus:
                    T = pair_ft(ea, A, funcs[mu][3], eb, B[None, :] + L, funcs[nu][3], kappa)
                    yield mu, nu, phase @ T


def bloch_pair_table(lattice, atoms, shell_atom, shell_l, shell_exp, kpts, kappa,
                     cut=LATTICE_CUT):
    """B[k][G][mu][nu] (see `bloch_pair_blocks`)."""
    kpts = np.atleast_2d(np.asarray(kpts, float))
    kappa = np.atleast_2d(np.asarray(kappa, float))
    nb = len(basis_functions(shell_atom, shell_l, shell_exp))
    out = np.zeros((kpts.shape[0], kappa.shape[0], nb, nb), complex)
    for mu, nu, blk in bloch_pair_blocks(lattice, atoms, shell_atom, shell_l, shell_exp,
                                         kpts, kappa, cut):
        out[:, :, mu, nu] = blk
    return out


def overlap(lattice, atoms, shell_atom, shell_l, shell_exp, kpts):
    """S_{mu nu}(k) = B_{mu nu}(k; 0): the Bloch-sum overlap matrix."""
    return bloch_pair_table(lattice, atoms, shell_atom, shell_l, shell_exp, kpts,
                            np.zeros((1, 3)))[:, 0]


# --------------------------------------------------------------------------
# the method
# --------------------------------------------------------------------------
def pair_density(Btab, Ck, Ckq):
    """rho[t][G], t = (k, v, c):  sum_{mu nu} conj(Ckq[k,mu,c]) B[k,G,mu,nu] Ck[k,nu,v].

    Btab: [nk][nG][nb][nb]; Ck: [nk][nb][nv]; Ckq: [nk][nb][nc]."""
    # [k,G,mu,v] = B @ Ck, then [k,G,c,v] = Ckq^H @ that
    BC = np.einsum("kgmn,knv->kgmv", Btab, Ck)
    r = np.einsum("kmc,kgmv->kvcg", Ckq.conj(), BC)
    nk, nv, nc, ng = r.shape
    return r.reshape(nk * nv * nc, ng)


def pair_density_lean(lattice, atoms, shell_atom, shell_l, shell_exp, kpts, kappa, Ck, Ckq,
                      cut=LATTICE_CUT):
    """Same rho[t][G] as `pair_density(bloch_pair_table(...), Ck, Ckq)` without
    holding the whole B table: Y[k,G,mu,v] = sum_nu B_{mu nu} Ck[nu,v] is
    accumulated pair by pair, then rho = Ckq^H Y."""
    nk, nb, nv = Ck.shape
    nc = Ckq.shape[2]
    ng = np.atleast_2d(kappa).shape[0]
    Y = np.zeros((nk, ng, nb, nv), complex)
    for mu, nu, blk in bloch_pair_blocks(lattice, atoms, shell_atom, shell_l, shell_exp,
                                         kpts, kappa, cut):
        Y[:, :, mu, :] += blk[:, :, None] * Ck[:, None, nu, :]
    r = np.einsum("kmc,kgmv->kvcg", Ckq.conj(), Y, optimize=True)
    return r.reshape(nk * nv * nc, ng)


def transition_energies(Ek, Ekq):
    """dE_t = E_{c,k+q} - E_{v,k}, t = (k, v, c)."""
    return (Ekq[:, None, :] - Ek[:, :, None]).reshape(-1)


def transition_weights(dE, w, eta):
    """W[w][t] = 1/(w - dE + i eta) - 1/(w + dE + i eta)."""
    w = np.asarray(w, float)[:, None]
    return 1.0 / (w - dE[None, :] + 1j * eta) - 1.0 / (w + dE[None, :] + 1j * eta)


def chi0(rho, W, nk, vcell):
    """chi0[w][G][G'] = 2/(nk V) sum_t W[w,t] conj(rho[t,G]) rho[t,G']  (Eq. (RPA), f_v - f_c = 2)."""
    pref = 2.0 / (nk * vcell)
    rh = rho.conj().T                                                # [G][t]
    out = np.empty((W.shape[0], rho.shape[1], rho.shape[1]), complex)
    for iw in range(W.shape[0]):
        out[iw] = pref * ((rh * W[iw][None, :]) @ rho)
    return out


def coulomb_sqrt(q, Gcart):
    """v^{1/2}(q+G) = sqrt(4 pi)/|q+G|."""
    return np.sqrt(4.0 * np.pi) / np.linalg.norm(np.asarray(q)[None, :] + Gcart, axis=1)


def dielectric_matrix(chi, vs):
    """eps = delta - v^{1/2} chi0 v^{1/2}  (Eq. (RPA))."""
    n = vs.shape[0]
    return np.eye(n)[None] - vs[None, :, None] * chi * vs[None, None, :]


def inverse_lu(eps):
    """Route 1: eps^{-1} by LU with partial pivoting (LAPACK via numpy)."""
    return np.linalg.inv(eps)


def inverse_dyson(chi, vs):
    """Route 2: solve chi = chi0 + chi0 v chi, then eps^{-1} = 1 + v^{1/2} chi v^{1/2}."""
    n = vs.shape[0]
    v = vs * vs
    lhs = np.eye(n)[None] - chi * v[None, None, :]
    full = np.linalg.solve(lhs, chi)
    return np.eye(n)[None] + vs[None, :, None] * full * vs[None, None, :]


def loss_functions(eps, eps_inv=None):
    """L_LFE[w][G] = -Im [eps^{-1}]_{GG} (Eq. (eps_LFE)); L_noLFE[w][G] =
    -Im (1/eps_{GG}) = Im eps_GG / |eps_GG|^2 (Eq. (eps_noLFE))."""
    if eps_inv is None:
        eps_inv = inverse_lu(eps)
    dinv = np.einsum("wgg->wg", eps_inv)
    d = np.einsum("wgg->wg", eps)
    return -dinv.imag, (-(1.0 / d)).imag, dinv, d


# --------------------------------------------------------------------------
# states (test set-up): S(k)-orthonormal coefficients from raw draws
# --------------------------------------------------------------------------
def orthonormalise(S, Z):
    """C = L^{-H} Q with S = L L^H and Q the orthonormal factor of L^H Z,
    so that C^H S C = 1.  S: [nk][nb][nb]; Z: [nk][nb][m]."""
    out = np.empty_like(Z)
    for k in range(S.shape[0]):
        L = np.linalg.cholesky(S[k])
        Q, _ = np.linalg.qr(L.conj().T @ Z[k])
        out[k] = np.linalg.solve(L.conj().T, Q)
    return out


def states(problem, iq=None, cut=LATTICE_CUT):
    """Orthonormal coefficients at k (and at k+q for q number iq) for a
    `synth.Problem`: C_k [nk][nb][nv] and C_kq [nk][nb][nc]."""
    c = problem.cell
    b = problem.basis
    Sk = overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, problem.kpts)
    Ck = orthonormalise(Sk, problem.Zk)
    if iq is None:
        return Ck
    kq = problem.kpts + problem.qpts[iq][None, :]
    Skq = overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, kq)
    return Ck, orthonormalise(Skq, problem.zkq(iq))


def solve_q(problem, iq, Ck=None, Ckq=None, w=None):
    """The whole path for one q: rho, chi0, eps, eps^{-1} diagonal, losses.

    Returns a dict with rho [nt][nG], chi0 [nw][nG][nG], eps, L_lfe, L_nolfe,
    eps_inv_diag, eps_diag."""
    c = problem.cell
    b = problem.basis
    if Ck is None or Ckq is None:
        Ck, Ckq = states(problem, iq)
    w = problem.w if w is None else np.asarray(w)
    q = problem.qpts[iq]
    Gc = problem.G_int @ c.recip
    kappa = q[None, :] + Gc
    rho = pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp,
                            problem.kpts, kappa, Ck, Ckq)
    dE = transition_energies(problem.Ek, problem.Ekq[iq])
    W = transition_weights(dE, w, problem.eta)
    chi = chi0(rho, W, problem.nk, c.volume)
    vs = coulomb_sqrt(q, Gc)
    eps = dielectric_matrix(chi, vs)
    L_lfe, L_nolfe, dinv, d = loss_functions(eps)
    return {"rho": rho, "chi0": chi, "eps": eps, "L_lfe": L_lfe, "L_nolfe": L_nolfe,
            "eps_inv_diag": dinv, "eps_diag": d, "dE": dE, "vs": vs, "Ck": Ck, "Ckq": Ckq}


# --------------------------------------------------------------------------
# uneven instances: one (q, w) block each, G set {G : |q+G| < G_max}
# --------------------------------------------------------------------------
def g_ball(recip, q, gmax):
    """Integer G (rows of `recip` as basis) with |q + G| < gmax, in the order
    of a plain scan over a bounding box (any order serves: the head is found
    by its value G = 0)."""
    recip = np.asarray(recip, float)
    # |n_i| = |a_i . G| / (2 pi) <= |a_i| |G| / (2 pi), |G| < gmax + |q|
    lat = 2.0 * np.pi * np.linalg.inv(recip).T
    reach = gmax + np.linalg.norm(q)
    m = [int(np.ceil(np.linalg.norm(lat[i]) * reach / (2.0 * np.pi))) + 1 for i in range(3)]
    out = []
    for n1 in range(-m[0], m[0] + 1):
        for n2 in range(-m[1], m[1] + 1):
            for n3 in range(-m[2], m[2] + 1):
                k = np.asarray(q) + n1 * recip[0] + n2 * recip[1] + n3 * recip[2]
                if np.dot(k, k) < gmax * gmax:
                    out.append((n1, n2, n3))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def solve_instances(problem, inst_q, inst_w, inst_gmax, states_by_q):
    """Heads of the loss functions of independent (q, w) blocks whose G sets
    are {G : |q+G| < G_max} (uneven sizes): per instance the steps of
    `solve_q` (Eq. (RPA), the Dyson step, Eqs. (eps_LFE), (eps_noLFE)) for one
    frequency, returning L_LFE = -Im [eps^{-1}]_{00} and L_noLFE =
    -Im (1/eps_00) at the head G = 0, and N_G.  Pair densities are formed once
    per q on the largest of that q's G sets and restricted by G value.
    states_by_q: {iq: (Ck, Ckq)}."""
    c = problem.cell
    b = problem.basis
    inst_q = np.asarray(inst_q)
    n = inst_q.shape[0]
    L1 = np.empty(n)
    L2 = np.empty(n)
    ngs = np.empty(n, dtype=np.int64)
    for iq in np.unique(inst_q):
        sel = np.nonzero(inst_q == iq)[0]
        q = problem.qpts[iq]
        Ck, Ckq = states_by_q[int(iq)]
        Gu = g_ball(c.recip, q, float(np.max(np.asarray(inst_gmax)[sel])))
        col = {tuple(g): j for j, g in enumerate(Gu)}
        kappa = q[None, :] + Gu @ c.recip
        rho_u = pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp,
                                  problem.kpts, kappa, Ck, Ckq)
        dE = transition_energies(problem.Ek, problem.Ekq[iq])
        for i in sel:
            Gi = g_ball(c.recip, q, float(inst_gmax[i]))
            cols = np.array([col[tuple(g)] for g in Gi])
            head = int(np.nonzero(np.all(Gi == 0, axis=1))[0][0])
            W = transition_weights(dE, [inst_w[i]], problem.eta)
            chi = chi0(rho_u[:, cols], W, problem.nk, c.volume)
            eps = dielectric_matrix(chi, coulomb_sqrt(q, Gi @ c.recip))
            Lf, Ln, _, _ = loss_functions(eps)
            L1[i] = Lf[0, head]
            L2[i] = Ln[0, head]
            ngs[i] = Gi.shape[0]
    return L1, L2, ngs


# --------------------------------------------------------------------------
# kinetic matrix (for the f-sum check only)
# --------------------------------------------------------------------------
def _gauss_moment(n, p):
    """int u^n e^{-p u^2} du."""
    if n % 2:
        return 0.0
    df = 1.0
    for m in range(n - 1, 0, -2):
        df *= m
    return np.sqrt(np.pi / p) * df / (2.0 * p) ** (n // 2)


def _overlap_1d(la, lb, A, B, a, b):
    """int (x-A)^la (x-B)^lb e^{-a(x-A)^2 - b(x-B)^2} dx, la, lb >= 0 (B may be an array)."""
    from math import comb
    if la < 0 or lb < 0:
        return np.zeros_like(np.asarray(B, float))
    p = a + b
    B = np.asarray(B, float)
    P = (a * A + b * B) / p
    PA, PB = P - A, P - B
    tot = np.zeros_like(B)
    for i in range(la + 1):
        for j in range(lb + 1):
            tot = tot + comb(la, i) * comb(lb, j) * PA ** (la - i) * PB ** (lb - j) * _gauss_moment(i + j, p)
    return np.exp(-a * b / p * (A - B) ** 2) * tot


def _laplace_1d(la, lb, A, B, a, b):
    """int (x-A)^la e^{-a(x-A)^2} d^2/dx^2 [(x-B)^lb e^{-b(x-B)^2}] dx."""
    return (lb * (lb - 1) * _overlap_1d(la, lb - 2, A, B, a, b)
            - 2.0 * b * (2 * lb + 1) * _overlap_1d(la, lb, A, B, a, b)
            + 4.0 * b * b * _overlap_1d(la, lb + 2, A, B, a, b))


def kinetic(lattice, atoms, shell_atom, shell_l, shell_exp, kpts, cut=LATTICE_CUT):
    """T_{mu nu}(k) = sum_L e^{ik.L} (1/2) int grad chi_mu(r - tau_mu) . grad chi_nu(r - tau_nu - L) dr."""
    atoms = np.asarray(atoms, float)
    kpts = np.atleast_2d(np.asarray(kpts, float))
    funcs = basis_functions(shell_atom, shell_l, shell_exp)
    nb = len(funcs)
    out = np.zeros((kpts.shape[0], nb, nb), complex)
    for mu, (_, at_a, ea, la) in enumerate(funcs):
        A = atoms[at_a]
        for nu, (_, at_b, eb, lb) in enumerate(funcs):
            B = atoms[at_b]
            radius = np.sqrt(cut * (ea + eb) / (ea * eb))
            L = lattice_translations(lattice, A - B, radius)
            Bp = B[None, :] + L
            S1 = [_overlap_1d(la[x], lb[x], A[x], Bp[:, x], ea, eb) for x in range(3)]
            D1 = [_laplace_1d(la[x], lb[x], A[x], Bp[:, x], ea, eb) for x in range(3)]
            lap = D1[0] * S1[1] * S1[2] + S1[0] * D1[1] * S1[2] + S1[0] * S1[1] * D1[2]
            val = -0.5 * primitive_norm(ea, max(la)) * primitive_norm(eb, max(lb)) * lap
            out[:, mu, nu] = np.exp(1j * (kpts @ L.T)) @ val
    return out
