"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test names the paper passage it relies on and the kind of mistake it
catches.  None of these compares the oracle with a retyped copy of itself:
the references are real-space quadrature, closed forms of textbook limits,
sum rules, analyticity (Kramers-Kronig), eigenvalue problems solved by LAPACK,
and brute-force velocity integrals.
"""
import numpy as np
import pytest

import synth
from oracle import rate, rpa
from tests import realspace


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _tiny_states(p, iq=0):
    Ck, Ckq = rpa.states(p, iq)
    return Ck, Ckq


def _funcs(b):
    return rpa.basis_functions(b.shell_atom, b.shell_l, b.shell_exp)


# ---------------------------------------------------------------------------
# 1. closed-form Gaussian-product integrals vs real-space quadrature
# ---------------------------------------------------------------------------
def test_pair_ft_isolated_vs_quadrature():
    """Eq. (RPA) matrix elements start from int chi_a e^{i kappa.r} chi_b dr.
    Compare the closed form with a dense Cartesian-grid quadrature for every
    s/p combination (catches wrong E(1,1) terms, normalisation, phase sign)."""
    rng = np.random.default_rng(3)
    h = 0.2
    x = np.arange(-8.0, 8.0, h)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r = np.stack([X, Y, Z], -1).reshape(-1, 3)
    A = rng.uniform(-0.6, 0.6, 3)
    Bc = rng.uniform(-0.6, 0.6, 3)
    a, b = 0.9, 1.4
    kap = np.array([[0.0, 0.0, 0.0], [0.7, -0.4, 1.1], [2.0, 0.3, -1.5]])
    ls = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    worst = 0.0
    for la in ls:
        fa = realspace.primitive_values(r, A, a, la)
        for lb in ls:
            fb = realspace.primitive_values(r, Bc, b, lb)
            ref = [(fa * fb * np.exp(1j * (r @ k))).sum() * h ** 3 for k in kap]
            got = rpa.pair_ft(a, A, la, b, Bc[None, :], lb, kap)[0]
            worst = max(worst, np.max(np.abs(got - np.array(ref))))
    assert worst < 1e-9


def test_bloch_pair_table_vs_periodic_quadrature():
    """Check 1: the Bloch-sum matrix element <phi_{mu,k+q}|e^{i(q+G).r}|phi_{nu k}>
    (Eq. (RPA) numerator; Bloch form of Appendix C) against quadrature of the
    quasi-periodic Bloch sums over one cell.  Catches the phase convention
    (e^{ik.L} vs e^{i(k+q).L}), the lattice-sum truncation and the G folding."""
    p = synth.make_tiny(shells_per_atom=1)
    c, b = p.cell, p.basis
    funcs = _funcs(b)
    # generic k (not a half reciprocal vector, where e^{ik.L} = +-1 would hide the phase sign)
    kgen = np.array([[0.11, -0.07, 0.19], [0.31, 0.05, -0.23]])
    for ik, iq in [(0, 0), (1, 1)]:
        k, q = kgen[ik], p.qpts[iq]
        kap = q[None, :] + p.G_int[[0, 3, 7]] @ c.recip
        Bq, *_ = realspace.matrix_elements(c.lattice, c.atoms, funcs, k, q, kap, n=32, reach=18.0)
        Bo = rpa.bloch_pair_table(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp,
                                  k[None, :], kap)[0]
        assert np.max(np.abs(Bq - Bo)) < 1e-10 * np.max(np.abs(Bo))


def test_pair_density_vs_quadrature_of_states():
    """rho_vck(q+G) = <c,k+q|e^{i(q+G).r}|v,k> computed from Bloch states
    tabulated on the grid (catches conj on the wrong coefficient set and the
    t = (k, v, c) ordering)."""
    p = synth.make_tiny(shells_per_atom=1, nv=2, nc=2, ng=9)
    c, b = p.cell, p.basis
    Ck, Ckq = _tiny_states(p, 0)
    funcs = _funcs(b)
    ik = 3
    k, q = p.kpts[ik], p.qpts[0]
    kap = q[None, :] + p.G_int @ c.recip
    _, fk, fkq, r, vol = realspace.matrix_elements(c.lattice, c.atoms, funcs, k, q, kap[:1], n=32, reach=18.0)
    psi_v = Ck[ik].T @ fk                   # [nv][N]
    psi_c = Ckq[ik].T @ fkq                 # [nc][N]
    Bt = rpa.bloch_pair_table(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts, kap)
    rho = rpa.pair_density(Bt, Ck, Ckq)
    for v in range(p.nv):
        for cc in range(p.nc):
            t = (ik * p.nv + v) * p.nc + cc
            for g in range(p.ng):
                ref = (psi_c[cc].conj() * np.exp(1j * (r @ kap[g])) * psi_v[v]).sum() * vol / r.shape[0]
                assert abs(rho[t, g] - ref) < 1e-10


def test_pair_density_lean_equals_table_route():
    p = synth.make_tiny(shells_per_atom=2)
    c, b = p.cell, p.basis
    Ck, Ckq = _tiny_states(p, 1)
    kap = p.qpts[1][None, :] + p.G_int @ c.recip
    Bt = rpa.bloch_pair_table(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts, kap)
    r1 = rpa.pair_density(Bt, Ck, Ckq)
    r2 = rpa.pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts, kap, Ck, Ckq)
    assert np.max(np.abs(r1 - r2)) < 1e-13 * np.max(np.abs(r1))


# ---------------------------------------------------------------------------
# 2. orthonormality
# ---------------------------------------------------------------------------
def test_states_orthonormal_and_rho_q0_is_identity():
    """Check 2: with q = 0 and G = 0, rho_{vck} = <c,k|v,k> = delta for
    S(k)-orthonormal states (catches normalisation of the overlap)."""
    p = synth.make_small(nq=1)
    c, b = p.cell, p.basis
    S = rpa.overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts[:6])
    Z = synth.random_coeffs(np.random.default_rng(0), (6, b.nbasis, 8))
    C = rpa.orthonormalise(S, Z)
    Bt = rpa.bloch_pair_table(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts[:6],
                              np.zeros((1, 3)))
    rho = rpa.pair_density(Bt, C, C).reshape(6, 8, 8)
    assert np.max(np.abs(rho - np.eye(8)[None])) < 1e-12
    # the overlap of one isolated tight s Gaussian with itself is 1
    assert abs(S[0, 0, 0] - 1.0) < 2e-2 and np.all(np.linalg.eigvalsh(S) > 0)


# ---------------------------------------------------------------------------
# 3-5. identities and signs of the dielectric matrix
# ---------------------------------------------------------------------------
def _small_q(iq=3, nw=50, ng=None):
    p = synth.make_small(nq=iq + 1, nw=nw)
    if ng is not None:
        p.G_int = p.G_int[:ng]
    return p, rpa.solve_q(p, iq)


def test_ng1_lfe_equals_nolfe():
    """Check 3: keeping only G = 0, eps^{-1}_{00} = 1/eps_00, so the
    loss with local fields equals the loss without them (Eqs. (eps_LFE),
    (eps_noLFE))."""
    _, r = _small_q(ng=1)
    assert np.max(np.abs(r["L_lfe"] - r["L_nolfe"])) <= 1e-14 * max(1.0, np.max(np.abs(r["L_lfe"])))


def test_loss_positive():
    """Check 5: for w > 0 the anti-Hermitian part of eps is positive
    semidefinite with retarded weights, so both loss functions are >= 0 for
    every G (catches a conjugated weight, the advanced sign of i eta, or a
    flipped Coulomb sign)."""
    for iq in (0, 4, 9):
        p = synth.make_small(nq=iq + 1, nw=50)
        r = rpa.solve_q(p, iq)
        assert r["L_lfe"][1:].min() >= -1e-14
        assert r["L_nolfe"][1:].min() >= -1e-14
        assert np.max(np.abs(r["L_lfe"][0])) < 1e-13   # w = 0: no absorption


def test_single_oscillator_peak():
    """Check 4: one transition, N_G = 1: eps = 1 - v (2/V)|rho|^2 2dE/((w+i eta)^2 - dE^2)
    is a Lorentz oscillator whose loss peak sits at w_L^2 = dE^2 + 2 dE v (2/V)|rho|^2
    (the textbook plasmon-shifted resonance).  The oracle's peak is located on
    a fine grid."""
    p = synth.make_tiny(n_k=1, nv=1, nc=1, ng=1, nq=1)
    c, b = p.cell, p.basis
    Ck, Ckq = _tiny_states(p, 0)
    p.w = np.linspace(0.01, 3.0, 60001)
    p.eta = 1e-5
    r = rpa.solve_q(p, 0, Ck, Ckq)
    dE = r["dE"][0]
    v = r["vs"][0] ** 2
    osc = v * 2.0 / c.volume * abs(r["rho"][0, 0]) ** 2
    wl = np.sqrt(dE ** 2 + 2.0 * dE * osc)
    wpk = p.w[np.argmax(r["L_lfe"][:, 0])]
    assert abs(wpk - wl) < 2 * (p.w[1] - p.w[0])
    # and the resonance itself is not a loss peak (it is screened away)
    assert r["L_lfe"][np.argmin(abs(p.w - dE)), 0] < 1e-3 * r["L_lfe"].max()


def test_hermitian_parts_and_reflection():
    """Check 11: chi0 built with the real weights Re W and Im W are Hermitian,
    and chi0(-w) = chi0(w)^H (catches rho rho instead of rho^* rho and a
    mis-indexed contraction)."""
    p = synth.make_small(nq=1, nw=8)
    r = rpa.solve_q(p, 0)
    W = rpa.transition_weights(r["dE"], p.w[:4], p.eta)
    pre = dict(nk=p.nk, vcell=p.cell.volume)
    for part in (W.real + 0j, W.imag + 0j):
        ch = rpa.chi0(r["rho"], part, **pre)
        assert np.max(np.abs(ch - ch.conj().transpose(0, 2, 1))) < 1e-13 * np.max(np.abs(ch))
    chp = rpa.chi0(r["rho"], W, **pre)
    chm = rpa.chi0(r["rho"], rpa.transition_weights(r["dE"], -p.w[:4], p.eta), **pre)
    assert np.max(np.abs(chm - chp.conj().transpose(0, 2, 1))) < 1e-13 * np.max(np.abs(chp))


def test_two_dyson_routes_agree():
    """Check 10: eps^{-1} by LU and by solving chi = chi0 + chi0 v chi agree."""
    p, r = _small_q(iq=6)
    a = rpa.inverse_lu(r["eps"])
    bb = rpa.inverse_dyson(r["chi0"], r["vs"])
    assert np.max(np.abs(a - bb)) < 1e-12 * np.max(np.abs(a))


# ---------------------------------------------------------------------------
# 6-7. analyticity and sum rules
# ---------------------------------------------------------------------------
def _hilbert_re_from_im(w, im, x):
    """Re f(x) from the odd extension of a piecewise-linear Im f on [0, w_max]:
    Re f(x) = (1/pi) P int Im f(w')/(w' - x) dw', integrated exactly per
    linear segment (x must not be a grid point)."""
    ws = np.concatenate([-w[::-1], w[1:]])
    ims = np.concatenate([-im[::-1], im[1:]])
    a, b = ws[:-1], ws[1:]
    ga, gb = ims[:-1], ims[1:]
    s = (gb - ga) / (b - a)
    out = np.empty(len(x))
    for i, xv in enumerate(x):
        out[i] = np.sum(s * (b - a) + (ga + s * (xv - a)) * np.log(np.abs((b - xv) / (a - xv))))
    return out / np.pi


def test_kramers_kronig_of_inverse_diagonal():
    """Check 6: f(w) = [eps^{-1}]_GG - 1 is analytic in the upper half plane
    (retarded weights), f(-w) = conj f(w), so Re f follows from Im f by the
    Kramers-Kronig transform (the paper obtains the principal-value part this
    way, Section II.D footnote).  Catches a missing antiresonant term, the
    advanced sign of i eta and a wrong conjugation."""
    p = synth.make_tiny(n_k=2, nv=2, nc=3, ng=4, nq=1)
    Ck, Ckq = _tiny_states(p, 0)
    p.eta = 0.02
    w = np.linspace(0.0, 60.0, 120001)
    p.w = w
    r = rpa.solve_q(p, 0, Ck, Ckq)
    idx = np.linspace(50, 6000, 40).astype(int)          # probe points below 3 Ha
    x = 0.5 * (w[idx] + w[idx + 1])
    for g in range(p.ng):
        f = r["eps_inv_diag"][:, g] - 1.0
        re = _hilbert_re_from_im(w, f.imag, x)
        ref = 0.5 * (f.real[idx] + f.real[idx + 1])
        assert np.max(np.abs(re - ref)) < 2e-3 * np.max(np.abs(f))


def test_first_moment_sum_rule_all_three():
    """Check 7: int_0^inf w Im eps_GG dw = int w L_LFE dw = int w L_noLFE dw
    = (pi/2) Omega_G^2 with Omega_G^2 = v(q+G) 2/(N_k V) sum_t 2 dE_t |rho_t(G)|^2,
    for any eta: local fields redistribute spectral weight without changing
    the first moment (the structure of Eq. (sum_rule)).  The tail beyond the
    grid is added from the 1/w^3 asymptote of Im eps."""
    p = synth.make_tiny(n_k=2, nv=2, nc=3, ng=9, nq=1)
    Ck, Ckq = _tiny_states(p, 0)
    p.eta = 0.01
    wmax = 40.0
    p.w = np.linspace(0.0, wmax, 200001)
    r = rpa.solve_q(p, 0, Ck, Ckq)
    v = r["vs"] ** 2
    rho2 = np.abs(r["rho"]) ** 2
    pref = 2.0 / (p.nk * p.cell.volume)
    omega2 = v * pref * np.sum(2.0 * r["dE"][:, None] * rho2, axis=0)
    # tail: Im eps_GG ~ v pref sum_t 4 eta dE |rho|^2 / w^3  ->  int_wmax^inf w (.) dw
    tail = v * pref * np.sum(4.0 * p.eta * r["dE"][:, None] * rho2, axis=0) / wmax
    m_eps = np.trapezoid(p.w[:, None] * r["eps_diag"].imag, p.w, axis=0) + tail
    m_lfe = np.trapezoid(p.w[:, None] * r["L_lfe"], p.w, axis=0) + tail
    m_no = np.trapezoid(p.w[:, None] * r["L_nolfe"], p.w, axis=0) + tail
    target = 0.5 * np.pi * omega2
    for m in (m_eps, m_lfe, m_no):
        assert np.max(np.abs(m / target - 1.0)) < 2e-3


def test_fsum_within_basis_truncation():
    """Check 8 (Eq. (sum_rule)): for eigenstates of the free-electron
    Hamiltonian in the Gaussian basis, the Thomas-Reiche-Kuhn sum over all
    final bands, sum_j (E_j - E_i)|<j,k+q|e^{i kappa.r}|i,k>|^2, approaches
    kappa^2/2 as the basis grows.  Then the high-frequency limit of the
    oracle's own chi0, w^2 v(q) chi0_00(w) -> Omega^2, approaches the plasma
    frequency omega_p^2 = 4 pi n_e with n_e = 2 N_v / V: this pins the
    1/(N_k V), spin and 4 pi factors of Eq. (RPA) and the scale of rho."""
    trk, plasma = [], []
    for shells in (2, 4, 6):
        p = synth.make_tiny(shells_per_atom=shells, n_k=2, nv=1, nc=1, ng=1, nq=1, lo=0.08, hi=3.0, seed=11)
        c, b = p.cell, p.basis
        q = np.array([0.25, 0.1, -0.15])
        kq = p.kpts + q[None, :]
        def eig(kk):
            S = rpa.overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, kk)
            T = rpa.kinetic(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, kk)
            E, C = [], []
            for i in range(S.shape[0]):
                L = np.linalg.cholesky(S[i])
                Li = np.linalg.inv(L)
                e, u = np.linalg.eigh(Li @ T[i] @ Li.conj().T)
                E.append(e)
                C.append(Li.conj().T @ u)
            return np.array(E), np.array(C)
        Ek, Ck = eig(p.kpts)
        Ekq, Ckq = eig(kq)
        nv = 2
        kap = q[None, :]
        Bt = rpa.bloch_pair_table(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts, kap)
        rho = rpa.pair_density(Bt, Ck[:, :, :nv], Ckq)            # all bands at k+q
        dE = rpa.transition_energies(Ek[:, :nv], Ekq)
        trk.append(np.sum(dE * np.abs(rho[:, 0]) ** 2) / (p.nk * nv) / (0.5 * q @ q))
        wbig = np.array([1.0e5])
        ch = rpa.chi0(rho, rpa.transition_weights(dE, wbig, 1e-3), p.nk, c.volume)[0, 0, 0]
        vq = rpa.coulomb_sqrt(q, np.zeros((1, 3)))[0] ** 2
        omega2 = (wbig[0] ** 2 * vq * ch).real
        plasma.append(omega2 / (4.0 * np.pi * 2.0 * nv / c.volume))
    for r in (np.array(trk), np.array(plasma)):
        err = np.abs(r - 1.0)
        assert err[-1] < 0.05
        assert err[-1] < err[0]


def test_casida_poles():
    """Check 9: with eta -> 0 the poles of eps^{-1} are the roots of
    det(w^2 - D^2 - 2 D^{1/2} K D^{1/2}) with D = diag(dE) and
    K = 2/(N_k V) R v R^H (R[t][G] = rho_t(G)), a Hermitian eigenproblem
    solved by LAPACK.  Every loss peak of the head must sit on one of them
    (catches errors in the full local-field matrix path)."""
    p = synth.make_tiny(n_k=1, nv=2, nc=2, ng=4, nq=1)
    Ck, Ckq = _tiny_states(p, 0)
    p.eta = 2e-5
    p.w = np.linspace(0.01, 2.5, 250001)
    r = rpa.solve_q(p, 0, Ck, Ckq)
    R = r["rho"]
    v = r["vs"] ** 2
    K = 2.0 / (p.nk * p.cell.volume) * (R * v[None, :]) @ R.conj().T
    D = np.diag(r["dE"])
    Dh = np.sqrt(D)
    poles = np.sqrt(np.linalg.eigvalsh(D @ D + 2.0 * Dh @ K @ Dh))
    L = r["L_lfe"][:, 0]
    pk = [i for i in range(1, len(L) - 1) if L[i] > L[i - 1] and L[i] >= L[i + 1] and L[i] > 1e-6 * L.max()]
    assert len(pk) >= 1
    dw = p.w[1] - p.w[0]
    for i in pk:
        assert np.min(np.abs(poles - p.w[i])) < 3 * dw
    # the strongest peak is at a pole that is NOT a bare transition energy
    top = p.w[pk[int(np.argmax(L[pk]))]]
    assert np.min(np.abs(r["dE"] - top)) > 100 * dw


# ---------------------------------------------------------------------------
# rate
# ---------------------------------------------------------------------------
def _eta_quadrature(vmin, v0, vesc, vE, n=4000):
    """Brute-force eta: spherical coordinates in the lab frame."""
    vmax = vesc + vE
    if vmin >= vmax:
        return 0.0
    v = np.linspace(vmin, vmax, n)
    ct = np.linspace(-1.0, 1.0, 2001)
    V, CT = np.meshgrid(v, ct, indexing="ij")
    u2 = V * V + vE * vE + 2 * V * vE * CT
    f = np.exp(-u2 / v0 ** 2) * (u2 < vesc * vesc)
    inner = np.trapezoid(f, ct, axis=1) * 2 * np.pi
    from math import erf, exp, pi, sqrt
    z = vesc / v0
    norm = pi ** 1.5 * v0 ** 3 * (erf(z) - 2 / sqrt(pi) * z * exp(-z * z))
    return np.trapezoid(v * inner, v) / norm


def test_eta_closed_form_vs_quadrature():
    """Check 12: the truncated-Maxwellian eta(v_min) closed form against direct
    integration of f(v)/v over the lab-frame velocity ball."""
    c = rate.C_KM_S
    v0, vesc, vE = 238 / c, 544 / c, 250.2 / c
    for vmin_kms in (0.0, 150.0, 300.0, 450.0, 600.0, 760.0):
        vm = vmin_kms / c
        ref = _eta_quadrature(vm, v0, vesc, vE)
        got = rate.eta_shm(vm, v0, vesc, vE)
        assert abs(got - ref) <= 2e-4 * rate.eta_shm(0.0, v0, vesc, vE)
    assert rate.eta_shm(800 / c, v0, vesc, vE) == 0.0


def test_rate_scalings_and_form_factor_limits():
    """Rate is linear in sigma_e and in rho_chi, and for a loss confined to one
    momentum the light/heavy ratio is |F_light(q)|^2 = (alpha m_e/q)^4
    (Eq. (F_DM_limits))."""
    q = np.linspace(0.5, 3.0, 6)
    w = np.linspace(0.0, 40.0, 41) / rate.HARTREE_EV
    L = np.zeros((6, 41))
    L[2, 10:30] = 0.3
    ph = rate.HaloParams()
    r1 = rate.dR_dw(q, w, L, ph)
    ph2 = rate.HaloParams(sigma_e_cm2=2e-39, rho_chi_GeV_cm3=0.6)
    assert np.allclose(rate.dR_dw(q, w, L, ph2), 4.0 * r1, rtol=1e-13, atol=0)
    light = rate.HaloParams(m_med_eV=0.0)
    rl = rate.dR_dw(q, w, L, light)
    nz = r1 > 0
    assert np.allclose(rl[nz] / r1[nz], (1.0 / q[2]) ** 4, rtol=1e-12)
    # recoil spectrum collects every omega bin exactly once
    spec = rate.recoil_spectrum(w, r1, ph, 20)
    dw = (w[1] - w[0]) * rate.HARTREE_EV
    wev = w * rate.HARTREE_EV
    assert np.isclose(spec.sum(), np.sum(r1[wev >= ph.w_gap_eV]) * dw, rtol=1e-13)


def test_recoil_spectrum_assigns_each_frequency_to_its_ionisation_step():
    """Eq. (excitation_rate) with the step model Q(w) = 1 + floor((w - w_gap)/w_pp)
    (0 below the gap): hand-checked values on both sides of each step, and a
    rate that is nonzero at single frequencies lands in exactly those Q."""
    gap, pp = 1.1, 3.75
    for wv, q in ((0.5, 0), (1.0999, 0), (1.1, 1), (4.8499, 1), (4.8501, 2), (8.6001, 3), (12.34, 3), (12.36, 4)):
        assert rate.ionisation_q(wv, gap, pp) == q, (wv, q)
    ph = rate.HaloParams()
    w = np.linspace(0.0, 30.0, 301) / rate.HARTREE_EV        # 0.1 eV steps
    dR = np.zeros(301)
    dR[[5, 20, 60, 100, 250]] = [7.0, 1.0, 2.0, 3.0, 4.0]     # 0.5, 2.0, 6.0, 10.0, 25.0 eV
    spec = rate.recoil_spectrum(w, dR, ph, 8)
    dw = 0.1
    want = np.zeros(8)
    want[0] += 1.0 * dw          # 2.0 eV -> Q = 1
    want[1] += 2.0 * dw          # 6.0 eV -> Q = 1 + floor(4.9 / 3.75) = 2
    want[2] += 3.0 * dw          # 10.0 eV -> Q = 1 + floor(8.9 / 3.75) = 3
    want[6] += 4.0 * dw          # 25.0 eV -> Q = 1 + floor(23.9 / 3.75) = 7
    assert np.allclose(spec, want, rtol=1e-12, atol=1e-15)   # 0.5 eV is below the gap


def test_rate_units_against_an_si_evaluation():
    """The natural-unit rate (eV, hbar = c = 1; Eq. (general_rate) with
    Eq. (dynamic_structure_factor)) against the same formula written in SI
    units with scipy's constants: a rate density with dimensions
    kg m^5 s^-3 carries the factor 1/(hbar^3 c) to become events per
    (kg s J).  Momenta in bohr^-1 are hbar q / a_0, frequencies in Hartree are
    w E_h, masses in eV are m e / c^2; heavy and light mediators."""
    sc = pytest.importorskip("scipy.constants")
    hbar, c, e = sc.hbar, sc.c, sc.e
    a0 = sc.physical_constants["Bohr radius"][0]
    Eh = sc.physical_constants["Hartree energy"][0]
    me = sc.m_e
    yr = 365.25 * 24 * 3600.0
    qb = np.linspace(0.4, 3.2, 15)                  # bohr^-1
    w = np.linspace(0.0, 30.0, 31) / rate.HARTREE_EV
    rng = np.random.default_rng(5)
    L = rng.uniform(0.0, 0.5, (15, 31))
    for m_med in (-1.0, 0.0):
        ph = rate.HaloParams(m_chi_eV=5e7, m_med_eV=m_med)
        got = rate.dR_dw(qb, w, L, ph)                                   # events/(kg yr eV)
        m_chi = ph.m_chi_eV * e / c ** 2                                  # kg
        mu = m_chi * me / (m_chi + me)
        n_chi = ph.rho_chi_GeV_cm3 * 1e9 / ph.m_chi_eV * 1e6              # m^-3
        rho_T = ph.rho_T_g_cm3 * 1e3                                      # kg m^-3
        sigma = ph.sigma_e_cm2 * 1e-4                                     # m^2
        q = hbar * qb / a0                                                # kg m s^-1
        want = np.zeros(w.shape[0])
        for iw, wh in enumerate(w):
            E = wh * Eh                                                    # J
            g = np.zeros(q.shape[0])
            for iq, qv in enumerate(q):
                vmin = qv / (2 * m_chi) + E / qv                           # m s^-1
                eta = rate.eta_shm(vmin / c, ph.v0_kms * 1e3 / c, ph.vesc_kms * 1e3 / c, ph.vE_kms * 1e3 / c) / c
                F2 = 1.0 if m_med < 0 else (sc.alpha * me * c / qv) ** 4
                g[iq] = qv ** 3 * F2 * L[iq, iw] * eta
            si = n_chi / rho_T * sigma / (8 * np.pi ** 2 * sc.alpha * mu ** 2) * np.trapezoid(g, q) / (hbar ** 3 * c)
            want[iw] = si * yr * e                                         # events/(kg yr eV)
        nz = want > 0
        assert nz.sum() > 10
        # scipy's constants (CODATA 2022) differ from the oracle's (2018) by ~1e-9; near the velocity cutoff
        # eta's steep fall magnifies that to ~2e-7, far below what a wrong power of hbar or c would give
        assert np.allclose(got[nz], want[nz], rtol=1e-6, atol=0)
        assert np.all(got[~nz] == 0)


def test_kinetic_textbook_values():
    """The kinetic matrix used by the f-sum pin: for a tight isolated
    normalised s Gaussian <T> = 3a/2, for p it is 5a/2; for two s Gaussians
    T_ab = m(3 - 2 m R^2) S_ab with m = ab/(a+b)."""
    cell = synth.diamond_cell()
    a = 30.0
    sa = np.array([0, 0, 1], np.int32)
    sl = np.array([0, 1, 0], np.int32)
    se = np.array([a, a, 25.0])
    T = rpa.kinetic(cell.lattice, cell.atoms, sa, sl, se, np.zeros((1, 3)))[0]
    assert abs(T[0, 0] - 1.5 * a) < 1e-10 * a
    assert abs(T[1, 1] - 2.5 * a) < 1e-10 * a
    # two s functions at moderate distance (same cell)
    atoms = np.array([[0.0, 0.0, 0.0], [1.3, 0.2, -0.4]])
    se2 = np.array([0.7, 1.1])
    sa2 = np.array([0, 1], np.int32)
    sl2 = np.array([0, 0], np.int32)
    big = np.eye(3) * 60.0
    T2 = rpa.kinetic(big, atoms, sa2, sl2, se2, np.zeros((1, 3)))[0]
    S2 = rpa.overlap(big, atoms, sa2, sl2, se2, np.zeros((1, 3)))[0]
    m = 0.7 * 1.1 / 1.8
    R2 = np.sum((atoms[0] - atoms[1]) ** 2)
    assert abs(T2[0, 1] - m * (3 - 2 * m * R2) * S2[0, 1]) < 1e-12


# ---------------------------------------------------------------------------
# workload geometry
# ---------------------------------------------------------------------------
def test_g_shell_counts():
    """Reading of 'reciprocal units' as 2 pi/a: the BCC reciprocal shells of
    the diamond cell close at 15, 27, 181, 339 and 531 vectors."""
    cell = synth.diamond_cell()
    _, g2 = synth.g_sorted(cell)
    unit2 = (2 * np.pi / cell.a) ** 2
    for bound, n in ((4, 15), (8, 27), (32, 181), (48, 339), (59, 531)):
        assert int(np.sum(g2 / unit2 <= bound + 1e-9)) == n
    assert cell.volume == pytest.approx(cell.a ** 3 / 4)


def test_loss_as_quadratic_form_of_the_anti_hermitian_part():
    """-Im [A^-1]_jj = [A^-1 B A^-H]_jj with B = (A - A^H)/(2i) for any
    invertible A (A^-1 - A^-H = A^-1 (A^H - A) A^-H).  The mixed GPU path
    evaluates L_LFE this way, so that a small loss is formed from the small
    anti-Hermitian part instead of the imaginary part of an O(1) number; here
    the identity is checked on the oracle's dielectric matrices, plain and
    transposed (the GPU stores eps^T), and a planted transpose of the inverse
    in the quadratic form fails."""
    p = synth.make_tiny(seed=3, shells_per_atom=2, n_k=2, nv=2, nc=3, ng=9, nq=1, nw=6)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq)
    for A in (o["eps"], np.transpose(o["eps"], (0, 2, 1))):
        X = np.linalg.inv(A)
        B = (A - np.conj(np.transpose(A, (0, 2, 1)))) / 2j
        quad = np.einsum("wjk,wkl,wjl->wj", X, B, np.conj(X))
        assert np.max(np.abs(quad.imag)) < 1e-12 * np.max(np.abs(quad))
        assert np.allclose(quad.real, o["L_lfe"], rtol=1e-10, atol=1e-14)
        bad = np.einsum("wkj,wkl,wjl->wj", X, B, np.conj(X))
        assert not np.allclose(bad.real, o["L_lfe"], rtol=1e-3)


def test_bin_loss_by_hand():
    """The |q| binning that feeds the rate integral (the momentum grid of the
    q integral of the rate, Appendix A): bins are half-open [e_i, e_(i+1)), a
    value on an inner edge belongs to the bin above it, values on or past the
    last edge and below the first are dropped, a bin holds the MEAN of its
    rows (not their sum), an empty bin is 0, and the centres are the edge
    midpoints.  Expected values are written out by hand."""
    edges = np.array([0.0, 0.1, 0.2, 0.3, 0.4])
    qmag = np.array([0.05, 0.1, 0.15, 0.35, 0.4, 0.5, -0.01, 0.0])
    L = np.array([[1.0, 10.0],       # 0.05 -> bin 0
                  [2.0, 20.0],       # 0.1 (inner edge) -> bin 1
                  [4.0, 40.0],       # 0.15 -> bin 1
                  [8.0, 80.0],       # 0.35 -> bin 3
                  [16.0, 160.0],     # 0.4 (last edge) -> dropped
                  [32.0, 320.0],     # past the last edge -> dropped
                  [64.0, 640.0],     # below the first edge -> dropped
                  [128.0, 1280.0]])  # 0.0 (first edge) -> bin 0
    out, centres, cnt = rate.bin_loss(qmag, L, edges)
    assert np.array_equal(cnt, [2, 2, 0, 1])
    assert np.array_equal(out, [[64.5, 645.0], [3.0, 30.0], [0.0, 0.0], [8.0, 80.0]])
    assert np.allclose(centres, [0.05, 0.15, 0.25, 0.35], rtol=0, atol=1e-15)
