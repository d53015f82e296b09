"""Pins of the optical-limit oracle (Appendix C): the gradient integrals
against numerical quadrature and against the centre derivative of the pinned
overlap, the anti-Hermitian momentum matrix, the assembled q -> 0 matrix
against the appendix's head and wing sums written out separately (with the
sign readings stated in oracle/optical.py), and positivity of the loss."""
import numpy as np
import pytest

import synth
from oracle import optical, rpa


def test_gradient_integral_against_quadrature():
    """int (x-A)^la e^{-a(x-A)^2} d/dx[(x-B)^lb e^{-b(x-B)^2}] dx: the closed form
    against a quadrature whose derivative is a central difference."""
    from scipy.integrate import quad
    rng = np.random.default_rng(5)
    h = 1e-5
    for _ in range(12):
        la, lb = int(rng.integers(0, 2)), int(rng.integers(0, 2))
        a, b = float(rng.uniform(0.2, 3.0)), float(rng.uniform(0.2, 3.0))
        A, B = float(rng.uniform(-1.0, 1.0)), float(rng.uniform(-1.0, 1.0))

        def gb(x):
            return (x - B) ** lb * np.exp(-b * (x - B) ** 2)

        def f(x):
            return (x - A) ** la * np.exp(-a * (x - A) ** 2) * (gb(x + h) - gb(x - h)) / (2.0 * h)

        want, _ = quad(f, -30.0, 30.0, epsabs=1e-13, epsrel=1e-12, limit=400)
        got = float(optical._deriv_1d(la, lb, A, np.array([B]), a, b)[0])
        assert got == pytest.approx(want, rel=1e-8, abs=1e-11), (la, lb, a, b, A, B)


@pytest.fixture(scope="module")
def tiny():
    return synth.make_tiny(seed=11, n_k=2)


def test_momentum_matrix_is_anti_hermitian(tiny):
    c, b = tiny.cell, tiny.basis
    k = np.array([[0.13, -0.21, 0.07], [0.0, 0.0, 0.0]])
    P = optical.momentum_matrix(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, k)
    top = np.max(np.abs(P))
    assert top > 0
    for i in range(k.shape[0]):
        for x in range(3):
            assert np.max(np.abs(P[i, x] + P[i, x].conj().T)) <= 1e-12 * top


def test_momentum_matrix_is_minus_the_centre_derivative_of_the_overlap(tiny):
    """For mu on atom 0 and nu on atom 1, moving atom 1 by h along x moves every
    chi_nu(r - tau_nu - L): dS_{mu nu}/d tau_x = -P_{mu nu}[x]."""
    c, b = tiny.cell, tiny.basis
    k = np.array([[0.13, -0.21, 0.07]])
    P = optical.momentum_matrix(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, k)[0]
    funcs = rpa.basis_functions(b.shell_atom, b.shell_l, b.shell_exp)
    on0 = [i for i, f in enumerate(funcs) if f[1] == 0]
    on1 = [i for i, f in enumerate(funcs) if f[1] == 1]
    h = 1e-5
    for x in range(3):
        d = np.zeros(3)
        d[x] = h
        at_p = np.array(c.atoms, float)
        at_m = np.array(c.atoms, float)
        at_p[1] += d
        at_m[1] -= d
        Sp = rpa.overlap(c.lattice, at_p, b.shell_atom, b.shell_l, b.shell_exp, k)[0]
        Sm = rpa.overlap(c.lattice, at_m, b.shell_atom, b.shell_l, b.shell_exp, k)[0]
        dS = (Sp - Sm) / (2.0 * h)
        blk = np.ix_(on0, on1)
        assert np.max(np.abs(dS[blk] + P[x][blk])) <= 1e-7 * np.max(np.abs(P[x][blk]))


@pytest.fixture(scope="module")
def optical_small():
    p = synth.make_optical("small", nw=24)
    Cv, Cc = optical.states_joint(p)
    qhat = np.array([1.0, 0.4, -0.3])
    return p, Cv, Cc, qhat / np.linalg.norm(qhat), optical.solve_optical(p, qhat, Cv, Cc)


def test_joint_states_are_orthonormal_together(optical_small):
    p, Cv, Cc, _, _ = optical_small
    c, b = p.cell, p.basis
    S = rpa.overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts)
    C = np.concatenate([Cv, Cc], axis=2)
    for k in range(p.nk):
        assert np.allclose(C[k].conj().T @ S[k] @ C[k], np.eye(C.shape[2]), atol=1e-10)


def test_head_and_wings_are_the_appendix_sums(optical_small):
    """The appendix's head and wings, written as sums over transitions (i = v,
    j = c with the antiresonant partner in W, m_e = 1, 4 pi alpha -> 4 pi, the
    k sum normalised by N_k), against the column-replacement construction.
    Sign readings: the head with "1 -" (the q -> 0 limit of Eq. (RPA); "1 +" as
    printed gives Im eps_00 < 0) and eps_G0 with "+i" (as printed, "-i", it is not
    the conjugate partner of eps_0G')."""
    p, Cv, Cc, qhat, o = optical_small
    c = p.cell
    W = rpa.transition_weights(o["dE"], p.w, p.eta)                      # [nw][nt]
    pc = o["p"] @ qhat                                                   # qhat . <c|grad|v>
    pv = -np.conj(o["p"]) @ qhat                                         # qhat . <v|grad|c>
    dE = o["dE"]
    g0 = o["g0"]
    Gn = np.linalg.norm(p.G_int @ c.recip, axis=1)
    pref = 4.0 * np.pi / c.volume * 2.0 / p.nk
    head = 1.0 - pref * W @ (np.abs(pc) ** 2 / dE ** 2)
    rho = o["rho"]
    others = [g for g in range(p.ng) if g != g0]
    wing_0G = 1j * pref * (W * (pv / dE)[None, :]) @ rho[:, others] / Gn[others][None, :]
    wing_G0 = 1j * pref * (W * (pc / dE)[None, :]) @ rho[:, others].conj() / Gn[others][None, :]
    eps = o["eps"]
    top = np.max(np.abs(eps))
    assert np.max(np.abs(eps[:, g0, g0] - head)) <= 1e-12 * top
    assert np.max(np.abs(eps[:, g0, others] - wing_0G)) <= 1e-12 * top
    assert np.max(np.abs(eps[:, others, g0] - wing_G0)) <= 1e-12 * top


def test_optical_loss_is_positive(optical_small):
    p, _, _, _, o = optical_small
    g0 = o["g0"]
    assert np.all(o["eps"][1:, g0, g0].imag > 0)
    assert np.all(o["L_nolfe"][1:, g0] > 0)
    assert np.all(o["L_lfe"][1:] > -1e-12)
