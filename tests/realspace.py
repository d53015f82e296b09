"""Brute-force real-space quadrature of Bloch-sum matrix elements.

An independent route to the closed-form Gaussian-product integrals used by
the oracle: the Bloch sums f_{mu k}(r) = sum_R e^{ik.R} chi_mu(r - tau_mu - R)
are tabulated on a uniform grid over one unit cell and
int_cell conj(f_{mu,k+q}) e^{i kappa.r} f_{nu k} dr is evaluated with the
periodic trapezoid rule (spectrally accurate for smooth periodic integrands).
"""
import numpy as np


def cell_grid(lattice, n):
    s = (np.arange(n) + 0.0) / n
    f = np.stack(np.meshgrid(s, s, s, indexing="ij"), -1).reshape(-1, 3)
    return f @ lattice


def primitive_values(r, centre, a, lvec):
    """Normalised Cartesian primitive at points r [N][3]."""
    d = r - centre[None, :]
    n = (2 * a / np.pi) ** 0.75
    val = n * np.exp(-a * np.sum(d * d, axis=1))
    for x in range(3):
        if lvec[x]:
            val = val * 2.0 * np.sqrt(a) * d[:, x]
    return val


def bloch_sums(lattice, atoms, funcs, k, r, reach):
    """f[mu][N] = sum_R e^{ik.R} chi_mu(r - tau_mu - R) over |R| <= reach."""
    nm = int(np.ceil(reach / np.min(np.linalg.norm(lattice, axis=1)))) + 2
    rr = np.arange(-nm, nm + 1)
    n = np.stack(np.meshgrid(rr, rr, rr, indexing="ij"), -1).reshape(-1, 3)
    R = n @ lattice
    R = R[np.linalg.norm(R, axis=1) <= reach]
    out = np.zeros((len(funcs), r.shape[0]), complex)
    for mu, (_, at, a, lv) in enumerate(funcs):
        for Rv in R:
            out[mu] += np.exp(1j * (k @ Rv)) * primitive_values(r, atoms[at] + Rv, a, lv)
    return out


def matrix_elements(lattice, atoms, funcs, k, q, kappas, n=36, reach=24.0):
    """B[G][mu][nu] = int_cell conj(f_{mu,k+q}) e^{i kappa_G.r} f_{nu k} dr."""
    r = cell_grid(lattice, n)
    vol = abs(np.linalg.det(lattice))
    fk = bloch_sums(lattice, atoms, funcs, k, r, reach)
    fkq = bloch_sums(lattice, atoms, funcs, k + q, r, reach)
    out = []
    for kap in np.atleast_2d(kappas):
        ph = np.exp(1j * (r @ kap))
        out.append((fkq.conj() * ph[None, :]) @ fk.T * (vol / r.shape[0]))
    return np.array(out), fk, fkq, r, vol
