"""ctypes binding of libqcx (include/qcx.h): argument marshalling only.

The raw entry points are available under their C names (``qcx_create``,
``qcx_pair_density``, ...) once ``load()`` has run; ``Context`` wraps them
for numpy arrays (host memory) and torch tensors (device memory, passed by
``data_ptr()``).  Loading fails loudly when the library has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
import re

import numpy as np

QCX_FP64 = 0
QCX_MIXED = 1
STATUS = {0: "QCX_OK", 1: "QCX_ERR_ARG", 2: "QCX_ERR_ALLOC", 3: "QCX_ERR_CUDA", 4: "QCX_ERR_SINGULAR",
          5: "QCX_ERR_NOT_CONVERGED", 6: "QCX_ERR_TIMEOUT", 7: "QCX_ERR_STATE", 8: "QCX_ERR_UNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
P = ct.c_void_p
I = ct.c_int
D = ct.c_double


class HaloParams(ct.Structure):
    _fields_ = [(n, ct.c_double) for n in ("m_chi_eV", "sigma_e_cm2", "rho_chi_GeV_cm3", "v0_kms", "vesc_kms",
                                            "vE_kms", "rho_T_g_cm3", "m_med_eV", "w_gap_eV", "w_pp_eV")]


def halo_params(m_chi_eV=1e9, sigma_e_cm2=1e-39, rho_chi_GeV_cm3=0.3, v0_kms=238.0, vesc_kms=544.0,
                vE_kms=250.2, rho_T_g_cm3=2.329, m_med_eV=-1.0, w_gap_eV=1.1, w_pp_eV=3.75) -> HaloParams:
    return HaloParams(m_chi_eV, sigma_e_cm2, rho_chi_GeV_cm3, v0_kms, vesc_kms, vE_kms, rho_T_g_cm3, m_med_eV,
                      w_gap_eV, w_pp_eV)


class Screening(ct.Structure):
    """qcx_screening."""
    _fields_ = [("model", ct.c_int), ("eps0", ct.c_double), ("tau", ct.c_double), ("wp_eV", ct.c_double),
                ("qtf_eV", ct.c_double), ("ne_bohr3", ct.c_double), ("fp", ct.c_double)]


SCREEN_SELF, SCREEN_NONE, SCREEN_MTF, SCREEN_LINDHARD = 0, 1, 2, 3


def screening(model=SCREEN_SELF, eps0=11.3, tau=1.563, wp_eV=16.6, qtf_eV=4130.0, ne_bohr3=0.0, fp=0.1):
    return Screening(model, eps0, tau, wp_eV, qtf_eV, ne_bohr3, fp)


class RateParams(ct.Structure):
    """qcx_rate_params."""
    _fields_ = [("m_chi_eV", ct.c_double), ("sigma_e_cm2", ct.c_double), ("m_med_eV", ct.c_double),
                ("mediator", ct.c_int), ("rho_T_g_cm3", ct.c_double), ("w_gap_eV", ct.c_double),
                ("w_pp_eV", ct.c_double), ("exposure_kg_yr", ct.c_double), ("n_events", ct.c_double)]


def rate_params(m_chi_eV=1e9, sigma_e_cm2=1e-39, m_med_eV=-1.0, mediator=0, rho_T_g_cm3=2.329, w_gap_eV=1.1,
                w_pp_eV=3.75, exposure_kg_yr=1.0, n_events=2.3):
    return RateParams(m_chi_eV, sigma_e_cm2, m_med_eV, mediator, rho_T_g_cm3, w_gap_eV, w_pp_eV, exposure_kg_yr,
                      n_events)


_SIGS = {
    "qcx_create": (I, [ct.POINTER(P), I, P]),
    "qcx_destroy": (None, [P]),
    "qcx_last_error": (ct.c_char_p, [P]),
    "qcx_sync": (I, [P]),
    "qcx_set_basis": (I, [P, P, I, P, I, P, P, P]),
    "qcx_nbasis": (I, [P]),
    "qcx_overlap": (I, [P, I, P, P]),
    "qcx_set_states": (I, [P, I, P, I, P, P, I, P, I, P, P]),
    "qcx_pair_density": (I, [P, I, I, P, I, P]),
    "qcx_chi0": (I, [P, I, I, P, D, I, P]),
    "qcx_pair_density_optical": (I, [P, I, I, P, P, I, P]),
    "qcx_chi0_spectral": (I, [P, I, I, P, D, D, D, I, I, P, P]),
    "qcx_spectral_grid": (I, [P, I, D, ct.POINTER(D), ct.POINTER(I)]),
    "qcx_set_spectral_chunk": (I, [P, I]),
    "qcx_set_spectral_engine": (I, [P, I]),
    "qcx_spectral_timings": (I, [P, P]),
    "qcx_invert_eps": (I, [P, I, I, P, P, P]),
    "qcx_set_refine_threshold": (I, [P, D]),
    "qcx_set_wait_limit": (I, [P, ct.c_longlong]),
    "qcx_set_fault_injection": (I, [P, I]),
    "qcx_loss_function": (I, [P, I, P, P]),
    "qcx_bin_loss": (I, [P, I, P, I, I, P, P, P]),
    "qcx_rate": (I, [P, I, P, I, P, P, ct.POINTER(HaloParams), P, I, P]),
    "qcx_bin_eps3d": (I, [P, I, P, D, I, D, I, I, I, P, P]),
    "qcx_loss_isotropic": (I, [P, I, I, I, I, P, D, P, P, ct.POINTER(Screening), P, P]),
    "qcx_rate_general": (I, [P, I, P, I, P, P, I, P, P, ct.POINTER(RateParams), P, I, P, P]),
    "qcx_solve_batch": (I, [P, I, P, P, P, D, I, P, P, P]),
    "qcx_batch_info": (I, [P, I, P]),
    "qcx_batch_autotune": (I, [P, I]),
    "qcx_mlp_nparam": (I, []),
    "qcx_mlp_set_params": (I, [P, P]),
    "qcx_mlp_get_params": (I, [P, P, P]),
    "qcx_mlp_grad": (I, [P, I, P, P, P, P]),
    "qcx_mlp_train": (I, [P, I, P, P, P, P]),
    "qcx_mlp_predict": (I, [P, I, P, P, P]),
    "qcx_head_nolfe": (I, [P, I, I, P, D, P]),
    "qcx_surrogate_features": (I, [P, I, P, P, P, P, D, D, P, P]),
    "qcx_surrogate_heads": (I, [P, I, P, I, P, I, P, D, I, P, P, P, P, P]),
    "qcx_eps_inverse_diag_noalloc": (I, [P, I, I, P, P, P, P, P]),
}


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libqcx.so")


def load():
    """Load libqcx.so and bind every entry point under its C name."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libqcx is not built ({path} missing): run __graft_entry__.build()")
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
        globals()[name] = f
    _lib = lib
    return lib


def declared_symbols(header: str | None = None) -> list[str]:
    """Names of the functions declared in include/qcx.h."""
    header = header or os.path.join(os.path.dirname(_HERE), "include", "qcx.h")
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qcx_[a-z0-9_]+)\s*\(", txt)))


class MlpOpts(ct.Structure):
    """qcx_mlp_opts."""
    _fields_ = [("epochs", ct.c_int), ("batch", ct.c_int), ("lr", ct.c_float), ("beta1", ct.c_float),
                ("beta2", ct.c_float), ("eps", ct.c_float), ("seed", ct.c_ulonglong)]


def mlp_opts(epochs=100, batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=1):
    return MlpOpts(epochs, batch, lr, beta1, beta2, eps, seed)


class SurrogateOpts(ct.Structure):
    """qcx_surrogate_opts."""
    _fields_ = [("q_max", ct.c_double), ("w_max", ct.c_double), ("sigma_accept", ct.c_double),
                ("check_frac", ct.c_double), ("check_tol", ct.c_double), ("seed", ct.c_ulonglong)]


class QcxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Arg:
    """Pointer to host (numpy) or device (torch) memory of the right dtype."""

    def __init__(self, x, dtype):
        self.keep = None
        if x is None:
            self.ptr = None
        elif hasattr(x, "data_ptr"):
            import torch
            want = {np.float64: torch.float64, np.complex128: torch.complex128, np.int32: torch.int32,
                    np.float32: torch.float32}[dtype]
            if x.dtype != want or not x.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}")
            self.ptr = P(x.data_ptr())
            self.keep = x
        else:
            arr = np.ascontiguousarray(x, dtype=dtype)
            self.keep = arr
            self.ptr = P(arr.ctypes.data)


def _out(shape, dtype, out):
    if out is not None:
        return out
    return np.zeros(shape, dtype=dtype)


class Context:
    """One libqcx context on `device` (optionally on an existing CUDA stream)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        load()
        h = P()
        st = qcx_create(ct.byref(h), device, P(stream) if stream else None)
        if st:
            raise QcxError(st, "qcx_create failed")
        self.h = h
        self.nk = self.nv = self.nc = self.nq = 0
        self._ng = {}
        self._nw = {}

    def close(self):
        if self.h:
            qcx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st:
            raise QcxError(st, qcx_last_error(self.h).decode())

    # ---------------------------------------------------------- system
    def set_basis(self, lattice, atom_xyz, shell_atom, shell_l, shell_exp):
        a = [_Arg(lattice, np.float64), _Arg(atom_xyz, np.float64), _Arg(shell_atom, np.int32),
             _Arg(shell_l, np.int32), _Arg(shell_exp, np.float64)]
        natom = len(np.asarray(atom_xyz).reshape(-1, 3)) if not hasattr(atom_xyz, "data_ptr") else atom_xyz.shape[0]
        nshell = len(shell_atom)
        self._check(qcx_set_basis(self.h, a[0].ptr, natom, a[1].ptr, nshell, a[2].ptr, a[3].ptr, a[4].ptr))
        self.nb = qcx_nbasis(self.h)

    def overlap(self, kpts, out=None):
        kp = _Arg(kpts, np.float64)
        nk = len(kpts)
        o = _out((nk, self.nb, self.nb), np.complex128, out)
        oa = _Arg(o, np.complex128)
        self._check(qcx_overlap(self.h, nk, kp.ptr, oa.ptr))
        return o

    def set_states(self, kpts, C_k, E_k, qpts, C_kq, E_kq):
        nk, nb, nv = C_k.shape
        nq, _, _, nc = C_kq.shape
        a = [_Arg(kpts, np.float64), _Arg(C_k, np.complex128), _Arg(E_k, np.float64), _Arg(qpts, np.float64),
             _Arg(C_kq, np.complex128), _Arg(E_kq, np.float64)]
        self._check(qcx_set_states(self.h, nk, a[0].ptr, nv, a[1].ptr, a[2].ptr, nq, a[3].ptr, nc, a[4].ptr,
                                   a[5].ptr))
        self.nk, self.nv, self.nc, self.nq = nk, nv, nc, nq

    # --------------------------------------------------------- the path
    def pair_density(self, iq, G_int, prec=QCX_FP64, want=False, out=None):
        g = _Arg(G_int, np.int32)
        ng = len(G_int)
        self._ng[prec] = ng
        o = _out((self.nk * self.nv * self.nc, ng), np.complex128, out) if (want or out is not None) else None
        oa = _Arg(o, np.complex128)
        self._check(qcx_pair_density(self.h, iq, ng, g.ptr, prec, oa.ptr))
        return o

    def pair_density_optical(self, iq, G_int, qhat, prec=QCX_FP64, want=False, out=None):
        """qcx_pair_density_optical: q number iq must be zero; G = 0 row = the q -> 0 limit along qhat."""
        g = _Arg(G_int, np.int32)
        qa = _Arg(np.asarray(qhat, np.float64), np.float64)
        ng = len(G_int)
        self._ng[prec] = ng
        o = _out((self.nk * self.nv * self.nc, ng), np.complex128, out) if (want or out is not None) else None
        oa = _Arg(o, np.complex128)
        self._check(qcx_pair_density_optical(self.h, iq, ng, g.ptr, qa.ptr, prec, oa.ptr))
        return o

    def chi0(self, iq, w, eta, prec=QCX_FP64, want=False, out=None):
        wa = _Arg(w, np.float64)
        nw = len(w)
        self._nw[prec] = nw
        ng = self._ng.get(prec, 0)
        o = _out((nw, ng, ng), np.complex128, out) if (want or out is not None) else None
        oa = _Arg(o, np.complex128)
        self._check(qcx_chi0(self.h, iq, nw, wa.ptr, float(eta), prec, oa.ptr))
        return o

    def chi0_spectral(self, iq, w, eta, E0, step, nbin, prec=QCX_FP64, want=False, want_S=False, out=None):
        """qcx_chi0_spectral; returns chi0 [nw][ng][ng] (if wanted) and the spectral weights
        [nbin][ng][ng] (if wanted)."""
        wa = _Arg(w, np.float64)
        nw = len(w)
        self._nw[prec] = nw
        ng = self._ng.get(prec, 0)
        o = _out((nw, ng, ng), np.complex128, out) if (want or out is not None) else None
        oa = _Arg(o, np.complex128)
        S = np.zeros((int(nbin), ng, ng), np.complex128) if want_S else None
        sa = _Arg(S, np.complex128)
        self._check(qcx_chi0_spectral(self.h, iq, nw, wa.ptr, float(eta), float(E0), float(step), int(nbin), prec,
                                      oa.ptr, sa.ptr))
        return o, S

    def spectral_grid(self, iq, step):
        """(E0, nbin) of qcx_spectral_grid."""
        e0, nb = ct.c_double(0.0), ct.c_int(0)
        self._check(qcx_spectral_grid(self.h, iq, float(step), ct.byref(e0), ct.byref(nb)))
        return e0.value, nb.value

    def set_spectral_chunk(self, bins):
        self._check(qcx_set_spectral_chunk(self.h, int(bins)))

    def set_spectral_engine(self, cuda_cores: bool):
        self._check(qcx_set_spectral_engine(self.h, 1 if cuda_cores else 0))

    def spectral_timings(self):
        """Stage times (ms) of the last chi0_spectral call: grouping, gather + K table,
        spectral weights, contraction, Dyson step."""
        ms = np.zeros(5, np.float64)
        self._check(qcx_spectral_timings(self.h, P(ms.ctypes.data)))
        return dict(zip(("grouping", "gather", "weights", "contraction", "dyson"), ms.tolist()))

    def invert_eps(self, iq, prec=QCX_FP64, want=True):
        nw, ng = self._nw[prec], self._ng[prec]
        if want:
            d = np.zeros((nw, ng), np.complex128)
            e = np.zeros((nw, ng), np.complex128)
            r = np.zeros(nw, np.float64)
            self._check(qcx_invert_eps(self.h, iq, prec, P(d.ctypes.data), P(e.ctypes.data), P(r.ctypes.data)))
            return d, e, r
        self._check(qcx_invert_eps(self.h, iq, prec, None, None, None))
        return None

    def set_refine_threshold(self, kappa1):
        self._check(qcx_set_refine_threshold(self.h, float(kappa1)))

    def set_wait_limit(self, cycles):
        self._check(qcx_set_wait_limit(self.h, int(cycles)))

    def set_fault_injection(self, withhold_copies: bool):
        self._check(qcx_set_fault_injection(self.h, 1 if withhold_copies else 0))

    def loss_function(self, iq, prec=QCX_FP64, out_lfe=None, out_nolfe=None):
        nw, ng = self._nw[prec], self._ng[prec]
        a = _out((nw, ng), np.float64, out_lfe)
        b = _out((nw, ng), np.float64, out_nolfe)
        aa, bb = _Arg(a, np.float64), _Arg(b, np.float64)
        self._check(qcx_loss_function(self.h, iq, aa.ptr, bb.ptr))
        return a, b

    def bin_loss(self, iq_list, which, edges, nw):
        iq = _Arg(np.asarray(iq_list, np.int32), np.int32)
        ed = _Arg(edges, np.float64)
        nbin = len(edges) - 1
        out = np.zeros((nbin, nw), np.float64)
        cnt = np.zeros(nbin, np.float64)
        self._check(qcx_bin_loss(self.h, len(iq_list), iq.ptr, which, nbin, ed.ptr, P(out.ctypes.data),
                                 P(cnt.ctypes.data)))
        return out, cnt

    def rate(self, qbin, w, L, params: HaloParams, nQ=0):
        qa, wa, La = _Arg(qbin, np.float64), _Arg(w, np.float64), _Arg(L, np.float64)
        dR = np.zeros(len(w), np.float64)
        dQ = np.zeros(max(nQ, 1), np.float64)
        self._check(qcx_rate(self.h, len(qbin), qa.ptr, len(w), wa.ptr, La.ptr, ct.byref(params),
                             P(dR.ctypes.data), nQ, P(dQ.ctypes.data) if nQ else None))
        return dR, dQ[:nQ]

    # ------------------------------------------------ rate end: 3-D tables
    def bin_eps3d(self, iq_list, q_lfe, nshell, dq, n_theta, n_phi, nw, fill=True):
        """Composite eps binned in (|q|, theta, phi): (eps [nshell][nth][nph][nw], count [nshell][nth][nph])."""
        iq = np.ascontiguousarray(iq_list, np.int32)
        eps = np.zeros((nshell, n_theta, n_phi, nw), np.complex128)
        cnt = np.zeros((nshell, n_theta, n_phi), np.float64)
        self._check(qcx_bin_eps3d(self.h, len(iq), P(iq.ctypes.data), float(q_lfe), nshell, float(dq), n_theta,
                                  n_phi, 1 if fill else 0, P(eps.ctypes.data), P(cnt.ctypes.data)))
        return eps, cnt

    def loss_isotropic(self, eps, count, w, dq, scr: Screening):
        """Isotropic loss [nshell][nw] of 3-D tables and the cells used per shell."""
        nshell, nth, nph, nw = eps.shape
        e, c, wa = _Arg(eps, np.complex128), _Arg(count, np.float64), _Arg(w, np.float64)
        L = np.zeros((nshell, nw), np.float64)
        nc = np.zeros(nshell, np.float64)
        self._check(qcx_loss_isotropic(self.h, nshell, nth, nph, nw, wa.ptr, float(dq), e.ptr, c.ptr, ct.byref(scr),
                                       P(L.ctypes.data), P(nc.ctypes.data)))
        return L, nc

    def rate_general(self, qbin, w, L, v, dphidv, params: RateParams, nQ=0, want_reach=False):
        """(dR/dw [nw], dR_Q [nQ], reach [nQ] or None) of the general rate."""
        qa, wa, La = _Arg(qbin, np.float64), _Arg(w, np.float64), _Arg(L, np.float64)
        va, fa = _Arg(v, np.float64), _Arg(dphidv, np.float64)
        dR = np.zeros(len(w), np.float64)
        dQ = np.zeros(max(nQ, 1), np.float64)
        rc = np.zeros(max(nQ, 1), np.float64) if want_reach else None
        self._check(qcx_rate_general(self.h, len(qbin), qa.ptr, len(w), wa.ptr, La.ptr, len(v), va.ptr, fa.ptr,
                                     ct.byref(params), P(dR.ctypes.data), nQ, P(dQ.ctypes.data) if nQ else None,
                                     P(rc.ctypes.data) if want_reach else None))
        return dR, dQ[:nQ], (rc[:nQ] if want_reach else None)

    # ------------------------------------------------- batched instances
    def solve_batch(self, inst_q, inst_w, inst_gmax, eta, prec=QCX_MIXED, out_lfe=None, out_nolfe=None,
                    want_ng=True):
        """Heads (L_LFE, L_noLFE) of uneven (q, w, G_max) instances; returns
        (L_lfe[n], L_nolfe[n], N_G[n] or None).  Outputs may be device tensors."""
        n = len(inst_q)
        qa = _Arg(np.asarray(inst_q, np.int32) if not hasattr(inst_q, "data_ptr") else inst_q, np.int32)
        wa, ga = _Arg(inst_w, np.float64), _Arg(inst_gmax, np.float64)
        a = _out((n,), np.float64, out_lfe)
        b = _out((n,), np.float64, out_nolfe)
        ng = np.zeros(n, np.int32) if want_ng else None
        aa, bb, na = _Arg(a, np.float64), _Arg(b, np.float64), _Arg(ng, np.int32)
        self._check(qcx_solve_batch(self.h, n, qa.ptr, wa.ptr, ga.ptr, float(eta), prec, aa.ptr, bb.ptr, na.ptr))
        return a, b, ng

    def batch_info(self):
        """Facts about the current batch plan (see qcx_batch_info)."""
        out = (ct.c_longlong * 13)()
        self._check(qcx_batch_info(self.h, 13, out))
        keys = ["tile_cap", "tiles", "tc_ctas", "solve_ctas", "kernels_per_replay", "autotuned", "distinct_q",
                "max_ng", "autotune_us", "precision", "cap_ng65_128", "cap_ng129_192", "cap_ng193_up"]
        return dict(zip(keys, list(out)))

    def batch_autotune(self, enable: bool):
        self._check(qcx_batch_autotune(self.h, 1 if enable else 0))

    # ------------------------------------------- learned LFE correction
    def mlp_set_params(self, params):
        pa = _Arg(np.asarray(params, np.float32) if not hasattr(params, "data_ptr") else params, np.float32)
        self._check(qcx_mlp_set_params(self.h, pa.ptr))

    def mlp_get_params(self):
        """(FP32 masters, values the kernels compute with)."""
        n = qcx_mlp_nparam()
        a = np.zeros(n, np.float32)
        c = np.zeros(n, np.float32)
        self._check(qcx_mlp_get_params(self.h, P(a.ctypes.data), P(c.ctypes.data)))
        return a, c

    def mlp_grad(self, X, y):
        Xa, ya = _Arg(X, np.float32), _Arg(y, np.float32)
        g = np.zeros(qcx_mlp_nparam(), np.float32)
        loss = ct.c_double()
        self._check(qcx_mlp_grad(self.h, len(y), Xa.ptr, ya.ptr, P(g.ctypes.data), ct.byref(loss)))
        return loss.value, g

    def mlp_train(self, X, y, opts: MlpOpts):
        Xa, ya = _Arg(X, np.float32), _Arg(y, np.float32)
        curve = np.zeros(opts.epochs, np.float32)
        self._check(qcx_mlp_train(self.h, len(y), Xa.ptr, ya.ptr, ct.byref(opts), P(curve.ctypes.data)))
        return curve

    def mlp_predict(self, X, out_mu=None, out_logvar=None):
        n = len(X)
        Xa = _Arg(X, np.float32)
        mu = _out((n,), np.float32, out_mu)
        lv = _out((n,), np.float32, out_logvar)
        ma, la = _Arg(mu, np.float32), _Arg(lv, np.float32)
        self._check(qcx_mlp_predict(self.h, n, Xa.ptr, ma.ptr, la.ptr))
        return mu, lv

    def head_nolfe(self, iq, w, eta):
        wa = _Arg(w, np.float64)
        out = np.zeros(len(w), np.float64)
        self._check(qcx_head_nolfe(self.h, iq, len(w), wa.ptr, float(eta), P(out.ctypes.data)))
        return out

    def surrogate_features(self, qvec, w, L_nolfe, q_max, w_max, L_lfe=None):
        """Network inputs X [n][6] and, with L_lfe, the targets y [n] (else None)."""
        n = len(w)
        qa, wa, La = _Arg(qvec, np.float64), _Arg(w, np.float64), _Arg(L_nolfe, np.float64)
        L1 = _Arg(L_lfe, np.float64)
        X = np.zeros((n, 6), np.float32)
        y = np.zeros(n, np.float32) if L_lfe is not None else None
        self._check(qcx_surrogate_features(self.h, n, qa.ptr, wa.ptr, La.ptr, L1.ptr, float(q_max), float(w_max),
                                           P(X.ctypes.data), P(y.ctypes.data) if y is not None else None))
        return X, y

    def surrogate_heads(self, iq_list, G_int, w, eta, opts: SurrogateOpts, fallback_prec=QCX_MIXED):
        """(L_lfe [nsel][nw], L_nolfe, source, largest spot-check miss)."""
        iq = np.ascontiguousarray(iq_list, np.int32)
        G = np.ascontiguousarray(G_int, np.int32)
        wa = np.ascontiguousarray(w, np.float64)
        nsel, nw = len(iq), len(wa)
        L1 = np.zeros((nsel, nw), np.float64)
        L2 = np.zeros((nsel, nw), np.float64)
        src = np.zeros((nsel, nw), np.int32)
        chk = ct.c_double()
        self._check(qcx_surrogate_heads(self.h, nsel, P(iq.ctypes.data), len(G), P(G.ctypes.data), nw,
                                        P(wa.ctypes.data), float(eta), fallback_prec, ct.byref(opts),
                                        P(L1.ctypes.data), P(L2.ctypes.data), P(src.ctypes.data), ct.byref(chk)))
        return L1, L2, src, chk.value

    def sync(self):
        self._check(qcx_sync(self.h))
