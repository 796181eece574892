"""FP64 CPU oracle for the ENUF-DPD hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path in
``paper_1303_4523_gb300``; neither imports the other. The arithmetic lives in
``enuf_oracle.c`` (plain C, FP64), which cites the equations of Wang,
Laaksonen & Lu (arXiv 1303.4523) it follows; this module only marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enuf_oracle.c")
_LIB = os.path.join(_HERE, "liborc_enuf.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "enuf_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("L", C.c_double), ("alpha", C.c_double), ("r_cut", C.c_double),
                ("beta", C.c_double), ("kappa", C.c_double), ("M", C.c_int),
                ("p", C.c_int), ("sigma_s", C.c_int), ("kmask", C.c_int),
                ("deriv", C.c_int), ("slater_k", C.c_int)]


class _DpdParams(C.Structure):
    _fields_ = [("ntypes", C.c_int), ("a", C.POINTER(C.c_double)), ("gamma", C.c_double),
                ("sigma", C.c_double), ("dt", C.c_double), ("lambda_vv", C.c_double),
                ("K_bond", C.c_double), ("r0_bond", C.c_double), ("seed", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, pd, pi = C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)
        pp = C.POINTER(_Params)
        _lib.orc_wrap.restype = d
        _lib.orc_wrap.argtypes = [d, d]
        for nm in ("orc_B1", "orc_B2", "orc_slater_energy", "orc_slater_force"):
            getattr(_lib, nm).restype = d
            getattr(_lib, nm).argtypes = [d, d]
        for nm in ("orc_real_space", "orc_recip_direct"):
            getattr(_lib, nm).restype = i
            getattr(_lib, nm).argtypes = [pp, i, pd, pd, pd, pd, pi, i]
        _lib.orc_recip_enuf.restype = i
        _lib.orc_recip_enuf.argtypes = [pp, i, pd, pd, pd, pd, pd, pd, pi, i]
        _lib.orc_self_neutral.restype = None
        _lib.orc_self_neutral.argtypes = [pp, i, pd, pd]
        _lib.orc_philox4x32_10.restype = None
        _lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        _lib.orc_theta.restype = d
        _lib.orc_theta.argtypes = [C.c_uint64, C.c_uint64, i, i]
        pdp = C.POINTER(_DpdParams)
        _lib.orc_dpd_forces.restype = i
        _lib.orc_dpd_forces.argtypes = [pp, pdp, i, pd, pd, pi, i, pi, C.c_uint64, pd, pd, pi, i]
        _lib.orc_total_forces.restype = i
        _lib.orc_total_forces.argtypes = [pp, pdp, i, pd, pd, pi, pd, i, pi, C.c_uint64, pd, pd]
        _lib.orc_dpd_run.restype = i
        _lib.orc_dpd_run.argtypes = [pp, pdp, i, pd, pd, pd, pi, pd, i, pi,
                                     C.POINTER(C.c_uint64), i, pd]
    return _lib


@dataclass
class EwaldParams:
    """Parameters of one electrostatics evaluation (reduced DPD units)."""
    L: float
    alpha: float
    r_cut: float
    beta: float          # R_c / lambda_e; <= 0 means point charges
    kappa: float         # 1/(4 pi eps0 eps_r) in reduced units
    M: int               # base grid per dimension; n_c = M/2 - 1
    p: int               # NFFT window cutoff
    sigma_s: int = 2
    kmask: int = 0
    deriv: int = 0       # ENUF forces: 0 ik-differentiation (Eq. 24-25), 1 analytic gradient
    slater_k: int = 0    # Slater smearing: 0 real-space correction, 1 k-space form factor

    def c(self) -> _Params:
        return _Params(self.L, self.alpha, self.r_cut, self.beta, self.kappa,
                       self.M, self.p, self.sigma_s, self.kmask, self.deriv,
                       self.slater_k)

    @property
    def ng(self) -> int:
        return self.sigma_s * self.M


@dataclass
class DpdParams:
    a: np.ndarray        # ntypes x ntypes
    gamma: float
    sigma: float
    dt: float
    lambda_vv: float = 0.65
    K_bond: float = 0.0
    r0_bond: float = 0.0
    seed: int = 0
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _DpdParams:
        a = np.ascontiguousarray(self.a, dtype=np.float64)
        self._keep = [a]
        return _DpdParams(a.shape[0], _pd(a), self.gamma, self.sigma, self.dt,
                          self.lambda_vv, self.K_bond, self.r0_bond, self.seed)


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def wrap(x: float, L: float) -> float:
    return lib().orc_wrap(x, L)


def B1(beta, r):
    return lib().orc_B1(beta, r)


def B2(beta, r):
    return lib().orc_B2(beta, r)


def slater_energy(beta, r):
    return lib().orc_slater_energy(beta, r)


def slater_force(beta, r):
    return lib().orc_slater_force(beta, r)


def _sampled(fn, P, pos, q, sample):
    pos, q = _f64(pos), _f64(q)
    n = q.shape[0]
    s = _i32(sample)
    nout = n if s is None else s.shape[0]
    F = np.zeros((nout, 3))
    EW = np.zeros(2)
    _check(fn(C.byref(P.c()), n, _pd(pos), _pd(q), _pd(F), _pd(EW), _pi(s),
              0 if s is None else s.shape[0]), fn.__name__)
    return F, EW


def real_space(P: EwaldParams, pos, q, sample=None):
    """Real-space erfc + Slater-correction sum (Eq. 31, Eq. 27-28): (F, [E, W])."""
    return _sampled(lib().orc_real_space, P, pos, q, sample)


def recip_direct(P: EwaldParams, pos, q, sample=None):
    """Direct reciprocal Ewald sum over integer k (Eq. 18-19, 22-24): (F, [E, W])."""
    return _sampled(lib().orc_recip_direct, P, pos, q, sample)


def recip_enuf(P: EwaldParams, pos, q, sample=None, want_grid=False, want_h=False):
    """Naive ENUF reciprocal sum (Table 2 step 4(ii)).

    Returns (F, [E, W], grid or None, hfield or None)."""
    pos, q = _f64(pos), _f64(q)
    n = q.shape[0]
    s = _i32(sample)
    nout = n if s is None else s.shape[0]
    F = np.zeros((nout, 3))
    EW = np.zeros(2)
    ng = P.ng
    grid = np.zeros((ng, ng, ng)) if want_grid else None
    h = np.zeros((1 if P.deriv else 3, ng, ng, ng)) if want_h else None
    _check(lib().orc_recip_enuf(C.byref(P.c()), n, _pd(pos), _pd(q), _pd(F), _pd(EW),
                                _pd(grid), _pd(h), _pi(s), 0 if s is None else s.shape[0]),
           "recip_enuf")
    return F, EW, grid, h


def slater_I(P: EwaldParams, r, rho_one=False):
    """(I(r), I'(r)) of the k-space Slater kernel (orc_slater_I)."""
    I, dI = C.c_double(), C.c_double()
    lib().orc_slater_I(C.byref(P.c()), C.c_double(r), int(rho_one), C.byref(I), C.byref(dI))
    return I.value, dI.value


def self_neutral(P: EwaldParams, q):
    """[E_self, E_neutral, W_neutral] (Eq. 16 third term; background term)."""
    q = _f64(q)
    out = np.zeros(3)
    lib().orc_self_neutral(C.byref(P.c()), q.shape[0], _pd(q), _pd(out))
    return out


def electrostatics(P: EwaldParams, pos, q, recip="enuf", sample=None):
    """Total electrostatic force and energies: F = F_real + F_recip;
    E = [E_real, E_recip, E_self + E_neutral, E_total]; W = total virial."""
    Fr, ER = real_space(P, pos, q, sample)
    if recip == "enuf":
        Fk, EK, _, _ = recip_enuf(P, pos, q, sample)
    else:
        Fk, EK = recip_direct(P, pos, q, sample)
    ES = self_neutral(P, q)
    E = np.array([ER[0], EK[0], ES[0] + ES[1], ER[0] + EK[0] + ES[0] + ES[1]])
    W = ER[1] + EK[1] + ES[2]
    return Fr + Fk, E, W


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def theta(seed, step, i, j):
    return lib().orc_theta(seed, step, i, j)


def dpd_forces(P: EwaldParams, D: DpdParams, pos, vel, types, bonds=None, step=0, sample=None):
    """DPD C + D + R/sqrt(dt) pair forces and bond forces (Eq. 2-7, Sec. 2).
    Returns (F, [E_conservative, E_bond] or None when sampled)."""
    pos, vel = _f64(pos), _f64(vel)
    types = _i32(types)
    n = types.shape[0]
    b = _i32(bonds) if bonds is not None and len(bonds) else None
    nb = 0 if b is None else b.shape[0]
    s = _i32(sample)
    nout = n if s is None else s.shape[0]
    F = np.zeros((nout, 3))
    E2 = np.zeros(2)
    Dc = D.c()
    _check(lib().orc_dpd_forces(C.byref(P.c()), C.byref(Dc), n, _pd(pos), _pd(vel), _pi(types),
                                nb, _pi(b), step, _pd(F), _pd(E2), _pi(s),
                                0 if s is None else s.shape[0]), "dpd_forces")
    return F, (E2 if s is None else None)


def total_forces(P, D, pos, vel, types, q, bonds=None, step=0):
    """Table 2 steps 3-5: DPD + bonds + electrostatics. Returns (F, E[6])."""
    pos, vel, q = _f64(pos), _f64(vel), _f64(q)
    types = _i32(types)
    n = q.shape[0]
    b = _i32(bonds) if bonds is not None and len(bonds) else None
    nb = 0 if b is None else b.shape[0]
    F = np.zeros((n, 3))
    E = np.zeros(6)
    Dc = D.c()
    _check(lib().orc_total_forces(C.byref(P.c()), C.byref(Dc), n, _pd(pos), _pd(vel), _pi(types),
                                  _pd(q), nb, _pi(b), step, _pd(F), _pd(E)), "total_forces")
    return F, E


def dpd_run(P, D, pos, vel, F, types, q, bonds=None, step=0, nsteps=1):
    """Table 2 modified velocity-Verlet, nsteps. Returns (pos, vel, F, step, E[6])."""
    pos, vel, F, q = _f64(pos).copy(), _f64(vel).copy(), _f64(F).copy(), _f64(q)
    types = _i32(types)
    n = q.shape[0]
    b = _i32(bonds) if bonds is not None and len(bonds) else None
    nb = 0 if b is None else b.shape[0]
    st = C.c_uint64(step)
    E = np.zeros(6)
    Dc = D.c()
    _check(lib().orc_dpd_run(C.byref(P.c()), C.byref(Dc), n, _pd(pos), _pd(vel), _pd(F), _pi(types),
                             _pd(q), nb, _pi(b), C.byref(st), nsteps, _pd(E)), "dpd_run")
    return pos, vel, F, st.value, E
