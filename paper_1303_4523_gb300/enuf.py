"""ctypes binding of libenuf.so (include/enuf.h): argument marshalling only.

Every step of the ENUF-DPD path runs in the library's CUDA kernels; this
module converts torch tensors / numpy arrays to pointers and status codes to
exceptions. The function names are the C names. ``Plan``, ``DpdSystem`` and
``Batch`` are thin owners of the C handles.

If the shared library is missing the import of this module raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ENUF_CHECK=1 in the environment loads the debug build (device index checks)
LIB_PATH = os.path.join(_HERE, "libenuf_check.so" if os.environ.get("ENUF_CHECK") == "1" else "libenuf.so")

ENUF_FP64, ENUF_FP32 = 0, 1
ENUF_OK, ENUF_ERR_INVALID, ENUF_ERR_OOM, ENUF_ERR_CUDA, ENUF_ERR_TIMEOUT, ENUF_ERR_UNSUPPORTED = range(6)
ENUF_BUF_GRID, ENUF_BUF_FIELD = 0, 1
STAGES = {"bin": 0, "spread": 1, "fft": 2, "gather": 3, "real": 4, "dpd": 5, "all": 6, "cell": 7}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "device wait timed out", 5: "unsupported configuration"}


class EnufError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class enuf_params(C.Structure):
    _fields_ = [("L", C.c_double), ("alpha", C.c_double), ("r_cut", C.c_double),
                ("beta", C.c_double), ("kappa", C.c_double), ("M", C.c_int), ("p", C.c_int),
                ("sigma_s", C.c_int), ("kmask", C.c_int), ("prec", C.c_int), ("tile", C.c_int),
                ("deriv", C.c_int), ("slater_k", C.c_int), ("fft_path", C.c_int), ("fft_radix", C.c_int),
                ("spread", C.c_int), ("pairs", C.c_int)]


class enuf_plan_info(C.Structure):
    _fields_ = [("M", C.c_int), ("n", C.c_int), ("n_c", C.c_int), ("tile", C.c_int),
                ("n_tiles", C.c_int), ("n_max", C.c_int), ("fft_kernels", C.c_int),
                ("device_bytes", C.c_size_t), ("fft_stages", C.c_int), ("fft_radix", C.c_int * 8),
                ("fft_two_factor", C.c_int), ("spread", C.c_int), ("brick_x", C.c_int),
                ("pairs", C.c_int)]


class dpd_params(C.Structure):
    _fields_ = [("ntypes", C.c_int), ("a", C.POINTER(C.c_double)), ("gamma", C.c_double),
                ("sigma", C.c_double), ("dt", C.c_double), ("lambda_vv", C.c_double),
                ("K_bond", C.c_double), ("r0_bond", C.c_double), ("seed", C.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1303_4523_gb300.build.build() "
                          "(the ENUF-DPD path has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, st = C.c_void_p, C.c_int, C.c_double, C.c_int
    pd = C.POINTER(C.c_double)
    sig = {
        "enuf_plan": (st, [C.POINTER(enuf_params), i, vp, C.POINTER(vp)]),
        "enuf_footprint": (st, [C.POINTER(enuf_params), i, C.POINTER(C.c_size_t)]),
        "enuf_get_info": (st, [vp, C.POINTER(enuf_plan_info)]),
        "enuf_plan_shape": (st, [C.POINTER(enuf_params), i, C.POINTER(enuf_plan_info)]),
        "enuf_accuracy_params": (st, [d, C.POINTER(enuf_params)]),
        "enuf_energy_forces": (st, [vp, i, vp, vp, vp, pd, pd]),
        "enuf_energy_forces_host": (st, [vp, i, vp, vp, vp, pd, pd]),
        "enuf_last_energies": (st, [vp, pd, pd]),
        "enuf_debug_buffer": (st, [vp, i, vp, C.c_size_t]),
        "enuf_enable_timing": (st, [vp, i]),
        "enuf_stage_time": (st, [vp, i, C.POINTER(C.c_float)]),
        "enuf_launches_per_eval": (i, [vp]),
        "enuf_destroy": (None, [vp]),
        "enuf_status_string": (C.c_char_p, [st]),
        "enuf_last_error": (C.c_char_p, [vp]),
        "dpd_create": (st, [vp, C.POINTER(dpd_params), i, vp, vp, vp, vp, i, vp, C.POINTER(vp)]),
        "dpd_step": (st, [vp, i, pd]),
        "dpd_copy_energies": (st, [vp]),
        "dpd_get_state": (st, [vp, vp, vp, vp, C.POINTER(C.c_uint64)]),
        "dpd_set_state": (st, [vp, vp, vp, vp, C.c_uint64]),
        "dpd_get_forces": (st, [vp, vp]),
        "dpd_step_host": (st, [vp, C.c_int, vp, vp, vp, C.POINTER(C.c_double)]),
        "enuf_check_word": (st, [vp, C.POINTER(C.c_uint), C.c_int]),
        "enuf_built_with_checks": (C.c_int, []),
        "enuf_debug_fail_allocs": (st, [i, i]),
        "dpd_device_state": (st, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
        "dpd_destroy": (None, [vp]),
        "enuf_batch_plan": (st, [i, C.POINTER(enuf_params), C.POINTER(C.c_int), vp, C.POINTER(vp)]),
        "enuf_batch_energy_forces": (st, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), pd]),
        "enuf_batch_launches": (i, [vp]),
        "enuf_batch_mode": (i, [vp]),
        "enuf_batch_destroy": (None, [vp]),
        "enuf_spread_noalloc": (st, [C.POINTER(enuf_params), i, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()

EXPORTED = ("enuf_plan", "enuf_footprint", "enuf_get_info", "enuf_plan_shape", "enuf_accuracy_params",
            "enuf_energy_forces",
            "enuf_last_energies",
            "enuf_energy_forces_host", "enuf_debug_buffer", "enuf_enable_timing",
            "enuf_stage_time", "enuf_launches_per_eval", "enuf_destroy", "enuf_status_string",
            "enuf_last_error", "dpd_create", "dpd_step", "dpd_copy_energies", "dpd_get_state", "dpd_set_state",
            "dpd_get_forces", "dpd_step_host", "dpd_device_state", "enuf_check_word",
            "enuf_built_with_checks", "enuf_debug_fail_allocs", "dpd_destroy", "enuf_batch_plan",
            "enuf_batch_energy_forces", "enuf_batch_launches", "enuf_batch_mode", "enuf_batch_destroy",
            "enuf_spread_noalloc")


def _check(status, handle=None, what=""):
    if status != 0:
        msg = lib.enuf_last_error(handle).decode() if handle else what
        raise EnufError(status, msg or what)


def make_params(L, alpha, r_cut, beta, kappa, M=0, p=4, sigma_s=2, kmask=0,
                prec="fp64", tile=0, deriv=0, slater_k=0, fft_path=0, fft_radix=0, spread=0,
                pairs=0) -> enuf_params:
    pr = {"fp64": ENUF_FP64, "fp32": ENUF_FP32}[prec] if isinstance(prec, str) else int(prec)
    return enuf_params(float(L), float(alpha), float(r_cut), float(beta), float(kappa), int(M),
                       int(p), int(sigma_s), int(kmask), pr, int(tile), int(deriv), int(slater_k),
                       int(fft_path), int(fft_radix), int(spread), int(pairs))


def _ptr(x):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous(), "tensors must be contiguous"
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def _torch_stream():
    """A dedicated torch CUDA stream for a plan (None when torch/CUDA is absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.Stream()
    except ImportError:
        pass
    return None


class _Fence:
    """Orders a plan's stream after torch's current stream on entry and torch's
    current stream after the plan's stream on exit (tensors are produced and
    consumed on torch's stream)."""

    def __init__(self, stream):
        self.s = stream

    def __enter__(self):
        if self.s is not None:
            import torch
            self.cur = torch.cuda.current_stream()
            self.s.wait_stream(self.cur)

    def __exit__(self, *exc):
        if self.s is not None:
            self.cur.wait_stream(self.s)
        return False


def debug_fail_allocs(count: int, after: int = 0) -> None:
    """Failure injection: after `after` more device allocations of the
    library, the next `count` fail as out of memory (count 0 ends it)."""
    _check(lib.enuf_debug_fail_allocs(int(after), int(count)), what="enuf_debug_fail_allocs")


def accuracy_params(delta: float, params: enuf_params) -> enuf_params:
    """A copy of params with alpha and M chosen for accuracy delta by the two
    conditions of Eq. 29 (from params.L and params.r_cut)."""
    out = enuf_params()
    C.memmove(C.byref(out), C.byref(params), C.sizeof(enuf_params))
    _check(lib.enuf_accuracy_params(float(delta), C.byref(out)), what="enuf_accuracy_params")
    return out


def plan_shape(params: enuf_params, n_max: int) -> enuf_plan_info:
    """Derived sizes of a plan with these parameters (tile edge, grid, FFT
    kernels and radices, device bytes), from the host logic alone."""
    info = enuf_plan_info()
    _check(lib.enuf_plan_shape(C.byref(params), int(n_max), C.byref(info)), what="enuf_plan_shape")
    return info


def enuf_footprint(params: enuf_params, n_max: int) -> int:
    b = C.c_size_t()
    _check(lib.enuf_footprint(C.byref(params), n_max, C.byref(b)), what="enuf_footprint")
    return b.value


class Plan:
    """Owner of an enuf_plan_t (Table 2 step 4 on one system shape)."""

    def __init__(self, params: enuf_params, n_max: int, stream=None):
        self.params = params
        self.h = C.c_void_p()
        self.stream = stream if stream is not None else _torch_stream()
        _check(lib.enuf_plan(C.byref(params), int(n_max), _stream_handle(self.stream), C.byref(self.h)),
               what="enuf_plan failed (see stderr)")
        info = enuf_plan_info()
        _check(lib.enuf_get_info(self.h, C.byref(info)), self.h)
        self.info = info
        self.n_max = n_max
        self.dtype_np = np.float32 if params.prec == ENUF_FP32 else np.float64

    @property
    def torch_dtype(self):
        import torch
        return torch.float32 if self.params.prec == ENUF_FP32 else torch.float64

    def energy_forces(self, pos, q, F, want_energy=True):
        """Device tensors pos [n,3], q [n], F [n,3] (overwritten). Returns (E[4], virial) or None."""
        n = q.shape[0]
        E = (C.c_double * 4)()
        W = C.c_double()
        with _Fence(self.stream):
            _check(lib.enuf_energy_forces(self.h, n, _ptr(pos), _ptr(q), _ptr(F),
                                          E if want_energy else None, C.byref(W) if want_energy else None),
                   self.h)
        return (np.array(E[:]), W.value) if want_energy else None

    def enqueue(self, pos, q, F):
        """Enqueue one evaluation on the plan's stream and return at once (no
        synchronisation, no fence against torch's stream: the caller orders
        its inputs and outputs). Energies: last_energies() once it completed."""
        n = q.shape[0]
        _check(lib.enuf_energy_forces(self.h, n, _ptr(pos), _ptr(q), _ptr(F), None, None), self.h)

    def last_energies(self):
        E = (C.c_double * 8)()
        _check(lib.enuf_last_energies(self.h, E, None), self.h)
        return np.array(E[:])

    def energy_forces_host(self, pos, q, F):
        """Host numpy arrays (dtype of the plan). Returns (E[4], virial)."""
        n = q.shape[0]
        E = (C.c_double * 4)()
        W = C.c_double()
        _check(lib.enuf_energy_forces_host(self.h, n, _ptr(pos), _ptr(q), _ptr(F), E, C.byref(W)), self.h)
        return np.array(E[:]), W.value

    def debug_buffer(self, which):
        n = self.info.n
        shape = (n, n, n) if which == ENUF_BUF_GRID else (1 if self.params.deriv else 3, n, n, n)
        out = np.empty(shape, dtype=self.dtype_np)
        _check(lib.enuf_debug_buffer(self.h, which, _ptr(out), out.nbytes), self.h)
        return out

    def enable_timing(self, on=True):
        _check(lib.enuf_enable_timing(self.h, int(on)), self.h)

    def stage_time(self, stage):
        ms = C.c_float()
        _check(lib.enuf_stage_time(self.h, STAGES[stage] if isinstance(stage, str) else stage, C.byref(ms)),
               self.h)
        return ms.value

    def launches(self):
        return lib.enuf_launches_per_eval(self.h)

    def check_word(self, reset=True):
        """Failure bits of the device index checks (debug build; 0 otherwise)."""
        m = C.c_uint()
        _check(lib.enuf_check_word(self.h, C.byref(m), int(reset)), self.h)
        return m.value

    def close(self):
        if self.h:
            lib.enuf_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DpdSystem:
    """Owner of a dpd_system_t: device-resident DPD state on a plan."""

    def __init__(self, plan: Plan, a, gamma, sigma, dt, pos, vel, types, q, bonds=None,
                 lambda_vv=0.65, K_bond=0.0, r0_bond=0.0, seed=0):
        self.plan = plan
        dt_np = plan.dtype_np
        a = np.ascontiguousarray(a, dtype=np.float64)
        self._a = a
        prm = dpd_params(a.shape[0], a.ctypes.data_as(C.POINTER(C.c_double)), gamma, sigma, dt,
                         lambda_vv, K_bond, r0_bond, seed)
        pos = np.ascontiguousarray(pos, dtype=dt_np)
        vel = np.ascontiguousarray(vel, dtype=dt_np)
        q = np.ascontiguousarray(q, dtype=dt_np)
        types = np.ascontiguousarray(types, dtype=np.int32)
        b = None if bonds is None or len(bonds) == 0 else np.ascontiguousarray(bonds, dtype=np.int32)
        self.N = q.shape[0]
        self.h = C.c_void_p()
        _check(lib.dpd_create(plan.h, C.byref(prm), self.N, _ptr(pos), _ptr(vel), _ptr(types), _ptr(q),
                              0 if b is None else b.shape[0], _ptr(b), C.byref(self.h)), plan.h)

    def step(self, nsteps=1, want_energy=False):
        E = (C.c_double * 8)() if want_energy else None
        _check(lib.dpd_step(self.h, int(nsteps), E), self.plan.h)
        return np.array(E[:]) if want_energy else None

    def copy_energies(self):
        """Enqueue the copy of the last step's energies to the plan's host buffer
        (read with Plan.last_energies() once the work has completed)."""
        _check(lib.dpd_copy_energies(self.h), self.plan.h)

    def get_state(self):
        dt = self.plan.dtype_np
        pos = np.empty((self.N, 3), dt)
        vel = np.empty((self.N, 3), dt)
        F = np.empty((self.N, 3), dt)
        st = C.c_uint64()
        _check(lib.dpd_get_state(self.h, _ptr(pos), _ptr(vel), _ptr(F), C.byref(st)), self.plan.h)
        return pos, vel, F, st.value

    def set_state(self, pos, vel, F=None, step=0):
        dt = self.plan.dtype_np
        pos = np.ascontiguousarray(pos, dtype=dt)
        vel = np.ascontiguousarray(vel, dtype=dt)
        F = None if F is None else np.ascontiguousarray(F, dtype=dt)
        _check(lib.dpd_set_state(self.h, _ptr(pos), _ptr(vel), _ptr(F), int(step)), self.plan.h)

    def set_state_device(self, pos, vel, step):
        """Upload pos/vel from HOST buffers (pinned torch tensors or numpy) keeping F."""
        _check(lib.dpd_set_state(self.h, _ptr(pos), _ptr(vel), None, int(step)), self.plan.h)

    def device_state(self):
        p, v, f = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib.dpd_device_state(self.h, C.byref(p), C.byref(v), C.byref(f)), self.plan.h)
        return p.value, v.value, f.value

    def step_host(self, pos, vel, F, nsteps=1, want_energy=False):
        """Upload the HOST state (arrays of the plan's dtype, pinned tensors or numpy),
        advance nsteps, copy the new state back into the same arrays; one host
        synchronisation. Returns the energies (as step) or None."""
        E = (C.c_double * 8)() if want_energy else None
        _check(lib.dpd_step_host(self.h, int(nsteps), _ptr(pos), _ptr(vel), _ptr(F), E), self.plan.h)
        return np.array(E[:]) if want_energy else None

    def get_state_into(self, pos=None, vel=None, F=None):
        """Copy state into caller-provided HOST buffers; returns the step."""
        st = C.c_uint64()
        _check(lib.dpd_get_state(self.h, _ptr(pos), _ptr(vel), _ptr(F), C.byref(st)), self.plan.h)
        return st.value

    def close(self):
        if self.h:
            lib.dpd_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owner of an enuf_batch_t: many systems, one captured graph (one launch
    sequence over all systems where every plan qualifies, see mode())."""

    def __init__(self, params_list, n_list, stream=None):
        ns = len(params_list)
        arr = (enuf_params * ns)(*params_list)
        nn = (C.c_int * ns)(*[int(v) for v in n_list])
        self.h = C.c_void_p()
        self.ns = ns
        self.n = list(n_list)
        self.stream = stream if stream is not None else _torch_stream()
        _check(lib.enuf_batch_plan(ns, arr, nn, _stream_handle(self.stream), C.byref(self.h)),
               what="enuf_batch_plan failed (see stderr)")

    def energy_forces(self, pos_list, q_list, F_list, want_energy=True):
        ns = self.ns
        P = (C.c_void_p * ns)(*[_ptr(x) for x in pos_list])
        Q = (C.c_void_p * ns)(*[_ptr(x) for x in q_list])
        Fp = (C.c_void_p * ns)(*[_ptr(x) for x in F_list])
        E = (C.c_double * (4 * ns))() if want_energy else None
        with _Fence(self.stream):
            _check(lib.enuf_batch_energy_forces(self.h, P, Q, Fp, E), what="enuf_batch_energy_forces")
        return np.array(E[:]).reshape(ns, 4) if want_energy else None

    def launches(self):
        return lib.enuf_batch_launches(self.h)

    def mode(self):
        """1: one launch sequence over all systems; 0: one graph branch per system."""
        return lib.enuf_batch_mode(self.h)

    def close(self):
        if self.h:
            lib.enuf_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
