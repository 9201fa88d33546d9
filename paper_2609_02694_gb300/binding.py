"""Thin ctypes binding of the RBE C ABI (include/rbe.h).

Argument marshalling only. Every step of the force path runs in the CUDA library
`_build/librbe_gb300.so`. If that library is missing, `lib()` raises instead of falling
back to anything else. Build the library with `paper_2609_02694_gb300.build.build()`.
"""
from __future__ import annotations

import ctypes as ct
import os
import re

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "rbe.h")

RBE_OK = 0
PRECISION = {"fp32_comp": 0, "fp32": 1, "fp64": 2}
ENERGY_KEYS = ("real", "lj", "kspace", "self", "total", "kinetic")
VIRIAL_KEYS = ("real", "lj", "kspace", "total")
TUNABLES = {"pair_test16": 0, "sf_tile": 1, "rbl_eager": 2, "rbl_span": 3, "pair_cluster": 4}
PHASES = ("kick_drift", "bin", "sample", "sf", "list", "pair", "pair2", "gather", "tail")


class RBEError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = lib().rbe_error_string(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{what}: {msg} (code {code})")
        self.code = code


class Params(ct.Structure):
    _fields_ = [
        ("alpha", ct.c_double), ("r_c", ct.c_double), ("r_core", ct.c_double),
        ("p_rbl", ct.c_int32), ("P", ct.c_int32), ("seed", ct.c_uint64),
        ("replica", ct.c_uint32), ("precision", ct.c_int32), ("coulomb_C", ct.c_double),
        ("dt", ct.c_double), ("kappa", ct.c_double), ("n_types", ct.c_int32),
        ("lj_eps", ct.POINTER(ct.c_double)), ("lj_sigma", ct.POINTER(ct.c_double)),
        ("cell_sub", ct.c_int32),
    ]


_LIB = None
_vp = ct.c_void_p


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load the CUDA library; raise if it is not built (no fallback path exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"RBE CUDA library not built: {path} (run build.build())")
    L = ct.CDLL(path)
    h = ct.c_void_p
    L.rbe_init.argtypes = [ct.POINTER(h), ct.POINTER(Params), ct.c_int64, _vp, _vp, _vp, _vp,
                           _vp, _vp, _vp]
    L.rbe_sample_k.argtypes = [h, ct.c_uint64, _vp, _vp]
    L.rbe_set_positions.argtypes = [h, _vp, ct.c_int]
    L.rbe_forces.argtypes = [h, ct.c_uint64, _vp, ct.c_int, _vp, _vp]
    L.rbe_forces_f64.argtypes = [h, ct.c_uint64, _vp, _vp, _vp]
    L.rbe_step.argtypes = [h, ct.c_int]
    L.rbe_get_energies.argtypes = [h, _vp, _vp]
    L.rbe_get_step.argtypes = [h, _vp]
    L.rbe_get_state.argtypes = [h, _vp, _vp, _vp]
    L.rbe_get_cells.argtypes = [h, _vp, _vp, _vp]
    L.rbe_get_rho.argtypes = [h, _vp, _vp]
    L.rbe_get_neighbor_counts.argtypes = [h, _vp, _vp]
    L.rbe_get_rbl_partners.argtypes = [h, _vp]
    L.rbe_get_memory.argtypes = [h, _vp]
    L.rbe_set_profiling.argtypes = [h, ct.c_int]
    L.rbe_get_profile.argtypes = [h, _vp, _vp]
    L.rbe_check_device.argtypes = [h]
    L.rbe_batch_create.argtypes = [ct.POINTER(ct.c_void_p), ct.c_int, ct.POINTER(ct.c_void_p), _vp]
    L.rbe_batch_step.argtypes = [ct.c_void_p, ct.c_int]
    L.rbe_batch_destroy.argtypes = [ct.c_void_p]
    L.rbe_batch_info.argtypes = [ct.c_void_p, _vp, _vp, _vp]
    L.rbe_measure_peak.argtypes = [ct.c_int, _vp, _vp]
    L.rbe_set_thermostat.argtypes = [ct.c_void_p, ct.c_double, ct.c_double, ct.c_double]
    L.rbe_get_thermostat.argtypes = [ct.c_void_p, _vp]
    L.rbe_set_tuning.argtypes = [ct.c_void_p, ct.c_int, ct.c_int]
    L.rbe_get_tuning.argtypes = [ct.c_void_p, ct.c_int, _vp]
    L.rbe_autotune.argtypes = [ct.c_void_p, ct.c_int, _vp]
    L.rbe_set_neighbor_list.argtypes = [ct.c_void_p, ct.c_double, ct.c_int]
    L.rbe_get_neighbor_list.argtypes = [ct.c_void_p, _vp]
    L.rbe_structure_factor_noalloc.argtypes = [_vp, _vp, ct.c_int64, _vp, ct.c_int, _vp, _vp]
    L.rbe_save.argtypes = [h, ct.c_char_p]
    L.rbe_load.argtypes = [h, ct.c_char_p]
    L.rbe_destroy.argtypes = [h]
    L.rbe_decision_band.argtypes = [_vp, ct.c_double, _vp, ct.c_int]
    L.rbe_decision_band.restype = ct.c_double
    L.rbe_error_string.argtypes = [ct.c_int]
    L.rbe_error_string.restype = ct.c_char_p
    L.rbe_version.restype = ct.c_char_p
    for name in declared_functions():
        if name not in ("rbe_error_string", "rbe_version", "rbe_decision_band"):
            getattr(L, name).restype = ct.c_int
    _LIB = L
    return L


def declared_functions(header: str = HEADER) -> list[str]:
    """Names of the functions include/rbe.h declares."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rbe_[a-z0-9_]+)\s*\(", txt)))


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _check(rc: int, what: str):
    if rc != RBE_OK:
        raise RBEError(rc, what)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # noqa: BLE001 - torch is optional for the binding
        pass
    return None


class RBE:
    """One periodic system on the GPU (a handle of the C ABI)."""

    def __init__(self, box, pos, q, types=None, mass=None, vel=None, *, alpha: float,
                 r_c: float, P: int, eps, sigma, seed: int = 1, replica: int = 0,
                 precision: str = "fp32_comp", coulomb_C: float = 332.06371, dt: float = 1.0,
                 kappa: float = 4.184e-4, r_core: float = 0.0, p_rbl: int = 10,
                 cell_sub: int = 0, stream=None):
        L = lib()
        self.box = _f64(box).copy()
        pos = _f64(pos, (-1, 3))
        self.N = pos.shape[0]
        q = _f64(q)
        eps = _f64(np.atleast_1d(eps)).reshape(-1)
        sig = _f64(np.atleast_1d(sigma)).reshape(-1)
        nt = int(round(np.sqrt(eps.size)))
        self._keep = [eps, sig]
        p = Params(alpha=alpha, r_c=r_c, r_core=r_core, p_rbl=p_rbl, P=P, seed=seed,
                   replica=replica, precision=PRECISION[precision], coulomb_C=coulomb_C,
                   dt=dt, kappa=kappa, n_types=nt,
                   lj_eps=eps.ctypes.data_as(ct.POINTER(ct.c_double)),
                   lj_sigma=sig.ctypes.data_as(ct.POINTER(ct.c_double)), cell_sub=cell_sub)
        self.P = P
        self.p_rbl = p_rbl if r_core > 0 else 0
        self.precision = precision
        t = None if types is None else np.ascontiguousarray(types, np.int32)
        m = None if mass is None else _f64(mass)
        v = None if vel is None else _f64(vel, (-1, 3))
        if stream is None:
            stream = _current_stream()
        self._h = ct.c_void_p()
        rc = L.rbe_init(ct.byref(self._h), ct.byref(p), self.N, self.box.ctypes.data,
                        pos.ctypes.data, q.ctypes.data, _ptr(t), _ptr(m), _ptr(v), stream)
        _check(rc, "rbe_init")

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rbe_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def sample_k(self, step: int):
        m = np.zeros((self.P, 3), np.int32)
        S = ct.c_double()
        _check(lib().rbe_sample_k(self._h, step, m.ctypes.data, ct.addressof(S)), "rbe_sample_k")
        return m, S.value

    def set_positions(self, pos):
        if isinstance(pos, np.ndarray):
            pos = _f64(pos, (-1, 3))
            _check(lib().rbe_set_positions(self._h, pos.ctypes.data, 0), "rbe_set_positions")
        else:  # torch tensor: host (pinned or not) or device, float64 (N, 3)
            _check(lib().rbe_set_positions(self._h, pos.data_ptr(), int(pos.is_cuda)),
                   "rbe_set_positions")

    def forces(self, step: int, out=None, energies: bool = True):
        """FP32 forces (N, 3) in id order; `out` may be a numpy array or a torch tensor."""
        if out is None:
            out = np.zeros((self.N, 3), np.float32)
        on_dev = 0 if isinstance(out, np.ndarray) else int(out.is_cuda)
        e = np.zeros(6, np.float64) if energies else None
        w = np.zeros(4, np.float64) if energies else None
        _check(lib().rbe_forces(self._h, step, _ptr(out), on_dev, _ptr(e), _ptr(w)), "rbe_forces")
        if not energies:
            return out
        return out, dict(zip(ENERGY_KEYS, e)), dict(zip(VIRIAL_KEYS, w))

    def forces_f64(self, step: int):
        F = np.zeros((self.N, 3), np.float64)
        e = np.zeros(6, np.float64)
        w = np.zeros(4, np.float64)
        _check(lib().rbe_forces_f64(self._h, step, F.ctypes.data, e.ctypes.data, w.ctypes.data),
               "rbe_forces_f64")
        return F, dict(zip(ENERGY_KEYS, e)), dict(zip(VIRIAL_KEYS, w))

    def step(self, n: int = 1):
        _check(lib().rbe_step(self._h, n), "rbe_step")

    def energies(self):
        e = np.zeros(6, np.float64)
        w = np.zeros(4, np.float64)
        _check(lib().rbe_get_energies(self._h, e.ctypes.data, w.ctypes.data), "rbe_get_energies")
        return dict(zip(ENERGY_KEYS, e)), dict(zip(VIRIAL_KEYS, w))

    def step_count(self) -> int:
        s = ct.c_uint64()
        _check(lib().rbe_get_step(self._h, ct.addressof(s)), "rbe_get_step")
        return s.value

    def state(self):
        pos = np.zeros((self.N, 3), np.float64)
        vel = np.zeros((self.N, 3), np.float64)
        s = np.zeros((self.N, 3), np.uint32)
        _check(lib().rbe_get_state(self._h, pos.ctypes.data, vel.ctypes.data, s.ctypes.data),
               "rbe_get_state")
        return pos, vel, s

    def cells(self):
        n = np.zeros(3, np.int32)
        _check(lib().rbe_get_cells(self._h, n.ctypes.data, None, None), "rbe_get_cells")
        cs = np.zeros(int(np.prod(n.astype(np.int64))) + 1, np.int64)
        ids = np.zeros(self.N, np.int64)
        _check(lib().rbe_get_cells(self._h, n.ctypes.data, cs.ctypes.data, ids.ctypes.data),
               "rbe_get_cells")
        return n, cs, ids

    def rho(self):
        r = np.zeros((self.P, 2), np.float64)
        m = np.zeros((self.P, 3), np.int32)
        _check(lib().rbe_get_rho(self._h, r.ctypes.data, m.ctypes.data), "rbe_get_rho")
        return r[:, 0] + 1j * r[:, 1], m

    def neighbor_counts(self):
        a = np.zeros(self.N, np.int32)
        b = np.zeros(self.N, np.int32)
        _check(lib().rbe_get_neighbor_counts(self._h, a.ctypes.data, b.ctypes.data),
               "rbe_get_neighbor_counts")
        return a, b

    def rbl_partners(self):
        out = np.zeros((self.N, self.p_rbl), np.int32)
        _check(lib().rbe_get_rbl_partners(self._h, out.ctypes.data), "rbe_get_rbl_partners")
        return out

    def set_profiling(self, enable: bool = True):
        _check(lib().rbe_set_profiling(self._h, int(enable)), "rbe_set_profiling")

    def profile(self):
        """(per-phase ms of the last evaluation or step, kernels per Verlet step)."""
        ms = np.zeros(len(PHASES), np.float64)
        k = ct.c_int64()
        _check(lib().rbe_get_profile(self._h, ms.ctypes.data, ct.addressof(k)), "rbe_get_profile")
        return dict(zip(PHASES, ms)), k.value

    def kernels_per_step(self) -> int:
        k = ct.c_int64()
        _check(lib().rbe_get_profile(self._h, None, ct.addressof(k)), "rbe_get_profile")
        return k.value

    def set_thermostat(self, T: float, tau: float, kB: float = 0.0019872067):
        """Nose-Hoover NVT at temperature T with relaxation time tau (tau <= 0: NVE)."""
        _check(lib().rbe_set_thermostat(self._h, float(T), float(tau), float(kB)),
               "rbe_set_thermostat")

    def thermostat(self):
        """(xi, eta, extended-energy term Q xi^2/2 + Nf kB T eta)."""
        out = np.zeros(3, np.float64)
        _check(lib().rbe_get_thermostat(self._h, out.ctypes.data), "rbe_get_thermostat")
        return tuple(out)

    def set_tuning(self, key: str, value: int):
        _check(lib().rbe_set_tuning(self._h, TUNABLES[key], int(value)), "rbe_set_tuning")

    def get_tuning(self, key: str) -> int:
        v = ct.c_int()
        _check(lib().rbe_get_tuning(self._h, TUNABLES[key], ct.addressof(v)), "rbe_get_tuning")
        return v.value

    def autotune(self, reps: int = 3) -> dict:
        ch = np.zeros(len(TUNABLES), np.int32)
        _check(lib().rbe_autotune(self._h, reps, ch.ctypes.data), "rbe_autotune")
        return {k: int(ch[v]) for k, v in TUNABLES.items()}

    def set_neighbor_list(self, skin: float, capacity: int = 0):
        """Verlet list at r_c + skin (skin 0: per-step cell traversal)."""
        _check(lib().rbe_set_neighbor_list(self._h, float(skin), int(capacity)),
               "rbe_set_neighbor_list")

    def neighbor_list_stats(self) -> dict:
        st = np.zeros(6, np.int64)
        _check(lib().rbe_get_neighbor_list(self._h, st.ctypes.data), "rbe_get_neighbor_list")
        return dict(builds=int(st[0]), evaluations=int(st[1]), max_len=int(st[2]),
                    max_len_charged=int(st[3]), capacity=int(st[4]),
                    capacity_charged=int(st[5]))

    def save(self, path: str):
        """Write the dynamic state (step, positions, velocities, thermostat) to a file."""
        _check(lib().rbe_save(self._h, os.fsencode(path)), "rbe_save")

    def load(self, path: str):
        """Resume from a file written by save() on a handle with the same system."""
        _check(lib().rbe_load(self._h, os.fsencode(path)), "rbe_load")

    def memory_bytes(self) -> int:
        b = ct.c_int64()
        _check(lib().rbe_get_memory(self._h, ct.addressof(b)), "rbe_get_memory")
        return b.value

    def check_device(self):
        _check(lib().rbe_check_device(self._h), "rbe_check_device")


class Batch:
    """Replicas advanced together: one CUDA graph launch per Verlet step for all of them."""

    def __init__(self, handles, stream=None):
        self.handles = list(handles)
        arr = (ct.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        if stream is None:
            stream = _current_stream()
        self._b = ct.c_void_p()
        _check(lib().rbe_batch_create(ct.byref(self._b), len(self.handles), arr, stream),
               "rbe_batch_create")

    def step(self, n: int = 1):
        _check(lib().rbe_batch_step(self._b, n), "rbe_batch_step")

    def info(self):
        """(classes, replicas run by the batched launches, kernel launches per step)."""
        k, nb, kern = ct.c_int32(), ct.c_int32(), ct.c_int64()
        _check(lib().rbe_batch_info(self._b, ct.addressof(k), ct.addressof(nb),
                                    ct.addressof(kern)), "rbe_batch_info")
        return k.value, nb.value, kern.value

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            lib().rbe_batch_destroy(self._b)
            self._b = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def measure_peak(kind: str) -> float:
    """Measured device throughput: 'fp32' (flop/s), 'sincos' (pairs/s) or 'fp64' (flop/s)."""
    v = ct.c_double()
    _check(lib().rbe_measure_peak({"fp32": 0, "sincos": 1, "fp64": 2}[kind], ct.addressof(v), None),
           "rbe_measure_peak")
    return v.value


def decision_band(X, r: float, box, wrap: bool = False) -> float:
    """Relative half-width of the exact-decision band the kernels use around r^2 for an FP32
    r^2 from frame coordinates bounded by X (per axis), in a box of edges box."""
    X = _f64(X).reshape(3).copy()
    b = _f64(box).reshape(3).copy()
    v = lib().rbe_decision_band(X.ctypes.data, float(r), b.ctypes.data, int(bool(wrap)))
    if v < 0:
        raise ValueError("rbe_decision_band: invalid argument")
    return v


def from_system(sy, *, P: int, alpha: float, r_c: float, **kw) -> RBE:
    """Handle for a `synth.System` (positions passed exactly on the 2^-32 grid)."""
    return RBE(sy.box, sy.positions(), sy.q, sy.types, sy.mass, sy.v, alpha=alpha, r_c=r_c,
               P=P, eps=sy.eps, sigma=sy.sig, **kw)
