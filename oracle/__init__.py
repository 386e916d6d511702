"""CPU oracle for the WMCD sweep — test infrastructure.

A plain sequential FP64 C++ statement of the method (``wmcd_oracle.cpp``), loaded with
ctypes. Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use it; the product package never imports it.

Parity note: every oracle function is pinned by ``tests/test_oracle_pins.py`` against
closed forms, printed values, invariants or brute force (see the header of that file).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "wmcd_oracle.cpp")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


class OParams(ctypes.Structure):
    _fields_ = [
        ("n_beads", ctypes.c_int64), ("box_L", ctypes.c_double),
        ("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double), ("A0", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("bond_type", ctypes.c_int32), ("bond_k", ctypes.c_double), ("bond_r0", ctypes.c_double),
        ("fene_R0", ctypes.c_double),
        ("wca_sigma", ctypes.c_double), ("wca_eps", ctypes.c_double), ("ext_kappa", ctypes.c_double),
        ("planewave_mode", ctypes.c_int32), ("lcut", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("sim_id", ctypes.c_uint64),
        ("colour_K", ctypes.c_int32), ("grid_f", ctypes.c_int32), ("n_cap", ctypes.c_int32),
        ("grid_layer", ctypes.c_int32 * 16), ("big_support", ctypes.c_int32),
        ("acceptance", ctypes.c_int32), ("centring", ctypes.c_int32), ("level2", ctypes.c_int32),
    ]


class OStats(ctypes.Structure):
    _fields_ = [
        ("attempts", ctypes.c_int64 * 16), ("accepts", ctypes.c_int64 * 16), ("deferred", ctypes.c_int64 * 16),
        ("pw_attempts", ctypes.c_int64), ("pw_accepts", ctypes.c_int64),
        ("bead_updates", ctypes.c_int64), ("accepted_total", ctypes.c_int64),
        ("sim_time", ctypes.c_double), ("sweeps", ctypes.c_int64), ("n_layers", ctypes.c_int64),
        ("dt_move", ctypes.c_double), ("p_fourier", ctypes.c_double), ("moved_beads", ctypes.c_int64),
    ]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, D, I64, I32, U64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    sig = {
        "oracle_create": ([P, P, P, I64, P], P),
        "oracle_destroy": ([P], None),
        "oracle_sweep": ([P, I64], ctypes.c_int),
        "oracle_planewave": ([P, I64], ctypes.c_int),
        "oracle_positions": ([P, P, ctypes.c_int], ctypes.c_int),
        "oracle_stats": ([P, P], ctypes.c_int),
        "oracle_trace_layer": ([P, ctypes.c_int, P, P, I64], I64),
        "oracle_trace_pw": ([P, P, P, I64], I64),
        "oracle_trace_du": ([P, ctypes.c_int, P, I64], I64),
        "oracle_trace_lam": ([P, ctypes.c_int, P, I64], I64),
        "oracle_philox": ([P, P, P], None),
        "oracle_phitilde": ([D], D),
        "oracle_moment": ([ctypes.c_int], D),
        "oracle_G": ([P, I64, P], None),
        "oracle_cos2pi": ([D], D),
        "oracle_sin2pi": ([D], D),
        "oracle_cos2pi_f": ([D], ctypes.c_float),
        "oracle_inv_cbrt": ([D, D], D),
        "oracle_lambda_a": ([], D),
        "oracle_layers": ([P, P, P, P, P, ctypes.c_int], ctypes.c_int),
        "oracle_slot_counts": ([P, ctypes.c_uint64, P], ctypes.c_int),
        "oracle_sample_slots": ([P, ctypes.c_int, I64, P, P], I64),
        "oracle_sample_ball": ([P, U64, I64, P], I64),
        "oracle_sample_polarisation": ([P, U64, I64, P], I64),
        "oracle_wavelet_field": ([P, P, D, P, D, P, P], None),
        "oracle_delta_u": ([P, I64, P, P], D),
        "oracle_total_energy": ([P], D),
        "oracle_pw_modes": ([P, P, P, I64, P, P], I64),
        "oracle_propose_moments": ([P, I64, U64, P], ctypes.c_int),
        "oracle_sweep_record": ([P, I64, P], ctypes.c_int),
        "oracle_pw_polarisation": ([P, D, P], None),
        "oracle_sweep_sample": ([P, I64], I64),
        "oracle_sample_threshold": ([P, U64, I64, P], I64),
        "oracle_pw_tables": ([P, P], None),
        "oracle_k_cdf_exact": ([D], D),
        "oracle_k_inverse": ([P, D], D),
        "oracle_solid_angle_in_cube": ([D], D),
        "oracle_sample_pw_k": ([P, U64, I64, P], I64),
        "oracle_trace_pw_k": ([P, P, I64], I64),
        "oracle_planewave_field": ([P, P, D, D, P, P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def make_params(**kw) -> OParams:
    p = OParams()
    layers = kw.pop("grid_layer", [])
    for k, v in kw.items():
        setattr(p, k, v)
    for i, g in enumerate(layers):
        p.grid_layer[i] = int(g)
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One simulation run by the oracle. ``params`` is a dict of parameter fields."""

    def __init__(self, params: dict, pos: np.ndarray, chain_len: np.ndarray):
        lib = _load()
        self._lib = lib
        pr = make_params(**dict(params))
        self.n = int(pr.n_beads)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        cl = np.ascontiguousarray(chain_len, dtype=np.int32)
        err = ctypes.c_int(0)
        self._keep = (pos, cl)
        self.h = lib.oracle_create(ctypes.byref(pr), _ptr(pos), _ptr(cl), len(cl), ctypes.byref(err))
        if not self.h:
            raise ValueError(f"oracle rejected the parameters (code {err.value})")

    def close(self):
        if self.h:
            self._lib.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1):
        self._lib.oracle_sweep(self.h, int(n))

    def sweep_sample(self, max_moves: int) -> int:
        """The first max_moves wavelet attempts of the next sweep (the rest of it skipped): a
        bounded sample for timing. Returns the attempts made."""
        return int(self._lib.oracle_sweep_sample(self.h, int(max_moves)))

    def planewave(self, n: int = 1):
        if self._lib.oracle_planewave(self.h, int(n)) != 0:
            raise ValueError("plane waves are off")

    def positions(self, unwrapped: bool = False) -> np.ndarray:
        out = np.zeros((self.n, 3), dtype=np.float64)
        self._lib.oracle_positions(self.h, _ptr(out), int(unwrapped))
        return out

    def stats(self) -> OStats:
        st = OStats()
        self._lib.oracle_stats(self.h, ctypes.byref(st))
        return st

    def trace_layer(self, l: int):
        cap = 4 * self.n + 16
        out = np.zeros(cap, dtype=np.uint8)
        nn = np.zeros(cap, dtype=np.int32)
        m = self._lib.oracle_trace_layer(self.h, int(l), _ptr(out), _ptr(nn), cap)
        return out[:m].copy(), nn[:m].copy()

    def trace_du(self, l: int):
        cap = 4 * self.n + 16
        out = np.zeros(cap)
        m = self._lib.oracle_trace_du(self.h, int(l), _ptr(out), cap)
        return out[:m].copy()

    def trace_lam(self, l: int):
        """The lambda each wavelet slot of layer l used in the last sweep (0: not attempted)."""
        cap = 4 * self.n + 16
        out = np.zeros(cap)
        m = self._lib.oracle_trace_lam(self.h, int(l), _ptr(out), cap)
        return out[:m].copy()

    def trace_pw(self):
        cap = 1 << 16
        out = np.zeros(cap, dtype=np.uint8)
        mode = np.zeros(cap, dtype=np.int32)
        m = self._lib.oracle_trace_pw(self.h, _ptr(out), _ptr(mode), cap)
        return out[:m].copy(), mode[:m].copy()

    def layers(self):
        lo, hi, mass, ex = (np.zeros(16) for _ in range(4))
        n = self._lib.oracle_layers(self.h, _ptr(lo), _ptr(hi), _ptr(mass), _ptr(ex), 16)
        return lo[:n], hi[:n], mass[:n], ex[:n]

    def slot_counts(self, sweep: int):
        """Slots of sweep `sweep`: per wavelet layer, and the plane-wave slots."""
        out = np.zeros(17, dtype=np.int64)
        n = self._lib.oracle_slot_counts(self.h, int(sweep), _ptr(out))
        return out[:n].copy(), int(out[16])

    def sample_slots(self, layer: int, n: int):
        lam = np.zeros(n)
        bead = np.zeros(n, dtype=np.int64)
        self._lib.oracle_sample_slots(self.h, int(layer), int(n), _ptr(lam), _ptr(bead))
        return lam, bead

    def sample_ball(self, sweep: int, n: int):
        out = np.zeros((n, 3))
        self._lib.oracle_sample_ball(self.h, int(sweep), int(n), _ptr(out))
        return out

    def sample_polarisation(self, sweep: int, n: int):
        out = np.zeros((n, 3))
        self._lib.oracle_sample_polarisation(self.h, int(sweep), int(n), _ptr(out))
        return out

    def wavelet_field(self, b, lam, p, Aw, pt):
        b = np.ascontiguousarray(b, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        pt = np.ascontiguousarray(pt, dtype=np.float64)
        out = np.zeros(3)
        self._lib.oracle_wavelet_field(self.h, _ptr(b), float(lam), _ptr(p), float(Aw), _ptr(pt), _ptr(out))
        return out

    def delta_u(self, ids, newpos) -> float:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        newpos = np.ascontiguousarray(newpos, dtype=np.float64).reshape(-1, 3)
        return float(self._lib.oracle_delta_u(self.h, len(ids), _ptr(ids), _ptr(newpos)))

    def total_energy(self) -> float:
        return float(self._lib.oracle_total_energy(self.h))

    def pw_modes(self):
        cap = 1 << 20
        modes = np.zeros((cap, 3), dtype=np.int32)
        prob = np.zeros(cap)
        R, PF = ctypes.c_double(), ctypes.c_double()
        m = self._lib.oracle_pw_modes(self.h, _ptr(modes), _ptr(prob), cap, ctypes.byref(R), ctypes.byref(PF))
        return modes[:m].copy(), prob[:m].copy(), R.value, PF.value

    def propose_moments(self, n: int, offset: int = 0):
        out = np.zeros(27)
        if self._lib.oracle_propose_moments(self.h, int(n), int(offset), _ptr(out)) != 0:
            raise ValueError("needs at least two beads")
        return out[:9].reshape(3, 3), out[9:18].reshape(3, 3), out[18:].reshape(3, 3)

    def planewave_field(self, l, phi, psi, pt):
        lv = np.ascontiguousarray(l, dtype=np.int32)
        pt = np.ascontiguousarray(pt, dtype=np.float64)
        out = np.zeros(3)
        self._lib.oracle_planewave_field(self.h, _ptr(lv), float(phi), float(psi), _ptr(pt), _ptr(out))
        return out

    def pw_tables(self):
        """(probability of the discrete cube, cube weight sum, shell weight integral, F(Q0))."""
        out = np.zeros(4)
        self._lib.oracle_pw_tables(self.h, _ptr(out))
        return tuple(out)

    def sample_threshold(self, sweep: int, n: int) -> np.ndarray:
        """Acceptance thresholds of n slots (accept iff dU <= threshold)."""
        out = np.zeros(n)
        self._lib.oracle_sample_threshold(self.h, int(sweep), int(n), _ptr(out))
        return out

    def k_inverse(self, u: float) -> float:
        return float(self._lib.oracle_k_inverse(self.h, float(u)))

    def sample_pw_k(self, ctr: int, n: int) -> np.ndarray:
        """n fresh plane-wave wave vectors (units of 2 pi / L) as the moves draw them."""
        out = np.zeros((n, 3))
        if self._lib.oracle_sample_pw_k(self.h, int(ctr), int(n), _ptr(out)) < 0:
            raise ValueError("plane waves are off")
        return out

    def trace_pw_k(self) -> np.ndarray:
        cap = 1 << 16
        out = np.zeros((cap, 3))
        m = self._lib.oracle_trace_pw_k(self.h, _ptr(out), cap)
        return out[:m].copy()

    def sweep_record(self, n: int):
        out = np.zeros((n, 3))
        self._lib.oracle_sweep_record(self.h, int(n), _ptr(out))
        return out


# ---- free functions ------------------------------------------------------------------

def philox(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def phitilde(k: float) -> float:
    return float(_load().oracle_phitilde(float(k)))


def moment(m: int) -> float:
    return float(_load().oracle_moment(int(m)))


def G(Q) -> np.ndarray:
    q = np.ascontiguousarray(np.atleast_1d(Q), dtype=np.float64)
    out = np.zeros_like(q)
    _load().oracle_G(_ptr(q), len(q), _ptr(out))
    return out


def cos2pi(t: float) -> float:
    return float(_load().oracle_cos2pi(float(t)))


def sin2pi(t: float) -> float:
    return float(_load().oracle_sin2pi(float(t)))


def cos2pi_f(t: float) -> float:
    return float(_load().oracle_cos2pi_f(float(t)))


def inv_cbrt(w: float, lo: float) -> float:
    return float(_load().oracle_inv_cbrt(float(w), float(lo)))


def k_cdf_exact(Q: float) -> float:
    return float(_load().oracle_k_cdf_exact(float(Q)))


def solid_angle_in_cube(t: float) -> float:
    return float(_load().oracle_solid_angle_in_cube(float(t)))


def pw_polarisation(l, psi: float) -> np.ndarray:
    lv = np.ascontiguousarray(l, dtype=np.int32)
    out = np.zeros(3)
    _load().oracle_pw_polarisation(_ptr(lv), float(psi), _ptr(out))
    return out


def lambda_a() -> float:
    return float(_load().oracle_lambda_a())
