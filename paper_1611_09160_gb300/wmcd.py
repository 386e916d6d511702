"""Python binding of the WMCD C ABI (include/wmcd.h): argument marshalling only.

Every step of the sweep runs in the CUDA library ``_build/libwmcd.so`` (sm_103a). There
is no CPU fallback: if the library is missing or no GPU is present, the calls fail.
PyTorch is used only for device buffers and streams.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import schedule as _schedule

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libwmcd.so")
_SOURCES = ["wmcd_kernels.cu", "wmcd_api.cu", "wmcd_batch.cu", "wmcd_noalloc.cu"]
_HEADERS = ["wmcd_device.cuh", "wmcd_internal.h", "wmcd_host.h"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]

MAX_LAYERS = 16
BOND_NONE, BOND_HARMONIC, BOND_FENE = 0, 1, 2
PLANEWAVE_OFF, PLANEWAVE_PERIODIC, PLANEWAVE_PERIODIC_FULL, PLANEWAVE_INFINITE = 0, 1, 2, 3
FP64, MIXED = 0, 1
ACCEPT_METROPOLIS, ACCEPT_GLAUBER = 0, 1
CENTRE_BEAD, CENTRE_UNIFORM = 0, 1
STATUS = {0: "WMCD_OK", -1: "WMCD_EINVAL", -2: "WMCD_ENOMEM", -3: "WMCD_ECUDA", -4: "WMCD_ETIMEOUT", -5: "WMCD_ESTATE",
          -6: "WMCD_EFULL"}
KERNEL_CLASSES = ["concurrent_wavelet", "serial_wavelet", "plane_wave", "cell_list", "schedule", "whole_gpu_serial"]


def _nvcc() -> str:
    for c in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.sep not in c or os.path.exists(c):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree for sm_103a (two translation units in parallel)."""
    inc = os.path.join(os.path.dirname(_HERE), "include", "wmcd.h")
    deps = [os.path.join(_CSRC, f) for f in _SOURCES + _HEADERS] + [inc]
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps):
        return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = [os.path.join(_BUILD, f.replace(".cu", f".{os.getpid()}.o")) for f in _SOURCES]

    def comp(i):
        cmd = [nvcc] + ARCH_FLAGS + NVCC_FLAGS + ["-c", os.path.join(_CSRC, _SOURCES[i]), "-o", objs[i]]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {_SOURCES[i]}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)

    with ThreadPoolExecutor(len(_SOURCES)) as ex:
        list(ex.map(comp, range(len(_SOURCES))))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc] + ARCH_FLAGS + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH


class Params(ctypes.Structure):
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
        ("grid_layer", ctypes.c_int32 * MAX_LAYERS), ("big_support", ctypes.c_int32),
        ("acceptance", ctypes.c_int32), ("centring", ctypes.c_int32), ("level2", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("attempts", ctypes.c_int64 * MAX_LAYERS), ("accepts", ctypes.c_int64 * MAX_LAYERS),
        ("deferred", ctypes.c_int64 * MAX_LAYERS),
        ("pw_attempts", ctypes.c_int64), ("pw_accepts", ctypes.c_int64),
        ("bead_updates", ctypes.c_int64), ("accepted_total", ctypes.c_int64),
        ("rechecks", ctypes.c_int64), ("partner_evals", ctypes.c_int64),
        ("sim_time", ctypes.c_double), ("sweeps", ctypes.c_int64), ("n_layers", ctypes.c_int64),
        ("dt_move", ctypes.c_double), ("p_fourier", ctypes.c_double), ("error_flags", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int64), ("conc_bead_updates", ctypes.c_int64),
        ("conc_moved_beads", ctypes.c_int64), ("conc_partner_evals", ctypes.c_int64),
        ("moved_beads", ctypes.c_int64),
    ]


class Audit(ctypes.Structure):
    _fields_ = [("decisions", ctypes.c_int64), ("outside", ctypes.c_int64), ("violations", ctypes.c_int64),
                ("flips", ctypes.c_int64), ("max_ratio", ctypes.c_double), ("records", ctypes.c_int64)]


_lib = None
_SIGS = {
    "wmcd_create": ["p", "p", "p", "i64", "p", "p"],
    "wmcd_sweep": ["p", "i64", "p"],
    "wmcd_planewave": ["p", "i64", "p"],
    "wmcd_positions": ["p", "p", "i", "p"],
    "wmcd_set_positions": ["p", "p", "p"],
    "wmcd_stats": ["p", "p", "p"],
    "wmcd_trace": ["p", "i", "p", "p", "i64", "p", "p"],
    "wmcd_trace_du": ["p", "i", "p", "i64", "p", "p"],
    "wmcd_trace_pw_k": ["p", "p", "i64", "p", "p"],
    "wmcd_state_size": ["p", "p"],
    "wmcd_get_state": ["p", "p", "i64", "p"],
    "wmcd_set_state": ["p", "p", "i64", "p"],
    "wmcd_profile": ["p", "i"],
    "wmcd_kernel_times": ["p", "p", "p", "i", "p"],
    "wmcd_device_bytes": ["p", "p"],
    "wmcd_audit": ["p", "i64", "p"],
    "wmcd_audit_read": ["p", "p", "p", "i64", "p"],
    "wmcd_destroy": ["p"],
    "wmcd_planewave_noalloc": ["p", "p", "p", "i64", "i64", "p", "i64", "p"],
    "wmcd_set_block": ["p", "i", "i"],
    "wmcd_batch_create": ["i", "i64", "p"],
    "wmcd_batch_need": ["p", "p"],
    "wmcd_batch_admit": ["p", "p", "p", "p", "i64", "p"],
    "wmcd_batch_step": ["p", "i64", "p"],
    "wmcd_batch_handle": ["p", "i", "p"],
    "wmcd_batch_retire": ["p", "i", "p"],
    "wmcd_batch_set_block": ["p", "i", "i"],
    "wmcd_batch_info": ["p", "p", "p", "p", "p"],
    "wmcd_batch_destroy": ["p"],
    "wmcd_batch_profile": ["p", "i"],
    "wmcd_batch_kernel_times": ["p", "p", "p", "i", "p"],
}
EXPORTED = sorted(list(_SIGS) + ["wmcd_strerror"])


def load(path: str | None = None):
    """Load the compiled library (build it first with ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"WMCD CUDA library not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    tmap = {"p": ctypes.c_void_p, "i64": ctypes.c_int64, "i": ctypes.c_int}
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = [tmap[a] for a in args]
        f.restype = ctypes.c_int
    lib.wmcd_strerror.argtypes = [ctypes.c_int]
    lib.wmcd_strerror.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


class WMCDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().wmcd_strerror(code).decode() if _lib is not None else STATUS.get(code, str(code))
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


def _check(rc: int, where: str):
    if rc != 0:
        raise WMCDError(rc, where)


def make_params(fields: dict) -> Params:
    p = Params()
    fields = dict(fields)
    layers = fields.pop("grid_layer", [])
    for k, v in fields.items():
        setattr(p, k, v)
    for i, g in enumerate(layers):
        p.grid_layer[i] = int(g)
    return p


def planewave_noalloc(params: dict, pos, chain_len, call_index: int, carry, n_moves: int, stream=None):
    """Plane-wave moves on caller-owned device positions (a torch CUDA tensor of N x 3 doubles,
    updated in place) with no device allocation; ``carry`` is an int32 array of 4 (in/out)."""
    lib = load()
    pr = make_params(params)
    cl = np.ascontiguousarray(chain_len, dtype=np.int32)
    pp, _k = _buf_ptr(pos)
    _check(lib.wmcd_planewave_noalloc(ctypes.byref(pr), pp, cl.ctypes.data, len(cl), int(call_index),
                                      carry.ctypes.data, int(n_moves), _stream_ptr(stream)), "wmcd_planewave_noalloc")


def default_params(n_beads: int, box_L: float, *, lambda_min: float = 2.0, lambda_max: float | None = None,
                   A0: float = 0.5, kT: float = 1.0, bond_type: int = BOND_HARMONIC, bond_k: float = 100.0,
                   bond_r0: float = 2.0, fene_R0: float = 3.0, wca_sigma: float = 2.0, wca_eps: float = 1.0,
                   ext_kappa: float = 0.0, planewave_mode: int = PLANEWAVE_OFF, lcut: int = 8,
                   precision: int = FP64, seed: int = 1, sim_id: int = 0, colour_K: int = 2,
                   acceptance: int = ACCEPT_METROPOLIS, centring: int = CENTRE_BEAD, **sched) -> dict:
    """Parameter fields of the benchmark systems: beads of radius a = 1, harmonic bonds
    k = 100 kT/a^2 with rest length 2a, WCA sigma = 2a, eps = 1 kT, lambda_min = 2a,
    lambda_max = L/2, A0 = 0.5, plus the default concurrent schedule for the box."""
    lmax = box_L / 2 if lambda_max is None else lambda_max
    d = dict(n_beads=int(n_beads), box_L=float(box_L), lambda_min=lambda_min, lambda_max=lmax, A0=A0, kT=kT,
             bond_type=bond_type, bond_k=bond_k, bond_r0=bond_r0, fene_R0=fene_R0, wca_sigma=wca_sigma,
             wca_eps=wca_eps, ext_kappa=ext_kappa, planewave_mode=planewave_mode, lcut=lcut, precision=precision,
             seed=seed, sim_id=sim_id, acceptance=acceptance, centring=centring)
    sched.setdefault("n_beads", int(n_beads))
    d.update(_schedule.choose(box_L, lambda_min, lmax, A0, wca_sigma, wca_eps, colour_K=colour_K, **sched))
    return d


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _buf_ptr(x):
    """(pointer, keep-alive) for a numpy array or a torch tensor (host or CUDA)."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data), x
    return ctypes.c_void_p(x.data_ptr()), x


class Simulation:
    """One WMCD simulation held on the GPU (a wmcd_handle)."""

    _owned = True

    def __init__(self, params: dict, pos, chain_len, stream=None):
        lib = load()
        self._lib = lib
        self.params = dict(params)
        self.n = int(params["n_beads"])
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        cl = np.ascontiguousarray(chain_len, dtype=np.int32)
        pr = make_params(params)
        h = ctypes.c_void_p()
        pp, _keep = _buf_ptr(pos)
        rc = lib.wmcd_create(ctypes.byref(pr), pp, cl.ctypes.data, len(cl), _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "wmcd_create")
        self.h = h

    @classmethod
    def _borrowed(cls, lib, h, params: dict):
        """A view of a simulation owned by a batch (not released by close)."""
        sim = cls.__new__(cls)
        sim._lib, sim.h, sim.params, sim.n, sim._owned = lib, h, dict(params), int(params["n_beads"]), False
        return sim

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                self._lib.wmcd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1, stream=None):
        _check(self._lib.wmcd_sweep(self.h, int(n), _stream_ptr(stream)), "wmcd_sweep")

    def planewave(self, n: int = 1, stream=None):
        _check(self._lib.wmcd_planewave(self.h, int(n), _stream_ptr(stream)), "wmcd_planewave")

    def positions(self, unwrapped: bool = False, out=None, stream=None):
        if out is None:
            out = np.zeros((self.n, 3), dtype=np.float64)
        p, _k = _buf_ptr(out)
        _check(self._lib.wmcd_positions(self.h, p, int(unwrapped), _stream_ptr(stream)), "wmcd_positions")
        return out

    def set_positions(self, pos, stream=None):
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        p, _k = _buf_ptr(pos)
        _check(self._lib.wmcd_set_positions(self.h, p, _stream_ptr(stream)), "wmcd_set_positions")

    def stats(self, stream=None, check: bool = True) -> Stats:
        st = Stats()
        rc = self._lib.wmcd_stats(self.h, ctypes.byref(st), _stream_ptr(stream))
        if check:
            _check(rc, "wmcd_stats")
        return st

    def trace(self, layer: int, stream=None):
        cap = 4 * self.n + 4096
        out = np.zeros(cap, dtype=np.uint8)
        nn = np.zeros(cap, dtype=np.int32)
        cnt = ctypes.c_int64()
        _check(self._lib.wmcd_trace(self.h, int(layer), out.ctypes.data, nn.ctypes.data, cap, ctypes.byref(cnt),
                                    _stream_ptr(stream)), "wmcd_trace")
        m = min(cnt.value, cap)
        return out[:m].copy(), nn[:m].copy()

    def trace_du(self, layer: int, stream=None):
        cap = 4 * self.n + 4096
        out = np.zeros(cap)
        cnt = ctypes.c_int64()
        _check(self._lib.wmcd_trace_du(self.h, int(layer), out.ctypes.data, cap, ctypes.byref(cnt),
                                       _stream_ptr(stream)), "wmcd_trace_du")
        return out[:min(cnt.value, cap)].copy()

    def trace_pw_k(self, stream=None):
        """Wave vectors (units of 2 pi / L) of the last sweep's or call's plane waves, N x 3."""
        cap = 4 * self.n + 4096
        out = np.zeros((cap, 3))
        cnt = ctypes.c_int64()
        _check(self._lib.wmcd_trace_pw_k(self.h, out.ctypes.data, cap, ctypes.byref(cnt), _stream_ptr(stream)),
               "wmcd_trace_pw_k")
        return out[:min(cnt.value, cap)].copy()

    def get_state(self, stream=None) -> bytes:
        sz = ctypes.c_int64()
        _check(self._lib.wmcd_state_size(self.h, ctypes.byref(sz)), "wmcd_state_size")
        buf = ctypes.create_string_buffer(sz.value)
        _check(self._lib.wmcd_get_state(self.h, buf, sz.value, _stream_ptr(stream)), "wmcd_get_state")
        return buf.raw

    def set_state(self, state: bytes, stream=None):
        buf = ctypes.create_string_buffer(state, len(state))
        _check(self._lib.wmcd_set_state(self.h, buf, len(state), _stream_ptr(stream)), "wmcd_set_state")

    def profile(self, enable: bool = True):
        _check(self._lib.wmcd_profile(self.h, int(enable)), "wmcd_profile")

    def kernel_times(self, stream=None) -> dict:
        n = len(KERNEL_CLASSES)
        la = (ctypes.c_int64 * n)()
        ms = (ctypes.c_double * n)()
        _check(self._lib.wmcd_kernel_times(self.h, la, ms, n, _stream_ptr(stream)), "wmcd_kernel_times")
        return {KERNEL_CLASSES[i]: (int(la[i]), float(ms[i])) for i in range(n)}

    def audit(self, capacity: int = 0, stream=None):
        """Audit every mixed-precision decision (binary32 against binary64, see wmcd.h);
        capacity < 0 turns it off."""
        _check(self._lib.wmcd_audit(self.h, int(capacity), _stream_ptr(stream)), "wmcd_audit")

    def audit_read(self, cap: int = 0, stream=None):
        """(counters as a dict, records as an array of rows dU32, dU64, band, threshold)."""
        a = Audit()
        rec = np.zeros((max(int(cap), 0), 4))
        _check(self._lib.wmcd_audit_read(self.h, ctypes.byref(a), rec.ctypes.data, int(cap), _stream_ptr(stream)),
               "wmcd_audit_read")
        d = {k: getattr(a, k) for k, _ in Audit._fields_}
        return d, rec[:min(int(cap), a.records)]

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(self._lib.wmcd_device_bytes(self.h, ctypes.byref(b)), "wmcd_device_bytes")
        return b.value

    def set_block(self, stage_warps: int = 2, serial_threads: int = 512):
        """Launch shapes (results do not depend on them)."""
        _check(self._lib.wmcd_set_block(self.h, int(stage_warps), int(serial_threads)), "wmcd_set_block")


def batch_need(params: dict) -> int:
    """Pool bytes a simulation with these parameters takes in a batch."""
    lib = load()
    pr = make_params(params)
    b = ctypes.c_int64()
    _check(lib.wmcd_batch_need(ctypes.byref(pr), ctypes.byref(b)), "wmcd_batch_need")
    return b.value


class Batch:
    """Many simulations resident on the GPU, advanced together (a wmcd_batch): one launch per
    phase of a sweep over all of them, the sweep replayed as a CUDA graph."""

    def __init__(self, capacity: int, pool_bytes: int):
        lib = load()
        self._lib = lib
        b = ctypes.c_void_p()
        _check(lib.wmcd_batch_create(int(capacity), int(pool_bytes), ctypes.byref(b)), "wmcd_batch_create")
        self.b = b
        self.capacity = int(capacity)
        self._members = {}

    def admit(self, params: dict, pos, chain_len):
        """Admit a simulation; returns its slot, or None when the batch is full (no slot or no
        pool room). Other errors raise."""
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        cl = np.ascontiguousarray(chain_len, dtype=np.int32)
        pr = make_params(params)
        pp, _keep = _buf_ptr(pos)
        slot = ctypes.c_int()
        rc = self._lib.wmcd_batch_admit(self.b, ctypes.byref(pr), pp, cl.ctypes.data, len(cl), ctypes.byref(slot))
        if rc == -6:
            return None
        _check(rc, "wmcd_batch_admit")
        h = ctypes.c_void_p()
        _check(self._lib.wmcd_batch_handle(self.b, slot.value, ctypes.byref(h)), "wmcd_batch_handle")
        self._members[slot.value] = Simulation._borrowed(self._lib, h, params)
        return slot.value

    def sim(self, slot: int) -> Simulation:
        return self._members[slot]

    def step(self, n: int = 1, stream=None):
        _check(self._lib.wmcd_batch_step(self.b, int(n), _stream_ptr(stream)), "wmcd_batch_step")

    def retire(self, slot: int, stream=None):
        sim = self._members.pop(slot)
        sim.h = None
        _check(self._lib.wmcd_batch_retire(self.b, int(slot), _stream_ptr(stream)), "wmcd_batch_retire")

    def profile(self, enable: bool = True):
        _check(self._lib.wmcd_batch_profile(self.b, int(enable)), "wmcd_batch_profile")

    def kernel_times(self, stream=None) -> dict:
        n = len(KERNEL_CLASSES)
        la = (ctypes.c_int64 * n)()
        ms = (ctypes.c_double * n)()
        _check(self._lib.wmcd_batch_kernel_times(self.b, la, ms, n, _stream_ptr(stream)), "wmcd_batch_kernel_times")
        return {KERNEL_CLASSES[i]: (int(la[i]), float(ms[i])) for i in range(n)}

    def set_block(self, stage_warps: int = 2, serial_threads: int = 512):
        """Launch shapes for the whole batch (results do not depend on them)."""
        _check(self._lib.wmcd_batch_set_block(self.b, int(stage_warps), int(serial_threads)), "wmcd_batch_set_block")

    def info(self) -> dict:
        r, f, lg, lp = (ctypes.c_int64() for _ in range(4))
        _check(self._lib.wmcd_batch_info(self.b, ctypes.byref(r), ctypes.byref(f), ctypes.byref(lg), ctypes.byref(lp)),
               "wmcd_batch_info")
        return {"resident": r.value, "pool_free": f.value, "largest_free": lg.value, "launches_per_sweep": lp.value}

    @property
    def slots(self):
        return sorted(self._members)

    def close(self):
        if getattr(self, "b", None):
            for sim in self._members.values():
                sim.h = None
            self._members.clear()
            self._lib.wmcd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
