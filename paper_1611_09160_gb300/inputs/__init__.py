"""Seeded synthetic inputs: initial bead configurations for the WMCD workloads.

This module places beads and nothing else; it contains none of the simulation
method's arithmetic. It is the one input source shared by the CUDA path and the
CPU oracle, so both always start from identical positions.

Workloads follow the shapes of the paper's validation systems (bead-spring chains in
a periodic cube, Sec. II) and the configurations used by the tests and the
benchmark: single chains, dilute and semi-dilute chain solutions, free spheres and
ensembles of uneven chain lengths. Chains are self-avoiding random walks with a
fixed step (the bond rest length); no bead is placed closer than ``min_dist`` to
another (minimum image), which keeps the initial WCA energy finite.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libwmcdgen.so")
_lib = None

SPHERE_VOLUME = 4.0 / 3.0 * math.pi  # volume of a bead of radius a = 1


def build(force: bool = False) -> str:
    """Compile the generator (plain C, no contraction so output is identical on every machine)."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.wmcd_gen_system.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]
        _lib.wmcd_gen_system.restype = ctypes.c_int
        _lib.wmcd_gen_loguniform_lengths.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.c_uint64, ctypes.c_void_p]
        _lib.wmcd_gen_loguniform_lengths.restype = ctypes.c_int
    return _lib


@dataclass
class System:
    """An initial configuration: positions (N, 3) float64 wrapped into [0, L), chain lengths
    (chains are consecutive bead ids; free spheres are chains of length 1) and the box side."""
    pos: np.ndarray
    chain_len: np.ndarray
    box_L: float

    @property
    def n_beads(self) -> int:
        return int(self.pos.shape[0])


def make_system(chain_lengths, n_spheres: int, box_L: float, seed: int,
                bond: float = 2.0, min_dist: float = 2.0) -> System:
    """Place chains (self-avoiding random walks of step ``bond``) then free spheres."""
    lib = _load()
    cl = np.ascontiguousarray(np.asarray(chain_lengths, dtype=np.int32).reshape(-1))
    n = int(cl.sum()) + int(n_spheres)
    out = np.zeros((n, 3), dtype=np.float64)
    rc = lib.wmcd_gen_system(len(cl), cl.ctypes.data if len(cl) else None, int(n_spheres), float(box_L),
                             float(bond), float(min_dist), int(seed) & (2**64 - 1), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"input generator failed (code {rc}): box too crowded for min_dist={min_dist}")
    chains = np.concatenate([cl, np.ones(int(n_spheres), dtype=np.int32)]) if n_spheres else cl
    return System(out, chains.astype(np.int32), float(box_L))


def box_for_volume_fraction(n_beads: int, phi: float, radius: float = 1.0) -> float:
    """Side of the periodic cube holding ``n_beads`` spheres of ``radius`` at volume fraction ``phi``."""
    return (n_beads * SPHERE_VOLUME * radius ** 3 / phi) ** (1.0 / 3.0)


def loguniform_lengths(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(n, dtype=np.int32)
    lib.wmcd_gen_loguniform_lengths(int(n), int(lo), int(hi), int(seed) & (2**64 - 1), out.ctypes.data)
    return out


# ---- the named workloads -------------------------------------------------------------

def single_chain(n: int = 32, box_L: float = 64.0, seed: int = 1) -> System:
    """One self-avoiding chain of ``n`` beads in a periodic cube (the small parity case)."""
    return make_system([n], 0, box_L, seed)


def dilute_chains(n_chains: int = 256, chain_len: int = 64, phi: float = 1e-3, seed: int = 1) -> System:
    """Chains at uniform random starting points at volume fraction ``phi``
    (256 x 64 = 16,384 beads at phi = 1e-3 gives L = 409.5)."""
    L = box_for_volume_fraction(n_chains * chain_len, phi)
    return make_system([chain_len] * n_chains, 0, L, seed)


def semidilute_chains(n_chains: int = 4096, chain_len: int = 256, phi: float = 0.05, seed: int = 1) -> System:
    """Homogeneous semi-dilute solution (4,096 x 256 = 1,048,576 beads at phi = 0.05, L = 444.6)."""
    L = box_for_volume_fraction(n_chains * chain_len, phi)
    return make_system([chain_len] * n_chains, 0, L, seed)


def free_spheres(n: int, phi: float, seed: int = 1) -> System:
    L = box_for_volume_fraction(n, phi)
    return make_system([], n, L, seed)


def suspension(n_spheres: int = 4_000_000, n_chains: int = 1000, chain_len: int = 1024, phi: float = 1e-3,
               seed: int = 1) -> System:
    """Large dilute suspension: free spheres plus chains at volume fraction ``phi``."""
    L = box_for_volume_fraction(n_spheres + n_chains * chain_len, phi)
    return make_system([chain_len] * n_chains, n_spheres, L, seed)


def ensemble(n_sims: int = 1024, lo: int = 16, hi: int = 2048, phi: float = 1e-3, seed: int = 1):
    """Independent single-chain systems with log-uniform chain lengths, box scaled to ``phi``."""
    lens = loguniform_lengths(n_sims, lo, hi, seed)
    out = []
    for s, n in enumerate(lens):
        L = box_for_volume_fraction(int(n), phi)
        out.append(make_system([int(n)], 0, L, seed * 1_000_003 + s))
    return out
