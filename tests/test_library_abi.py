"""CPU checks of the C-ABI library and the host logic (no compute calls, no GPU needed)."""
import math
import os
import re

import numpy as np
import pytest

from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import schedule as S
from paper_1611_09160_gb300 import wmcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "wmcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wmcd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    wmcd.build()
    return wmcd.load()


def test_library_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert declared == wmcd.EXPORTED
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_and_struct_layout_match_the_header(lib, tmp_path):
    import ctypes
    import subprocess
    assert lib.wmcd_strerror(0) == b"ok"
    assert lib.wmcd_strerror(-1).startswith(b"invalid")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "wmcd.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(wmcd_params), offsetof(wmcd_params, seed),'
        ' offsetof(wmcd_params, grid_layer), sizeof(wmcd_stats_t), offsetof(wmcd_stats_t, sim_time),'
        ' offsetof(wmcd_stats_t, error_flags)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(wmcd.Params), wmcd.Params.seed.offset, wmcd.Params.grid_layer.offset,
            ctypes.sizeof(wmcd.Stats), wmcd.Stats.sim_time.offset, wmcd.Stats.error_flags.offset]
    assert got == want


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    import ctypes
    p = wmcd.make_params(wmcd.default_params(10, 50.0))
    h = ctypes.c_void_p()
    pos = np.zeros((10, 3))
    cl = np.array([10], np.int32)
    bad = [dict(lambda_max=30.0), dict(lambda_min=0.0), dict(A0=-1.0), dict(colour_K=5), dict(n_cap=257),
           dict(grid_f=100),       # L/grid_f below the WCA cutoff
           dict(acceptance=2), dict(centring=-1), dict(level2=0x10000), dict(level2=-1), dict(planewave_mode=4)]
    for b in bad:
        q = wmcd.make_params(dict(wmcd.default_params(10, 50.0), **b))
        rc = lib.wmcd_create(ctypes.byref(q), pos.ctypes.data, cl.ctypes.data, 1, None, ctypes.byref(h))
        assert rc == -1, b
    # chain lengths that do not add up to N
    rc = lib.wmcd_create(ctypes.byref(p), pos.ctypes.data, np.array([4, 4], np.int32).ctypes.data, 2, None,
                         ctypes.byref(h))
    assert rc == -1


def test_schedule_choice():
    for L in [64.0, 409.5, 444.6, 2761.0]:
        for K in (2, 3, 4):
            sch = S.choose(L, 2.0, L / 2, 0.5, 2.0, 1.0, colour_K=K)
            assert sch["grid_f"] >= 1 and L / sch["grid_f"] >= 2 ** (1 / 6) * 2.0
            lo, hi = S.layer_bounds(2.0, L / 2)
            for l, G in enumerate(sch["grid_layer"][:len(hi)]):
                if G:
                    assert G % K == 0 and G >= 2 * K
                    # the region margin covers the influence of a move plus the slack
                    assert (K - 1) * (L / G) / 2 >= 2 * hi[l] + 0.125 * hi[l] + 2 ** (1 / 6) * 2.0
            assert all(g == 0 for g in sch["grid_layer"][len(hi):])
    lo, hi = S.layer_bounds(2.0, 32.0)
    assert lo == [2.0, 4.0, 8.0, 16.0] and hi == [4.0, 8.0, 16.0, 32.0]


def test_input_generator_geometry():
    s = I.dilute_chains(n_chains=8, chain_len=40, phi=1e-3, seed=4)
    L = s.box_L
    assert L == pytest.approx((320 * 4 / 3 * math.pi / 1e-3) ** (1 / 3))
    assert np.all((s.pos >= 0) & (s.pos < L))
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(len(s.pos)) * 1e9
    assert r.min() >= 2.0 - 1e-12
    starts = np.concatenate([[0], np.cumsum(s.chain_len)[:-1]])
    for a, n in zip(starts, s.chain_len):
        bonds = r[np.arange(a, a + n - 1), np.arange(a + 1, a + n)]
        assert np.allclose(bonds, 2.0, atol=1e-12)
    # same seed, same system
    s2 = I.dilute_chains(n_chains=8, chain_len=40, phi=1e-3, seed=4)
    assert np.array_equal(s.pos, s2.pos)


def test_noalloc_entry_refuses_bad_parameters_and_carry_before_any_cuda_call(lib):
    """The allocation-free plane-wave entry point checks its parameters as wmcd_create does
    (plus its own limits) and refuses a carried wave vector that is not in the mode table, all
    before it makes any CUDA call (so these run without a GPU)."""
    import ctypes
    base = wmcd.default_params(10, 50.0, planewave_mode=wmcd.PLANEWAVE_PERIODIC, lcut=6)
    pos = np.zeros((10, 3))
    cl = np.array([10], np.int32)

    def call(p, carry):
        q = wmcd.make_params(p)
        c = np.ascontiguousarray(carry, dtype=np.int32)
        return lib.wmcd_planewave_noalloc(ctypes.byref(q), pos.ctypes.data, cl.ctypes.data, 1, 0, c.ctypes.data, 1,
                                          None)
    ok_carry = [0, 0, 0, 0]
    for b in [dict(bond_type=wmcd.BOND_FENE, fene_R0=0.0), dict(lambda_min=0.0), dict(colour_K=7),
              dict(lcut=9), dict(planewave_mode=wmcd.PLANEWAVE_OFF), dict(n_beads=20000)]:
        assert call(dict(base, **b), ok_carry) == -1, b
    for carry in ([2, 0, 0, 0], [-1, 1, 0, 0], [1, 0, 0, 0], [1, 7, 0, 0], [1, 4, 4, 3]):
        assert call(base, carry) == -1, carry
