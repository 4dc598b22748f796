"""C-ABI library checks that need no GPU: it loads, exports every entry point
the header declares, and its host-side helpers (the tile cost model of
Section 2, Table 1, and the tile schedules) are right."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "corr.h")


@pytest.fixture(scope="module")
def L():
    from paper_1702_00844_gb300 import lib
    return lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(corr_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert {"corr_create", "corr_correlate", "corr_correlate_batched", "corr_gain_backward",
            "corr_destroy"} <= set(names)
    for n in names:
        assert hasattr(L, n), f"{n} not exported"


def test_status_strings(L):
    for s in range(6):
        assert L.corr_status_string(s)


def test_table1_cost_model(L):
    golden = os.path.join(ROOT, "tests", "golden", "table1_tile_sizes.txt")
    rows = [ln.split() for ln in open(golden) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8
    for w, h, flops, nbytes, ai, regs in rows:
        f, b, r = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        L.corr_tile_cost(int(w), int(h), ctypes.byref(f), ctypes.byref(b), ctypes.byref(r))
        assert (f.value, b.value, r.value) == (int(flops), int(nbytes), int(regs))
        assert f"{f.value / b.value:.2f}" == ai


def test_tc_tile_schedule_covers_triangle(L):
    for S in (1, 63, 64, 65, 150, 256, 576):
        n = L.corr_tc_tiles(S)
        nb = (S + 63) // 64
        assert n == nb * (nb + 1) // 2
        seen = set()
        rb, cb = ctypes.c_int(), ctypes.c_int()
        for k in range(n):
            assert L.corr_tc_tile_decode(S, k, ctypes.byref(rb), ctypes.byref(cb)) == 0
            assert 0 <= rb.value <= cb.value < nb
            seen.add((rb.value, cb.value))
        assert len(seen) == n
        assert L.corr_tc_tile_decode(S, n, ctypes.byref(rb), ctypes.byref(cb)) == -1
        # every baseline s1 <= s2 lies in exactly one tile
        covered = 0
        for (r, c) in seen:
            for s2 in range(c * 64, min(S, c * 64 + 64)):
                covered += max(0, min(s2, r * 64 + 63) - r * 64 + 1)
        assert covered == S * (S + 1) // 2


def _schedule(L, variant, tail, S):
    n = L.corr_tc_schedule(variant, tail, S, 0, None)
    assert n > 0
    buf = (ctypes.c_int * (4 * n))()
    assert L.corr_tc_schedule(variant, tail, S, n - 1, buf) == -1          # too small
    assert L.corr_tc_schedule(variant, tail, S, n, buf) == n
    return [tuple(buf[4 * k:4 * k + 4]) for k in range(n)]


@pytest.mark.parametrize("variant,tail", [(0, 1), (1, 1), (2, 0), (2, 1)])
def test_tc_work_schedules_cover_each_baseline_once(L, variant, tail):
    """Every tile configuration's work tiles (the pair variant's two lists
    included, with either tail kind) hold each baseline s1 <= s2 of a channel
    exactly once; blocks that hold no stations appear only where a pair tile
    needs a partner row block."""
    for S in (1, 40, 64, 65, 128, 129, 150, 192, 200, 256, 320, 576, 600):
        nb = (S + 63) // 64
        tiles = _schedule(L, variant, tail, S)
        count = np.zeros((S, S), dtype=np.int64)
        for rb, cb0, ncb, lst in tiles:
            rows = [rb, rb + 1] if variant == 2 and lst == 0 else [rb]
            cols = list(range(cb0, cb0 + ncb))
            assert 1 <= ncb <= 2 and rb <= cb0 and cb0 + ncb <= nb
            if variant != 2:
                assert lst == 0
            for r in rows:
                for c in cols:
                    lo1, hi1 = r * 64, min(S, r * 64 + 64)
                    lo2, hi2 = c * 64, min(S, c * 64 + 64)
                    if lo1 < hi1 and lo2 < hi2:
                        count[lo1:hi1, lo2:hi2] += 1
        upper = np.triu(np.ones((S, S), dtype=bool))
        assert (count[upper] == 1).all(), (variant, tail, S)
        if variant == 2:
            second = [t for t in tiles if t[3] == 1]
            if nb % 2 == 0:
                assert second == []
            elif tail == 1:   # block 0's row as wide tiles
                assert second == [(0, 0, 1, 1)] + [(0, c, 2, 1) for c in range(1, nb, 2)]
            else:             # the last block column as narrow tiles
                assert second == [(r, nb - 1, 1, 1) for r in range(nb)]
    assert L.corr_tc_schedule(2, 3, 64, 0, None) == -1   # unknown tail kind


def test_fp32_subtile_schedule_covers_triangle(L):
    for S in (1, 3, 8, 9, 64, 150):
        n = L.corr_fp32_subtiles(S)
        nq = (S + 3) // 4
        assert n == nq * (nq + 1) // 2
        i, j = ctypes.c_int(), ctypes.c_int()
        pairs = set()
        for k in range(n):
            assert L.corr_fp32_subtile_decode(S, k, ctypes.byref(i), ctypes.byref(j)) == 0
            assert i.value <= j.value
            for a in range(4):
                for b in range(4):
                    s1, s2 = 4 * i.value + a, 4 * j.value + b
                    if s1 <= s2 < S:
                        assert (s1, s2) not in pairs
                        pairs.add((s1, s2))
        assert len(pairs) == S * (S + 1) // 2


def test_create_rejects_bad_descriptions_without_gpu(L):
    from paper_1702_00844_gb300.corr import Desc
    h = ctypes.c_void_p()
    bad = [Desc(0, 2, 1, 1, 1, 0, 0, 0),    # no stations
           Desc(4, 2, 0, 1, 1, 0, 0, 0),    # no channels
           Desc(4, 2, 1, -1, 1, 0, 0, 0),   # negative samples
           Desc(4, 2, 1, 1, 0, 0, 0, 0),    # no integrations
           Desc(4, 2, 1, 1, 1, 7, 0, 0),    # bad dtype
           Desc(4, 2, 1, 1, 1, 0, 9, 0)]    # bad path
    for d in bad:
        assert L.corr_create(ctypes.byref(d), ctypes.byref(h)) == 1
        assert not h.value
    unsupported = [Desc(4, 3, 1, 1, 1, 0, 0, 0),   # three polarisations
                   Desc(4, 1, 1, 1, 1, 0, 1, 4 | 1),  # one pol with gain calibration
                   Desc(4, 2, 1, 1, 1, 1, 1, 0),   # FP16 on the FP32 path
                   Desc(4, 1, 1, 1, 1, 0, 2, 0),   # FP32 on the tensor path with one pol
                   Desc(4, 2, 1, 70000, 1, 2, 0, 0)]  # int8 with T beyond the INT32 range
    for d in unsupported:
        assert L.corr_create(ctypes.byref(d), ctypes.byref(h)) == 2
    assert L.corr_create(None, ctypes.byref(h)) == 1
    assert L.corr_correlate(None, None, None, None) == 1
    assert L.corr_destroy(None) == 0


def test_roofline_examples_from_the_paper():
    from paper_1702_00844_gb300.metrics import perf_max
    golden = os.path.join(ROOT, "tests", "golden", "roofline_examples.txt")
    for ln in open(golden):
        if not ln.strip() or ln.startswith("#"):
            continue
        name, peak, ai, bw, printed = ln.split()
        assert round(perf_max(float(peak), float(ai), float(bw))) == int(printed), name


def test_global_arithmetic_intensity():
    """AI_global = nrStations + 1 (Section 3.6): 32 flops per baseline over 16
    bytes per station per sample."""
    from paper_1702_00844_gb300.metrics import ai_global, correlator_ops
    assert ai_global(64) == 65
    assert correlator_ops(8, 256, 16) == 32 * 36 * 256 * 16
    assert correlator_ops(256, 1024, 480) == pytest.approx(5.174e11, rel=1e-3)


def test_reorder_rejects_bad_arguments_without_gpu(L):
    """corr_reorder's argument checks run before any CUDA call."""
    a, b = ctypes.c_void_p(4096), ctypes.c_void_p(1 << 30)
    ok_args = (8, 2, 16, 1, 2, 0, 1)          # S, C, T, I, ci8, cst -> cts
    bad = [(-1, 2, 16, 1, 2, 0, 1), (8, 2, 16, 0, 2, 0, 1), (8, 2, 16, 1, 3, 0, 1),
           (8, 2, 16, 1, 2, 3, 1), (8, 2, 16, 1, 2, 0, -1)]
    for args in bad:
        assert L.corr_reorder(*args, a, b, None) == 1
    assert L.corr_reorder(*ok_args, None, b, None) == 1                  # NULL input
    assert L.corr_reorder(*ok_args, ctypes.c_void_p(4098), b, None) == 1  # misaligned (4-byte elements)
    assert L.corr_reorder(*ok_args, a, ctypes.c_void_p(4096 + 64), None) == 1  # overlapping
    assert L.corr_reorder(0, 2, 16, 1, 2, 0, 1, None, None, None) == 0   # nothing to move
