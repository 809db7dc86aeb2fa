"""The C-ABI library builds, loads and exports every entry point its header
declares; host-side argument checks return the documented status codes.
No test here launches GPU work."""
import ctypes
import os
import re

import pytest

from paper_1806_05713_gb300 import build as lj_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lj_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    path = lj_build.build()
    return ctypes.CDLL(path), path


def test_header_declares_entry_points():
    names = _declared()
    for must in ("lj_build_pairlist", "lj_force", "lj_energy", "lj_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    cdll, path = lib
    for name in sorted(_declared()):
        assert hasattr(cdll, name), f"{name} declared in include/ but not exported by {path}"


def test_binding_covers_every_declared_symbol():
    from paper_1806_05713_gb300 import lj
    assert _declared() == set(lj.SIGNATURES)


def test_binding_has_a_same_named_function_for_every_entry_point():
    from paper_1806_05713_gb300 import lj
    for name in _declared():
        assert callable(getattr(lj, name, None)), f"lj.{name} missing"


def test_status_strings_and_version():
    from paper_1806_05713_gb300 import lj
    L = lj.load()
    assert L.lj_version() >= 10000
    for code in range(7):
        assert L.lj_status_string(code).decode().startswith("LJ_")
    assert b"unknown" in L.lj_status_string(99)


def test_host_argument_checks_without_gpu():
    from paper_1806_05713_gb300 import lj
    L = lj.load()
    box = lj._box3([10.0, 10.0, 10.0])
    nnz, mrow = ctypes.c_int64(), ctypes.c_int64()
    # n < 0
    assert L.lj_build_pairlist(None, -1, box, 3.3, 1, None, None, 0, None, 0, ctypes.byref(nnz),
                               ctypes.byref(mrow), None) == lj.LJ_ERR_ARG
    # box shorter than 2 r_s
    assert L.lj_build_pairlist(None, 0, lj._box3([6.0, 10, 10]), 3.3, 1, ctypes.c_void_p(16),
                               None, 0, None, 0, ctypes.byref(nnz), ctypes.byref(mrow),
                               None) == lj.LJ_ERR_BOX
    # non-finite search length
    assert L.lj_build_pairlist(None, 0, box, float("nan"), 1, ctypes.c_void_p(16), None, 0, None,
                               0, ctypes.byref(nnz), ctypes.byref(mrow), None) == lj.LJ_ERR_ARG
    # force: bad precision, bad cutoff, box too small, bad eps
    fake = ctypes.c_void_p(256)
    args = lambda **k: dict(dict(q=fake, p=fake, n=10, rp=fake, col=fake, nnz=10, half=1, dt=0.01,
                                 rc=3.0, box=box, eps=1.0, sig=1.0, prec=0, tpi=0), **k)

    def force(ws=None, wsb=0, **k):
        a = args(**k)
        return L.lj_force(a["q"], a["p"], a["n"], a["rp"], a["col"], a["nnz"], a["half"], a["dt"],
                          a["rc"], a["box"], a["eps"], a["sig"], a["prec"], a["tpi"], ws, wsb, None)
    assert force(prec=7) == lj.LJ_ERR_ARG
    assert force(rc=-1.0) == lj.LJ_ERR_ARG
    assert force(rc=6.0) == lj.LJ_ERR_BOX
    assert force(eps=0.0) == lj.LJ_ERR_ARG
    assert force(q=None) == lj.LJ_ERR_ARG
    assert force(tpi=3) == lj.LJ_ERR_ARG
    # retired schedule codes (group refill 64, lane queue 256, compaction
    # 4096, two entries per lane on the fixed-point rows) are refused
    for retired in (64 | 8, 256 | 8, 4096 | 8, lj.LJ_SCHED_FIXED | lj.LJ_SCHED_SWP2 | 8):
        assert force(prec=0, tpi=retired, ws=fake, wsb=1 << 40) == lj.LJ_ERR_ARG
    # the stream walk indexes entries in 32 bits with up to 128 of padding:
    # lists within 256 of 2^31 entries are refused before any launch
    stream32 = lj.LJ_SCHED_FIXED | lj.LJ_SCHED_STREAM | 32
    assert force(prec=0, tpi=stream32, nnz=(1 << 31) - 200, ws=fake, wsb=1 << 40) == \
        lj.LJ_ERR_CAPACITY
    # the space-filling row order excludes the length-sorted one and the
    # stream walk
    C = lj.LJ_SCHED_CELLS
    for bad in (C | lj.LJ_SCHED_SORTED | 8, C | lj.LJ_SCHED_FIXED | lj.LJ_SCHED_STREAM | 8):
        assert force(prec=0, tpi=bad, ws=fake, wsb=1 << 40) == lj.LJ_ERR_ARG
    # mixed precision, or the FP64 fixed-point schedule, without a workspace
    assert force(prec=1, tpi=8) == lj.LJ_ERR_CAPACITY
    assert force(prec=0, tpi=lj.LJ_SCHED_FIXED | 8) == lj.LJ_ERR_CAPACITY
    assert force(prec=0, tpi=8) == lj.LJ_ERR_CAPACITY
    # double-float form: 4, 8 or 16 lanes (optionally length-sorted), a
    # workspace with the fixed-point records, K = 24 eps sigma^6 dt / lambda^7
    # within its exponent range (checked before any launch)
    assert force(prec=2, tpi=2) == lj.LJ_ERR_ARG
    assert force(prec=2, tpi=lj.LJ_SCHED_SWP2 | 2) == lj.LJ_ERR_ARG
    assert force(prec=2, tpi=lj.LJ_SCHED_IMAGES | 8) == lj.LJ_ERR_ARG
    assert force(prec=2, tpi=8) == lj.LJ_ERR_CAPACITY
    assert force(prec=2, tpi=8, dt=1e-250, ws=fake, wsb=1 << 40) == lj.LJ_ERR_ARG
    # the fixed-point FP64 schedules need a box at most 1024 r_c wide
    wide = lj._box3([4000.0, 4000.0, 4000.0])
    assert force(tpi=lj.LJ_SCHED_FIXED | 8, box=wide, ws=fake, wsb=1 << 40) == lj.LJ_ERR_ARG
    assert force(tpi=lj.LJ_SCHED_FIXED | 2, ws=fake, wsb=1 << 40) == lj.LJ_ERR_ARG
    # empty work is a no-op that succeeds
    assert force(n=0, nnz=0) == lj.LJ_OK
    # lj_md_steps: its own arguments, then every force check, before any launch

    def md(steps=3, state=fake, rs=3.3, ws=fake, wsb=1 << 40, flags=0, qb=None, en=None, **k):
        a = args(**k)
        return L.lj_md_steps(a["q"], a["p"], a["n"], a["rp"], a["col"], a["nnz"], a["half"],
                             a["dt"], a["rc"], rs, a["box"], a["eps"], a["sig"], a["prec"],
                             a["tpi"], steps, flags, qb, en, state, ws, wsb, None)
    assert md(steps=-1) == lj.LJ_ERR_ARG
    assert md(state=None) == lj.LJ_ERR_ARG
    assert md(state=ctypes.c_void_p(260)) == lj.LJ_ERR_ARG
    assert md(rs=3.0) == lj.LJ_ERR_ARG
    assert md(rs=float("nan")) == lj.LJ_ERR_ARG
    assert md(prec=7) == lj.LJ_ERR_ARG
    assert md(tpi=3) == lj.LJ_ERR_ARG
    assert md(rc=6.0, rs=6.3) == lj.LJ_ERR_BOX
    assert md(ws=None, wsb=0) == lj.LJ_ERR_CAPACITY
    assert md(prec=2, dt=1e-250) == lj.LJ_ERR_ARG
    assert md(flags=2) == lj.LJ_ERR_ARG
    assert md(qb=ctypes.c_void_p(264)) == lj.LJ_ERR_ARG
    assert md(en=ctypes.c_void_p(260)) == lj.LJ_ERR_ARG
    assert md(en=fake, prec=2) == lj.LJ_ERR_ARG
    assert md(steps=0) == lj.LJ_OK
    # force + energy (+ virial): outputs required and 8-byte aligned, before any launch

    def fev(e=fake, w=fake, **k):
        a = args(**k)
        return L.lj_force_energy_virial(a["q"], a["p"], a["n"], a["rp"], a["col"], a["nnz"],
                                        a["half"], a["dt"], a["rc"], a["box"], a["eps"], a["sig"],
                                        1, e, w, fake, 1 << 40, None)
    assert fev(w=None) == lj.LJ_ERR_ARG
    assert fev(e=None) == lj.LJ_ERR_ARG
    assert fev(w=ctypes.c_void_p(260)) == lj.LJ_ERR_ARG
    assert fev(rc=6.0) == lj.LJ_ERR_BOX
    assert L.lj_force_energy(fake, fake, 10, fake, fake, 10, 1, 0.01, 3.0, box, 1.0, 1.0, 1, None,
                             fake, 1 << 40, None) == lj.LJ_ERR_ARG
    assert md(steps=0, flags=lj.LJ_MD_LAST_HALF_KICK, qb=fake, en=fake) == lj.LJ_OK


def test_workspace_sizes_are_sane():
    from paper_1806_05713_gb300 import lj
    L = lj.load()
    b = lj._box3([49.2, 49.2, 49.2])
    w1 = L.lj_pairlist_workspace_bytes(119164, b, 3.3)
    # two-walk scratch (~100 B per atom) plus the one-walk row slabs: 1.5 times
    # the mean full row (150 at density 1, r_s = 3.3) + 32, rounded to 32 -> 288
    assert 119164 * (32 + 4 * 288) <= w1 < 119164 * (200 + 4 * 288)
    assert L.lj_force_workspace_bytes(1000, b, 0) >= 256 + 8 * 1000
    assert L.lj_force_workspace_bytes(1000, b, 1) >= 24000
    assert L.lj_force_workspace_bytes(1000, b, 2) >= 40000
    assert L.lj_energy_workspace_bytes(1000) >= 8


def test_product_path_has_no_cpu_fallback(monkeypatch):
    """Without the built library the binding raises instead of computing."""
    from paper_1806_05713_gb300 import lj
    monkeypatch.setattr(lj, "_lib", None)
    monkeypatch.setattr(lj, "_LIB_PATH", "/nonexistent/liblj_gb300.so")
    with pytest.raises(RuntimeError, match="not built"):
        lj.load()


def test_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1806_05713_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "lj_oracle" not in text, f


def test_measurement_entry_points_check_arguments_without_gpu():
    """lj_measure_peak and lj_eval_reciprocal refuse bad arguments before any
    CUDA call (so these run on a machine without a GPU)."""
    from paper_1806_05713_gb300 import lj
    L = lj.load()
    rate, ms = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    peak = lambda kind=lj.LJ_PEAK_DFMA, buf=None, nb=0, work=1, r=True, m=True: L.lj_measure_peak(
        kind, buf, nb, work, ctypes.byref(rate) if r else None, ctypes.byref(ms) if m else None, None)
    assert peak(kind=-1) == lj.LJ_ERR_ARG
    assert peak(kind=4) == lj.LJ_ERR_ARG
    assert peak(work=0) == lj.LJ_ERR_ARG
    assert peak(r=False) == lj.LJ_ERR_ARG
    assert peak(m=False) == lj.LJ_ERR_ARG
    # the L2 probe needs a 256-byte aligned buffer, a multiple of 4096 bytes
    assert peak(kind=lj.LJ_PEAK_L2_READ) == lj.LJ_ERR_ARG
    assert peak(kind=lj.LJ_PEAK_L2_READ, buf=ctypes.c_void_p(4096), nb=4000) == lj.LJ_ERR_ARG
    assert peak(kind=lj.LJ_PEAK_L2_READ, buf=ctypes.c_void_p(4096 + 64), nb=8192) == lj.LJ_ERR_ARG
    assert rate.value == 0.0 and ms.value == 0.0
    fake = ctypes.c_void_p(4096)
    assert L.lj_eval_reciprocal(-1, fake, 10, fake, None, None) == lj.LJ_ERR_ARG
    # kind 0 (a double-float seed with an FP64 Newton step) is retired
    assert L.lj_eval_reciprocal(0, fake, 10, fake, None, None) == lj.LJ_ERR_ARG
    assert L.lj_eval_reciprocal(7, fake, 10, fake, None, None) == lj.LJ_ERR_ARG
    assert L.lj_eval_reciprocal(lj.LJ_RCP_FP32, fake, -1, fake, None, None) == lj.LJ_ERR_ARG
    assert L.lj_eval_reciprocal(lj.LJ_RCP_FP32, None, 10, fake, None, None) == lj.LJ_ERR_ARG
    assert L.lj_eval_reciprocal(lj.LJ_RCP_FP32, ctypes.c_void_p(4100), 10, fake, None, None) == \
        lj.LJ_ERR_ARG
    assert L.lj_eval_reciprocal(lj.LJ_RCP_DF2, None, 0, None, None, None) == lj.LJ_OK
