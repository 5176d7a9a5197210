"""Host-side checks that need no GPU: the C-ABI library builds, loads, exports
every symbol the headers declare, and rejects invalid arguments before
touching the device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_symbols():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(nacc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2305_04966_gb300 import build, _abi
    build.build()
    return _abi.load()


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for n in ("nacc_march_grid", "nacc_update_grid", "nacc_sample_pdf", "nacc_render_fwd",
              "nacc_render_bwd", "nacc_grid_points", "nacc_last_error"):
        assert n in names
    assert len(names) >= 13
    assert len(HEADERS) >= 3  # the method, the harness, the learned proposal
    assert "nacc_mlp_forward" in names and "nacc_render_fwd_ckpt" in names


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """Each entry point's comment names the passage of the paper it follows
    (equation, section, table, algorithm, appendix), or says that it is
    library plumbing, harness, size arithmetic, or has no counterpart."""
    missing = []
    for h in HEADERS:
        src = open(h).read()
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(nacc_\w+)\s*\(", src, flags=re.M):
            before = src[:m.start()]
            j = before.rfind("*/")
            com = before[before.rfind("/*", 0, j):j] if j >= 0 else ""
            if not re.search(r"Eq\.|Sec\.|Table|Algorithm|Appendix|no counterpart|plumbing|harness|size arithmetic",
                             com):
                missing.append(f"{os.path.basename(h)}:{m.group(1)}")
    assert not missing, missing


def test_library_exports_every_declared_symbol(lib):
    from paper_2305_04966_gb300 import _abi
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"{name} has no ctypes signature"


def test_struct_layouts_match_header(lib):
    from paper_2305_04966_gb300 import _abi
    assert ctypes.sizeof(_abi.Grid) == 6 * 4 + 2 * 4 + 8
    assert ctypes.sizeof(_abi.MarchParams) == 24
    assert ctypes.sizeof(_abi.BlobField) == 8 + 4 * 8
    assert ctypes.sizeof(_abi.Packed) == 6 * 8


def test_scratch_sizes(lib):
    assert lib.nacc_march_scratch_bytes(0) >= 256
    assert lib.nacc_march_scratch_bytes(640000) >= 2 * 4 * 640000
    assert lib.nacc_march_scratch_bytes(640000) % 256 == 0
    assert lib.nacc_update_grid_scratch_bytes(4 * 128 ** 3) >= 16
    assert lib.nacc_version() >= 100


def test_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_2305_04966_gb300 import _abi
    g = _abi.Grid()
    g.aabb_min[:] = [-1.0, -1.0, -1.0]
    g.aabb_max[:] = [1.0, 1.0, 1.0]
    g.res, g.n_levels, g.bits = 16, 1, None
    p = _abi.MarchParams(0.01, 1024, 0.0, 1e10, 1e-4)
    out = _abi.Packed()
    # NULL grid
    rc = lib.nacc_march_grid(None, None, None, 10, ctypes.byref(p), None, ctypes.byref(out), None, 0, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG
    assert b"grid" in lib.nacc_last_error()
    # NULL bits
    rc = lib.nacc_march_grid(ctypes.byref(g), None, None, 10, ctypes.byref(p), None, ctypes.byref(out),
                             None, 0, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG and b"bits" in lib.nacc_last_error()
    # bad levels / res
    g.bits = 1
    g.n_levels = 9
    assert lib.nacc_march_grid(ctypes.byref(g), None, None, 10, ctypes.byref(p), None,
                               ctypes.byref(out), None, 0, None) == _abi.NACC_ERR_INVALID_ARG
    g.n_levels, g.res = 1, 5  # 125 cells, not a multiple of 32
    assert lib.nacc_march_grid(ctypes.byref(g), None, None, 10, ctypes.byref(p), None,
                               ctypes.byref(out), None, 0, None) == _abi.NACC_ERR_INVALID_ARG
    g.res = 16
    bad = _abi.MarchParams(-1.0, 1024, 0.0, 1e10, 1e-4)
    assert lib.nacc_march_grid(ctypes.byref(g), None, None, 10, ctypes.byref(bad), None,
                               ctypes.byref(out), None, 0, None) == _abi.NACC_ERR_INVALID_ARG
    assert b"step" in lib.nacc_last_error()
    # sample arrays not 16-byte aligned (the fill writes 128-bit stores): rejected before any launch
    unaligned = _abi.Packed(256, 260, 512, 768, 10, 1024)
    assert lib.nacc_march_grid(ctypes.byref(g), None, None, 10, ctypes.byref(p), None,
                               ctypes.byref(unaligned), None, 0, None) == _abi.NACC_ERR_INVALID_ARG
    assert b"16-byte" in lib.nacc_last_error()
    up = _abi.MarchParams(0.01, 1024, 0.2, 1000.0, 1e-4)
    unaligned = _abi.Packed(256, 256, 520, 768, 10, 1024)
    assert lib.nacc_march_unbounded(ctypes.byref(g), None, None, 10, ctypes.byref(up), None,
                                    ctypes.byref(unaligned), None, 0, None) == _abi.NACC_ERR_INVALID_ARG
    assert b"16-byte" in lib.nacc_last_error()
    # render: NULL offsets / bg
    bg = (ctypes.c_float * 3)(1, 1, 1)
    assert lib.nacc_render_fwd(4, None, None, None, None, None, bg, 0.0, None, None, None, None, None,
                               None) == _abi.NACC_ERR_INVALID_ARG
    assert lib.nacc_render_bwd(4, 1, 1, 1, 1, 1, None, 0.0, None, None, None, 1, 1, None) == _abi.NACC_ERR_INVALID_ARG
    # sample_pdf bin limits
    assert lib.nacc_sample_pdf(4, 0, 1, 1, 8, 0, 0, 1, None) == _abi.NACC_ERR_INVALID_ARG
    assert lib.nacc_sample_pdf(4, 8, 1, 1, 5000, 0, 0, 1, None) == _abi.NACC_ERR_INVALID_ARG
    # update_grid decay range and scratch
    assert lib.nacc_update_grid(ctypes.byref(g), 1, 1, 1.5, 0.01, 0.0, 1, 1, 1 << 20, None) == _abi.NACC_ERR_INVALID_ARG
    assert lib.nacc_update_grid(ctypes.byref(g), 1, 1, 0.5, 0.01, 0.0, 1, 1, 8, None) == _abi.NACC_ERR_INVALID_ARG
    assert b"scratch" in lib.nacc_last_error()


def test_error_messages_are_thread_local(lib):
    import threading
    from paper_2305_04966_gb300 import _abi
    lib.nacc_sample_pdf(4, 0, 1, 1, 8, 0, 0, 1, None)
    msgs = []

    def other():
        msgs.append(lib.nacc_last_error())

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert msgs == [b""]
    assert b"n_bins" in lib.nacc_last_error()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2305_04966_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "lib_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _abi.load()


def test_render_rejects_misaligned_sample_arrays(lib):
    from paper_2305_04966_gb300 import _abi
    bg = (ctypes.c_float * 3)(1, 1, 1)
    ok, bad = 1 << 20, (1 << 20) + 4
    rc = lib.nacc_render_fwd(4, ok, bad, ok, ok, ok, bg, 0.0, ok, ok, ok, ok, None, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG and b"16-byte" in lib.nacc_last_error()
    rc = lib.nacc_render_bwd(4, ok, ok, ok, ok, bad, bg, 0.0, None, None, None, ok, ok, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG
    assert lib.nacc_selftest_wait_timeout(0, None) == _abi.NACC_ERR_INVALID_ARG


def test_render_ckpt_arguments(lib):
    """The checkpointed render pair: 64 bytes of record per ray; a NULL or
    misaligned record buffer is rejected on the host before any launch."""
    from paper_2305_04966_gb300 import _abi
    assert lib.nacc_render_ckpt_bytes(0) == 0 and lib.nacc_render_ckpt_bytes(-3) == 0
    assert lib.nacc_render_ckpt_bytes(640000) == 640000 * 64
    bg = (ctypes.c_float * 3)(1, 1, 1)
    ok, bad = 1 << 20, (1 << 20) + 4
    rc = lib.nacc_render_fwd_ckpt(4, ok, ok, ok, ok, ok, bg, 0.0, ok, ok, ok, ok, None, None, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG and b"ckpt_out" in lib.nacc_last_error()
    rc = lib.nacc_render_fwd_ckpt(4, ok, ok, ok, ok, ok, bg, 0.0, ok, ok, ok, ok, None, bad, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG and b"16-byte" in lib.nacc_last_error()
    rc = lib.nacc_render_bwd_ckpt(4, ok, ok, ok, ok, ok, bg, 0.0, None, None, None, None, ok, ok, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG and b"ckpt" in lib.nacc_last_error()
    rc = lib.nacc_render_bwd_ckpt(4, ok, ok, ok, ok, ok, bg, 0.0, None, None, None, bad, ok, ok, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG and b"16-byte" in lib.nacc_last_error()
    rc = lib.nacc_render_bwd_ckpt(4, ok, bad, ok, ok, ok, bg, 0.0, None, None, None, ok, ok, ok, None)
    assert rc == _abi.NACC_ERR_INVALID_ARG  # the plain pair's checks still apply


def test_march_count_event_hook_arguments(lib):
    from paper_2305_04966_gb300 import _abi
    assert lib.nacc_set_march_count_events(1 << 20, None) == _abi.NACC_ERR_INVALID_ARG
    assert lib.nacc_set_march_count_events(None, None) == _abi.NACC_OK
