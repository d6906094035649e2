"""The C-ABI library builds, loads, exports every symbol include/cgs.h declares, and
rejects bad arguments before touching a GPU (CPU only: no compute call runs)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "cgs.h"


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(cgs_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def native():
    from paper_2410_00486_gb300 import build as B
    B.build()
    from paper_2410_00486_gb300 import _native as N
    N.lib()
    return N


def test_every_declared_symbol_is_exported(native):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(str(native.LIB_PATH))
    for name in names:
        assert hasattr(lib, name), name
    assert set(native.EXPORTS) == set(names)


def test_struct_sizes_match_header(native):
    assert ctypes.sizeof(native.cgs_camera) == 80
    assert ctypes.sizeof(native.cgs_config) == 4 * 13


def test_host_only_queries(native):
    cfg = native.make_config(1200, 680, 16, 64, 3)
    assert native.cgs_param_count(300_000, 3) == 59 * 300_000
    assert native.cgs_param_count(10, 0) == 140
    assert native.cgs_tiles_per_view(cfg) == 75 * 43
    assert native.cgs_bin_sort_workspace(1000, 300_000, 16, cfg) > 16 * 75 * 43 * 8
    bad = native.make_config(1200, 680, 12, 64, 3)
    assert native.cgs_tiles_per_view(bad) == -1
    assert native.status_string(-4).startswith("tile instance capacity")


def test_argument_validation_needs_no_gpu(native):
    L = native.lib()
    cfg = native.make_config(64, 48, 16, 64, 1)
    # null pointers / bad sizes / bad options are refused before any CUDA call
    assert L.cgs_preprocess(None, 10, None, 1, ctypes.byref(cfg), None, None, None, None) == native.CGS_ERR_ARG
    bad = native.make_config(64, 48, 16, 48, 1)
    assert L.cgs_preprocess(8, 10, 16, 1, ctypes.byref(bad), 16, None, None, None) == native.CGS_ERR_ARG
    bad = native.make_config(64, 48, 16, 64, 1, batch_depth_bwd=48)
    assert L.cgs_preprocess(8, 10, 16, 1, ctypes.byref(bad), 16, None, None, None) == native.CGS_ERR_ARG
    assert L.cgs_preprocess(8, 0, 16, 1, ctypes.byref(cfg), 16, None, None, None) == native.CGS_ERR_ARG
    assert L.cgs_preprocess(8, 10, 16, 1, ctypes.byref(cfg), 8, None, None, None) == native.CGS_ERR_ARG  # unaligned
    assert L.cgs_bin_sort(16, 10, 1, ctypes.byref(cfg), 256, 0, 100, 16, 16, None, 16, None, None) == \
        native.CGS_ERR_WORKSPACE
    assert L.cgs_adam(None, None, None, None, 10, 1, None, 0.9, 0.999, 1e-15, 1, None, 0.0, None, None) == \
        native.CGS_ERR_ARG
    lr = (ctypes.c_float * 6)()
    assert L.cgs_adam(16, 16, 16, 16, 10, 1, ctypes.cast(lr, ctypes.c_void_p), 0.9, 0.999, 1e-15, 0, None,
                      0.0, None, None) == native.CGS_ERR_ARG   # step < 1 without a device counter


def test_scheduler_matches_oracle(native):
    """The library's host scheduler draws exactly like the oracle's (Eqs. 5-8)."""
    import numpy as np
    from oracle import oracle as O
    rng = np.random.default_rng(0)
    lib_s, orc_s = native.Scheduler(4), O.Scheduler(4)
    for step in range(400):
        if step % 23 == 0:
            k = len(orc_s.K)
            r0 = 8 if k % 2 else 2
            assert lib_s.add(k, r0) == k
            orc_s.add(k, r0)
        u = int(rng.integers(0, 2 ** 32))
        a, b = lib_s.draw(u), orc_s.draw(u)
        assert a == b
        loss = float(rng.uniform(0, 1)) if rng.uniform() > 0.1 else 0.5
        lib_s.report(a, loss)
        orc_s.report(b, loss)
        ids, r, l = lib_s.state()
        assert r == orc_s.R


def test_scheduler_batched_calls_match_single_calls(native):
    """cgs_sched_draw_n / cgs_sched_report_n act exactly as the same single calls in a row."""
    import numpy as np
    rng = np.random.default_rng(5)
    a, b = native.Scheduler(4), native.Scheduler(4)
    for k in range(16):
        a.add(k, 8 if k % 2 else 2)
        b.add(k, 8 if k % 2 else 2)
    for _ in range(60):
        u = rng.integers(0, 2 ** 32, 16, dtype=np.uint64).astype(np.uint32)
        ia = a.draw_n(u)
        ib = np.array([b.draw(int(x)) for x in u], dtype=np.int32)
        assert np.array_equal(ia, ib)
        loss = rng.uniform(0, 1, 16)
        a.report_n(ia, loss)
        for i, l in zip(ib, loss):
            b.report(int(i), float(l))
        assert a.state() == b.state()
    assert a.draw_n(np.zeros(0, np.uint32)).size == 0
    with pytest.raises(native.CgsError):
        a.report_n([99], [0.5])



def test_render_entry_points_share_argument_checks(native):
    """cgs_render_fwd and cgs_render_fwd_noalloc refuse the same bad configurations and view
    counts before any CUDA call."""
    L = native.lib()
    P = 16                                    # a 16-byte aligned stand-in pointer (never dereferenced)
    bads = [native.make_config(64, 48, 16, 64, 1, batch_depth_bwd=48), native.make_config(64, 48, 16, 64, 5),
            native.make_config(64, 48, 16, 64, 1, near_z=0.0), native.make_config(64, 48, 12, 64, 1),
            native.make_config(64, 48, 16, 48, 1), native.make_config(0, 48, 16, 64, 1)]
    good = native.make_config(64, 48, 16, 64, 1)
    cases = [(c, 1) for c in bads] + [(good, 1025), (good, 0)]
    for cfg, V in cases:
        c = ctypes.byref(cfg)
        assert L.cgs_render_fwd(P, P, P, None, V, c, None, None, None, P, P, P, P, None, None, P, 1 << 20,
                                None, None) == native.CGS_ERR_ARG
        assert L.cgs_render_fwd_noalloc(P, P, P, None, V, c, None, None, None, P, P, P, P, None, None, None,
                                        None) == native.CGS_ERR_ARG
    # unaligned records, targets without loss outputs
    c = ctypes.byref(good)
    assert L.cgs_render_fwd_noalloc(8, P, P, None, 1, c, None, None, None, P, P, P, P, None, None, None,
                                    None) == native.CGS_ERR_ARG
    assert L.cgs_render_fwd_noalloc(P, P, P, None, 1, c, None, P, None, P, P, P, P, None, None, None,
                                    None) == native.CGS_ERR_ARG


def test_commit_window_needs_a_fresh_staging():
    """commit_window() refuses when nothing was staged since the last commit (before any GPU
    work), so a window never trains on the previous keyframes' inputs by mistake."""
    from paper_2410_00486_gb300.window import MappingWindow
    w = object.__new__(MappingWindow)
    with pytest.raises(RuntimeError, match="stage_window"):
        w.commit_window()
    w._pending = False                        # the state right after a commit
    with pytest.raises(RuntimeError, match="stage_window"):
        w.commit_window()
