"""Host-side checks of the C ABI (no GPU): the library loads, exports every symbol that
include/fif.h declares, and its host-only entry points validate arguments."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2008_03324_gb300 import build as B
    B.build()
    from paper_2008_03324_gb300 import fif
    fif.lib()
    return fif


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fif.h")).read()
    return sorted(set(re.findall(r"FIF_API\s+[\w\s\*]+?\b(fif_\w+)\s*\(", txt)))


def test_header_declares_the_four_calls():
    names = declared_symbols()
    for n in ("fif_build", "fif_query", "fif_query_backward", "fif_pointcloud_fim"):
        assert n in names


def test_library_exports_every_declared_symbol(F):
    lib = ctypes.CDLL(F.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) == set(F.SYMBOLS)


def test_status_strings(F):
    assert F.status_str(0) == "ok"
    assert "wait" in F.status_str(F.ETIMEOUT)
    assert F.status_str(12345) == "unknown status"
    assert F.lib().fif_version() == 10100


def test_field_bytes_and_init_validation(F):
    g = F.make_grid((0, 0, 0), 0.5, (21, 21, 7))
    assert F.field_bytes(g, F.STORAGE_F32) == 21 * 21 * 7 * 216 * 4
    assert F.field_bytes(g, F.STORAGE_BF16) == 21 * 21 * 7 * 224 * 2
    assert F.field_bytes(g, 7) == 0
    bad = F.make_grid((0, 0, 0), 0.5, (1, 21, 7))
    assert F.field_bytes(bad, F.STORAGE_F32) == 0
    assert F.field_bytes(F.make_grid((0, 0, 0), -1.0, (2, 2, 2)), 0) == 0
    p = F.make_params()
    f = F.FieldC()
    lib = F.lib()
    nbytes = F.field_bytes(g, 0)
    fake = ctypes.c_void_p(0x100000)   # never dereferenced by fif_field_init
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0, fake, nbytes) == F.OK
    assert f.stride == 216
    # k from Eq. quadratic_conditions with alpha = 45 deg, v_alpha = 0.5
    assert f.k[1] == pytest.approx(0.5)
    assert f.k[2] == pytest.approx(0.7071067811865476)
    assert f.k[0] == pytest.approx(-0.20710678118654757)
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0, fake, nbytes - 1) == F.ESIZE
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0,
                              ctypes.c_void_p(0x100004), nbytes) == F.EALIGN
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0, None, nbytes) == F.EINVAL
    p2 = F.make_params(r_max=0.05)   # r_max <= r_min
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p2), 0, fake, nbytes) == F.EINVAL
    p3 = F.make_params(half_fov=4.0)
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p3), 0, fake, nbytes) == F.EINVAL


def test_workspace_bytes_host_only(F):
    g = F.make_grid((0.125, 0.125, 0.125), 0.25, (200, 200, 40))
    p = F.make_params(r_max=10.0)
    f = F.FieldC()
    fake = ctypes.c_void_p(0x100000)
    assert F.lib().fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0, fake,
                                  F.field_bytes(g, 0)) == F.OK
    ws = F.build_workspace_bytes(f, 200_000)
    assert ws >= 200_000 * 20
    assert F.build_workspace_bytes(f, -1) == 0


def test_calls_reject_bad_arguments_before_any_launch(F):
    lib = F.lib()
    g = F.make_grid((0, 0, 0), 0.5, (4, 4, 4))
    p = F.make_params()
    f = F.FieldC()
    fake = ctypes.c_void_p(0x100000)
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0, fake, F.field_bytes(g, 0)) == 0
    assert lib.fif_query(ctypes.byref(f), None, -1, F.Q_METRICS, None, None, None, None, None) == F.EINVAL
    assert lib.fif_query(ctypes.byref(f), None, 5, F.Q_METRICS, None, None, None, None, None) == F.EINVAL
    assert lib.fif_query(ctypes.byref(f), fake, 5, 0x1000, None, None, None, None, None) == F.EINVAL
    # the compensated contraction is a GP-field option only
    assert lib.fif_query(ctypes.byref(f), fake, 5, F.Q_METRICS | F.Q_GP_COMPENSATED, None, fake, None, None,
                         None) == F.EINVAL
    assert lib.fif_query(ctypes.byref(f), fake, 0, F.Q_METRICS, None, fake, None, None, None) == F.OK
    assert lib.fif_query_backward(ctypes.byref(f), fake, 5, F.Q_NEAREST, fake, fake, fake, None) == F.EINVAL
    assert lib.fif_build(ctypes.byref(f), None, 5, fake, 1 << 20, None) == F.EINVAL
    assert lib.fif_build(ctypes.byref(f), fake, 5, fake, 16, None) == F.ESIZE
    cam = F.make_pinhole(width=0)
    assert lib.fif_pointcloud_fim(fake, 5, ctypes.byref(p), ctypes.byref(cam), fake, 5, F.Q_METRICS,
                                  None, fake, None, None, None) == F.EINVAL
    assert lib.fif_device_error(None, 0, None) == F.EINVAL
    assert lib.fif_field_load(None, b"/nonexistent", fake, 16, None, None) == F.EINVAL
    f2 = F.FieldC()
    assert lib.fif_field_load(ctypes.byref(f2), b"/nonexistent/x.fif", fake, 16, None, None) == F.EIO


def test_query_host_checks_and_staging_size(F):
    """fif_query_host's argument checks return before any CUDA call; its staging is two buffers of
    poses + FIM + metrics + sign + status per pose, each array rounded up to 256 bytes."""
    up = lambda x: (x + 255) // 256 * 256
    assert F.query_host_staging_bytes(1000) == 2 * (up(28000) + up(84000) + up(24000) + up(1000) + up(4000))
    assert F.query_host_staging_bytes(0) == 0 and F.query_host_staging_bytes(-3) == 0
    lib = F.lib()
    g = F.make_grid((0, 0, 0), 0.5, (4, 4, 4))
    p = F.make_params()
    f = F.FieldC()
    fake = ctypes.c_void_p(0x100000)
    s1, s2 = ctypes.c_void_p(0x10), ctypes.c_void_p(0x20)   # never used: every call below fails its checks
    assert lib.fif_field_init(ctypes.byref(f), ctypes.byref(g), ctypes.byref(p), 0, fake, F.field_bytes(g, 0)) == 0
    need = F.query_host_staging_bytes(64)
    q = lib.fif_query_host
    assert q(ctypes.byref(f), fake, -1, F.Q_METRICS, None, fake, None, None, 64, fake, need, s1, s2) == F.EINVAL
    assert q(ctypes.byref(f), None, 5, F.Q_METRICS, None, fake, None, None, 64, fake, need, s1, s2) == F.EINVAL
    assert q(ctypes.byref(f), fake, 0, F.Q_METRICS, None, fake, None, None, 64, fake, need, s1, s2) == F.OK
    assert q(ctypes.byref(f), fake, 5, F.Q_METRICS, None, fake, None, None, 0, fake, need, s1, s2) == F.EINVAL
    assert q(ctypes.byref(f), fake, 5, F.Q_METRICS, None, fake, None, None, 64, None, need, s1, s2) == F.EINVAL
    assert q(ctypes.byref(f), fake, 5, F.Q_METRICS, None, fake, None, None, 64, fake, need, s1, s1) == F.EINVAL
    assert q(ctypes.byref(f), fake, 5, F.Q_METRICS, None, fake, None, None, 64, fake, need - 1, s1, s2) == F.ESIZE
    assert q(ctypes.byref(f), fake, 5, F.Q_METRICS, None, fake, None, None, 64, ctypes.c_void_p(0x100004), need,
             s1, s2) == F.EALIGN


def test_c_client_compiles_and_links(F, tmp_path):
    """include/fif.h is plain C and libfif.so links from a C program (no Python, no PyTorch); the
    GPU tests run the same program."""
    from tests import _fixtures as X
    exe = X.build_c_client(tmp_path)
    assert os.access(exe, os.X_OK)


def test_field_load_rejects_bad_files_before_any_copy(F, tmp_path):
    """fif_field_load validates the file (magic, version, sizes, checksum) before it touches the
    device: a foreign file, a truncated header and an empty file give FIF_EFORMAT; a missing file
    FIF_EIO."""
    lib = F.lib()
    fake = ctypes.c_void_p(0x100000)
    f = F.FieldC()
    cases = {"foreign.fif": b"NOTAFIELD" + bytes(200), "short.fif": b"FIFFIELD" + bytes(8), "empty.fif": b""}
    for name, data in cases.items():
        p = tmp_path / name
        p.write_bytes(data)
        assert lib.fif_field_load(ctypes.byref(f), str(p).encode(), fake, 1 << 20, None, None) == F.EFORMAT, name
    assert lib.fif_field_load(ctypes.byref(f), str(tmp_path / "none.fif").encode(), fake, 1 << 20, None,
                              None) == F.EIO


def test_fma_probe_is_outside_the_product_library(F):
    """The FP32 FMA throughput probe lives in the benchmark's own libfif_probe.so: the product
    library does not export it, and the probe's argument checks return before any launch."""
    import bench
    assert not hasattr(F.lib(), "fif_fma_probe")
    P = bench.probe_lib()
    fake = ctypes.c_void_p(0x100000)
    assert P.fif_fma_probe(None, 4, 10, 0, None) == F.EINVAL
    assert P.fif_fma_probe(fake, 0, 10, 0, None) == F.EINVAL
    assert P.fif_fma_probe(fake, 4, 0, 1, None) == F.EINVAL
    assert P.fif_fma_probe(ctypes.c_void_p(0x100002), 4, 10, 0, None) == F.EALIGN


def test_wait_limit_setter(F):
    """fif_set_wait_limit accepts any limit (0 restores the default) and needs no GPU."""
    lib = F.lib()
    assert lib.fif_set_wait_limit(1000) == F.OK
    assert lib.fif_set_wait_limit(0) == F.OK
