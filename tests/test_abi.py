"""The C library builds, loads and exports every function include/dust.h
declares (no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dust.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dust_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_10793_gb300 import build as B
    path = B.build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_interface():
    names = declared_functions()
    for required in ("dust_create", "dust_set_gas", "dust_load_particles", "dust_step",
                     "dust_sync", "dust_get_deposit", "dust_get_particles", "dust_get_gas",
                     "dust_last_error", "dust_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_has_every_declared_name():
    from paper_1908_10793_gb300 import dust as D
    for name in declared_functions():
        assert callable(getattr(D, name)), name


def test_create_error_path_without_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_1908_10793_gb300 import dust as D
    D.load_library()
    with pytest.raises(D.DustError) as e:
        D.dust_create(D.dust_geometry(kind=7), D.dust_grid(), [D.dust_species(mass=1.0)],
                      D.dust_options())
    assert e.value.code == D.DUST_EINVAL


def test_semi_implicit_pusher_rejected_for_curvilinear_grids(lib):
    # checked with the other descriptors, before any CUDA call
    from paper_1908_10793_gb300 import dust as D
    from paper_1908_10793_gb300 import inputs as I
    w = I.cyldisk("small")
    geo, grid, sp, opt, keep = D.make_descriptors(w, pusher=D.DUST_PUSHER_SEMI_IMPLICIT)
    with pytest.raises(D.DustError) as e:
        D.dust_create(geo, grid, sp, opt)
    assert e.value.code == D.DUST_EINVAL and "semi-implicit" in str(e.value)
    geo, grid, sp, opt, keep = D.make_descriptors(w, pusher=7)
    with pytest.raises(D.DustError) as e:
        D.dust_create(geo, grid, sp, opt)
    assert e.value.code == D.DUST_EINVAL


def test_host_io_async_option_validated_without_gpu(lib):
    from paper_1908_10793_gb300 import dust as D
    from paper_1908_10793_gb300 import inputs as I
    w = I.box2d("small")
    geo, grid, sp, opt, keep = D.make_descriptors(w, host_io_async=2)
    with pytest.raises(D.DustError) as e:
        D.dust_create(geo, grid, sp, opt)
    assert e.value.code == D.DUST_EINVAL and "host_io_async" in str(e.value)


def test_test_wait_timeout_option_validated_without_gpu(lib):
    from paper_1908_10793_gb300 import dust as D
    from paper_1908_10793_gb300 import inputs as I
    w = I.box2d("small")
    geo, grid, sp, opt, keep = D.make_descriptors(w, test_wait_timeout=3)
    with pytest.raises(D.DustError) as e:
        D.dust_create(geo, grid, sp, opt)
    assert e.value.code == D.DUST_EINVAL and "test_wait_timeout" in str(e.value)


@pytest.mark.parametrize("tile", [(2048, 1, 1), (8, -1, 8), (8, 8, 1024)])
def test_tile_option_validated_without_gpu(lib, tile):
    from paper_1908_10793_gb300 import dust as D
    from paper_1908_10793_gb300 import inputs as I
    w = I.box2d("small")
    geo, grid, sp, opt, keep = D.make_descriptors(w, tile=tile)
    with pytest.raises(D.DustError) as e:
        D.dust_create(geo, grid, sp, opt)
    assert e.value.code == D.DUST_EINVAL and "tile[" in str(e.value)


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    # no fallback: with libdust.so missing, the first call raises
    from paper_1908_10793_gb300 import dust as D
    monkeypatch.setattr(D, "LIB_PATH", str(tmp_path / "libdust.so"))
    monkeypatch.setattr(D, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        D.load_library()
