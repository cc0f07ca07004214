"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/stab.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "stab.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stab_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1502_03701_gb300 import binding, build
    build.build()
    lib = ctypes.CDLL(binding.LIB_PATH)
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(binding.SYMBOLS) == names


def test_default_opts_and_create_rejects_bad_grid():
    from paper_1502_03701_gb300 import binding
    o = binding.default_opts()
    assert o.gamma == 1.4 and o.gmres_m == 30 and o.tile[0] == 8 and o.precond_prec == 32
    L = binding.load()
    h = ctypes.c_void_p()
    g = binding.Grid(2, 4, 64, 1, 1.0, -1.0, 1.0, 1.0, 0.0)  # nx < 6: rejected before any CUDA call
    st = L.stab_create(ctypes.byref(h), ctypes.c_void_p(1), 0, ctypes.byref(g), 0.3, 1000.0, 0.71, None, None)
    assert st == 1 and not h.value
    assert b"nx" in L.stab_last_error(None)


def test_autotune_cache_file_roundtrip(tmp_path):
    """The tuning cache file format reads back (no GPU needed)."""
    from paper_1502_03701_gb300 import binding
    src = tmp_path / "tune.txt"
    # seven columns: an FP64-stencil entry; the eighth marks the pair stencil
    src.write_text("256 512 7 1 32 4 1\n512 256 5 0 16 2 2 1\nbad line\n512 256 5 0 16 2 2 7\n")
    assert binding.autotune_load(str(src)) == 2
    dst = tmp_path / "out.txt"
    assert binding.autotune_save(str(dst)) >= 2
    lines = set(dst.read_text().split("\n"))
    assert "256 512 7 1 32 4 1 0" in lines and "512 256 5 0 16 2 2 1" in lines
    assert binding.autotune_load(str(tmp_path / "missing.txt")) == -1


def test_memory_estimate_grows_with_the_problem():
    """stab_estimate_bytes (host arithmetic only)."""
    import stab_inputs as si
    from paper_1502_03701_gb300 import estimate_bytes
    g, _ = si.mixing_layer_2d(32, 64, Ma=0.3)
    g2, _ = si.mixing_layer_2d(64, 128, Ma=0.3)
    base = estimate_bytes(g, 4, 30, precond=0)
    n = 4 * 32 * 64
    assert base > (30 + 31 + 3) * n * 16        # Arnoldi and GMRES bases at least
    assert estimate_bytes(g, 4, 40, precond=0) - base == 10 * n * 16 + (10 * n * 16) // 10
    assert estimate_bytes(g, 4, 30, precond=1, tile=(8, 8)) > base + 32 * 256 * 256 * 8
    fixed = 8 << 20                              # tables and alignment allowance
    assert estimate_bytes(g2, 4, 30, precond=0) - fixed > 3.5 * (base - fixed)
    assert estimate_bytes(g, 4, 30, yonly=False, precond=0) > base


def test_batch_binding_checks_arguments_before_calling_the_library():
    """JvBatch refuses mismatched lists and closed handles on the host (no GPU needed)."""
    from paper_1502_03701_gb300 import JvBatch, StabError

    class FakeHandle:
        _h = object()
        n = 8

    B = JvBatch.__new__(JvBatch)
    B.handles = [FakeHandle(), FakeHandle()]
    B._b = object()
    with pytest.raises(ValueError):
        B.apply([1], [1, 2])
    with pytest.raises(ValueError):
        B.precond_apply([1, 2], [1])
    with pytest.raises(ValueError):
        B.orthogonalize([1, 2], [3], [1, 2])
    import torch
    ok = torch.zeros(8, dtype=torch.complex128)
    with pytest.raises(ValueError, match="CUDA"):  # host tensors are refused before any library call
        B.apply([ok, ok], [ok, ok])
    with pytest.raises(ValueError, match="complex128"):
        B.precond_apply([torch.zeros(8), ok], [ok, ok])
    B.handles[1]._h = None
    with pytest.raises(StabError, match="closed"):
        B.apply([1, 2], [1, 2])
    B._b = None


def test_memory_estimate_of_the_reduced_preconditioner():
    """The reduced-operator factors take three m x m level blocks per level (m = nv * 2 * tx * tz), so
    their estimate does not grow with the tile height, while the dense tile inverses grow with its square."""
    import stab_inputs as si
    from paper_1502_03701_gb300 import estimate_bytes
    g, _ = si.mixing_layer_2d(64, 128, Ma=0.3)
    n = 4 * 64 * 128
    base = estimate_bytes(g, 4, 30, precond=0)
    short = estimate_bytes(g, 4, 30, precond=2, tile=(8, 16)) - base
    tall = estimate_bytes(g, 4, 30, precond=2, tile=(8, 128)) - base
    m = 4 * 2 * 8
    assert short >= n * 3 * m * 8 and tall >= n * 3 * m * 8      # FP32 factors: 3 m complex per unknown
    assert tall < 1.2 * short + (2 << 20)
    dense = estimate_bytes(g, 4, 30, precond=1, tile=(8, 16)) - base
    assert dense > n * 4 * 8 * 16 * 8                            # b complex per unknown, b = 512
