"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every symbol include/gmg.h declares, and rejects bad
configurations before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1208_4247_gb300 import build, gmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return gmg.lib()


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            syms |= set(re.findall(r"\b(gmg_[a-z0-9_]+)\s*\(", text))
    return syms


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert "gmg_solve" in syms and "gmg_create" in syms and "gmg_destroy" in syms
    for s in sorted(syms):
        assert hasattr(L, s), s
    # the binding knows every declared symbol's signature
    assert syms <= set(gmg.SIGNATURES)


def test_abi_version(L):
    assert L.gmg_abi_version() == 2


def test_config_defaults(L):
    c = gmg.Config()
    assert L.gmg_config_init(ctypes.byref(c), 3, 256) == 0
    assert (c.d, c.n, c.levels, c.smoother, c.nu1, c.nu2, c.precision, c.maxit) == \
        (3, 256, 0, 1, 2, 2, 0, 100)
    assert c.omega == pytest.approx(0.8)


@pytest.mark.parametrize("field,value,status", [
    ("d", 4, 1), ("n", 100, 1), ("n", 1, 1), ("levels", 9, 1), ("smoother", 7, 1),
    ("omega", 2.5, 1), ("nu1", -1, 1), ("nu2", 17, 1), ("cycle", 2, 1),
    ("maxit", -3, 1), ("precision", 9, 8), ("transfer", 2, 1), ("smoother", 4, 1),
])
def test_bad_config_rejected_before_device_use(L, field, value, status):
    c = gmg.Config()
    L.gmg_config_init(ctypes.byref(c), 3, 256)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert L.gmg_create(ctypes.byref(c), None, ctypes.byref(h)) == status
    assert not h.value
    assert len(L.gmg_last_error()) > 0


def test_null_arguments(L):
    assert L.gmg_create(None, None, None) == 1
    assert L.gmg_solve(None, None, None, 1e-10, None, None) == 1
    assert L.gmg_destroy(None) == 0
    assert L.gmg_config_init(None, 3, 8) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gmg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gmg, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        gmg.lib()


def test_learned_smoother_needs_fp64(L):
    c = gmg.Config()
    L.gmg_config_init(ctypes.byref(c), 3, 64)
    c.smoother = 2
    c.precision = 1
    h = ctypes.c_void_p()
    assert L.gmg_create(ctypes.byref(c), None, ctypes.byref(h)) == 8
    assert b"FP64" in L.gmg_last_error()


def test_learned_calls_reject_bad_sizes(L):
    w = (ctypes.c_float * (2 * 8 * 27))()
    assert L.gmg_learned_conv(4, 16, w, None, None, 0, None) == 1
    assert L.gmg_learned_conv(3, 12, w, None, None, 1, None) == 1
    loss = ctypes.c_double()
    assert L.gmg_learned_loss_grad(3, 2, w, None, 10, ctypes.byref(loss), None, None) == 1
    assert L.gmg_learned_train(3, 64, 0, 1, 1, 10, 1e-3, 1, w, w, None, None) == 1
    assert L.gmg_smoother_select(None, None, None, 0, 8, 2, None, None, None) == 1
    assert L.gmg_measure_fp64_rate(2, ctypes.byref(loss), None) == 1
    assert L.gmg_measure_fp64_rate(0, None, None) == 1


def test_batch_and_fft_reject_bad_arguments(L):
    c = gmg.Config()
    L.gmg_config_init(ctypes.byref(c), 3, 16)
    c.precision = 1
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 2)(3, 2)
    n = (ctypes.c_int * 2)(16, 100)
    assert L.gmg_batch_create(2, d, n, ctypes.byref(c), 0, 0, None, ctypes.byref(h)) == 1
    assert b"solve 1" in L.gmg_last_error()
    n[1] = 64
    c.precision = 0
    assert L.gmg_batch_create(2, d, n, ctypes.byref(c), 0, 0, None, ctypes.byref(h)) == 8
    c.precision = 1
    c.smoother, c.nu1, c.nu2 = 0, 1, 2
    assert L.gmg_batch_create(2, d, n, ctypes.byref(c), 0, 0, None, ctypes.byref(h)) == 8
    assert L.gmg_batch_solve(None, None, None, 1e-10, None, None, None) == 1
    assert L.gmg_batch_destroy(None) == 0
    assert L.gmg_fft_create(3, 100, None, ctypes.byref(h)) == 1
    assert L.gmg_fft_create(4, 64, None, ctypes.byref(h)) == 1
    assert L.gmg_fft_solve(None, None, None) == 1
    assert L.gmg_fft_destroy(None) == 0


def test_fmg_needs_plain_fp64(L):
    c = gmg.Config()
    L.gmg_config_init(ctypes.byref(c), 3, 64)
    c.cycle = 1
    c.precision = 1
    h = ctypes.c_void_p()
    assert L.gmg_create(ctypes.byref(c), None, ctypes.byref(h)) == 8


def test_problem_statement_entry_points_reject_bad_arguments(L):
    """gmg_solve_strided, gmg_create_batched, gmg_smoother_{train,save,load}:
    argument checks that need no GPU."""
    st = (ctypes.c_int64 * 3)(1, 20, 400)
    assert L.gmg_solve_strided(None, None, None, st, 1e-10, None, None) == 1
    out = ctypes.c_void_p()
    assert L.gmg_create_batched(0, None, None, ctypes.byref(out)) == 1
    c = (gmg.Config * 2)()
    L.gmg_config_init(ctypes.byref(c[0]), 3, 16)
    L.gmg_config_init(ctypes.byref(c[1]), 2, 64)
    c[0].precision = c[1].precision = 1
    c[1].nu1 = 1  # differs from solve 0
    assert L.gmg_create_batched(2, c, None, ctypes.byref(out)) == 1
    assert b"differ" in L.gmg_last_error()
    size = ctypes.c_size_t(0)
    assert L.gmg_smoother_save(None, None, 0, ctypes.byref(size)) == 1
    assert L.gmg_smoother_load(None, None, 0) == 1
    assert L.gmg_smoother_train(None, None, None, None) == 1


def test_paper_variant_needs_plain_fp64(L):
    """The paper's multi-colour smoother and transfers run in the plain FP64
    form only; the defaults select full weighting."""
    c = gmg.Config()
    L.gmg_config_init(ctypes.byref(c), 2, 64)
    assert c.transfer == 0
    h = ctypes.c_void_p()
    for smoother, transfer in ((3, 0), (1, 1)):
        c.smoother, c.transfer, c.precision = smoother, transfer, 1
        assert L.gmg_create(ctypes.byref(c), None, ctypes.byref(h)) == 8
        assert not h.value
    c.smoother, c.transfer, c.precision = 2, 1, 0
    assert L.gmg_create(ctypes.byref(c), None, ctypes.byref(h)) == 8
