"""The C ABI without a GPU: the library loads, exports every entry point that
include/lbm.h declares, the ctypes mirror of lbm_params has the C layout, and
invalid parameters are rejected on the host before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")
HEADERS = [os.path.join(ROOT, "include", h) for h in ("lbm.h", "lbm_nn.h")]


@pytest.fixture(scope="module")
def L():
    from paper_2103_02119_gb300 import build
    build.build()
    from paper_2103_02119_gb300 import lbm
    return lbm


def declared():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L.lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (lbm_\w+)", out))
    assert set(names) <= exported


def test_params_layout_matches_header(L, tmp_path):
    fields = [f for f, _ in L.lbm_params._fields_]
    src = tmp_path / "off.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\nint main(void){\n'
                   + "".join(f'printf("{f} %zu\\n", offsetof(lbm_params, {f}));\n' for f in fields)
                   + 'printf("sizeof %zu\\n", sizeof(lbm_params));\nreturn 0;}\n')
    exe = tmp_path / "off"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                      text=True).stdout.splitlines())
    for f in fields:
        assert int(got[f]) == getattr(L.lbm_params, f).offset, f
    assert int(got["sizeof"]) == ctypes.sizeof(L.lbm_params)


def test_params_init_defaults(L):
    p = L.lbm_params_init()
    assert (p.nx, p.ny, p.precision, p.periodic_x, p.periodic_y) == (64, 64, 32, 1, 1)
    assert p.a == 1.0 and abs(p.cs2 - 1 / 3) < 1e-15 and p.rho0 == 1.0
    assert list(p.omega) == [1.0] * 9


BAD = [
    ("nx", 2, "nx and ny"),
    ("ny", 0, "nx and ny"),
    ("a", 0.0, "a must"),
    ("a", float("nan"), "a must"),
    ("cs2", 0.3, "cs2"),          # with a = 0.5: cs2 >= a^2
    ("cs2", -1.0, "cs2"),
    ("precision", 16, "precision"),
    ("periodic_x", 2, "periodic"),
    ("block_x", 48, "block_x"),
    ("bands", -1, "bands"),
    ("rho0", -1.0, "rho0"),
    ("Fx", float("inf"), "force"),
    ("use_gi_corr", 3, "correction"),
    ("scheme", 2, "scheme"),
]


@pytest.mark.parametrize("field,value,msg", BAD)
def test_invalid_params_rejected_on_host(L, field, value, msg):
    p = L.lbm_params_init()
    p.a, p.cs2 = 0.5, 0.1
    setattr(p, field, value)
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(p)
    assert e.value.status == L.LBM_ERR_INVALID
    assert msg in str(e.value)


@pytest.mark.parametrize("j,value", [(3, 0.0), (4, 0.0), (5, 2.5), (0, -0.1)])
def test_invalid_relaxation_rates(L, j, value):
    p = L.lbm_params_init()
    p.omega[j] = value
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(p)
    assert e.value.status == L.LBM_ERR_INVALID


def test_null_arguments(L):
    p = L.lbm_params_init()
    assert L.lib.lbm_create(ctypes.byref(p), None, None, None) == L.LBM_ERR_INVALID
    assert L.lib.lbm_create(None, None, None, ctypes.byref(ctypes.c_void_p())) == L.LBM_ERR_INVALID
    assert "params is NULL" in L.lbm_last_error(None)
    assert L.lib.lbm_step(None, 1) == L.LBM_ERR_INVALID
    assert L.lib.lbm_diagnostics(None, None) == L.LBM_ERR_INVALID
    L.lib.lbm_destroy(None)  # ignored
    assert L.lib.lbm_step_count(None) == -1


def test_batch_invalid_params_rejected_on_host(L):
    good = L.lbm_params_init()
    bad = L.lbm_params_init()
    bad.precision = 64
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_create([good, bad])
    assert e.value.status == L.LBM_ERR_INVALID
    assert "lattice 1" in str(e.value) and "FP32" in str(e.value)
    bad = L.lbm_params_init()
    bad.nx = 2
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_create([bad, good])
    assert "lattice 0" in str(e.value) and "nx and ny" in str(e.value)
    big = L.lbm_params_init()
    big.nx, big.ny = 65536, 4096          # 9 x 65536 x 4096 >= 2^31 values
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_create([good, big])
    assert "2^31" in str(e.value)
    with pytest.raises(ValueError):
        L.lbm_batch_create([good], masks=[np.zeros(5, np.uint8)])


def test_batch_null_arguments(L):
    p = L.lbm_params_init()
    out = ctypes.c_void_p()
    assert L.lib.lbm_batch_create(ctypes.byref(p), 1, None, None, None) == L.LBM_ERR_INVALID
    assert L.lib.lbm_batch_create(None, 1, None, None, ctypes.byref(out)) == L.LBM_ERR_INVALID
    assert L.lib.lbm_batch_create(ctypes.byref(p), 0, None, None, ctypes.byref(out)) == \
        L.LBM_ERR_INVALID
    assert L.lib.lbm_batch_step(None, 1) == L.LBM_ERR_INVALID
    assert L.lib.lbm_batch_run(None, 1e-8, 100, 100, None) == L.LBM_ERR_INVALID
    assert L.lib.lbm_batch_count(None) == -1
    assert L.lib.lbm_batch_is_active(None, 0) == -1
    assert L.lib.lbm_batch_step_count(None, 0) == -1
    L.lib.lbm_batch_destroy(None)  # ignored


def test_nn_invalid_shapes_rejected_on_host(L):
    for args in [([8, 16], 0, 16, 16), ([8, 16], 2, 15, 16), ([8, 0], 2, 16, 16),
                 ([8] * 7, 2, 128, 128), ([600], 2, 16, 16)]:
        with pytest.raises(L.LbmError) as e:
            L.lbm_nn_create(*args)
        assert e.value.status == L.LBM_ERR_INVALID
    assert L.lib.lbm_nn_param_count(None) == 0
    assert L.lib.lbm_nn_forward(None, None, 1, None) == L.LBM_ERR_INVALID
    L.lib.lbm_nn_destroy(None)


def test_peak_probes_reject_bad_arguments_on_host(L):
    out = ctypes.c_double(-1.0)
    for nbytes, iters in [(0, 1), (8, 1), (1000, 1), (1 << 20, 0)]:
        assert L.lib.lbm_peak_copy_gbs(nbytes, iters, None, ctypes.byref(out)) == L.LBM_ERR_INVALID
    assert L.lib.lbm_peak_copy_gbs(1 << 20, 1, None, None) == L.LBM_ERR_INVALID
    assert L.lib.lbm_peak_fp64_gflops(0, None, ctypes.byref(out)) == L.LBM_ERR_INVALID
    assert L.lib.lbm_peak_fp64_gflops(10, None, None) == L.LBM_ERR_INVALID
    assert out.value == -1.0


def test_allocation_failure_hook_gives_oom_on_the_host(L):
    """lbm_debug_fail_alloc(1) fails the next device allocation before any
    CUDA call: lbm_create's first allocation is a population buffer, so it
    returns LBM_ERR_OOM, frees what it holds and names the allocation."""
    p = L.lbm_params_init()
    L.lbm_debug_fail_alloc(1)
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(p)
    assert e.value.status == L.LBM_ERR_OOM
    assert "distributions" in str(e.value)
    assert "distributions" in L.lbm_last_error(None)
    # the hook fired once and is disarmed; bad arguments are rejected
    assert L.lib.lbm_debug_fail_alloc(-1) == L.LBM_ERR_INVALID
    assert L.lib.lbm_debug_fail_alloc(0) == L.LBM_OK


def test_wait_limit_rejects_bad_arguments_on_host(L):
    assert L.lib.lbm_set_wait_limit(None, 10) == L.LBM_ERR_INVALID
    assert L.lib.lbm_batch_set_wait_limit(None, 10) == L.LBM_ERR_INVALID
