"""CPU checks of the boundary: the library loads and exports every symbol the
header declares; pure-host calls behave (no GPU needed, no compute calls)."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libreg():
    from paper_1812_06765_gb300 import build
    build.build()
    from paper_1812_06765_gb300 import _lib
    return _lib


def test_exports_every_header_symbol(libreg):
    names = libreg.header_functions()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", libreg.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = libreg.lib()
    for n in names:
        assert hasattr(L, n)


def test_config_default_and_version(libreg):
    cfg = libreg.reg_config_default()
    assert cfg.tau == 0.01 and cfg.rho == 0.01 and cfg.alpha == 10.0
    assert cfg.lbfgs_mem == 5 and cfg.max_backtracks == 20 and cfg.levels == 1
    assert list(cfg.max_iter) == [50] * 8 and cfg.start_level == -1
    assert cfg.autotune == 1 and cfg.fused_tz == 0 and cfg.use_graph == 1 and cfg.image_dtype == 0
    assert cfg.test_expire_wait == 0
    assert libreg.reg_version() >= 10000
    assert ctypes.sizeof(libreg.RegConfig) == 8 * 6 + 4 * 6 + 4 * 8 + 4 * 24 + 4 * 12
    assert list(cfg.fused_split) == [0] * 5


def test_create_rejects_bad_config_before_touching_the_gpu(libreg):
    for field, value in (("levels", 0), ("levels", 9), ("lbfgs_mem", 0), ("tau", 0.0), ("c1", 1.5),
                         ("max_backtracks", 0), ("eval_impl", 7), ("autotune", 2), ("fused_tz", 7),
                         ("fused_tz", 514), ("fused_tz", -2), ("eval_impl", -1), ("test_expire_wait", 2)):
        cfg = libreg.reg_config_default()
        setattr(cfg, field, value)
        with pytest.raises(libreg.RegError) as ei:
            libreg.reg_create(cfg)
        assert ei.value.code == libreg.REG_ERR_ARG
        assert libreg.reg_last_error(None)
    for split in ((3, 1, 0, 0, 0), (4, -1, 0, 0, 0), (0, 0, 0, 0, 7), (4, 1, 514, 1, 0), (0, 1, 0, 0, 0)):
        cfg = libreg.reg_config_default()
        cfg.fused_split[:] = list(split)
        with pytest.raises(libreg.RegError) as ei:
            libreg.reg_create(cfg)
        assert ei.value.code == libreg.REG_ERR_ARG


def test_null_handle_calls_are_safe(libreg):
    L = libreg.lib()
    assert L.reg_destroy(None) == 0
    assert L.reg_eval_objective_grad(None, 0, None, None, None, None, None) == libreg.REG_ERR_ARG
    assert L.reg_register(None, None, 0, None, None) == libreg.REG_ERR_ARG
    assert b"NULL" in L.reg_last_error(None)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle; its binding fails loudly without the library."""
    pkg = os.path.join(ROOT, "paper_1812_06765_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
    code = ("import sys; sys.path.insert(0, %r); from paper_1812_06765_gb300 import _lib; "
            "_lib.LIB_PATH = '/nonexistent/libreg.so'\n"
            "try:\n    _lib.lib()\nexcept RuntimeError as e:\n    print('raised', e)\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised" in out.stdout, out.stdout + out.stderr
