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


def test_noalloc_refuses_oversized_dims_before_touching_the_gpu(libreg):
    """The allocation-free entry point checks its fixed capacity (3 floats per node of
    the Laplacian, at most 4096 voxels per side) before any CUDA call, so sizes
    whose products overflow 32 bits are refused with REG_ERR_ARG; the pointers
    are never dereferenced."""
    fake = 256   # non-NULL, 8-byte aligned, never read
    for dims in ((1 << 30, 4, 4), (4098, 4, 4), (4, 4, 4096 + 2), (1 << 20, 1 << 20, 1 << 20), (200, 200, 200)):
        with pytest.raises(libreg.RegError) as ei:
            libreg.reg_eval_objective_grad_noalloc(fake, fake, dims, (1.0, 1.0, 1.0), fake, fake, 0.1, 0.1, 1.0, fake)
        assert ei.value.code == libreg.REG_ERR_ARG
        assert "node floats" in libreg.reg_last_error(None)


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


def _golden_pt_rows():
    with open(os.path.join(ROOT, "tests", "golden", "pt_tables.txt")) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_axis_tables_match_the_hand_derived_eq3_tables(libreg):
    """The P^T index sets and weights the library uploads equal the hand-derived
    Eq. 3 tables (unit spacing; FP32 weights)."""
    from fractions import Fraction
    rows = _golden_pt_rows()
    assert rows
    for r in rows:
        m, n, k, first = int(r[0]), int(r[1]), int(r[2]), int(r[3])
        w_ref = [float(Fraction(w)) for w in r[4:]]
        _, _, f, cnt, w = libreg.reg_axis_tables(m, 1.0, n)
        assert f[k] == first and cnt[k] == len(w_ref), r
        assert abs(w[k, :cnt[k]] - w_ref).max() <= 1e-7, r
        assert not w[k, cnt[k]:].any()


@pytest.mark.parametrize("m,h,n", [(256, 1.0, 129), (112, 2.5, 57), (1577, 0.75, 789), (33, 1.5, 9),
                                   (37, 1.1, 19), (8, 0.97, 3)])
def test_axis_tables_agree_with_the_oracle_and_with_each_other(libreg, m, h, n):
    """P^T tables against the FP64 oracle's; the P entries (k0, w1) are the
    same weights seen from the voxel side: voxel i has 1 - w1 at node k0 and w1
    at k0 + 1, and nothing elsewhere."""
    import numpy as np
    import oracle
    oracle.build()
    k0, w1, first, cnt, w = libreg.reg_axis_tables(m, h, n)
    dense = np.zeros((n, m))
    for k in range(n):
        f_o, w_o = oracle.PT_table(m, h, n, k)
        assert first[k] == f_o and cnt[k] == len(w_o), k
        assert np.abs(w[k, :cnt[k]] - w_o).max() <= 1e-6
        dense[k, first[k]:first[k] + cnt[k]] = w[k, :cnt[k]]
    from_p = np.zeros((n, m))
    from_p[k0, np.arange(m)] += 1.0 - w1
    from_p[k0 + 1, np.arange(m)] += w1
    assert k0.min() >= 0 and k0.max() <= n - 2
    assert np.abs(dense - from_p).max() <= 1e-6
    np.testing.assert_allclose(dense.sum(axis=0), 1.0, atol=1e-6)   # partition of unity at every voxel


def test_axis_tables_reject_bad_arguments(libreg):
    L = libreg.lib()
    for m, h, n in ((3, 1.0, 3), (16, 0.0, 9), (16, float("inf"), 9), (16, 1.0, 2)):
        assert L.reg_axis_tables(m, h, n, None, None, None, None, None, 0, None) == libreg.REG_ERR_ARG
    import ctypes
    import numpy as np
    w = np.zeros((9, 3), np.float32)
    assert L.reg_axis_tables(16, 1.0, 9, None, None, None, None, ctypes.c_void_p(w.ctypes.data), 3,
                             None) == libreg.REG_ERR_ARG   # 4 weights per node needed


def test_header_limits_match_the_binding(libreg):
    import re
    text = open(libreg.HEADER).read()
    limits = dict(re.findall(r"#define (REG_MAX_\w+) (\d+)", text))
    assert int(limits["REG_MAX_VOXELS"]) == libreg.MAX_VOXELS == 2**31 - 1
    assert int(limits["REG_MAX_PLANES"]) == libreg.MAX_PLANES == 65535
    assert int(limits["REG_MAX_LEVELS"]) == libreg.MAX_LEVELS and int(limits["REG_MAX_MEM"]) == libreg.MAX_MEM


def test_header_entries_cite_their_passage_or_say_they_have_none(libreg):
    """Every compute or geometry entry point of the header cites the passage of
    the paper that defines it (Sec. / Eq.), or states that it has no counterpart
    there; the plain utilities (version, defaults, destroy, last error) are exempt."""
    import re
    text = open(libreg.HEADER).read()
    found = {}
    for m in re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*\n((?:[^;/]|/(?!\*))*?\b(reg_\w+)\s*\([^;]*;)", text, re.S):
        found[m.group(3)] = re.sub(r"\s*\n\s*\*?\s*", " ", m.group(1))
    exempt = {"reg_version", "reg_destroy", "reg_last_error"}
    assert set(found) >= set(libreg.header_functions())
    for name, comment in found.items():
        if name in exempt:
            continue
        assert re.search(r"Sec\. [0-9]|Eq\. [0-9]|counterpart in the paper|paper reports", comment), name


def test_plain_c_client_compiles_links_and_runs(libreg, tmp_path):
    """The header is plain C (C99, -pedantic): a C program includes it, links
    libreg.so and calls the host-only entry points."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = tmp_path / "client.c"
    src.write_text(r"""
#include <stdio.h>
#include "reg.h"
int main(void)
{
    reg_config cfg;
    int dims[3] = {256, 256, 256}, split[5], first[9], cnt[9], need = 0;
    double steps = 0.0;
    float w[9 * 4];
    reg_config_default(&cfg);
    if (cfg.levels != 1 || cfg.lbfgs_mem != 5) return 1;
    if (reg_fused_split_plan(dims, 152, split, &steps) != REG_OK) return 2;
    if (reg_axis_tables(16, 1.0, 9, NULL, NULL, first, cnt, w, 4, &need) != REG_OK || need != 4) return 3;
    if (reg_axis_tables(3, 1.0, 9, NULL, NULL, NULL, NULL, NULL, 0, NULL) != REG_ERR_ARG) return 4;
    printf("%d %d %d %d %d %.1f %d %d %s\n", split[0], split[1], split[2], split[3], split[4], steps, first[1],
           cnt[1], reg_last_error(NULL));
    return 0;
}
""")
    libdir = os.path.dirname(libreg.LIB_PATH)
    exe = tmp_path / "client"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lreg", "-Wl,-rpath," + libdir,
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    fields = out.stdout.split()
    assert tuple(int(v) for v in fields[:5]) == libreg.reg_fused_split_plan((256, 256, 256), 152)[0]
    assert fields[6:8] == ["0", "4"] and "reg_axis_tables" in out.stdout
