"""Marshalling of the Python binding on CPU: the arguments it hands to the C
library, with the library call replaced by a recorder (no GPU, no compute)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
reg = pytest.importorskip("paper_1812_06765_gb300")
from paper_1812_06765_gb300 import _lib  # noqa: E402


def _stats(levels=2):
    st = _lib.RegStats()
    st.levels = levels
    for lv in range(levels):
        st.iters[lv], st.evals[lv], st.J[lv], st.level_seconds[lv], st.tiling[lv] = 10 + lv, 11 + lv, 1.5, 0.25, 16
    st.J_final, st.D_final, st.S_final, st.seconds, st.kernel_launches = 1.0, 0.75, 0.005, 0.5, 321
    return st


class _NoLibHandle(reg.Registration):
    """A Registration whose handle value is a placeholder that never reaches the library."""

    def close(self):
        self.h = None


def _handle(monkeypatch, calls):
    r = object.__new__(_NoLibHandle)
    r.h = ctypes.c_void_p(1234)
    monkeypatch.setattr(reg.Registration, "node_shape", lambda self, level=0: (3, 5, 4, 3))

    def fake_register(h, uptr, dev, iptr):
        calls.append((h, uptr, dev, iptr))
        return 0, _stats()
    monkeypatch.setattr(_lib, "reg_register", fake_register)
    return r


def test_register_numpy_output_and_initial_field(monkeypatch):
    calls = []
    r = _handle(monkeypatch, calls)
    u, st = r.register(out="numpy")
    assert isinstance(u, np.ndarray) and u.shape == (3, 5, 4, 3) and u.dtype == np.float32
    assert calls[-1] == (r.h, u.ctypes.data, False, None)
    assert st == dict(status=0, iters=[10, 11], evals=[11, 12], level_status=[0, 0], J=[1.5, 1.5], J_final=1.0,
                      D_final=0.75, S_final=0.005, seconds=0.5, kernel_launches=321, level_seconds=[0.25, 0.25],
                      tiling=[16, 16])
    u0 = torch.arange(180, dtype=torch.float64).reshape(3, 5, 4, 3)   # any dtype, any host array kind
    r.register(out="numpy", u_init=u0)
    assert calls[-1][3] != 0 and calls[-1][2] is False


def test_register_rejects_unknown_output_kind(monkeypatch):
    r = _handle(monkeypatch, [])
    with pytest.raises(ValueError):
        r.register(out="cuda")
    with pytest.raises(ValueError):
        reg.register_batch([r], out="host")


def test_config_fields_follow_the_arguments():
    cfg = reg.make_config(levels=3, tau=0.1, alpha=50.0, mem=8, max_iter=[60, 70], node_dims=[(9, 13, 5)],
                          fused_split=(160, 1, 80, 1, 16), image_dtype="bf16", autotune=False)
    assert (cfg.levels, cfg.tau, cfg.rho, cfg.alpha, cfg.lbfgs_mem) == (3, 0.1, 0.1, 50.0, 8)
    assert list(cfg.max_iter) == [60] + [70] * 7
    assert list(cfg.node_dims[0]) == [9, 13, 5] and list(cfg.node_dims[1]) == [0, 0, 0]
    assert list(cfg.fused_split) == [160, 1, 80, 1, 16] and cfg.image_dtype == 1 and cfg.autotune == 0
    with pytest.raises(ValueError):
        reg.make_config(image_dtype="f16")
