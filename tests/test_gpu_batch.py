"""Batched registration of pairs of uneven size against one-at-a-time registration.

Each batched item runs the per-pair code with the pair's own buffers, tiling and
block counts, and reductions keep a fixed order, so a pair's displacement from
the batch equals, bit for bit, the one reg_register gives for it alone.
"""
import numpy as np
import pytest

from synth import CONFIGS, make_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def reg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06765_gb300 as reg
    return reg


SIZES = [(48, 40, 32), (64, 64, 48), (32, 32, 32), (56, 48, 40), (40, 40, 64)]


def _pairs():
    return [make_pair(4, pair=i, dims=d) for i, d in enumerate(SIZES)]


def _cfg(reg_mod, **kw):
    c = CONFIGS[4]
    args = dict(levels=c["levels"], tau=c["eta"], alpha=c["alpha"], mem=c["mem"], max_iter=25, c1=c["c1"])
    args.update(kw)
    return reg_mod.make_config(**args)


@pytest.mark.parametrize("image_dtype", ["f32", "bf16"])
def test_batch_equals_single_registrations(reg_mod, image_dtype):
    # the batch tiles every level by the throughput rule and forms the curvature
    # sum in the fused pass; single registrations with that rule (fused_tz = -1)
    # must give the same result bit for bit
    pairs = _pairs()
    single = []
    for p in pairs:
        r = reg_mod.Registration(_cfg(reg_mod, image_dtype=image_dtype, fused_tz=-1)).set_images(p["R"], p["T"],
                                                                                              p["spacing"])
        single.append(r.register(out="numpy"))
        r.close()
    regs = [reg_mod.Registration(_cfg(reg_mod, image_dtype=image_dtype, fused_tz=-1)).set_images(
        p["R"], p["T"], p["spacing"]) for p in pairs]
    batch = reg_mod.register_batch(regs, out="numpy")
    assert all(s["tiling"] == [-1, -1, -1] for _, s in batch)
    for (u1, s1), (u2, s2) in zip(single, batch):
        np.testing.assert_array_equal(u1, u2)
        assert s1["iters"] == s2["iters"] and s1["evals"] == s2["evals"]
        assert s1["J"] == s2["J"]
    # (launch counts no longer order the two forms: a single registration runs
    # each small level as one whole-level kernel)
    assert batch[0][1]["kernel_launches"] > 0
    for r in regs:
        r.close()


def test_batch_rejects_mixed_or_repeated_inputs(reg_mod):
    from paper_1812_06765_gb300 import _lib
    pairs = _pairs()[:2]
    regs = [reg_mod.Registration(_cfg(reg_mod)).set_images(p["R"], p["T"], p["spacing"]) for p in pairs]
    with pytest.raises(_lib.RegError) as ei:
        reg_mod.register_batch([regs[0], regs[0]])
    assert ei.value.code == _lib.REG_ERR_ARG
    odd = make_pair(4, pair=9, dims=(33, 32, 32))   # odd dimension: not a ratio-2 grid
    r_odd = reg_mod.Registration(_cfg(reg_mod)).set_images(odd["R"], odd["T"], odd["spacing"])
    with pytest.raises(_lib.RegError) as ei:
        reg_mod.register_batch([regs[0], r_odd])
    assert ei.value.code == _lib.REG_ERR_ARG
    r_lv = reg_mod.Registration(_cfg(reg_mod, levels=2)).set_images(pairs[1]["R"], pairs[1]["T"], pairs[1]["spacing"])
    with pytest.raises(_lib.RegError):
        reg_mod.register_batch([regs[0], r_lv])
    for r in regs + [r_odd, r_lv]:
        r.close()


def test_batch_host_driven_equals_graph(reg_mod):
    """use_graph = 0 queues the batched level's kernels from the host in the
    graph's order (for profilers): the same result bit for bit."""
    pairs = _pairs()[:3]
    out = []
    for graph in (1, 0):
        regs = [reg_mod.Registration(_cfg(reg_mod, use_graph=graph)).set_images(p["R"], p["T"], p["spacing"])
                for p in pairs]
        out.append(reg_mod.register_batch(regs, out="numpy"))
        for r in regs:
            r.close()
    for (u1, s1), (u2, s2) in zip(*out):
        np.testing.assert_array_equal(u1, u2)
        assert s1["iters"] == s2["iters"] and s1["evals"] == s2["evals"]
        assert s1["kernel_launches"] == s2["kernel_launches"]


def test_batch_autotuned_tiling(reg_mod):
    """Without a forced rule the batch autotuner picks the tiling of each level
    (cached per batch geometry); the handles keep their own tiling."""
    pairs = _pairs()[:4]
    regs = [reg_mod.Registration(_cfg(reg_mod)).set_images(p["R"], p["T"], p["spacing"]) for p in pairs]
    own = [[r.level_tiling(lv) for lv in range(3)] for r in regs]
    first = reg_mod.register_batch(regs, out="numpy")
    assert own == [[r.level_tiling(lv) for lv in range(3)] for r in regs]
    rules = first[0][1]["tiling"]
    assert all(rule in (0, -1, 16, 32, 64, 128) for rule in rules)
    again = reg_mod.register_batch(regs, out="numpy")
    for (u1, s1), (u2, s2) in zip(first, again):
        assert s1["tiling"] == s2["tiling"] == rules
        np.testing.assert_array_equal(u1, u2)
    for r in regs:
        r.close()



def test_batch_reports_numeric_error(reg_mod):
    from paper_1812_06765_gb300 import _lib
    pairs = _pairs()[:2]
    bad = dict(pairs[1])
    bad["T"] = bad["T"].copy()
    bad["T"][5, 6, 7] = np.nan
    regs = [reg_mod.Registration(_cfg(reg_mod)).set_images(p["R"], p["T"], p["spacing"]) for p in (pairs[0], bad)]
    with pytest.raises(_lib.RegError) as ei:
        reg_mod.register_batch(regs, out="numpy")
    assert ei.value.code == _lib.REG_ERR_NUMERIC
    for r in regs:
        r.close()


def test_batch_matches_oracle_per_pair(reg_mod, orc):
    """Each pair of an uneven batch (one of the batch workload's sizes, 96^3, and three
    smaller shapes) registered together through register_batch, against the FP64
    oracle registering that pair alone: a fixed number of accepted steps on each of
    3 levels, mean |u - u_oracle| <= 0.02 voxel, and J to 1e-4 on every level where
    the two took the same number of evaluations (otherwise an Armijo test that FP32
    and FP64 decided differently branched the search: J to 1e-2)."""
    c = CONFIGS[4]
    sizes = [(96, 96, 96), (64, 48, 40), (40, 56, 32), (32, 32, 48)]
    pairs = [make_pair(4, pair=20 + i, dims=d) for i, d in enumerate(sizes)]
    kw = dict(levels=c["levels"], tau=c["eta"], alpha=c["alpha"], mem=c["mem"], c1=c["c1"], max_iter=[6, 8, 8],
              fixed_iters=True)
    regs = [reg_mod.Registration(reg_mod.make_config(**kw)).set_images(p["R"], p["T"], p["spacing"]) for p in pairs]
    batch = reg_mod.register_batch(regs, out="numpy")
    for p, (u, st) in zip(pairs, batch):
        uo, sto = orc.register(p["dims"], p["spacing"], p["R"], p["T"], orc.make_config(**kw))
        assert st["status"] == 0 and sto["status"] == 0
        assert st["iters"] == sto["iters"] == [6, 8, 8]
        du = np.sqrt(((u.astype(np.float64) - uo) ** 2).sum(axis=0)).mean() / min(p["spacing"])
        assert du <= 0.02, (p["dims"], du, st, sto)
        for lv in range(c["levels"]):
            tol = 1e-4 if st["evals"][lv] == sto["evals"][lv] else 1e-2
            assert abs(st["J"][lv] - sto["J"][lv]) <= tol * abs(sto["J"][lv]), (p["dims"], lv, st, sto)
    for r in regs:
        r.close()
