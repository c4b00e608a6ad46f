"""Pins of the oracle's L-BFGS rules (Sec. 2.1 "L-BFGS"; readings R9, R10).

The rules the paper leaves open are fixed by readings R9 and R10: the first
step, the curvature test that decides whether a pair is stored, the retry
after a failed line search and the two stopping tests.  Each test runs the
oracle's L-BFGS driver on an objective built by hand (a small quadratic, or a
scripted sequence of values and gradients), where the iterates, evaluation
counts or stopping index follow from the rule by hand.  A plausible slip in
any rule (the 2-norm for the infinity norm in the first step, a dropped or
inverted curvature test, a stopping test against the previous iterate instead
of the first, a counter that is not reset) changes a checked value.
"""
import numpy as np
import pytest


def quad(A):
    A = np.asarray(A, np.float64)
    return lambda x: (0.5 * x @ (A @ x), A @ x)


def scripted(Js, gs):
    """Objective whose k-th evaluation returns Js[k] and gs[k] (whatever x is)."""
    calls = []

    def fun(x):
        k = len(calls)
        calls.append(x.copy())
        return Js[k], np.asarray(gs[k], np.float64)
    return fun, calls


def test_first_step_is_g_scaled_to_one_node_spacing_in_the_inf_norm(orc):
    # f = x'Ax / 2, A = diag(1, 2, 1/2), x0 = (3, -1, 2): g0 = (3, -2, 1), ||g0||_inf = 3.
    # With Hmin = 0.6 the first direction is -0.2 g0 = (-0.6, 0.4, -0.2); t = 1 passes
    # Armijo (f drops by 2.45, c1 g'p = -2.8e-4), so x1 = (2.4, -0.6, 1.8) after 2 evaluations.
    cfg = orc.make_config(mem=5, fixed_iters=True)
    x, st = orc.lbfgs(quad(np.diag([1.0, 2.0, 0.5])), [3.0, -1.0, 2.0], 0.6, cfg, 1)
    assert st["iters"] == 1 and st["evals"] == 2 and st["status"] == 0
    np.testing.assert_allclose(x, [2.4, -0.6, 1.8], rtol=0, atol=1e-15)
    # the step's largest entry is exactly Hmin (a 2-norm scaling would give 0.6 * 3 / sqrt(14))
    assert abs(np.max(np.abs(x - [3.0, -1.0, 2.0])) - 0.6) <= 1e-15


@pytest.mark.parametrize("delta,stored", [(1e-11, False), (-1e-3, False), (1e-3, True)])
def test_pair_is_stored_only_if_it_passes_the_curvature_test(orc, delta, stored):
    # f = (x1^2 - a x2^2) / 2 with a^3 = 1 - delta, x0 = (1, 1), Hmin = 1.
    # g0 = (1, -a), ||g0||_inf = 1 (a < 1) or a (a > 1); the first step is accepted at t = 1
    # and the pair is s = p0, y = A s with s'y = (1 - a^3) / ||g0||_inf^2 (one node spacing).
    # The test keeps it only if s'y > 1e-10 ||s|| ||y||:
    #   delta = 1e-11: s'y = 1e-11 < 2e-10 (just below), not stored;
    #   delta = -1e-3: s'y < 0, not stored;
    #   delta = 1e-3: stored.
    # Without a stored pair the second step is the first-step rule again at
    # x1 = x0 + p0: g1 = (x1_1, -a x1_2), and x2 = x1 - g1 / ||g1||_inf.
    a = (1.0 - delta) ** (1.0 / 3.0)
    A = np.diag([1.0, -a])
    cfg = orc.make_config(mem=5, fixed_iters=True)
    x1, st1 = orc.lbfgs(quad(A), [1.0, 1.0], 1.0, cfg, 1)
    g0 = np.array([1.0, -a])
    p0 = -g0 / np.max(np.abs(g0))
    np.testing.assert_allclose(x1, [1.0, 1.0] + p0, rtol=0, atol=1e-15)
    s, y = p0, A @ p0
    assert (s @ y > 1e-10 * np.linalg.norm(s) * np.linalg.norm(y)) == stored
    x2, st2 = orc.lbfgs(quad(A), [1.0, 1.0], 1.0, cfg, 2)
    assert st2["iters"] == 2 and st2["status"] == 0
    g1 = A @ x1
    memoryless = x1 - g1 / np.max(np.abs(g1))
    if stored:
        assert np.max(np.abs(x2 - memoryless)) > 1e-3
    else:
        assert st2["evals"] == 3
        np.testing.assert_allclose(x2, memoryless, rtol=0, atol=1e-14)


def test_gradient_stopping_rule_compares_with_the_first_gradient(orc):
    # Scripted: J falls by 100 per evaluation (every step is accepted at t = 1) and the
    # gradients point along e1 with norms 1, 0.1, 1e-3, 2e-5, 9e-6, 1e-7.  The rule
    # ||g_k|| <= 1e-5 ||g_0|| first holds at k = 4 (9e-6); a comparison with the previous
    # gradient (9e-6 / 2e-5) would not stop there, a missing rule would run to the cap.
    norms = [1.0, 0.1, 1e-3, 2e-5, 9e-6, 1e-7, 1e-8, 1e-9]
    Js = [1000.0 - 100.0 * k for k in range(len(norms))]
    fun, calls = scripted(Js, [[c, 0.0] for c in norms])
    cfg = orc.make_config(mem=5, tol_grad_rel=1e-5, tol_j_rel=1e-7, tol_j_count=3)
    x, st = orc.lbfgs(fun, [0.0, 0.0], 0.5, cfg, 7)
    assert st["status"] == 0 and st["iters"] == 4 and st["evals"] == 5
    assert st["J"] == Js[4]
    # with the rules switched off the driver runs to the cap
    fun, calls = scripted(Js, [[c, 0.0] for c in norms])
    x, st = orc.lbfgs(fun, [0.0, 0.0], 0.5, orc.make_config(mem=5, fixed_iters=True), 7)
    assert st["iters"] == 7 and st["evals"] == 8


def test_objective_stopping_rule_counts_consecutive_small_changes_against_J0(orc):
    # Scripted: J0 = 1000, so a change is small when |J_{k-1} - J_k| <= 1e-7 (1 + 1000)
    # = 1.001e-4.  Changes: 999 (large), 5e-5, 5e-5 (small, small), 0.5 (large: the count
    # restarts), then 5e-5 three times: the third consecutive small change stops the level
    # at k = 7.  Without the restart it would stop at k = 5, with a threshold relative to
    # |J_k| (~1) never (the cap, 12), after two small changes at k = 3.
    # The gradient is constant, so y = 0, no pair is stored and every step is
    # -Hmin e1 (g'p = -0.1; Armijo needs a drop of 1e-5 <= 5e-5).
    d = [999.0, 5e-5, 5e-5, 0.5, 5e-5, 5e-5, 5e-5, 5e-5, 5e-5, 5e-5, 5e-5, 5e-5, 5e-5]
    Js = [1000.0]
    for v in d:
        Js.append(Js[-1] - v)
    fun, calls = scripted(Js, [[1.0, 0.0]] * len(Js))
    cfg = orc.make_config(mem=5, tol_grad_rel=1e-5, tol_j_rel=1e-7, tol_j_count=3)
    x, st = orc.lbfgs(fun, [0.0, 0.0], 0.1, cfg, 12)
    assert st["status"] == 0 and st["iters"] == 7 and st["evals"] == 8
    np.testing.assert_allclose(x, [-0.7, 0.0], rtol=0, atol=1e-14)


def test_failed_search_with_memory_retries_once_from_the_first_step_rule(orc):
    # Scripted: evaluation 0 at x0 = 0 (J 10, g (1, 0)), evaluation 1 at the first step
    # x1 = (-Hmin, 0) (J 9, g (0.5, 0)): the pair s = (-Hmin, 0), y = (-0.5, 0) is stored.
    # The next direction comes from the stored pair; its line search sees J = 100 on all
    # 5 trials and fails.  The driver then forgets the pair and retries once with the
    # first-step rule, -Hmin g1 / ||g1||_inf = (-Hmin, 0), whose first trial (J 8) is
    # accepted: x2 = (-2 Hmin, 0) after 2 + 5 + 1 evaluations.
    Hmin, nb = 0.25, 5
    Js = [10.0, 9.0] + [100.0] * nb + [8.0]
    gs = [[1.0, 0.0], [0.5, 0.0]] + [[0.3, 0.0]] * nb + [[0.2, 0.0]]
    fun, calls = scripted(Js, gs)
    cfg = orc.make_config(mem=5, max_backtracks=nb, fixed_iters=True)
    x, st = orc.lbfgs(fun, [0.0, 0.0], Hmin, cfg, 2)
    assert st["status"] == 0 and st["iters"] == 2 and st["evals"] == 2 + nb + 1
    np.testing.assert_allclose(x, [-2 * Hmin, 0.0], rtol=0, atol=1e-15)
    # the failed search halved t from 1: its trial points are x1 + t p, t = 1, 1/2, ...
    steps = [calls[2 + j][0] - calls[1][0] for j in range(nb)]
    np.testing.assert_allclose(np.array(steps[1:]) / np.array(steps[:-1]), 0.5, rtol=1e-12)
    # a second failure ends the level with the warning and leaves x at x1
    Js2 = [10.0, 9.0] + [100.0] * (2 * nb)
    gs2 = [[1.0, 0.0], [0.5, 0.0]] + [[0.3, 0.0]] * (2 * nb)
    fun, calls = scripted(Js2, gs2)
    x, st = orc.lbfgs(fun, [0.0, 0.0], Hmin, cfg, 2)
    assert st["status"] == 1 and st["iters"] == 1 and st["evals"] == 2 + 2 * nb
    np.testing.assert_allclose(x, [-Hmin, 0.0], rtol=0, atol=1e-15)


def dense_bfgs_inverse(pairs, gamma, n):
    """H of the BFGS inverse update applied to H0 = gamma I, pairs oldest first."""
    H = gamma * np.eye(n)
    for s, y in pairs:
        r = 1.0 / (s @ y)
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    return H


def test_retry_after_a_failed_search_forgets_the_old_pairs(orc):
    # As above in 2-D, one iteration further.  Evaluation 0: x0 = 0, g0 = (1, 0);
    # evaluation 1: x1 = (-H, 0), g1 = (0.5, 0.5), pair 1 s1 = (-H, 0), y1 = (-0.5, 0.5)
    # (s'y = H/2 > 0, stored).  The direction from pair 1 fails all 5 trials; the retry
    # takes -H g1 / ||g1||_inf = (-H, -H) to x2 = (-2H, -H) with g2 = (0.2, 0.1), and
    # stores pair 2 s2 = (-H, -H), y2 = (-0.3, -0.4).  The memory was reset before the
    # retry, so the third direction uses pair 2 alone: x3 = x2 - H2 g2 with H2 the BFGS
    # inverse of pair 2 on gamma = s2'y2 / y2'y2 (the dense formula).
    Hm, nb = 0.25, 5
    Js = [10.0, 9.0] + [100.0] * nb + [8.0, 7.0]
    gs = [[1.0, 0.0], [0.5, 0.5]] + [[0.3, 0.0]] * nb + [[0.2, 0.1], [0.0, 0.0]]
    fun, calls = scripted(Js, gs)
    cfg = orc.make_config(mem=5, max_backtracks=nb, fixed_iters=True)
    x, st = orc.lbfgs(fun, [0.0, 0.0], Hm, cfg, 3)
    assert st["status"] == 0 and st["iters"] == 3 and st["evals"] == 2 + nb + 2
    x2 = np.array([-2 * Hm, -Hm])
    np.testing.assert_allclose(calls[-2], x2, rtol=0, atol=1e-15)
    s1, y1 = np.array([-Hm, 0.0]), np.array([-0.5, 0.5])
    s2, y2 = np.array([-Hm, -Hm]), np.array([-0.3, -0.4])
    g2 = np.array([0.2, 0.1])
    gamma = (s2 @ y2) / (y2 @ y2)
    x3 = x2 - dense_bfgs_inverse([(s2, y2)], gamma, 2) @ g2
    np.testing.assert_allclose(x, x3, rtol=0, atol=1e-13)
    # keeping pair 1 would give a different third step
    x3_kept = x2 - dense_bfgs_inverse([(s1, y1), (s2, y2)], gamma, 2) @ g2
    assert np.max(np.abs(x3_kept - x3)) > 1e-3
