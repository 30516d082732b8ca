"""Pins of the oracle's NUTS move (CPU only).

The move doubles a leapfrog trajectory in random directions until a U-turn, a divergent
point or the maximum depth, and draws the new point with weights exp(-H) (uniform
progressive sampling inside a doubling, biased progressive sampling at the merge).  Its
random numbers come in as arguments, so each pin fixes them:
  * one doubling is a Metropolis step to the one-step leapfrog point in the drawn direction
    (that point from the plain forward leapfrog by time reversal: a backward step from
    (theta, v) is a forward step from (theta, -v) with the velocity negated);
  * where it stops (point, kind) and how deep it gets equal a recursive reference written
    from the textbook definition (each sub-trajectory checked when it is complete, the first
    failing one ending the move) for every direction sequence;
  * the probabilities of each point being selected equal those of the sampling rules,
    enumerated, against frequencies over many uniforms;
  * inside the sampler, with the exact Gaussian likelihood, the weighted posterior recovers
    the closed-form mean and variance (a wrong selection or merge rule changes the spread);
  * special cases: a divergent first point, a start whose log pi is not finite, and the
    follow mode (a near decision follows the hint and counts a tie, a far one a mismatch).
"""
import itertools
import math

import numpy as np

import oracle.smc2 as smc2


def _gauss(mu, sd):
    """log N(theta; mu, diag(sd^2)) up to a constant, its gradient, and the (ll, g) payload
    (the point index s that the move passes is not needed)."""
    def fn(th, s=None):
        z = (th - mu) / sd
        lp = float(-0.5 * np.sum(z * z))
        g = -z / sd
        return lp, g, (lp, g)
    return fn


def _H(lp, v, gamma):
    return -lp + 0.5 * float(v @ v) / gamma ** 2


def test_one_doubling_is_a_metropolis_step_to_the_leapfrog_point():
    rng = np.random.default_rng(11)
    mu, sd = np.array([0.3, -0.4]), np.array([0.7, 0.5])
    fn = _gauss(mu, sd)
    gamma = 0.4
    moved = 0
    for trial in range(200):
        th0 = rng.standard_normal(2)
        v0 = gamma * rng.standard_normal(2)
        d = 1 if rng.random() < 0.5 else -1
        u_merge = float(rng.random()) or 0.5
        lp0, g0, pay0 = fn(th0)
        res = smc2.nuts_move(th0, v0, lp0, g0, pay0, fn, gamma, 1, [d], [0.5], [u_merge])
        # the leapfrog point in direction d by time reversal of the forward leapfrog
        thL, vL, lpL, _, _ = smc2.leapfrog(th0, d * v0, g0, 1, gamma, lambda t, l: fn(t)[:2])
        v1 = d * vL
        accept = math.log(u_merge) <= _H(lp0, v0, gamma) - _H(lpL, v1, gamma)
        want = thL if accept else th0
        np.testing.assert_allclose(res["theta"], want, rtol=0, atol=1e-13)
        np.testing.assert_allclose(res["v"], v1 if accept else v0, rtol=0, atol=1e-13)
        assert res["depth"] == 1 and res["stats"]["points"] == 1
        moved += int(accept)
    assert 20 < moved < 200  # both outcomes occur


def _recursive_nuts_stop(th0, v0, g0, fn, gamma, J, dirs):
    """Where the textbook recursion stops: build_tree(z, d, j) builds the two halves of depth
    j - 1 one after the other (the second from the end of the first), returns at once when a
    half is invalid, and checks the whole sub-trajectory for a U-turn when both are done.
    Returns (stop point, kind, depth, points built)."""
    half = 0.5 * gamma * gamma
    count = [0]
    H0 = _H(fn(th0)[0], v0, gamma)

    def step(z, d):
        th, v, g = z
        vh = v + d * half * g
        th2 = th + d * vh
        lp, g2, _ = fn(th2)
        v2 = vh + d * half * g2
        count[0] += 1
        return (th2, v2, g2), lp

    def uturn(d, first, last):
        dth = d * (last[0] - first[0])
        return float(dth @ first[1]) < 0.0 or float(dth @ last[1]) < 0.0

    def build(z, d, j):
        """-> (first, last, status) with status None (valid) or (point index, kind)"""
        if j == 0:
            z2, lp = step(z, d)
            if not np.isfinite(lp) or _H(lp, z2[1], gamma) - H0 > smc2.NUTS_DELTA_MAX:
                return z2, z2, (count[0] - 1, 2)
            return z2, z2, None
        f1, l1, st = build(z, d, j - 1)
        if st is not None:
            return f1, l1, st
        f2, l2, st = build(l1, d, j - 1)
        if st is not None:
            return f1, l2, st
        if uturn(d, f1, l2):
            return f1, l2, (count[0] - 1, 1)
        return f1, l2, None

    ends = {+1: (th0, v0, g0), -1: (th0, v0, g0)}
    for j in range(J):
        d = dirs[j]
        first, last, st = build(ends[d], d, j)
        if st is not None:
            return st[0], st[1], j, count[0]
        ends[d] = last
        if uturn(+1, ends[-1], ends[+1]):
            return count[0] - 1, 3, j + 1, count[0]
    return count[0] - 1, 0, J, count[0]


def test_stop_point_and_depth_match_the_recursive_definition():
    """All 2^5 direction sequences from several starts on an anisotropic Gaussian (trajectories
    that turn inside a sub-trajectory, at a merge, or reach the depth limit)."""
    rng = np.random.default_rng(2)
    mu, sd = np.array([0.0, 0.5, -0.2]), np.array([1.0, 0.3, 0.6])
    fn = _gauss(mu, sd)
    J = 5
    kinds = set()
    for start in range(6):
        th0 = mu + sd * rng.standard_normal(3)
        gamma = [0.15, 0.3, 0.05][start % 3]
        v0 = gamma * rng.standard_normal(3)
        lp0, g0, pay0 = fn(th0)
        for dirs in itertools.product([-1, 1], repeat=J):
            res = smc2.nuts_move(th0, v0, lp0, g0, pay0, fn, gamma, J, list(dirs), [0.5] * (2 ** J - 1),
                                 [0.5] * J)
            want = _recursive_nuts_stop(th0, v0, g0, fn, gamma, J, dirs)
            got = (res["stop"][0], res["stop"][1], res["depth"], res["stats"]["points"])
            assert got == want, (start, dirs, got, want)
            kinds.add(want[1])
    assert {0, 1, 3} <= kinds, kinds


def test_selection_probabilities_follow_the_sampling_rules():
    """Two doublings (directions +1, +1; no U-turn in 3 points): point weights w = exp(-H).
    Doubling 0 merges {p0} into {z0}: p0 is taken with probability min(1, w_p0 / w_z0).
    Doubling 1 builds {p1, p2}: its candidate is p2 with probability w_p2 / (w_p1 + w_p2)
    (uniform progressive sampling), and it replaces the selected point with probability
    min(1, (w_p1 + w_p2) / (w_z0 + w_p0)) (biased progressive sampling)."""
    mu, sd = np.zeros(2), np.array([1.0, 0.8])
    fn = _gauss(mu, sd)
    gamma = 0.45
    th0, v0 = np.array([0.6, -0.3]), np.array([0.1, 0.25])
    lp0, g0, pay0 = fn(th0)
    # the three points and their weights (forward leapfrog, one step at a time)
    pts, H = [], []
    z = (th0, v0, g0)
    for _ in range(3):
        thL, vL, lpL, gL, _ = smc2.leapfrog(z[0], z[1], z[2], 1, gamma, lambda t, l: fn(t)[:2])
        pts.append(thL)
        H.append(_H(lpL, vL, gamma))
        z = (thL, vL, gL)
    w0 = math.exp(-_H(lp0, v0, gamma))
    wp = [math.exp(-h) for h in H]
    a0 = min(1.0, wp[0] / w0)
    c2 = wp[2] / (wp[1] + wp[2])
    a1 = min(1.0, (wp[1] + wp[2]) / (w0 + wp[0]))
    want = {0: (1 - a0) * (1 - a1), 1: a0 * (1 - a1), 2: a1 * (1 - c2), 3: a1 * c2}
    rng = np.random.default_rng(4)
    n = 20000
    counts = {k: 0 for k in want}
    for _ in range(n):
        u_sel = [float(1.0 - rng.random()) for _ in range(3)]
        u_merge = [float(1.0 - rng.random()) for _ in range(2)]
        res = smc2.nuts_move(th0, v0, lp0, g0, pay0, fn, gamma, 2, [1, 1], u_sel, u_merge)
        assert res["stop"] == (2, 0), res["stop"]  # maximum depth, no U-turn
        k = 0 if np.array_equal(res["theta"], th0) else 1 + [np.array_equal(res["theta"], p) for p in pts].index(True)
        counts[k] += 1
    for k, p in want.items():
        sd_k = math.sqrt(p * (1 - p) / n)
        assert abs(counts[k] / n - p) < 4 * sd_k + 1e-3, (k, counts[k] / n, p)


def _gauss_ll(mu_l, s_l):
    def fn(th):
        z = (th - mu_l) / s_l
        return float(np.sum(-0.5 * z * z)), -z / s_l
    return fn


def test_nuts_sampler_recovers_conjugate_gaussian_posterior():
    """NUTS moves with the exact Gaussian likelihood (NUTS-reversal weights): the recycled
    estimate and the weighted spread match the closed-form posterior.  Taking every new
    point as the candidate, or accepting every merge, leaves a spread 13-21% too wide."""
    mu_l = np.array([0.8, -0.5, 0.3])
    s_l = np.array([0.3, 0.4, 0.25])
    prec = 1.0 + 1.0 / s_l ** 2
    post_mean = (mu_l / s_l ** 2) / prec
    post_var = 1.0 / prec
    N = 3000
    recs, rec_mean = smc2.run(0, 1, 1, None, np.zeros((1, 1), np.float32), N, 1, 15, 0.3, "nuts", 124,
                              loglik_grad_fn=_gauss_ll(mu_l, s_l), D=3, nuts_depth=4)
    assert np.all(np.abs(rec_mean - post_mean) < 0.1 * np.sqrt(post_var))
    last = recs[-1]
    w = np.exp(last["logw"] - last["logw"].max())
    w /= w.sum()
    var = w @ (last["theta"] - last["mean"]) ** 2
    assert np.all((var / post_var > 0.9) & (var / post_var < 1.1)), var / post_var
    kinds = np.bincount([r["stop"][1] for r in last["nuts"]], minlength=5)
    assert kinds[1] > 0 and kinds[3] > 0  # U-turns inside doublings and of whole trajectories


def test_divergent_first_point_keeps_the_start():
    fn = _gauss(np.zeros(1), np.array([1e-3]))  # curvature 1e6: one step of 0.5 diverges
    th0, v0 = np.array([0.01]), np.array([0.3])
    lp0, g0, pay0 = fn(th0)
    res = smc2.nuts_move(th0, v0, lp0, g0, pay0, fn, 0.5, 3, [1, 1, 1], [0.5] * 7, [0.5] * 3)
    assert res["stop"] == (0, 2) and res["depth"] == 0
    np.testing.assert_array_equal(res["theta"], th0)


def test_start_without_finite_log_pi_is_not_moved():
    fn = _gauss(np.zeros(2), np.ones(2))
    th0 = np.array([0.1, 0.2])
    res = smc2.nuts_move(th0, np.array([0.1, 0.1]), -np.inf, np.zeros(2), (0.0, np.zeros(2)), fn, 0.3, 3,
                         [1, 1, 1], [0.5] * 7, [0.5] * 3)
    assert res["stop"] == (-1, 4) and res["stats"]["points"] == 0
    np.testing.assert_array_equal(res["theta"], th0)


def test_follow_mode_counts_ties_and_mismatches():
    """One doubling whose merge accepts by a margin of 1e-7 (log u just below H_0 - H_1): a hint
    that rejects is followed and counted as a tie.  The same hint against a margin of 1 is
    followed and counted as a mismatch."""
    fn = _gauss(np.zeros(2), np.array([1.0, 0.8]))
    gamma = 1.5
    th0, v0 = np.array([0.6, -0.3]), np.array([0.1, 0.25]) * (gamma / 0.45)
    lp0, g0, pay0 = fn(th0)
    thL, vL, lpL, _, _ = smc2.leapfrog(th0, v0, g0, 1, gamma, lambda t, l: fn(t)[:2])
    dH = _H(lp0, v0, gamma) - _H(lpL, vL, gamma)
    assert dH < -0.1  # the merge margin dH - log u is then adjustable through u in (0, 1]
    for log_u, kind in ((dH - 1e-7, "nuts_ties"), (dH - 1.0, "nuts_mismatch")):
        own = smc2.nuts_move(th0, v0, lp0, g0, pay0, fn, gamma, 1, [1], [0.5], [math.exp(log_u)])
        assert own["trace"]["merge"] == 1 and own["stats"]["nuts_ties"] == 0
        np.testing.assert_array_equal(own["theta"], thL)
        reject = dict(own["trace"], merge=0)  # the same decisions but the merge
        fol = smc2.nuts_move(th0, v0, lp0, g0, pay0, fn, gamma, 1, [1], [0.5], [math.exp(log_u)], hint=reject)
        assert fol["trace"]["merge"] == 0 and fol["stats"][kind] == 1, (kind, fol["stats"])
        assert fol["stats"]["nuts_ties"] + fol["stats"]["nuts_mismatch"] == 1
        np.testing.assert_array_equal(fol["theta"], th0)
