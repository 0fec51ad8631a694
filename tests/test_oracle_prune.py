"""Pins of the pruning oracle (Sec. III-C, Eq. 4, with the geometric
criteria) against hand-built cases and an independent float64 brute force."""
import math

import numpy as np
import pytest

import oracle

LS_SMALL = math.log(0.01)


def _scene(points, feats, logits, log_scales=None):
    p = np.asarray(points, np.float32)
    n = p.shape[0]
    ls = (np.full((n, 3), LS_SMALL, np.float32) if log_scales is None
          else np.asarray(log_scales, np.float32))
    return p, np.asarray(logits, np.float32), ls, np.asarray(feats, np.float32)


def test_pair_lower_opacity_is_pruned():
    f = np.eye(16)[[0, 0]]
    p, lg, ls, f = _scene([[0, 0, 0], [0.01, 0, 0]], f, [1.0, 0.5])
    assert list(oracle.prune(p, lg, ls, f, tau_dist=0.05, tau_sim=0.9)) == [0, 2]
    # swap the opacities: the other one goes
    assert list(oracle.prune(p, lg[::-1].copy(), ls, f, tau_dist=0.05, tau_sim=0.9)) == [2, 0]
    # equal opacity: the higher index goes
    assert list(oracle.prune(p, np.array([0.3, 0.3], np.float32), ls, f,
                             tau_dist=0.05, tau_sim=0.9)) == [0, 2]


def test_pair_distance_and_similarity_thresholds():
    f_same = np.eye(16)[[0, 0]]
    for dx, expect in ((0.049, [0, 2]), (0.051, [0, 0])):
        p, lg, ls, f = _scene([[0, 0, 0], [0, 0, dx]], f_same, [1.0, 0.0])
        assert list(oracle.prune(p, lg, ls, f, tau_dist=0.05, tau_sim=0.9)) == expect
    # cosine 0.91 / 0.89 against tau_sim = 0.9
    for c, expect in ((0.91, [0, 2]), (0.89, [0, 0])):
        f = np.stack([np.eye(16)[0], c * np.eye(16)[0] + math.sqrt(1 - c * c) * np.eye(16)[1]])
        p, lg, ls, f = _scene([[0, 0, 0], [0.01, 0, 0]], f, [1.0, 0.0])
        assert list(oracle.prune(p, lg, ls, f, tau_dist=0.05, tau_sim=0.9)) == expect
    # opposite features, zero feature: never similar
    for f in (np.stack([np.eye(16)[0], -np.eye(16)[0]]), np.stack([np.eye(16)[0], np.zeros(16)])):
        p, lg, ls, f = _scene([[0, 0, 0], [0.01, 0, 0]], f, [1.0, 0.0])
        assert list(oracle.prune(p, lg, ls, f, tau_dist=0.05, tau_sim=0.9)) == [0, 0]


def _satellites(k_sat=6, cphi=0.92):
    """A centre (highest opacity) and satellites at 1..k_sat cm along
    different directions, each similar to the centre (cos 0.92) but not to
    one another (cos 0.8464)."""
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    pts = [[0, 0, 0]] + [0.01 * (i + 1) * dirs[i] for i in range(k_sat)]
    sphi = math.sqrt(1 - cphi * cphi)
    f = [np.eye(16)[0]] + [cphi * np.eye(16)[0] + sphi * np.eye(16)[i + 1] for i in range(k_sat)]
    lg = [2.0] + [0.1 * i for i in range(k_sat)]
    return _scene(pts, f, lg)


def test_only_the_k_nearest_are_marked():
    p, lg, ls, f = _satellites()
    for k, expect in ((3, [0, 2, 2, 2, 0, 0, 0]), (1, [0, 2, 0, 0, 0, 0, 0]),
                      (8, [0, 2, 2, 2, 2, 2, 2])):
        assert list(oracle.prune(p, lg, ls, f, k=k, tau_dist=0.065, tau_sim=0.9)) == expect


def test_neighbour_ranking_ties_break_by_index():
    # two satellites at exactly the same distance: with K = 1 the lower index wins
    pts = [[0, 0, 0], [0.02, 0, 0], [-0.02, 0, 0]]
    f = np.eye(16)[[0, 0, 0]]
    p, lg, ls, f = _scene(pts, f, [3.0, 1.0, 1.0])
    # 1 and 2 are 4 cm apart; with tau 0.03 they do not see each other
    assert list(oracle.prune(p, lg, ls, f, k=1, tau_dist=0.03, tau_sim=0.9)) == [0, 2, 0]


def test_geometric_criteria():
    thr_lo, thr_hi = oracle.prune_thresholds(0.005, 0.5)
    assert thr_lo == pytest.approx(math.log(0.005 / 0.995), rel=1e-6)
    assert thr_hi == pytest.approx(math.log(0.5), rel=1e-6)
    pts = [[0, 0, 0], [1, 0, 0], [2, 0, 0], [3, 0, 0], [3.01, 0, 0]]
    lg = [math.log(0.004 / 0.996), 0.0, 0.0, 0.0, math.log(0.004 / 0.996)]
    ls = [[LS_SMALL] * 3, [LS_SMALL, math.log(0.6), LS_SMALL], [math.log(0.4)] * 3,
          [LS_SMALL] * 3, [LS_SMALL] * 3]
    f = np.eye(16)[[0, 1, 2, 3, 3]]
    p, lg, ls, f = _scene(pts, f, lg, ls)
    m = oracle.prune(p, lg, ls, f, tau_dist=0.05, tau_sim=0.9, min_opacity=0.005, max_scale=0.5)
    # 0 transparent, 1 too large, 2 fine, 4 transparent and redundant next to 3
    assert list(m) == [1, 1, 0, 0, 3]
    # switched off
    m = oracle.prune(p, lg, ls, f, tau_dist=0.05, tau_sim=0.9, min_opacity=0.0,
                     max_scale=float("inf"))
    assert list(m) == [0, 0, 0, 0, 2]


def _brute_force64(p, lg, f, k, tau, tau_sim):
    """Eq. 4 with the same readings, float64 throughout, written directly."""
    p = p.astype(np.float64)
    f = f.astype(np.float64)
    n = p.shape[0]
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    nf = np.linalg.norm(f, axis=1)
    cos = (f @ f.T) / np.maximum(np.outer(nf, nf), 1e-300)
    red = np.zeros(n, bool)
    for i in range(n):
        cand = [j for j in range(n) if j != i and d[i, j] < tau]
        cand.sort(key=lambda j: (d[i, j], j))
        for j in cand[:k]:
            if cos[i, j] > tau_sim and (lg[i] > lg[j] or (lg[i] == lg[j] and i < j)):
                red[j] = True
    return red, d, cos


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_against_float64_brute_force(seed):
    """Clustered random scenes on a 1/64 m lattice (squared distances exact
    in float32), 16-d features drawn around 6 centroids: the FP32 oracle must
    equal a float64 brute force wherever no cosine lies within 1e-5 of
    tau_sim (checked), for several K."""
    rng = np.random.default_rng(seed)
    n = 400
    centres = rng.integers(0, 16, size=(8, 3))
    p = (centres[rng.integers(0, 8, n)] + rng.integers(-3, 4, size=(n, 3))) / 64.0
    cent = rng.standard_normal((6, 16))
    f = cent[rng.integers(0, 6, n)] + 0.25 * rng.standard_normal((n, 16))
    lg = np.round(rng.standard_normal(n), 1)  # ties in opacity happen
    p, lg, ls, f = _scene(p, f, lg)
    tau, tau_sim = 0.05, 0.9
    red64, d, cos = _brute_force64(p, lg, f, 16, tau, tau_sim)
    near = (d < tau) & (np.abs(cos - tau_sim) < 1e-5)
    assert not near.any()
    for k in (1, 4, 16):
        red64, _, _ = _brute_force64(p, lg, f, k, tau, tau_sim)
        m = oracle.prune(p, lg, ls, f, k=k, tau_dist=tau, tau_sim=tau_sim, min_opacity=0.0)
        assert m.max() <= 2
        np.testing.assert_array_equal(m == 2, red64)
    assert 0.05 < red64.mean() < 0.9  # the scene exercises the rule


def test_sampled_decisions_equal_the_full_mask():
    rng = np.random.default_rng(7)
    n = 3000
    p = rng.random((n, 3)).astype(np.float32) * 0.4
    f = (np.eye(16)[rng.integers(0, 3, n)] + 0.2 * rng.standard_normal((n, 16))).astype(np.float32)
    lg = rng.standard_normal(n).astype(np.float32)
    ls = (math.log(0.01) + 0.8 * rng.standard_normal((n, 3))).astype(np.float32)
    full = oracle.prune(p, lg, ls, f, k=8, tau_dist=0.04, tau_sim=0.8, min_opacity=0.1,
                        max_scale=0.03)
    assert (full & 2).any() and (full & 1).any()
    idx = rng.integers(0, n, 200)
    np.testing.assert_array_equal(
        oracle.prune(p, lg, ls, f, k=8, tau_dist=0.04, tau_sim=0.8, min_opacity=0.1,
                     max_scale=0.03, idx=idx), full[idx])


def test_permutation_with_distinct_opacities():
    """With distinct logits the rule does not depend on storage order."""
    rng = np.random.default_rng(3)
    n = 500
    p = rng.random((n, 3)).astype(np.float32) * 0.3
    f = (np.eye(16)[rng.integers(0, 2, n)] + 0.08 * rng.standard_normal((n, 16))).astype(np.float32)
    lg = rng.permutation(n).astype(np.float32) / n
    ls = np.full((n, 3), LS_SMALL, np.float32)
    m = oracle.prune(p, lg, ls, f, k=6, tau_dist=0.04, tau_sim=0.85)
    perm = rng.permutation(n)
    mp = oracle.prune(p[perm], lg[perm], ls[perm], f[perm], k=6, tau_dist=0.04, tau_sim=0.85)
    np.testing.assert_array_equal(mp, m[perm])
    assert (m == 2).sum() > 10
