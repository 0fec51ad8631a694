"""Pins of the loop-signature and query oracle (Sec. III-D, Sec. I)."""
import numpy as np

from oracle import loop


def test_codewords_assign_to_themselves():
    rng = np.random.default_rng(0)
    c = rng.standard_normal((32, 512))
    idx, margin = loop.assign(c, c)
    np.testing.assert_array_equal(idx, np.arange(32))
    assert (margin > 0).all()


def test_two_codeword_bisector():
    """Points on either side of the perpendicular bisector of two codewords."""
    c = np.array([[1.0, 0.0], [0.0, 1.0]])
    x = np.array([[0.9, 0.1], [0.2, 0.7], [0.5, 0.5]])
    idx, margin = loop.assign(x, c)
    assert list(idx) == [0, 1, 0]  # the tie on the bisector goes to the lower index
    np.testing.assert_allclose(margin, [1.6, 1.0, 0.0], atol=1e-12)


def test_assignment_brute_force():
    rng = np.random.default_rng(1)
    x, c = rng.standard_normal((50, 20)), rng.standard_normal((7, 20))
    idx, _ = loop.assign(x, c)
    for i in range(50):
        d = [sum((x[i, j] - c[k, j]) ** 2 for j in range(20)) for k in range(7)]
        assert idx[i] == int(np.argmin(d))


def test_signature_and_cosine():
    rng = np.random.default_rng(2)
    c = rng.standard_normal((8, 16))
    x = c[rng.integers(0, 8, 1000)] + 0.01 * rng.standard_normal((1000, 16))
    s = loop.signature(x, c)
    assert abs(s.sum() - 1) < 1e-12
    h = loop.histogram(loop.assign(x, c)[0], 8)
    np.testing.assert_allclose(s, h / 1000)
    assert abs(loop.cosine(s, s)[0] - 1) < 1e-15
    a, b = np.array([1.0, 0, 2, 0]), np.array([[0, 3.0, 0, 1], [2, 0, 4, 0], [0, 0, 0, 0]])
    np.testing.assert_allclose(loop.cosine(a, b), [0.0, 1.0, 0.0], atol=1e-15)


def test_loop_candidates():
    sim = np.array([0.9, 0.95, 0.5, 0.95, 0.99, 0.97])
    centres = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.5, 0, 0], [10, 0, 0], [0, 0, 0.2]])
    cur = np.zeros(3)
    # 4 is the most similar but far away; 1 and 3 tie at 0.95 behind 5
    np.testing.assert_array_equal(loop.loop_candidates(sim, centres, cur, 0.8, 2.0), [5, 1])
    np.testing.assert_array_equal(loop.loop_candidates(sim, centres, cur, 0.8, 2.0, top=3),
                                  [5, 1, 3])
    np.testing.assert_array_equal(loop.loop_candidates(sim, centres, cur, 0.98, 2.0), [-1, -1])
    np.testing.assert_array_equal(loop.loop_candidates(sim, centres, cur, 0.96, 2.0), [5, -1])


def test_query_relevance():
    f = np.array([[1.0, 0, 0], [0, 2.0, 0], [3.0, 3.0, 0], [0, 0, 0]])
    q = np.array([[2.0, 0, 0], [0, 0, 1.0]])
    r = loop.query_relevance(f, q)
    np.testing.assert_allclose(r, [[1, 0], [0, 0], [np.sqrt(0.5), 0], [0, 0]], atol=1e-15)
    rng = np.random.default_rng(3)
    f, q = rng.standard_normal((20, 16)), rng.standard_normal((3, 16))
    np.testing.assert_allclose(loop.query_relevance(5 * f, 0.1 * q), loop.query_relevance(f, q),
                               rtol=1e-13)
