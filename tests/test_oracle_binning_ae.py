"""Pins of the oracle's binning definition and its FP64 autoencoder (no GPU).

Binning is checked against brute force on tiny inputs (Python's own tuple
ordering of every emitted (tile, depth bits, emission index) triple) and
against structural invariants.  The autoencoder is checked against the
standard normal CDF, explicit loops, finite differences on toy widths and the
closed form of Adam's first step.
"""
import math

import numpy as np
import pytest

from paper_2511_16144_gb300 import synth


def brute_force_bins(rect, depth, n, ncams, tx, ty):
    items = []
    e = 0
    for c in range(ncams):
        for i in range(n):
            x0, y0, x1, y1 = rect[c * n + i]
            bits = int(np.float32(depth[c * n + i]).view(np.uint32))
            for yy in range(y0, y1):
                for xx in range(x0, x1):
                    tile = c * tx * ty + yy * tx + xx
                    items.append((tile, bits, e, i))
                    e += 1
    items.sort()
    return items


@pytest.mark.parametrize("seed,n,ncams,tx,ty", [(0, 40, 1, 5, 4), (1, 60, 3, 4, 3),
                                                (2, 1, 1, 1, 1), (3, 30, 2, 7, 2)])
def test_bin_sort_brute_force(oracle_lib, seed, n, ncams, tx, ty):
    rng = np.random.default_rng(seed)
    rect, depth = synth.synthetic_projected(rng, n, ncams, tx, ty, max_extent=3, tie_frac=0.3)
    out = oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty)
    ref = brute_force_bins(rect, depth, n, ncams, tx, ty)
    assert len(out["ids"]) == len(ref)
    np.testing.assert_array_equal(out["ids"], [r[3] for r in ref])
    np.testing.assert_array_equal(out["keys"] >> np.uint64(32), [r[0] for r in ref])
    np.testing.assert_array_equal(out["keys"] & np.uint64(0xFFFFFFFF), [r[1] for r in ref])
    ntile = ncams * tx * ty
    for t in range(ntile):
        members = [k for k, r in enumerate(ref) if r[0] == t]
        if members:
            assert tuple(out["ranges"][t]) == (members[0], members[-1] + 1)
        else:
            assert tuple(out["ranges"][t]) == (0, 0)


def _kept_pairs(out, n, ncams, tx, ty):
    """(item, tile) pairs of a binning result (item = camera * n + index)."""
    tiles = (out["keys"] >> np.uint64(32)).astype(np.int64)
    cams = tiles // (tx * ty)
    return set(zip((cams * n + out["ids"].astype(np.int64)).tolist(), tiles.tolist()))


def _box_min_q(rec, t, tx):
    """min over the tile's pixel-centre square of a dx^2 + 2 b dx dy + c dy^2,
    d = (u - x, v - y), as a bounded linear least-squares problem (q = |L^T d|^2
    with L L^T the conic), solved by scipy in float64."""
    from scipy.optimize import lsq_linear
    u, v, a, b, c = (float(x) for x in rec[:5])
    x, y = t % tx, t // tx
    Q = np.array([[a, b], [b, c]])
    L = np.linalg.cholesky(Q)
    lo = [u - (16 * x + 15.5), v - (16 * y + 15.5)]
    hi = [u - (16 * x + 0.5), v - (16 * y + 0.5)]
    r = lsq_linear(L.T, np.zeros(2), bounds=(lo, hi), tol=1e-14, lsq_solver="exact")
    d = r.x
    return float(d @ Q @ d)


@pytest.mark.parametrize("seed", [0, 1])
def test_bin_sort_tile_test(oracle_lib, seed):
    """A tile of a record's rect is binned exactly when the record's ellipse
    q(d) <= cut meets the tile's pixel-centre square: the minimum of q over the
    square, found independently by bounded least squares, is below the cut
    (1e-5 relative band for the FP32 decision); the kept instances come out in
    the brute-force order."""
    rng = np.random.default_rng(40 + seed)
    n, ncams, tx, ty = 150, 2, 9, 7
    rect, depth = synth.synthetic_projected(rng, n, ncams, tx, ty, max_extent=4, tie_frac=0.2)
    rec = synth.synthetic_records(rng, rect, depth)
    out = oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty, proj=rec)
    kept = _kept_pairs(out, n, ncams, tx, ty)
    n_in, n_out = 0, 0
    for i in range(ncams * n):
        x0, y0, x1, y1 = rect[i]
        cam = i // n
        for yy in range(y0, y1):
            for xx in range(x0, x1):
                t = yy * tx + xx
                qmin = _box_min_q(rec[i], t, tx)
                cut = float(rec[i, 7])
                inside = (i, cam * tx * ty + t) in kept
                if qmin < cut * (1 - 1e-5) - 1e-6:
                    assert inside, (i, t, qmin, cut)
                    n_in += 1
                elif qmin > cut * (1 + 1e-5) + 1e-6:
                    assert not inside, (i, t, qmin, cut)
                    n_out += 1
    assert n_in > 100 and n_out > 100, (n_in, n_out)  # both sides exercised
    # order: the brute-force sort of the kept instances
    ref = [r for r in brute_force_bins(rect, depth, n, ncams, tx, ty)
           if ((r[0] // (tx * ty)) * n + r[3], r[0]) in kept]
    np.testing.assert_array_equal(out["ids"], [r[3] for r in ref])
    np.testing.assert_array_equal(out["keys"] >> np.uint64(32), [r[0] for r in ref])


def test_tile_test_keeps_every_contributing_pixel(oracle_lib):
    """Conservative: every pixel where a Gaussian passes the skip threshold
    (o exp(power) >= 1/255, FP64 projection) lies in a tile binned for it,
    with the records rounded to FP32 and the cutoff formed as the GPU forms
    it."""
    scene, cams = synth.tiny()
    cam = cams[0]
    o = oracle_lib.project(scene, cam)
    valid = o["valid"] == 1
    n = scene.n
    rec = np.zeros((n, 8), np.float32)
    rec[:, 0:2] = o["mean2d"]
    rec[:, 2:5] = o["conic"]
    rec[:, 5] = o["opacity"]
    rec[:, 6] = o["depth"]
    op32 = rec[:, 5]
    with np.errstate(divide="ignore"):
        rec[:, 7] = (np.float32(2) * np.log(np.float32(255) * op32)).astype(np.float32) * \
            np.float32(1.001) + np.float32(0.01)
    rect = np.where(valid[:, None], o["rect"], 0).astype(np.int32)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    out = oracle_lib.bin_sort(rect, rec[:, 6], n, 1, tx, ty, proj=rec)
    kept = _kept_pairs(out, n, 1, tx, ty)
    assert len(kept) < int(((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).sum())
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    px, py = xs + 0.5, ys + 0.5
    checked = 0
    for i in np.nonzero(valid)[0]:
        a, b, c = o["conic"][i]
        dx, dy = o["mean2d"][i, 0] - px, o["mean2d"][i, 1] - py
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        hit = o["opacity"][i] * np.exp(np.minimum(power, 0.0)) >= 1.0 / 255.0
        hit &= power <= 0.0
        for t in np.unique((ys[hit] // 16) * tx + xs[hit] // 16):
            assert (i, int(t)) in kept, (i, t)
            checked += 1
    assert checked > 1000


def test_bin_sort_invariants_and_ties(oracle_lib):
    rng = np.random.default_rng(7)
    n, ncams, tx, ty = 3000, 2, 12, 9
    rect, depth = synth.synthetic_projected(rng, n, ncams, tx, ty, tie_frac=0.2)
    out = oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty)
    keys, ids, ranges = out["keys"], out["ids"], out["ranges"]
    area = np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)
    assert keys.size == area.sum()
    assert np.all(np.diff(keys.astype(np.uint64)) >= 0) if keys.size else True
    # ties keep ascending Gaussian index inside a tile
    same = keys[1:] == keys[:-1]
    assert same.sum() > 0
    assert np.all(ids[1:][same] > ids[:-1][same])
    # ranges partition [0, K)
    nonempty = ranges[:, 1] > ranges[:, 0]
    spans = ranges[nonempty]
    assert spans[:, 1].max() == keys.size and spans[:, 0].min() == 0
    assert (spans[:, 1] - spans[:, 0]).sum() == keys.size


# ---------------------------------------------------------------- autoencoder

def test_gelu_tanh_form_against_normal_cdf():
    from oracle import ae
    from scipy.special import ndtr
    # the tanh form tracks x Phi(x) to within 4.73e-4, reached near x = 2.7;
    # a wrong constant (e.g. 0.044 or 0.045, or 0.8 for sqrt(2/pi)) or a
    # missing cubic term breaks the bound, a sign error breaks it by far
    x = np.linspace(-8, 8, 160001)
    dev = np.abs(ae.gelu(x) - x * ndtr(x))
    assert dev.max() <= 4.8e-4
    assert dev.max() >= 4.6e-4 and 2.4 < abs(x[dev.argmax()]) < 3.0
    np.testing.assert_allclose(ae.gelu(np.array([0.0, 40.0, -40.0])), [0.0, 40.0, 0.0],
                               atol=1e-12)
    # derivative against central differences
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(ae.gelu_grad(x), (ae.gelu(x + h) - ae.gelu(x - h)) / (2 * h),
                               rtol=1e-8, atol=1e-9)


def test_mlp_forward_matches_loops():
    from oracle import ae
    rng = np.random.default_rng(0)
    widths = (5, 4, 3)
    layers = [[rng.standard_normal((b, a)), rng.standard_normal(b)]
              for a, b in zip(widths[:-1], widths[1:])]
    x = rng.standard_normal((6, 5))
    y, _ = ae.mlp_forward(layers, x)
    for p in range(6):
        h = list(x[p])
        for li, (W, b) in enumerate(layers):
            out = []
            for o in range(W.shape[0]):
                acc = b[o]
                for i in range(W.shape[1]):
                    acc += W[o, i] * h[i]
                if li < len(layers) - 1:
                    u = math.sqrt(2 / math.pi) * (acc + 0.044715 * acc ** 3)
                    acc = 0.5 * acc * (1 + math.tanh(u))
                out.append(acc)
            h = out
        np.testing.assert_allclose(y[p], h, rtol=1e-13, atol=1e-14)


def _toy_ae(seed=0):
    enc, dec = synth.ae_init((16, 12, 8, 4), (4, 8, 12, 16), seed=seed)
    f64 = lambda L: [[W.astype(np.float64), b.astype(np.float64)] for W, b in L]
    return f64(enc), f64(dec)


def test_recon_loss_closed_forms():
    from oracle import ae
    rng = np.random.default_rng(1)
    x = synth.unit_rows(rng.standard_normal((7, 16)))
    assert ae.recon_loss(x, x)[0] == pytest.approx(0.0, abs=1e-15)
    # y = 2x: (y - x)^2 mean = |x|^2 / 16 = 1/16 per pixel, cos = 1
    assert ae.recon_loss(2 * x, x)[0] == pytest.approx(1.0 / 16, rel=1e-13)
    # y = -x: 4/16 + 2
    assert ae.recon_loss(-x, x)[0] == pytest.approx(0.25 + 2.0, rel=1e-13)


@pytest.mark.parametrize("mode", ["recon", "enc_adapt"])
def test_train_step_gradients_fd(mode):
    from oracle import ae
    enc, dec = _toy_ae()
    rng = np.random.default_rng(2)
    x = synth.unit_rows(rng.standard_normal((9, 16)))
    target = rng.standard_normal((9, 4))
    state = ae.new_state(enc, dec)
    enc0 = [[W.copy(), b.copy()] for W, b in enc]
    dec0 = [[W.copy(), b.copy()] for W, b in dec]
    _, grads = ae.train_step(enc, dec, state, x, target, mode, lr=0.0)

    def loss_of(e, d):
        z, _ = ae.mlp_forward(e, x)
        if mode == "recon":
            return ae.recon_loss(ae.mlp_forward(d, z)[0], x)[0]
        return ae.l1_loss(z, target)[0]

    params = enc0 + dec0
    n_checked = 0
    for li, (W, b) in enumerate(params):
        if grads[li] is None:
            assert mode == "enc_adapt" and li >= len(enc0)
            continue
        for j, arr in enumerate((W, b)):
            flat = arr.reshape(-1)
            for k in range(0, flat.size, max(1, flat.size // 7)):
                h = 1e-6
                old = flat[k]
                flat[k] = old + h
                lp = loss_of(enc0, dec0)
                flat[k] = old - h
                lm = loss_of(enc0, dec0)
                flat[k] = old
                fd = (lp - lm) / (2 * h)
                ana = grads[li][j].reshape(-1)[k]
                assert abs(fd - ana) <= 1e-6 * max(1.0, abs(fd)), (li, j, k, fd, ana)
                n_checked += 1
    assert n_checked > 40


def test_distill_gradient_fd():
    from oracle import ae
    _, dec = _toy_ae(3)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((5, 4))
    t = rng.standard_normal((5, 16))
    loss, df = ae.distill(dec, f, t)
    for p in range(5):
        for k in range(4):
            h = 1e-6
            f2 = f.copy()
            f2[p, k] += h
            lp = ae.l1_loss(ae.decode(dec, f2), t)[0]
            f2[p, k] -= 2 * h
            lm = ae.l1_loss(ae.decode(dec, f2), t)[0]
            assert abs((lp - lm) / (2 * h) - df[p, k]) <= 1e-7


def test_adam_first_step_closed_form():
    from oracle import ae
    # after one step m_hat = g and v_hat = g^2, so the update is lr g / (|g| + eps)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(50)
    p = rng.standard_normal(50)
    p0 = p.copy()
    m, v = np.zeros(50), np.zeros(50)
    ae.adam_update(p, g, m, v, 1, 1e-3)
    np.testing.assert_allclose(p, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    ae.adam_update(p, g, m, v, 2, 1e-3)
    np.testing.assert_allclose(p, p0 - 2e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_enc_adapt_leaves_decoder_untouched():
    from oracle import ae
    enc, dec = _toy_ae()
    dec0 = [[W.copy(), b.copy()] for W, b in dec]
    rng = np.random.default_rng(6)
    x = synth.unit_rows(rng.standard_normal((8, 16)))
    state = ae.new_state(enc, dec)
    ae.train_step(enc, dec, state, x, rng.standard_normal((8, 4)), "enc_adapt", 1e-2)
    for (W, b), (W0, b0) in zip(dec, dec0):
        np.testing.assert_array_equal(W, W0)
        np.testing.assert_array_equal(b, b0)


def test_cosine_error_closed_form():
    from oracle import ae
    a = np.array([[1.0, 0.0], [0.0, 2.0], [0.0, 0.0]])
    b = np.array([[1.0, 1.0], [0.0, 1.0], [0.0, 0.0]])
    m, excl = ae.cosine_error(a, b)
    assert excl == 1
    assert m == pytest.approx(((1 - 1 / math.sqrt(2)) + 0.0) / 2, rel=1e-14)
