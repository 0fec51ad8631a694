"""The fixtures under tests/golden (no GPU): the paper's stated constants
against the library and the oracle, and the FP64 oracle against the
regression fixture its generator script wrote."""
import importlib.util
import inspect
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _json(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_latent_width_and_loop_candidates():
    c = _json("paper_constants.json")
    from paper_2511_16144_gb300 import lgs
    from oracle import loop
    assert lgs.AE_WIDTHS[4] == c["feature_dim"]["value"]          # encoder output
    assert lgs.AE_WIDTHS[0] == lgs.AE_WIDTHS[-1]                    # decoder mirrors it
    top = inspect.signature(loop.loop_candidates).parameters["top"].default
    assert top == c["loop_top_candidates"]["value"]


def test_eq4_inequalities_are_strict():
    """Two Gaussians 0.0625 apart with identical basis-vector features
    (cosine exactly 1): at tau_dist = 0.0625 or tau_sim = 1 neither is
    redundant; just inside both thresholds the lower-opacity one is."""
    import oracle
    assert _json("paper_constants.json")["pruning_condition"]["value"].startswith("strict")
    means = np.array([[0, 0, 0], [0.0625, 0, 0]], np.float32)
    logits = np.array([1.0, 0.0], np.float32)                       # the second is fainter
    log_scales = np.full((2, 3), np.log(0.01), np.float32)
    feats = np.zeros((2, 16), np.float32)
    feats[:, 0] = 1.0
    kw = dict(k=1, min_opacity=0.005)
    assert oracle.prune(means, logits, log_scales, feats, tau_dist=0.0625, tau_sim=0.5,
                        **kw).tolist() == [0, 0]
    assert oracle.prune(means, logits, log_scales, feats, tau_dist=0.07, tau_sim=1.0,
                        **kw).tolist() == [0, 0]
    assert oracle.prune(means, logits, log_scales, feats, tau_dist=0.07, tau_sim=0.999,
                        **kw).tolist() == [0, 2]


def _bias_only(widths, rng):
    """Layers with zero weights and random biases: the network's output is
    the last bias whatever the input, so a loss on it has a closed form."""
    return [[np.zeros((b, a)), rng.standard_normal(b)] for a, b in zip(widths[:-1], widths[1:])]


def test_eq2_and_eq3_are_l1_losses():
    """Eq. 2 (distillation through the decoder) and Eq. 3 (encoder
    adaptation) as the oracle computes them are the mean absolute error, with
    the sign as gradient: checked on two pixels where the networks reduce to
    their last bias (the L2 value differs, so a squared loss would fail)."""
    from oracle import ae
    c = _json("paper_constants.json")
    assert c["distillation_loss"]["value"] == "L1"
    assert c["encoder_adaptation_loss"]["value"] == "L1"
    rng = np.random.default_rng(5)
    dec = _bias_only((16, 64, 128, 256, 512), rng)
    enc = _bias_only((512, 256, 128, 64, 16), rng)
    f_render = rng.standard_normal((2, 16))
    f_gt = rng.standard_normal((2, 512))
    loss, dz = ae.distill(dec, f_render, f_gt)
    y = dec[-1][1]
    assert np.isclose(loss, np.abs(y[None] - f_gt).mean(), rtol=1e-14, atol=0)
    assert not np.isclose(loss, ((y[None] - f_gt) ** 2).mean())
    assert np.all(dz == 0)  # nothing reaches z through zero weights
    x = rng.standard_normal((2, 512))
    state = ae.new_state(enc, dec)
    loss3, grads = ae.train_step(enc, dec, state, x, f_render, "enc_adapt", lr=0.0)
    z = enc[-1][1]
    assert np.isclose(loss3, np.abs(z[None] - f_render).mean(), rtol=1e-14, atol=0)
    # the latent bias gradient: the sum over pixels of sign(z - F_render) / (2 * 16)
    np.testing.assert_allclose(grads[3][1], np.sign(z[None] - f_render).sum(0) / 32.0,
                               rtol=1e-14, atol=0)
    assert all(g is None for g in grads[4:])  # the decoder is frozen in Eq. 3


def _compare(got, ref, path="fixture"):
    if isinstance(ref, dict):
        assert set(got) >= set(ref) - {"_about"}, path
        for k, v in ref.items():
            if k != "_about":
                _compare(got[k], v, f"{path}.{k}")
        return
    g, r = np.asarray(got), np.asarray(ref)
    assert g.shape == r.shape, (path, g.shape, r.shape)
    if r.dtype.kind in "iub":
        np.testing.assert_array_equal(g, r, err_msg=path)
    else:
        np.testing.assert_allclose(g, r, rtol=1e-9, atol=1e-12, err_msg=path)


def test_oracle_matches_its_regression_fixture():
    m = _maker()
    _compare(m.compute(m.inputs()), _json("oracle_regression.json"))
