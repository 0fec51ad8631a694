"""Writes ``oracle_regression.json``: what the FP64 oracle computes on small
seeded inputs.  Only ``oracle/`` produces the stored values; the inputs come
from the seeded generators (``paper_2511_16144_gb300.synth``, no method
arithmetic).  The test beside it regenerates the inputs and compares, so a
change to the oracle's arithmetic fails until the fixture is rewritten by
this script.  Run from the repository root:

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FIXTURE = os.path.join(HERE, "oracle_regression.json")


def inputs():
    """The seeded inputs of every fixture (also used by the test)."""
    from paper_2511_16144_gb300 import synth
    scene = synth.random_scene(np.random.default_rng(7), 12, (-0.5, -0.4, 1.5), (0.5, 0.4, 2.5),
                               math.log(0.08), 0.3, 3, feat_dim=4)
    cam = synth.Camera(40.0, 40.0, 8.0, 6.0, 16, 12, synth.identity_view())
    g = np.random.default_rng(8)
    upstream = dict(rgb=g.standard_normal((12, 16, 3)), depth=g.standard_normal((12, 16)),
                    feat=g.standard_normal((12, 16, 4)))
    enc, dec = synth.ae_init(seed=3003)
    x = synth.embedding_map(np.random.default_rng(9), synth.embedding_centroids(), 4, 2)
    x = x.reshape(-1, 512).astype(np.float64)
    f_gt = synth.embedding_map(np.random.default_rng(10), synth.embedding_centroids(), 4, 2)
    f_gt = f_gt.reshape(-1, 512).astype(np.float64)
    prune_scene = synth.random_scene(np.random.default_rng(11), 200, (0, 0, 0), (0.4, 0.4, 0.4),
                                     math.log(0.02), 0.5, 4, feat_dim=16, feat_noise=0.02)
    r = np.random.default_rng(12)
    codebook = synth.unit_rows(r.standard_normal((8, 16)))
    words = synth.unit_rows(codebook[r.integers(0, 8, 64)] + 0.5 * r.standard_normal((64, 16)))
    return dict(scene=scene, cam=cam, upstream=upstream, enc=enc, dec=dec, x=x, f_gt=f_gt,
                prune_scene=prune_scene, codebook=codebook, words=words)


def compute(inp):
    """The oracle's outputs on ``inputs()``, as plain lists."""
    import oracle
    from oracle import ae, loop
    sc, cam, up = inp["scene"], inp["cam"], inp["upstream"]
    p = oracle.project(sc, cam)
    r = oracle.render(sc, cam)
    b = oracle.render_backward(sc, cam, up["rgb"], up["depth"], up["feat"])
    enc = [[np.asarray(W, np.float64), np.asarray(bb, np.float64)] for W, bb in inp["enc"]]
    dec = [[np.asarray(W, np.float64), np.asarray(bb, np.float64)] for W, bb in inp["dec"]]
    z = ae.encode(enc, inp["x"])
    y = ae.decode(dec, z)
    d_loss, d_dz = ae.distill(dec, z, inp["f_gt"])
    t_loss, grads = ae.train_step(enc, dec, ae.new_state(enc, dec), inp["x"], None, "recon",
                                  lr=0.0)
    ps = inp["prune_scene"]
    mask = oracle.prune(ps.means, ps.opacity_logits, ps.log_scales, ps.feats, k=8,
                        tau_dist=0.05, tau_sim=0.9)
    assign, _ = loop.assign(inp["words"], inp["codebook"])
    out = {
        "project": {k: np.asarray(p[k]).tolist() for k in
                    ("mean2d", "depth", "conic", "opacity", "radius", "rect", "valid")},
        "render": {k: np.asarray(r[k]).tolist() for k in
                   ("rgb", "depth", "feat", "T_final", "n_contrib")},
        "render_backward": {k: np.asarray(b[k]).tolist() for k in
                            ("means", "quats", "log_scales", "opacity_logits", "colors",
                             "feats")},
        "ae": {
            "z": z.tolist(),
            "y_first8": y[:, :8].tolist(),
            "y_row_norms": np.linalg.norm(y, axis=1).tolist(),
            "distill_loss": float(d_loss),
            "distill_dz": np.asarray(d_dz).tolist(),
            "recon_loss": float(t_loss),
            "grad_norms": [[float(np.linalg.norm(gW)), float(np.linalg.norm(gb))]
                           for gW, gb in grads],
            "gW_row0_first4": [np.asarray(gW)[0, :4].tolist() for gW, _ in grads],
        },
        "prune_mask": mask.astype(int).tolist(),
        "codebook_assign": np.asarray(assign).astype(int).tolist(),
    }
    return out


def main():
    out = compute(inputs())
    out = {"_about": "FP64 oracle outputs on the seeded inputs of tests/golden/make_golden.py "
                     "(written by that script; regression fixture, not an independent pin)",
           **out}
    with open(FIXTURE, "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {FIXTURE} ({os.path.getsize(FIXTURE)} bytes)")


if __name__ == "__main__":
    main()
