"""What the trained autoencoder gains (marked gpu).

Setup (the benchmark's frame): 300k Gaussians in the 6x6x3 m room with
spatially coherent 512-d semantics (64 3D Voronoi cells); the plain path
renders all 512 channels for 8 keyframes at 640x480, and those rendered maps
are the autoencoder's online training data (200 Adam steps of 64k pixels,
lr 5e-3, L2 + (1 - cos)).  The Gaussians' 16-d features are the encoder prior
E(g_i) (Sec. III-B.2); the 16-d render is decoded by D and compared with the
plain 512-channel render pixel by pixel (1 - cos over pixels with a
non-zero reference).

Baselines: the untrained autoencoder, a random linear 512 -> 16 projection
with its pseudo-inverse as decoder, and an autoencoder trained on a different
scene (a frozen, non-adapted encoder).

The per-Gaussian N(0, 0.02) embedding noise sets a floor: a 16-d code cannot
carry it, and the plain render keeps what survives alpha blending (about
0.01-0.02 of cosine at this density, more for sparser maps).
"""
import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth

pytestmark = pytest.mark.gpu


def cosine_error(y, ref):
    nr = ref.norm(dim=1)
    keep = nr > 1e-6
    cos = (y * ref).sum(1)[keep] / (y.norm(dim=1)[keep] * nr[keep]).clamp_min(1e-30)
    return float((1 - cos).mean().item()), int((~keep).sum().item())


def semantic_scene(n, seed, sem_seed):
    scene, cams = synth.indoor(n=n, n_cams=8, seed=seed)
    g = synth.semantic_features(scene.means, synth.ROOM_LO, synth.ROOM_HI, seed=sem_seed)
    return scene.with_feats(g), cams


def render_feat(ds, cam):
    from paper_2511_16144_gb300.render import Frame
    fr = Frame(ds, [cam])
    return fr.out["feat"][0].reshape(-1, ds.feats.shape[1])


def train_ae(frames, seed, steps=200):
    from paper_2511_16144_gb300.ae import AutoEncoder
    enc, dec = synth.ae_init(seed=seed)
    model = AutoEncoder(enc, dec)
    data = torch.cat(frames).bfloat16()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    for _ in range(steps):
        idx = torch.randint(0, data.shape[0], (65536,), device="cuda", generator=gen)
        model.train_step(data[idx].contiguous(), lr=5e-3)
    return model


def decoded_error(model, ds512, ds_geom, cam, ref):
    from paper_2511_16144_gb300.render import DeviceScene
    f16 = model.encode(ds512.feats.bfloat16().contiguous())
    ds16 = DeviceScene(ds_geom.means, ds_geom.quats, ds_geom.log_scales, ds_geom.opacity_logits,
                       ds_geom.colors, f16.contiguous())
    y = model.decode(render_feat(ds16, cam).contiguous())
    return cosine_error(y, ref)


def test_trained_autoencoder_gain():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs
    from paper_2511_16144_gb300.ae import AutoEncoder
    from paper_2511_16144_gb300.render import DeviceScene
    build.build()
    lgs.load()
    scene, cams = semantic_scene(300_000, 1001, 1005)
    ds = DeviceScene.from_host(scene)
    frames = [render_feat(ds, c) for c in cams]
    model = train_ae(frames, 3003)
    errs = []
    for c, ref in zip(cams[::3], frames[::3]):
        errs.append(decoded_error(model, ds, ds, c, ref)[0])
    trained = float(np.mean(errs))

    # baselines on the same views
    untrained = np.mean([decoded_error(AutoEncoder(*synth.ae_init(seed=3003)), ds, ds, c, ref)[0]
                         for c, ref in zip(cams[::3], frames[::3])])
    gen = torch.Generator(device="cuda").manual_seed(5)
    Pm = torch.randn((512, 16), device="cuda", generator=gen) / np.sqrt(512)
    Pinv = torch.linalg.pinv(Pm)
    lin = []
    from paper_2511_16144_gb300.render import DeviceScene as DS
    for c, ref in zip(cams[::3], frames[::3]):
        ds16 = DS(ds.means, ds.quats, ds.log_scales, ds.opacity_logits, ds.colors,
                  (ds.feats @ Pm).contiguous())
        lin.append(cosine_error(render_feat(ds16, c) @ Pinv, ref)[0])
    linear = float(np.mean(lin))
    other_scene, other_cams = semantic_scene(300_000, 1011, 1015)
    ods = DeviceScene.from_host(other_scene)
    other = train_ae([render_feat(ods, c) for c in other_cams], 3013)
    frozen = np.mean([decoded_error(other, ds, ds, c, ref)[0]
                      for c, ref in zip(cams[::3], frames[::3])])
    print(f"decoded cosine error: trained {trained:.4f}; untrained {untrained:.4f}, "
          f"linear+pinv {linear:.4f}, other-scene encoder {frozen:.4f}")
    # the target of the learned part: mean (1 - cos) of the decoded 16-d
    # render against the plain 512-channel render at most 0.02 (training is
    # bit-reproducible, so this is one fixed number per build)
    assert trained <= 0.02, trained
    assert trained < 0.1 * min(untrained, linear, frozen)
