"""FP64 oracle of the compact-space query and the language loop signature
(TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the CPU legs of
the benchmark use it).

* Query (Sec. I): a text query's embedding is projected into the compact
  16-d space by the encoder (E(q)) and compared there with the map's
  features; the comparison is the cosine similarity, per pixel of a
  rendered feature map or per Gaussian.
* Loop signature (Sec. III-D): each keyframe's language features are assigned
  to their closest codeword of a codebook built offline by k-means; the
  normalised histogram of the assignments is the keyframe's signature; the
  cosine similarity to the signatures of spatially close past keyframes,
  above tau_hist, gives the loop candidates, of which the two most similar
  go on to geometric verification (Sec. IV-A).

Readings where the paper is silent: "closest" is the Euclidean distance
(argmin_k |x - c_k|^2, ties to the lower index); the cosine of a zero vector
is 0; "spatially close" is a camera-centre distance below a radius; ties in
similarity go to the lower keyframe index.
"""
from __future__ import annotations

import numpy as np


def assign(x, codebook):
    """Closest codeword of every row of x ([P, D]) and the margin between the
    best and the second best squared distance (float64)."""
    x = np.asarray(x, np.float64)
    c = np.asarray(codebook, np.float64)
    d2 = (x * x).sum(1)[:, None] - 2.0 * x @ c.T + (c * c).sum(1)[None, :]
    idx = np.argmin(d2, axis=1)  # first minimum: the lower index wins ties
    part = np.partition(d2, 1, axis=1)
    return idx.astype(np.int64), part[:, 1] - part[:, 0]


def histogram(idx, k):
    """Assignment counts per codeword."""
    return np.bincount(np.asarray(idx, np.int64), minlength=k).astype(np.int64)


def signature(x, codebook):
    """Normalised histogram of the keyframe's assignments."""
    idx, _ = assign(x, codebook)
    h = histogram(idx, codebook.shape[0]).astype(np.float64)
    return h / max(h.sum(), 1.0)


def cosine(a, b):
    """Cosine similarity of each row of b with a (0 when a norm is 0)."""
    a = np.asarray(a, np.float64)
    b = np.atleast_2d(np.asarray(b, np.float64))
    na, nb = np.linalg.norm(a), np.linalg.norm(b, axis=1)
    out = np.zeros(b.shape[0])
    ok = (na > 0) & (nb > 0)
    out[ok] = (b[ok] @ a) / (na * nb[ok])
    return out


def loop_candidates(sim, centres, cur_centre, tau_hist, radius, top=2):
    """Indices of past keyframes with similarity above tau_hist and camera
    centre within radius of the current one, most similar first (ties to
    the lower index), at most `top`; -1 pads."""
    sim = np.asarray(sim, np.float64)
    d = np.linalg.norm(np.asarray(centres, np.float64) - np.asarray(cur_centre, np.float64), axis=1)
    ok = np.flatnonzero((sim > tau_hist) & (d < radius))
    order = sorted(ok.tolist(), key=lambda i: (-sim[i], i))[:top]
    return np.array(order + [-1] * (top - len(order)), np.int64)


def query_relevance(feats, queries):
    """Cosine similarity [M, Q] between every feature row and every query."""
    f = np.asarray(feats, np.float64)
    q = np.atleast_2d(np.asarray(queries, np.float64))
    nf = np.linalg.norm(f, axis=1)[:, None]
    nq = np.linalg.norm(q, axis=1)[None, :]
    den = nf * nq
    out = np.zeros((f.shape[0], q.shape[0]))
    np.divide(f @ q.T, den, out=out, where=den > 0)
    return out
