"""ctypes binding of liblgs (the C ABI in include/lgs.h).

Each function here carries the C entry point's name and only marshals
arguments: torch CUDA tensors supply device memory and the current CUDA
stream, and every step runs in the library's kernels.  If liblgs.so is
missing, or no CUDA device is present, calls raise; there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgs.so")
MAX_CAMS = 16
TILE = 16
PROJ_STRIDE = 8
F32, BF16 = 0, 1
# lgs_status
OK, ERR_INVALID, ERR_CAPACITY, ERR_NONFINITE, ERR_TIMEOUT, ERR_CUDA = 0, 1, 2, 3, 4, 5

_lib = None


class LgsError(RuntimeError):
    """A liblgs call returned a non-zero lgs_status (``status``; ``detail``
    for a device-side error reported by lgs_sync_status)."""

    def __init__(self, msg, status=None, detail=None):
        super().__init__(msg)
        self.status, self.detail = status, detail


AE_LAYERS = 8
AE_WIDTHS = (512, 256, 128, 64, 16, 64, 128, 256, 512)
AE_ENCODE, AE_DECODE, AE_TRAIN = 0, 1, 2
AE_RECON, AE_ENC_ADAPT = 0, 1


class AeWeights(ctypes.Structure):
    _fields_ = [("W", ctypes.c_void_p * AE_LAYERS), ("Wt", ctypes.c_void_p * AE_LAYERS),
                ("b", ctypes.c_void_p * AE_LAYERS)]


class AeState(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p * AE_LAYERS)
                for name in ("W", "b", "mW", "vW", "mb", "vb", "gW", "gb", "Wbf", "Wtbf")] + \
               [("step", ctypes.c_int64)]


class PruneParams(ctypes.Structure):
    """lgs_prune_params."""
    _fields_ = [("k", ctypes.c_int), ("tau_dist", ctypes.c_float), ("tau_sim", ctypes.c_float),
                ("min_opacity", ctypes.c_float), ("max_scale", ctypes.c_float),
                ("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class LgsCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("viewmat", ctypes.c_float * 12), ("znear", ctypes.c_float)]


def load():
    """Opens liblgs.so (build it first with ``paper_2511_16144_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LgsError(f"{LIB_PATH} is missing: run paper_2511_16144_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    F = ctypes.c_float
    sig = {
        "lgs_version": ([], ctypes.c_char_p),
        "lgs_last_error": ([], ctypes.c_char_p),
        "gs_project": ([P, P, P, P, I64, P, I32, P, P, P], I32),
        "gs_bin_sort_workspace": ([I64, I32, I32, I32, I64], SZ),
        "gs_bin_sort": ([P, P, I64, I32, I32, I32, I64, P, P, P, P, P, SZ, P], I32),
        "gs_render_fwd": ([P, P, P, I64, P, I32, P, P, I32, I32, P, P, P, P, P, P, P, P], I32),
        "gs_render_bwd": ([P, P, P, P, P, P, P, I64, P, I32, P, P, I32, I32, P, P, P, P, P, P, P,
                           P, P, P, P, P, P, P], I32),
        "lgs_l1_loss": ([P, P, I32, I64, F, P, P, P], I32),
        "ae_workspace_bytes": ([I64, I32], SZ),
        "ae_encode": ([P, P, I64, P, P, SZ, P], I32),
        "ae_decode": ([P, P, I64, P, F, P, P, P, P, SZ, P], I32),
        "ae_decode_pack": ([P, P, SZ, P], I32),
        "ae_decode_packed": ([P, P, I64, P, F, P, P, P, SZ, P], I32),
        "ae_train_step": ([P, P, P, I64, I32, F, P, P, SZ, P], I32),
        "ae_pack": ([P, I32, I32, P], I32),
        "lgs_device_error": ([P], I32),
        "lgs_sync_status": ([P, P], I32),
        "lgs_set_sort_wait_limit": ([I64], None),
        "lgs_graph_kernel_nodes": ([P], I64),
        "lgs_zero": ([P, SZ, P], I32),
        "gs_render_bwd_static_capacity": ([], I64),
        "gs_render_bwd_static": ([P, P, P, P, P, P, P, I64, P, I32, P, P, I32, I32, P, P, P, P,
                                  P, P, P, P, P, P, P, P, P], I32),
        "gs_prune_workspace": ([I64], SZ),
        "gs_prune": ([P, P, P, P, I32, I32, I64, P, P, P, P, SZ, P], I32),
        "gs_compact_workspace": ([I64], SZ),
        "gs_compact_index": ([P, I64, P, P, P, SZ, P], I32),
        "gs_gather_rows": ([P, I64, I32, P, P, P], I32),
        "lgs_dssim_workspace": ([I32, I32, I32], SZ),
        "lgs_dssim_loss": ([P, P, I32, I32, I32, F, P, P, P, SZ, P], I32),
        "gs_pose_grad": ([P, P, P, P, I64, P, I32, P, P, P], I32),
        "lgs_codebook_workspace": ([I32], SZ),
        "lgs_codebook_assign": ([P, I64, I32, P, I32, P, P, P, SZ, P], I32),
        "lgs_hist_cosine": ([P, P, I32, I32, P, P], I32),
        "lgs_loop_candidates": ([P, P, I32, P, F, F, I32, P, P], I32),
        "gs_query_relevance": ([P, I32, I64, I32, P, I32, P, P], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return ["lgs_version", "lgs_last_error", "gs_project", "gs_bin_sort_workspace", "gs_bin_sort",
            "gs_render_fwd", "gs_render_bwd", "lgs_l1_loss", "ae_workspace_bytes", "ae_encode",
            "ae_decode", "ae_decode_pack", "ae_decode_packed", "ae_train_step", "ae_pack",
            "lgs_device_error", "lgs_sync_status",
            "lgs_set_sort_wait_limit", "lgs_graph_kernel_nodes", "lgs_zero",
            "gs_render_bwd_static_capacity", "gs_render_bwd_static", "gs_prune_workspace",
            "gs_prune", "gs_compact_workspace", "gs_compact_index", "gs_gather_rows",
            "lgs_dssim_workspace", "lgs_dssim_loss", "gs_pose_grad", "lgs_codebook_workspace",
            "lgs_codebook_assign", "lgs_hist_cosine", "lgs_loop_candidates",
            "gs_query_relevance"]


def _check(status, what):
    if status != 0:
        msg = load().lgs_last_error().decode()
        raise LgsError(f"{what} failed with status {status}: {msg}", status)


def _p(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if t.numel() and not t.is_contiguous():
            raise LgsError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def cameras(cams):
    """Packs camera objects (fx, fy, cx, cy, width, height, viewmat[3,4],
    znear) into an lgs_camera array."""
    arr = (LgsCamera * len(cams))()
    for k, c in enumerate(cams):
        vm = np.asarray(c.viewmat, np.float32).reshape(12)
        arr[k] = LgsCamera(float(c.fx), float(c.fy), float(c.cx), float(c.cy), int(c.width),
                           int(c.height), (ctypes.c_float * 12)(*vm.tolist()), float(c.znear))
    return arr


def _dtype_code(t):
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise LgsError(f"unsupported channel dtype {t.dtype}")


def tile_grid(cam):
    return (int(cam.width) + TILE - 1) // TILE, (int(cam.height) + TILE - 1) // TILE


# ---------------------------------------------------------------- entry points

def gs_project(means, quats, log_scales, opacity_logits, cams):
    """Returns proj [C*N, 8] float32 and rect [C*N, 4] int16 (uint16 bits)."""
    lib = load()
    n, c = means.shape[0], len(cams)
    dev = means.device
    proj = torch.empty((c * n, PROJ_STRIDE), dtype=torch.float32, device=dev)
    rect = torch.empty((c * n, 4), dtype=torch.int16, device=dev)
    ca = cameras(cams)
    _check(lib.gs_project(_p(means), _p(quats), _p(log_scales), _p(opacity_logits), n, ca, c,
                          _p(proj), _p(rect), _stream()), "gs_project")
    return proj, rect


class BinBuffers:
    """Caller-owned buffers of gs_bin_sort for one (n, cameras, grid),
    grown when the instance count exceeds the capacity."""

    def __init__(self, n, n_cams, tiles_x, tiles_y, capacity, device, want_keys=False):
        self.n, self.n_cams, self.tiles_x, self.tiles_y = n, n_cams, tiles_x, tiles_y
        self.device, self.want_keys = device, want_keys
        self.ranges = torch.empty((n_cams * tiles_x * tiles_y, 2), dtype=torch.int32, device=device)
        self.k_dev = torch.zeros(1, dtype=torch.int64, device=device)
        self.resize(capacity)

    def resize(self, capacity):
        lib = load()
        self.capacity = int(capacity)
        self.ids = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)
        self.keys = (torch.empty(max(self.capacity, 1), dtype=torch.int64, device=self.device)
                     if self.want_keys else None)
        ws = lib.gs_bin_sort_workspace(self.n, self.n_cams, self.tiles_x, self.tiles_y,
                                       self.capacity)
        self.workspace = torch.empty(max(int(ws), 256), dtype=torch.uint8, device=self.device)
        self.workspace_bytes = int(ws)


def gs_bin_sort(proj, rect, bufs: BinBuffers, stream=None):
    """Enqueues binning into ``bufs`` (no synchronisation)."""
    lib = load()
    _check(lib.gs_bin_sort(_p(proj), _p(rect), bufs.n, bufs.n_cams, bufs.tiles_x, bufs.tiles_y,
                           bufs.capacity, _p(bufs.ids), _p(bufs.ranges), _p(bufs.keys),
                           _p(bufs.k_dev), _p(bufs.workspace), bufs.workspace_bytes,
                           stream or _stream()), "gs_bin_sort")


def bin_sort_checked(proj, rect, bufs: BinBuffers, headroom=1.25):
    """gs_bin_sort, then reads K and re-runs with a larger capacity if it
    overflowed.  Returns K (this synchronises once)."""
    gs_bin_sort(proj, rect, bufs)
    k = int(bufs.k_dev.item())
    if k > bufs.capacity:
        bufs.resize(int(math.ceil(k * headroom)) + 1024)
        gs_bin_sort(proj, rect, bufs)
    return k


def gs_render_fwd(proj, bufs: BinBuffers, cams, colors, feats, bg=(0.0, 0.0, 0.0),
                  want_count=False):
    """Returns dict(rgb [C,H,W,3], depth [C,H,W], feat [C,H,W,D], T_final,
    last, n_contrib (if asked))."""
    lib = load()
    c = len(cams)
    h, w = int(cams[0].height), int(cams[0].width)
    d = int(feats.shape[1])
    dev = proj.device
    out = dict(rgb=torch.empty((c, h, w, 3), dtype=torch.float32, device=dev),
               depth=torch.empty((c, h, w), dtype=torch.float32, device=dev),
               feat=torch.empty((c, h, w, d), dtype=torch.float32, device=dev),
               T_final=torch.empty((c, h, w), dtype=torch.float32, device=dev),
               last=torch.empty((c, h, w), dtype=torch.int32, device=dev))
    out["n_contrib"] = (torch.empty((c, h, w), dtype=torch.int32, device=dev) if want_count
                        else None)
    bga = (ctypes.c_float * 3)(*[float(x) for x in bg])
    ca = cameras(cams)
    _check(lib.gs_render_fwd(_p(proj), _p(bufs.ids), _p(bufs.ranges), bufs.n, ca, c, _p(colors),
                             _p(feats), d, _dtype_code(feats), bga, _p(out["rgb"]),
                             _p(out["depth"]), _p(out["feat"]), _p(out["T_final"]),
                             _p(out["last"]), _p(out["n_contrib"]), _stream()), "gs_render_fwd")
    return out


def gs_render_bwd(params, proj, bufs: BinBuffers, cams, colors, feats, fwd, d_rgb, d_depth, d_feat,
                  grads, grad2d, bg=(0.0, 0.0, 0.0)):
    """Accumulates parameter gradients into ``grads`` (dict of tensors named
    means, quats, log_scales, opacity_logits, colors, feats).  ``params`` =
    (means, quats, log_scales, opacity_logits); ``grad2d`` [C*N, 8] scratch."""
    lib = load()
    means, quats, log_scales, logits = params
    c = len(cams)
    d = int(feats.shape[1])
    bga = (ctypes.c_float * 3)(*[float(x) for x in bg])
    ca = cameras(cams)
    _check(lib.gs_render_bwd(_p(means), _p(quats), _p(log_scales), _p(logits), _p(proj),
                             _p(bufs.ids), _p(bufs.ranges), bufs.n, ca, c, _p(colors), _p(feats), d,
                             _dtype_code(feats), bga, _p(fwd["T_final"]), _p(fwd["last"]),
                             _p(d_rgb), _p(d_depth), _p(d_feat), _p(grad2d), _p(grads["means"]),
                             _p(grads["quats"]), _p(grads["log_scales"]),
                             _p(grads["opacity_logits"]), _p(grads["colors"]), _p(grads["feats"]),
                             _stream()), "gs_render_bwd")


def gs_render_bwd_static(params, proj, bufs: BinBuffers, cams, colors, feats, fwd, d_rgb, d_depth,
                         d_feat, grads, bg=(0.0, 0.0, 0.0)):
    """gs_render_bwd with the library's fixed scratch instead of a
    caller-owned grad2d buffer (for callers that cannot allocate)."""
    lib = load()
    means, quats, log_scales, logits = params
    c = len(cams)
    d = int(feats.shape[1])
    bga = (ctypes.c_float * 3)(*[float(x) for x in bg])
    ca = cameras(cams)
    _check(lib.gs_render_bwd_static(_p(means), _p(quats), _p(log_scales), _p(logits), _p(proj),
                                    _p(bufs.ids), _p(bufs.ranges), bufs.n, ca, c, _p(colors),
                                    _p(feats), d, _dtype_code(feats), bga, _p(fwd["T_final"]),
                                    _p(fwd["last"]), _p(d_rgb), _p(d_depth), _p(d_feat),
                                    _p(grads["means"]), _p(grads["quats"]),
                                    _p(grads["log_scales"]), _p(grads["opacity_logits"]),
                                    _p(grads["colors"]), _p(grads["feats"]), _stream()),
           "gs_render_bwd_static")


def lgs_l1_loss(pred, target, weight, grad, loss_dev):
    """grad = weight sign(pred - target)/count; loss_dev += weight mean|.|."""
    lib = load()
    _check(lib.lgs_l1_loss(_p(pred), _p(target), _dtype_code(target), pred.numel(), float(weight),
                           _p(grad), _p(loss_dev), _stream()), "lgs_l1_loss")


# ---------------------------------------------------------------- autoencoder

def ae_workspace_bytes(P, what):
    return int(load().ae_workspace_bytes(int(P), int(what)))


def _workspace(P, what, device, cache=None):
    nbytes = ae_workspace_bytes(P, what)
    if cache is not None and cache.numel() >= nbytes:
        return cache, nbytes
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device), nbytes


def ae_encode(weights: AeWeights, x, z, ws=None):
    """z [P,16] f32 = E(x), x bf16 [P,512]."""
    P = x.shape[0]
    ws, nb = _workspace(P, AE_ENCODE, x.device, ws)
    _check(load().ae_encode(ctypes.byref(weights), _p(x), P, _p(z), _p(ws), nb, _stream()),
           "ae_encode")
    return ws


def ae_decode(weights: AeWeights, z, target=None, weight=1.0, loss=None, dz=None, y=None, ws=None):
    """Eq. 2 (loss += weight mean|D(z) - target|, dz = its gradient) and/or
    y = D(z)."""
    P = z.shape[0]
    ws, nb = _workspace(P, AE_DECODE, z.device, ws)
    _check(load().ae_decode(ctypes.byref(weights), _p(z), P, _p(target), float(weight), _p(loss),
                            _p(dz), _p(y), _p(ws), nb, _stream()), "ae_decode")
    return ws


def ae_decode_pack(weights: AeWeights, ws):
    """Packs the decoder weights into the workspace `ws` of a later
    ae_decode_packed call (the first half of ae_decode with a target)."""
    _check(load().ae_decode_pack(ctypes.byref(weights), _p(ws), ws.numel(), _stream()),
           "ae_decode_pack")


def ae_decode_packed(weights: AeWeights, z, target, weight, loss, dz, ws):
    """Eq. 2 as ae_decode with a target, from weights ae_decode_pack wrote
    into `ws`."""
    _check(load().ae_decode_packed(ctypes.byref(weights), _p(z), z.shape[0], _p(target),
                                   float(weight), _p(loss), _p(dz), _p(ws), ws.numel(),
                                   _stream()), "ae_decode_packed")


def ae_train_step(state: AeState, x, target, mode, lr, loss, ws=None):
    P = x.shape[0]
    ws, nb = _workspace(P, AE_TRAIN, x.device, ws)
    _check(load().ae_train_step(ctypes.byref(state), _p(x), _p(target), P, int(mode), float(lr),
                                _p(loss), _p(ws), nb, _stream()), "ae_train_step")
    return ws


def ae_pack(state: AeState, first=0, last=AE_LAYERS - 1):
    _check(load().ae_pack(ctypes.byref(state), first, last, _stream()), "ae_pack")


def lgs_zero(t):
    """Zero-fills a device tensor with a memset on the current stream."""
    _check(load().lgs_zero(_p(t), t.numel() * t.element_size(), _stream()), "lgs_zero")


def lgs_device_error():
    code = ctypes.c_int(0)
    _check(load().lgs_device_error(ctypes.byref(code)), "lgs_device_error")
    return code.value



def lgs_sync_status(stream=None):
    """(status, detail) of the device-side work: synchronises the current
    stream (or ``stream``) and returns one recorded error and its detail,
    clearing it (OK, 0 when none is pending)."""
    lib = load()
    d = ctypes.c_int64(0)
    st = lib.lgs_sync_status(_stream() if stream is None else stream, ctypes.byref(d))
    return int(st), int(d.value)


def check_device(what="device work"):
    """Raises LgsError for every error the device recorded (after
    synchronising the current stream)."""
    st, detail = lgs_sync_status()
    if st != OK:
        msg = load().lgs_last_error().decode()
        raise LgsError(f"{what}: status {st} (detail {detail}): {msg}", st, detail)


def lgs_set_sort_wait_limit(polls):
    """Polling rounds before the pruning sort's look-back gives up (<= 0:
    the default)."""
    load().lgs_set_sort_wait_limit(int(polls))

def prune_params(lo, hi, k=8, tau_dist=0.05, tau_sim=0.9, min_opacity=0.005,
                 max_scale=float("inf")):
    return PruneParams(int(k), float(tau_dist), float(tau_sim), float(min_opacity),
                       float(max_scale), (ctypes.c_float * 3)(*[float(v) for v in lo]),
                       (ctypes.c_float * 3)(*[float(v) for v in hi]))


def gs_prune(means, opacity_logits, log_scales, feats, params: PruneParams, mask=None,
             n_pruned=None, ws=None):
    """Enqueues gs_prune; returns (mask uint8 [n], n_pruned int64 [1]) on the device."""
    n, d = feats.shape
    dev = feats.device
    mask = torch.empty(n, dtype=torch.uint8, device=dev) if mask is None else mask
    n_pruned = torch.empty(1, dtype=torch.int64, device=dev) if n_pruned is None else n_pruned
    if ws is None:
        ws = torch.empty(max(int(load().gs_prune_workspace(n)), 256), dtype=torch.uint8, device=dev)
    _check(load().gs_prune(_p(means), _p(opacity_logits), _p(log_scales), _p(feats), d,
                           _dtype_code(feats), n, ctypes.byref(params), _p(mask), _p(n_pruned),
                           _p(ws), ws.numel(), _stream()), "gs_prune")
    return mask, n_pruned


def gs_compact(mask, tensors):
    """Keeps the rows whose mask is 0, in order, of every tensor in
    ``tensors`` (first dimension n).  Reads the kept count back (synchronises)."""
    L = load()
    n = mask.shape[0]
    dev = mask.device
    new_index = torch.empty(n, dtype=torch.int32, device=dev)
    n_kept = torch.empty(1, dtype=torch.int64, device=dev)
    ws = torch.empty(max(int(L.gs_compact_workspace(n)), 256), dtype=torch.uint8, device=dev)
    _check(L.gs_compact_index(_p(mask), n, _p(new_index), _p(n_kept), _p(ws), ws.numel(),
                              _stream()), "gs_compact_index")
    k = int(n_kept.item())
    out = []
    for t in tensors:
        dst = torch.empty((k,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
        out.append(dst)
        if k == 0:
            continue
        row = t[0].numel() * t.element_size()
        _check(L.gs_gather_rows(_p(t), n, row, _p(new_index), _p(dst), _stream()),
               "gs_gather_rows")
    return out, new_index


def lgs_dssim_loss(pred, target, weight, grad, loss_dev, ws=None):
    """loss_dev += weight (1 - mean SSIM(pred, target)); grad += its gradient.
    pred / target / grad: [C, H, W, 3] float32 on the device."""
    L = load()
    c, h, w = int(pred.shape[0]), int(pred.shape[1]), int(pred.shape[2])
    if ws is None:
        ws = torch.empty(max(int(L.lgs_dssim_workspace(c, h, w)), 4), dtype=torch.uint8,
                         device=pred.device)
    _check(L.lgs_dssim_loss(_p(pred), _p(target), c, h, w, float(weight), _p(grad), _p(loss_dev),
                            _p(ws), ws.numel(), _stream()), "lgs_dssim_loss")


def gs_pose_grad(means, quats, log_scales, opacity_logits, cams, grad2d, d_pose=None):
    """[n_cams, 6] gradient w.r.t. left se(3) perturbations (rho, phi) of each
    camera's world->camera transform, from gs_render_bwd's 2D records."""
    n = means.shape[0]
    d_pose = (torch.empty((len(cams), 6), dtype=torch.float32, device=means.device)
              if d_pose is None else d_pose)
    _check(load().gs_pose_grad(_p(means), _p(quats), _p(log_scales), _p(opacity_logits), n,
                               cameras(cams), len(cams), _p(grad2d), _p(d_pose), _stream()),
           "gs_pose_grad")
    return d_pose


def lgs_codebook_assign(x, codebook, hist=None, assign=None, ws=None):
    """Closest codeword per row of x (bf16 [P, D]); hist [K] uint32 += counts.
    Returns (assign int32 [P] or None, hist)."""
    L = load()
    P, D = x.shape
    K = codebook.shape[0]
    dev = x.device
    hist = torch.zeros(K, dtype=torch.int32, device=dev) if hist is None else hist
    if ws is None:
        ws = torch.empty(max(int(L.lgs_codebook_workspace(K)), 4), dtype=torch.uint8, device=dev)
    _check(L.lgs_codebook_assign(_p(x), P, D, _p(codebook), K, _p(assign), _p(hist), _p(ws),
                                 ws.numel(), _stream()), "lgs_codebook_assign")
    return assign, hist


def lgs_hist_cosine(hist, hists, out=None):
    M, K = hists.shape
    out = torch.empty(M, dtype=torch.float32, device=hists.device) if out is None else out
    _check(load().lgs_hist_cosine(_p(hist), _p(hists), M, K, _p(out), _stream()),
           "lgs_hist_cosine")
    return out


def lgs_loop_candidates(sim, centres, cur_centre, tau_hist, radius, top=2, out=None):
    out = torch.empty(top, dtype=torch.int32, device=sim.device) if out is None else out
    cur = (ctypes.c_float * 3)(*[float(v) for v in cur_centre])
    _check(load().lgs_loop_candidates(_p(sim), _p(centres), sim.shape[0], cur, float(tau_hist),
                                      float(radius), top, _p(out), _stream()),
           "lgs_loop_candidates")
    return out


def gs_query_relevance(feats, queries, out=None):
    """[M, Q] cosine of every feature row (fp32/bf16 [M, D]) with every
    compact-space query (fp32 [Q, D])."""
    M, D = feats.shape
    Q = queries.shape[0]
    out = torch.empty((M, Q), dtype=torch.float32, device=feats.device) if out is None else out
    _check(load().gs_query_relevance(_p(feats), _dtype_code(feats), M, D, _p(queries), Q, _p(out),
                                     _stream()), "gs_query_relevance")
    return out
