"""ctypes binding of the learned warm start (include/ni_cnn.h): marshalling only.

The network is trained and run by libni's BF16 tensor-core kernels; this module
passes device pointers of torch tensors and the current stream.
"""
from __future__ import annotations

import ctypes as C
import struct

import numpy as np
import torch

from . import ni

HALO = 6
MAGIC = b"NICNN001"


def _lib():
    L = ni.load()
    if not getattr(L, "_cnn_ready", False):
        vp = C.c_void_p
        L.ni_cnn_num_params.restype = C.c_int
        L.ni_cnn_create.argtypes = [C.c_int, C.c_int, C.c_uint64, C.POINTER(vp)]
        L.ni_cnn_destroy.argtypes = [vp]
        L.ni_cnn_get_params.argtypes = [vp, vp]
        L.ni_cnn_set_params.argtypes = [vp, vp]
        L.ni_cnn_forward.argtypes = [vp, vp, C.c_int, vp, vp]
        L.ni_cnn_loss_grad.argtypes = [vp, vp, vp, vp, vp, C.c_int, C.c_float, C.POINTER(C.c_double), vp, vp]
        L.ni_cnn_train_step.argtypes = [vp, vp, vp, vp, vp, C.c_int, C.c_float, C.c_float,
                                        C.POINTER(C.c_double), vp]
        L.ni_cnn_edge_targets.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.POINTER(ni.Camera), C.c_double, vp, vp]
        L.ni_cnn_make_tiles.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, vp, vp]
        for f in ("ni_cnn_create", "ni_cnn_destroy", "ni_cnn_get_params", "ni_cnn_set_params", "ni_cnn_forward",
                  "ni_cnn_loss_grad", "ni_cnn_train_step", "ni_cnn_edge_targets", "ni_cnn_make_tiles"):
            getattr(L, f).restype = C.c_int
        L._cnn_ready = True
    return L


def num_params() -> int:
    return _lib().ni_cnn_num_params()


def _ck(rc, what):
    if rc != 0:
        raise ni.NIError(rc, what)


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Net:
    """The 6-layer warm-start network on the current CUDA device."""

    def __init__(self, max_batch: int, tile: int, seed: int = 0):
        self.L = _lib()
        self.tile, self.max_batch = tile, max_batch
        h = C.c_void_p()
        _ck(self.L.ni_cnn_create(max_batch, tile, seed, C.byref(h)), "ni_cnn_create")
        self.h = h
        self.np = num_params()

    def close(self):
        if getattr(self, "h", None):
            self.L.ni_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.np, np.float32)
        _ck(self.L.ni_cnn_get_params(self.h, out.ctypes.data), "get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.np
        _ck(self.L.ni_cnn_set_params(self.h, p.ctypes.data), "set_params")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: float32 [B, T+12, T+12, 4] on the device -> [B, T, T, 5]."""
        B = x.shape[0]
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        assert tuple(x.shape[1:]) == (self.tile + 2 * HALO, self.tile + 2 * HALO, 4)
        out = torch.empty((B, self.tile, self.tile, 5), dtype=torch.float32, device=x.device)
        _ck(self.L.ni_cnn_forward(self.h, x.data_ptr(), B, out.data_ptr(), _stream()), "forward")
        return out

    def loss_grad(self, x, tz, tl, tw, w_weight=0.1, want_grad=True):
        B = x.shape[0]
        loss = (C.c_double * 3)()
        grad = np.zeros(self.np, np.float32) if want_grad else None
        _ck(self.L.ni_cnn_loss_grad(self.h, x.data_ptr(), tz.data_ptr(), tl.data_ptr(), tw.data_ptr(), B,
                                    w_weight, loss, grad.ctypes.data if want_grad else None, _stream()),
            "loss_grad")
        return (loss[0], loss[1], loss[2]), grad

    def train_step(self, x, tz, tl, tw, lr, w_weight=0.1):
        B = x.shape[0]
        loss = (C.c_double * 3)()
        _ck(self.L.ni_cnn_train_step(self.h, x.data_ptr(), tz.data_ptr(), tl.data_ptr(), tw.data_ptr(), B,
                                     w_weight, lr, loss, _stream()), "train_step")
        return loss[0], loss[1], loss[2]

    def save(self, path: str):
        p = self.get_params()
        with open(path, "wb") as f:
            f.write(MAGIC)
            f.write(struct.pack("<ii", self.np, self.tile))
            f.write(p.tobytes())


def edge_targets(normals: torch.Tensor, mask: torch.Tensor, logdepth: torch.Tensor, camera, k=2.0):
    H, W = mask.shape
    out = torch.empty((H, W, 4), dtype=torch.float32, device=normals.device)
    cam = ni.Camera(int(camera["camera"]), float(camera["fx"]), float(camera["fy"]), float(camera["cx"]),
                    float(camera["cy"]))
    _ck(_lib().ni_cnn_edge_targets(normals.data_ptr(), mask.data_ptr(), logdepth.data_ptr(), H, W, C.byref(cam),
                                   k, out.data_ptr(), _stream()), "edge_targets")
    return out


def make_tiles(normals: torch.Tensor, mask: torch.Tensor, tile: int) -> torch.Tensor:
    H, W = mask.shape
    nt = ((H + tile - 1) // tile) * ((W + tile - 1) // tile)
    out = torch.empty((nt, tile + 2 * HALO, tile + 2 * HALO, 4), dtype=torch.float32, device=normals.device)
    _ck(_lib().ni_cnn_make_tiles(normals.data_ptr(), mask.data_ptr(), H, W, tile, out.data_ptr(), _stream()),
        "make_tiles")
    return out
