"""Thin ctypes binding of libni (include/ni.h): argument marshalling only.

Every step of the integration runs in the library's CUDA kernels; this module
checks tensor dtypes, devices and layouts, passes raw device pointers and the
current torch stream, and turns status codes into exceptions.  There is no CPU
fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Tuple

import torch

from . import build as _build

NI_OK = 0
NI_ERR_NOT_CONVERGED = 4
STATUS = {0: "NI_OK", 1: "NI_ERR_INVALID_ARG", 2: "NI_ERR_CUDA", 3: "NI_ERR_OOM",
          4: "NI_ERR_NOT_CONVERGED", 5: "NI_ERR_TIMEOUT", 6: "NI_ERR_STATE", 7: "NI_ERR_NO_NET"}

EXPORTS = ["ni_config_default", "ni_create", "ni_destroy", "ni_seed_components",
           "ni_solve_components", "ni_solve_scales", "ni_merge", "ni_merge_residuals",
           "ni_integrate", "ni_integrate_host", "ni_get_logdepth", "ni_load_net", "ni_last_error",
           "ni_status_string", "ni_seed_components_noalloc", "ni_min_made", "ni_load_tuning"]


class Camera(C.Structure):
    _fields_ = [("camera", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double)]


class Config(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("cam", Camera), ("theta_c_deg", C.c_double),
                ("connectivity", C.c_int), ("k", C.c_double), ("L", C.c_double), ("U", C.c_double),
                ("T", C.c_int), ("dE_max", C.c_double), ("can_merge", C.c_int),
                ("freq_merging", C.c_int), ("n_fill_irls", C.c_int), ("cg_rtol", C.c_double),
                ("cg_maxit", C.c_int), ("scale_rtol", C.c_double), ("scale_maxit", C.c_int),
                ("precision", C.c_int), ("batched", C.c_int), ("use_graph", C.c_int),
                ("warm_start", C.c_int), ("hard_outliers", C.c_int), ("validate", C.c_int),
                ("ctas_per_sm", C.c_int), ("mg_coarse_sweeps", C.c_int), ("precond", C.c_int), ("mg_omega", C.c_double),
                ("mg_correction", C.c_double), ("mg_cta_cells", C.c_int), ("mg_flags", C.c_int),
                ("fill_kernels", C.c_int), ("scale_solver", C.c_int), ("bini_residual", C.c_int),
                ("learned_weights", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("ms_seed", C.c_double), ("ms_setup", C.c_double), ("ms_fill", C.c_double),
                ("ms_scale", C.c_double), ("ms_output", C.c_double), ("ms_total", C.c_double),
                ("n_valid", C.c_int64), ("K0", C.c_int32), ("K_final", C.c_int32),
                ("n_inter0", C.c_int32), ("merges", C.c_int32), ("scale_iters", C.c_int32),
                ("fill_iters", C.c_int32), ("fill_unconverged", C.c_int32),
                ("scale_cg_iters", C.c_int32), ("n_energy", C.c_int32), ("energy", C.c_double * 64),
                ("ms_fill_solve", C.c_double), ("fill_px_iters", C.c_int64), ("kernel_launches", C.c_int64),
                ("warm_fallbacks", C.c_int32), ("fill_fallbacks", C.c_int32),
                ("scale_cg_total", C.c_int64)]

    def as_dict(self) -> Dict[str, object]:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "energy"}
        d["energy"] = [self.energy[i] for i in range(self.n_energy)]
        return d


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libni.so (ctypes).  Raises if it is missing and not built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libni is not built ({path}); run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(path)
    vp, i32p = C.c_void_p, C.POINTER(C.c_int32)
    L.ni_config_default.argtypes = [C.POINTER(Config), C.c_int, C.c_int]
    L.ni_config_default.restype = None
    L.ni_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    L.ni_destroy.argtypes = [vp]
    L.ni_seed_components.argtypes = [vp, vp, vp, vp, i32p, vp]
    L.ni_solve_components.argtypes = [vp, vp, vp]
    L.ni_solve_scales.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_double), C.POINTER(C.c_int), vp]
    L.ni_merge.argtypes = [vp, vp, i32p, vp]
    L.ni_merge_residuals.argtypes = [vp, vp, vp, i32p, vp]
    L.ni_integrate.argtypes = [vp, vp, vp, vp, vp, C.POINTER(Stats), vp]
    L.ni_integrate_host.argtypes = [vp, vp, vp, vp, C.POINTER(Stats), vp]
    L.ni_get_logdepth.argtypes = [vp, vp, vp]
    L.ni_seed_components_noalloc.argtypes = [vp, vp, C.c_int, C.c_int, C.POINTER(Camera), C.c_double,
                                             vp, vp, vp]
    L.ni_load_net.argtypes = [vp, C.c_char_p]
    L.ni_load_tuning.argtypes = [vp, C.c_char_p]
    L.ni_min_made.argtypes = [vp, vp, C.c_int, vp, C.c_int32, vp, C.POINTER(C.c_double), vp, vp, vp]
    L.ni_last_error.argtypes = [vp]
    L.ni_last_error.restype = C.c_char_p
    L.ni_status_string.argtypes = [C.c_int]
    L.ni_status_string.restype = C.c_char_p
    for f in EXPORTS:
        if f not in ("ni_config_default", "ni_last_error", "ni_status_string"):
            getattr(L, f).restype = C.c_int
    _LIB = L
    return L


class NIError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_net_path() -> str:
    """The trained warm-start network shipped with the package."""
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "nets", "warmstart_256.bin")


def default_tuning_path() -> str:
    """The tuning table written by tune.py on GB300 and shipped with the package."""
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.txt")


def default_config(H: int, W: int) -> Config:
    cfg = Config()
    load().ni_config_default(C.byref(cfg), H, W)
    return cfg


def config_for(H: int, W: int, camera: Dict[str, float], params: Optional[Dict] = None, **over) -> Config:
    """Config for an H x W map with camera dict {"camera", "fx", "fy", "cx", "cy"}
    and method hyper-parameters (theta_c_deg None = pixel-level limit)."""
    cfg = default_config(H, W)
    cfg.cam.camera = int(camera["camera"])
    cfg.cam.fx, cfg.cam.fy = float(camera["fx"]), float(camera["fy"])
    cfg.cam.cx, cfg.cam.cy = float(camera["cx"]), float(camera["cy"])
    p = dict(params or {})
    p.update(over)
    for k, v in p.items():
        if k == "theta_c_deg":
            cfg.theta_c_deg = -1.0 if v is None else float(v)
        elif hasattr(cfg, k) and k not in ("cam", "H", "W"):
            setattr(cfg, k, type(getattr(cfg, k))(v))
    return cfg


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _check_dev(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Integrator:
    """One handle of libni for H x W maps (ni_create / ni_destroy)."""

    def __init__(self, cfg: Config):
        self.L = load()
        self.cfg = cfg
        self.H, self.W = cfg.H, cfg.W
        h = C.c_void_p()
        rc = self.L.ni_create(C.byref(cfg), C.byref(h))
        if rc != NI_OK:
            raise NIError(rc, "ni_create failed (invalid config or out of memory)")
        self.h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._inputs = None

    def close(self):
        if getattr(self, "h", None):
            self.L.ni_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, rc, allow=()):
        if rc != NI_OK and rc not in allow:
            raise NIError(rc, self.L.ni_last_error(self.h).decode())
        return rc

    # -- stage calls ---------------------------------------------------------
    def seed_components(self, normals: torch.Tensor, mask: torch.Tensor) -> Tuple[torch.Tensor, int]:
        _check_dev(normals, torch.float32, (self.H, self.W, 4), "normals")
        _check_dev(mask, torch.uint8, (self.H, self.W), "mask")
        self._inputs = (normals, mask)          # the handle reads them until the fill is done
        labels = torch.empty((self.H, self.W), dtype=torch.int32, device=normals.device)
        K = C.c_int32()
        self._raise(self.L.ni_seed_components(self.h, normals.data_ptr(), mask.data_ptr(),
                                              labels.data_ptr(), C.byref(K), _stream()))
        return labels, K.value

    def solve_components(self, allow_unconverged=False) -> torch.Tensor:
        z = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
        self._raise(self.L.ni_solve_components(self.h, z.data_ptr(), _stream()),
                    (NI_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return z

    def solve_scales(self, max_iters: int, logdepth: Optional[torch.Tensor] = None):
        """Returns (iterations run, energies, log-depth tensor)."""
        z = logdepth
        if z is None:
            z = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
            ptr = None
        else:
            _check_dev(z, torch.float32, (self.H, self.W), "logdepth")
            ptr = z.data_ptr()
        e = (C.c_double * max(1, max_iters))()
        it = C.c_int()
        self._raise(self.L.ni_solve_scales(self.h, max_iters, ptr, e, C.byref(it), _stream()))
        if ptr is None:
            self._raise(self.L.ni_get_logdepth(self.h, z.data_ptr(), _stream()))
        return it.value, [e[i] for i in range(it.value)], z

    def logdepth(self) -> torch.Tensor:
        z = torch.empty((self.H, self.W), dtype=torch.float32, device=self.device)
        self._raise(self.L.ni_get_logdepth(self.h, z.data_ptr(), _stream()))
        return z

    def merge(self) -> Tuple[torch.Tensor, int]:
        labels = torch.empty((self.H, self.W), dtype=torch.int32, device=self.device)
        K = C.c_int32()
        self._raise(self.L.ni_merge(self.h, labels.data_ptr(), C.byref(K), _stream()))
        return labels, K.value

    def merge_residuals(self, chi_abs: torch.Tensor) -> Tuple[torch.Tensor, int]:
        _check_dev(chi_abs, torch.float32, (self.H, self.W, 4 if self.cfg.connectivity == 8 else 2), "chi_abs")
        labels = torch.empty((self.H, self.W), dtype=torch.int32, device=self.device)
        K = C.c_int32()
        self._raise(self.L.ni_merge_residuals(self.h, chi_abs.data_ptr(), labels.data_ptr(), C.byref(K),
                                              _stream()))
        return labels, K.value

    def integrate(self, normals: torch.Tensor, mask: torch.Tensor, allow_unconverged=False):
        """Algorithm 1 end to end on device tensors: (depth, labels, stats dict)."""
        _check_dev(normals, torch.float32, (self.H, self.W, 4), "normals")
        _check_dev(mask, torch.uint8, (self.H, self.W), "mask")
        depth = torch.empty((self.H, self.W), dtype=torch.float32, device=normals.device)
        labels = torch.empty((self.H, self.W), dtype=torch.int32, device=normals.device)
        st = Stats()
        self._raise(self.L.ni_integrate(self.h, normals.data_ptr(), mask.data_ptr(), depth.data_ptr(),
                                        labels.data_ptr(), C.byref(st), _stream()),
                    (NI_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return depth, labels, st.as_dict()

    def integrate_host(self, normals: torch.Tensor, mask: torch.Tensor, depth_out: torch.Tensor,
                       allow_unconverged=False):
        """Algorithm 1 on HOST tensors (pinned for full copy speed); the copies run
        inside the library call.  Writes depth_out (float32 CPU tensor)."""
        for t, name in ((normals, "normals"), (mask, "mask"), (depth_out, "depth_out")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CPU tensor")
        st = Stats()
        self._raise(self.L.ni_integrate_host(self.h, normals.data_ptr(), mask.data_ptr(),
                                             depth_out.data_ptr(), C.byref(st), _stream()),
                    (NI_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return st.as_dict()

    def load_tuning(self, path: Optional[str] = None):
        """Knobs left at 0 in the config come from the tuning table at `path`
        (default: the table shipped for GB300) for every later map."""
        path = default_tuning_path() if path is None else path
        self._raise(self.L.ni_load_tuning(self.h, path.encode()))

    def load_net(self, path: str):
        self._raise(self.L.ni_load_net(self.h, path.encode()))

    # -- quality diagnostic ----------------------------------------------------
    def min_made(self, z: torch.Tensor, depth_gt: torch.Tensor, labels: Optional[torch.Tensor] = None,
                 K: int = 1, z_is_log: bool = True, per_component: bool = False):
        """ni_min_made: the minimum mean absolute depth error one scale per
        component reaches against depth_gt (labels None: the MADE after the best
        global scale).  Returns the MADE, or (MADE, per-component MADE [K],
        per-component scale [K]) as float64 CUDA tensors if per_component."""
        _check_dev(z, torch.float32, (self.H, self.W), "z")
        _check_dev(depth_gt, torch.float32, (self.H, self.W), "depth_gt")
        if labels is not None:
            _check_dev(labels, torch.int32, (self.H, self.W), "labels")
        else:
            K = 1
        made = C.c_double()
        comp = scale = None
        if per_component:
            comp = torch.empty(K, dtype=torch.float64, device=z.device)
            scale = torch.empty(K, dtype=torch.float64, device=z.device)
        self._raise(self.L.ni_min_made(self.h, z.data_ptr(), int(bool(z_is_log)),
                                       None if labels is None else labels.data_ptr(), K,
                                       depth_gt.data_ptr(), C.byref(made),
                                       None if comp is None else comp.data_ptr(),
                                       None if scale is None else scale.data_ptr(), _stream()))
        return (made.value, comp, scale) if per_component else made.value
