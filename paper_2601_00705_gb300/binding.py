"""ctypes binding of ``librgs.so`` (the C ABI in ``include/rgs.h``). Argument marshalling only:
every step of the render runs in the library's CUDA kernels.

The library is loaded from ``paper_2601_00705_gb300/_build/librgs.so`` (built by
``paper_2601_00705_gb300.build``). There is no fallback: if the library cannot be built or
loaded, importing it raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

RGS_MAX_VIEWS = 64
(RGS_OK, RGS_ERR_INVALID_ARG, RGS_ERR_CUDA, RGS_ERR_CAPACITY, RGS_ERR_NOMEM, RGS_ERR_STATE,
 RGS_ERR_TOO_LARGE) = range(7)
RGS_STATIC_SCAN_MAX_N = 1 << 26
GRAD_MEANS, GRAD_SCALES, GRAD_QUATS, GRAD_OPACITY, GRAD_SH, GRAD_POSE = 1, 2, 4, 8, 16, 32
GRAD_ALL = 63

# Every function the header declares (checked by the ABI tests).
EXPORTED = ("rgs_create", "rgs_destroy", "rgs_config_default", "rgs_last_error",
            "rgs_render_forward", "rgs_render_backward", "rgs_release_state", "rgs_reserve",
            "rgs_query_stats", "rgs_set_phase_timing", "rgs_phase_times", "rgs_radix_sort_u32",
            "rgs_exclusive_scan_u32", "rgs_exclusive_scan_u32_static", "rgs_copy_tile_lists",
            "rgs_copy_records", "rgs_autotune", "rgs_render_forward_posed",
            "rgs_track_config_default", "rgs_adam_config_default", "rgs_track_grad_weight",
            "rgs_track_loss", "rgs_pose_adam_step", "rgs_seed_config_default", "rgs_triangulate",
            "rgs_init_seeds", "rgs_covisibility", "rgs_render_backward_mapping", "rgs_map_ema",
            "rgs_prune_config_default", "rgs_prune_mask", "rgs_single_pass_scan_bytes",
            "rgs_exclusive_scan_u32_single_pass")

PHASES = ("preprocess", "compact", "depth_sort", "offsets", "duplicate", "tile_sort", "ranges",
          "blend_forward", "blend_backward", "preprocess_backward")


class Gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("world_to_cam", ctypes.c_float * 12)]


class Config(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("znear", ctypes.c_float), ("eps2d", ctypes.c_float),
                ("jac_clamp", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("pixels_per_thread", ctypes.c_int32),
                ("backward_pixels_per_thread", ctypes.c_int32),
                ("sh_ready_event", ctypes.c_void_p)]


class Images(ctypes.Structure):
    _fields_ = [("color", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("alpha", ctypes.c_void_p)]


class ImageGrads(ctypes.Structure):
    _fields_ = [("d_color", ctypes.c_void_p), ("d_depth", ctypes.c_void_p),
                ("d_alpha", ctypes.c_void_p)]


class TrackConfig(ctypes.Structure):
    _fields_ = [("tau_alpha", ctypes.c_float), ("tau_grad", ctypes.c_float),
                ("fit_exposure", ctypes.c_int32)]


class AdamConfig(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("iterations", ctypes.c_int32)]


class SeedConfig(ctypes.Structure):
    _fields_ = [("min_parallax", ctypes.c_float), ("max_reproj", ctypes.c_float),
                ("tie_eps", ctypes.c_float), ("plane_radius", ctypes.c_float),
                ("s_par_cap", ctypes.c_float), ("alpha_lo", ctypes.c_float),
                ("alpha_hi", ctypes.c_float), ("voxel", ctypes.c_float)]


class MapReg(ctypes.Structure):
    _fields_ = [("lambda_iso", ctypes.c_float), ("lambda_alpha", ctypes.c_float),
                ("lambda_mu", ctypes.c_float), ("ema_means", ctypes.c_void_p),
                ("obs_count", ctypes.c_void_p), ("vis_score", ctypes.c_void_p),
                ("value", ctypes.c_void_p)]


class PruneConfig(ctypes.Structure):
    _fields_ = [("min_opacity", ctypes.c_float), ("max_trace", ctypes.c_float),
                ("min_observations", ctypes.c_uint32), ("min_visibility", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [("n_visible", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("n_eval", ctypes.c_int64), ("n_contrib", ctypes.c_int64),
                ("n_nonfinite", ctypes.c_int64),
                ("pair_capacity", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
                ("status", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_needed: bool = True):
    """Loads librgs.so (building it first if it is missing or stale and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        lib = ctypes.CDLL(_build.LIB_PATH)
        P, I32, I64, U32, U64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                 ctypes.c_uint64)
        S = ctypes.c_int
        sig = {
            "rgs_create": (S, [ctypes.POINTER(P), ctypes.c_int]),
            "rgs_destroy": (None, [P]),
            "rgs_config_default": (None, [ctypes.POINTER(Config)]),
            "rgs_last_error": (ctypes.c_char_p, [P]),
            "rgs_render_forward": (S, [P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), I32,
                                       ctypes.POINTER(Config), ctypes.POINTER(Images),
                                       ctypes.POINTER(U64), P]),
            "rgs_render_backward": (S, [P, U64, ctypes.POINTER(ImageGrads), U32, P, P, P, P, P, P,
                                        P]),
            "rgs_release_state": (S, [P, U64]),
            "rgs_reserve": (S, [P, ctypes.POINTER(U64), I64, P]),
            "rgs_query_stats": (S, [P, U64, ctypes.POINTER(Stats), P]),
            "rgs_set_phase_timing": (S, [P, I32]),
            "rgs_phase_times": (S, [P, U64, ctypes.POINTER(ctypes.c_float), I32, P]),
            "rgs_radix_sort_u32": (S, [P, P, P, I64, I32, I32, P]),
            "rgs_exclusive_scan_u32": (S, [P, P, P, I64, P, P]),
            "rgs_exclusive_scan_u32_static": (S, [P, P, I64, P, P]),
            "rgs_single_pass_scan_bytes": (I64, [I64]),
            "rgs_exclusive_scan_u32_single_pass": (S, [P, P, I64, P, P, I64, P, P]),
            "rgs_copy_tile_lists": (S, [P, U64, P, I64, P, ctypes.POINTER(I64), P]),
            "rgs_copy_records": (S, [P, U64, P, P, P]),
            "rgs_autotune": (S, [P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), I32,
                                 ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_float), P]),
            "rgs_render_forward_posed": (S, [P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                             I32, P, ctypes.POINTER(Config),
                                             ctypes.POINTER(Images), ctypes.POINTER(U64), P]),
            "rgs_track_config_default": (None, [ctypes.POINTER(TrackConfig)]),
            "rgs_adam_config_default": (None, [ctypes.POINTER(AdamConfig)]),
            "rgs_track_grad_weight": (S, [P, ctypes.POINTER(Camera), I32, P, ctypes.c_float, P,
                                          P]),
            "rgs_track_loss": (S, [P, ctypes.POINTER(Camera), I32, ctypes.POINTER(TrackConfig),
                                   P, P, P, P, P, P, P, P]),
            "rgs_pose_adam_step": (S, [P, I32, ctypes.POINTER(AdamConfig), P, P, P, P, P]),
            "rgs_seed_config_default": (None, [ctypes.POINTER(SeedConfig)]),
            "rgs_covisibility": (S, [P, P, P, I64, I32, ctypes.c_float, P, P, P]),
            "rgs_render_backward_mapping": (S, [P, U64, ctypes.POINTER(ImageGrads), U32, P, P, P,
                                                P, P, P, ctypes.POINTER(MapReg), P]),
            "rgs_map_ema": (S, [P, I64, P, P, ctypes.c_float, P]),
            "rgs_prune_config_default": (None, [ctypes.POINTER(PruneConfig)]),
            "rgs_prune_mask": (S, [P, I64, P, P, P, P, ctypes.POINTER(PruneConfig), P, P, P]),
            "rgs_triangulate": (S, [P, ctypes.POINTER(Camera), I32, I64, I32, P, P, P, P, P,
                                    ctypes.POINTER(SeedConfig), P, P, P, P, P, P, P]),
            "rgs_init_seeds": (S, [P, ctypes.POINTER(Camera), I32, I64, I32, P, P, P, P, P, P, P,
                                   P, P, I32, ctypes.POINTER(SeedConfig), P, P, P, P, P, P, P,
                                   ctypes.POINTER(I64), P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return _lib


class RGSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"rgs error {status}: {message}")
        self.status = status


def default_config(**overrides) -> Config:
    cfg = Config()
    load().rgs_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "bg":
            cfg.bg = (ctypes.c_float * 3)(*[float(x) for x in v])
        else:
            setattr(cfg, k, v)
    return cfg


def default_track_config(**overrides) -> TrackConfig:
    cfg = TrackConfig()
    load().rgs_track_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def default_adam_config(**overrides) -> AdamConfig:
    cfg = AdamConfig()
    load().rgs_adam_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def default_prune_config(**overrides) -> PruneConfig:
    cfg = PruneConfig()
    load().rgs_prune_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def default_seed_config(**overrides) -> SeedConfig:
    cfg = SeedConfig()
    load().rgs_seed_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def make_cameras(cameras) -> ctypes.Array:
    """Camera dicts (width, height, fx, fy, cx, cy, R [3,3], t [3]) -> rgs_camera array."""
    arr = (Camera * len(cameras))()
    for k, c in enumerate(cameras):
        arr[k].width = int(c["width"])
        arr[k].height = int(c["height"])
        arr[k].fx, arr[k].fy = float(c["fx"]), float(c["fy"])
        arr[k].cx, arr[k].cy = float(c["cx"]), float(c["cy"])
        R = np.asarray(c["R"], dtype=np.float32).reshape(3, 3)
        t = np.asarray(c["t"], dtype=np.float32).reshape(3)
        Rt = np.concatenate([R, t[:, None]], axis=1).reshape(12)
        for j in range(12):
            arr[k].world_to_cam[j] = float(Rt[j])
    return arr


class Context:
    """Owns one rgs_ctx on a CUDA device. Methods take raw device pointers (ints)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.rgs_create(ctypes.byref(h), int(device))
        if st != RGS_OK:
            raise RGSError(st, f"rgs_create(device={device}) failed")
        self.handle = h

    def _check(self, st: int):
        if st != RGS_OK:
            msg = self.lib.rgs_last_error(self.handle)
            raise RGSError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, g: Gaussians, cams, cfg: Config, images: Images, state: int,
                stream: int) -> int:
        h = ctypes.c_uint64(state)
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        self._check(self.lib.rgs_render_forward(self.handle, ctypes.byref(g), cam_arr,
                                                len(cam_arr), ctypes.byref(cfg),
                                                ctypes.byref(images), ctypes.byref(h),
                                                ctypes.c_void_p(stream)))
        return h.value

    def forward_posed(self, g: Gaussians, cams, world_to_cam: int, cfg: Config, images: Images,
                      state: int, stream: int) -> int:
        h = ctypes.c_uint64(state)
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        self._check(self.lib.rgs_render_forward_posed(
            self.handle, ctypes.byref(g), cam_arr, len(cam_arr), ctypes.c_void_p(world_to_cam),
            ctypes.byref(cfg), ctypes.byref(images), ctypes.byref(h), ctypes.c_void_p(stream)))
        return h.value

    def track_grad_weight(self, cams, observed: int, tau_grad: float, w: int, stream: int):
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        self._check(self.lib.rgs_track_grad_weight(self.handle, cam_arr, len(cam_arr),
                                                   ctypes.c_void_p(observed), float(tau_grad),
                                                   ctypes.c_void_p(w), ctypes.c_void_p(stream)))

    def track_loss(self, cams, cfg: TrackConfig, color: int, alpha: int, observed: int,
                   w_grad: int, d_color: int, loss: int, gain_bias: int, stream: int):
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        P = ctypes.c_void_p
        self._check(self.lib.rgs_track_loss(self.handle, cam_arr, len(cam_arr), ctypes.byref(cfg),
                                            P(color), P(alpha), P(observed), P(w_grad or None),
                                            P(d_color), P(loss), P(gain_bias), P(stream)))

    def pose_adam_step(self, n_views: int, cfg: AdamConfig, d_pose: int, adam_state: int,
                       step: int, world_to_cam: int, stream: int):
        P = ctypes.c_void_p
        self._check(self.lib.rgs_pose_adam_step(self.handle, int(n_views), ctypes.byref(cfg),
                                                P(d_pose), P(adam_state), P(step),
                                                P(world_to_cam), P(stream)))

    def covisibility(self, alpha_a: int, alpha_b: int, n: int, n_pairs: int, tau: float,
                     counts: int, iou: int, stream: int):
        P = ctypes.c_void_p
        self._check(self.lib.rgs_covisibility(self.handle, P(alpha_a), P(alpha_b), int(n),
                                              int(n_pairs), float(tau), P(counts), P(iou),
                                              P(stream)))

    def triangulate(self, cams, m: int, k: int, ptrs: dict, cfg: SeedConfig, stream: int):
        """ptrs: device pointers ref_view, ref_xy, nb_view, nb_xy, nb_conf (inputs) and valid, X,
        best, err, angle, kappa (outputs)."""
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        P = ctypes.c_void_p
        self._check(self.lib.rgs_triangulate(
            self.handle, cam_arr, len(cam_arr), int(m), int(k), P(ptrs["ref_view"]),
            P(ptrs["ref_xy"]), P(ptrs["nb_view"]), P(ptrs["nb_xy"]), P(ptrs["nb_conf"]),
            ctypes.byref(cfg), P(ptrs["valid"]), P(ptrs["X"]), P(ptrs["best"]), P(ptrs["err"]),
            P(ptrs["angle"]), P(ptrs["kappa"]), P(stream)))

    def init_seeds(self, cams, m: int, k: int, ptrs: dict, sh_degree: int, cfg: SeedConfig,
                   stream: int) -> int:
        """ptrs: device pointers ref_view, nb_view, valid, X, err, angle, kappa, observed,
        gain_bias (inputs) and index, means, log_scales, quats, opacity_logits, sh, normals
        (outputs, capacity m). Returns the number of seeds written."""
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        P = ctypes.c_void_p
        n = ctypes.c_int64(0)
        self._check(self.lib.rgs_init_seeds(
            self.handle, cam_arr, len(cam_arr), int(m), int(k), P(ptrs["ref_view"]),
            P(ptrs["nb_view"]), P(ptrs["valid"]), P(ptrs["X"]), P(ptrs["err"]), P(ptrs["angle"]),
            P(ptrs["kappa"]), P(ptrs["observed"]), P(ptrs["gain_bias"]), int(sh_degree),
            ctypes.byref(cfg), P(ptrs["index"]), P(ptrs["means"]), P(ptrs["log_scales"]),
            P(ptrs["quats"]), P(ptrs["opacity_logits"]), P(ptrs["sh"]), P(ptrs["normals"]),
            ctypes.byref(n), P(stream)))
        return int(n.value)

    def backward_mapping(self, state: int, grads: ImageGrads, grad_mask: int, ptrs: list,
                         reg: MapReg, stream: int):
        """ptrs: d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_pose (0 = none)."""
        P = ctypes.c_void_p
        self._check(self.lib.rgs_render_backward_mapping(
            self.handle, ctypes.c_uint64(state), ctypes.byref(grads), grad_mask,
            *[P(p or None) for p in ptrs], ctypes.byref(reg), P(stream)))

    def map_ema(self, n: int, means: int, ema: int, eta: float, stream: int):
        P = ctypes.c_void_p
        self._check(self.lib.rgs_map_ema(self.handle, int(n), P(means), P(ema), float(eta),
                                         P(stream)))

    def prune_mask(self, n: int, log_scales: int, logits: int, obs_count: int, vis_score: int,
                   cfg: "PruneConfig", keep: int, n_keep: int, stream: int):
        P = ctypes.c_void_p
        self._check(self.lib.rgs_prune_mask(self.handle, int(n), P(log_scales), P(logits),
                                            P(obs_count), P(vis_score), ctypes.byref(cfg),
                                            P(keep), P(n_keep), P(stream)))

    def backward(self, state: int, grads: ImageGrads, grad_mask: int, d_means: int,
                 d_log_scales: int, d_quats: int, d_opacity_logits: int, d_sh: int, d_pose: int,
                 stream: int):
        P = ctypes.c_void_p
        self._check(self.lib.rgs_render_backward(
            self.handle, ctypes.c_uint64(state), ctypes.byref(grads), ctypes.c_uint32(grad_mask),
            P(d_means or None), P(d_log_scales or None), P(d_quats or None),
            P(d_opacity_logits or None), P(d_sh or None), P(d_pose or None), P(stream)))

    def autotune(self, g: Gaussians, cams, cfg: Config, stream: int) -> float:
        """Times every tile shape / pixels-per-thread choice and writes the fastest into cfg;
        returns its forward + backward milliseconds (0 when served from the cache)."""
        cam_arr = cams if isinstance(cams, ctypes.Array) else make_cameras(cams)
        ms = ctypes.c_float(0.0)
        self._check(self.lib.rgs_autotune(self.handle, ctypes.byref(g), cam_arr, len(cam_arr),
                                          ctypes.byref(cfg), ctypes.byref(ms),
                                          ctypes.c_void_p(stream)))
        return ms.value

    def release(self, state: int):
        if state:
            self._check(self.lib.rgs_release_state(self.handle, ctypes.c_uint64(state)))

    def reserve(self, state: int, pair_capacity: int, stream: int = 0) -> int:
        h = ctypes.c_uint64(state)
        self._check(self.lib.rgs_reserve(self.handle, ctypes.byref(h), int(pair_capacity),
                                         ctypes.c_void_p(stream)))
        return h.value

    def stats(self, state: int, stream: int = 0) -> dict:
        s = Stats()
        self._check(self.lib.rgs_query_stats(self.handle, ctypes.c_uint64(state), ctypes.byref(s),
                                             ctypes.c_void_p(stream)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def set_phase_timing(self, enable: bool):
        self._check(self.lib.rgs_set_phase_timing(self.handle, int(bool(enable))))

    def phase_times(self, state: int, stream: int = 0) -> dict:
        ms = (ctypes.c_float * len(PHASES))()
        self._check(self.lib.rgs_phase_times(self.handle, ctypes.c_uint64(state), ms, len(PHASES),
                                             ctypes.c_void_p(stream)))
        return dict(zip(PHASES, [float(x) for x in ms]))

    def tile_lists(self, state: int, total_tiles: int, stream: int = 0):
        """(pair values [P] u32, ranges [total_tiles, 2] u32) of a state's sorted pair list."""
        n = ctypes.c_int64()
        self._check(self.lib.rgs_copy_tile_lists(self.handle, ctypes.c_uint64(state), None, 0,
                                                 None, ctypes.byref(n), ctypes.c_void_p(stream)))
        vals = np.zeros(max(n.value, 1), dtype=np.uint32)
        ranges = np.zeros((max(total_tiles, 1), 2), dtype=np.uint32)
        self._check(self.lib.rgs_copy_tile_lists(
            self.handle, ctypes.c_uint64(state), vals.ctypes.data_as(ctypes.c_void_p), vals.size,
            ranges.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n), ctypes.c_void_p(stream)))
        return vals[:n.value], ranges[:total_tiles]

    def tile_ranges(self, state: int, total_tiles: int, stream: int = 0):
        """[first, last + 1) of every global tile's run in a state's sorted pair list."""
        n = ctypes.c_int64()
        ranges = np.zeros((max(total_tiles, 1), 2), dtype=np.uint32)
        self._check(self.lib.rgs_copy_tile_lists(
            self.handle, ctypes.c_uint64(state), None, 0, ranges.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(n), ctypes.c_void_p(stream)))
        return ranges[:total_tiles]

    def records(self, state: int, vn: int, stream: int = 0):
        """(records [vn, 12] f32, tile counts [vn] u32) of a state."""
        rec = np.zeros((max(vn, 1), 12), dtype=np.float32)
        nt = np.zeros(max(vn, 1), dtype=np.uint32)
        self._check(self.lib.rgs_copy_records(self.handle, ctypes.c_uint64(state),
                                              rec.ctypes.data_as(ctypes.c_void_p),
                                              nt.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.c_void_p(stream)))
        return rec[:vn], nt[:vn]

    def radix_sort_u32(self, keys: int, vals: int, n: int, begin_bit: int, end_bit: int,
                       stream: int = 0):
        self._check(self.lib.rgs_radix_sort_u32(self.handle, ctypes.c_void_p(keys),
                                                ctypes.c_void_p(vals or None), int(n),
                                                int(begin_bit), int(end_bit),
                                                ctypes.c_void_p(stream)))

    def exclusive_scan_u32(self, inp: int, out: int, n: int, total: int = 0, stream: int = 0):
        self._check(self.lib.rgs_exclusive_scan_u32(self.handle, ctypes.c_void_p(inp),
                                                    ctypes.c_void_p(out), int(n),
                                                    ctypes.c_void_p(total or None),
                                                    ctypes.c_void_p(stream)))
