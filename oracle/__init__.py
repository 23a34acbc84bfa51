"""FP64 CPU oracle of the differentiable Gaussian-splatting rasterizer (Section 3.1, Eq. proj and
Eq. alpha; Appendix C.1; pose Jacobians of Section 3.2.3).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. The product path (the CUDA library and its Python
binding) never imports, links or runs it, and the oracle imports nothing from the product package.

The arithmetic lives in ``rgs_oracle.cpp`` (plain C++17, double precision, std::thread over image
rows). This module compiles it with g++ and marshals numpy arrays through ctypes.

Inputs are plain numpy arrays (any float dtype; promoted to float64 here):
  means [N,3], log_scales [N,3], quats [N,4] (w, x, y, z; need not be unit), opacity_logits [N],
  sh [N,K,3] with K = (degree+1)^2;
  cameras: a sequence of dicts with width, height, fx, fy, cx, cy, R [3,3], t [3]
  (world-to-camera, mu^C = R mu^W + t);
  config: dict overriding DEFAULT_CONFIG.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgs_oracle.cpp")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "librgs_oracle.so")

DEFAULT_CONFIG = dict(
    alpha_min=1.0 / 255.0,
    alpha_max=0.99,
    t_min=1e-4,
    znear=0.2,
    eps2d=0.3,
    jac_clamp=1.3,
    bg=(0.0, 0.0, 0.0),
    # Ambiguity margins (relative) for the discrete decisions an FP32 renderer may take the other
    # way, on top of the modelled float32 error of each quantity (see rgs_oracle.cpp):
    # margin_alpha around alpha_min / alpha_max in ln(o G) (the hardware exponential's error),
    # margin_t around t_min in ln T, margin_z the oracle's own depth rounding.
    margin_alpha=2e-6,
    margin_t=5e-6,
    margin_z=1e-15,
    margin_g=1e-5,
    margin_effect=1e-5,
    margin_cont=3e-5,
)

# Pixel ambiguity bits (see rgs_oracle.cpp). FORWARD_AMBIGUOUS marks pixels where a discrete
# decision (coverage, stop, order, near plane) lies within FP32 rounding of its threshold, so an
# FP32 renderer may legitimately take the other branch; BACKWARD_AMBIGUOUS adds gradient kinks.
# AMB_COND (the propagated FP32 error bound of the colour exceeds margin_cont) involves no
# decision and excludes nothing: such pixels are compared at the full tolerance in both the
# forward and the backward comparison; the bit only reports where the bound is large.
AMB_ALPHA_MIN, AMB_ALPHA_MAX, AMB_T_MIN, AMB_DEPTH_TIE, AMB_NEAR, AMB_GRAD_KINK, AMB_COND = (
    1, 2, 4, 8, 16, 32, 64)
FORWARD_AMBIGUOUS = AMB_ALPHA_MIN | AMB_T_MIN | AMB_DEPTH_TIE | AMB_NEAR
BACKWARD_AMBIGUOUS = FORWARD_AMBIGUOUS | AMB_ALPHA_MAX | AMB_GRAD_KINK

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle shared library with g++ (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_sh_basis.argtypes = [I, I, P, P]
            lib.oracle_sh_basis.restype = None
            lib.oracle_quat_to_rotmat.argtypes = [I, P, P]
            lib.oracle_quat_to_rotmat.restype = None
            lib.oracle_project.argtypes = [I, I, P, P, P, P, P, I, P, P, P]
            lib.oracle_project.restype = None
            lib.oracle_render.argtypes = [I, I, P, P, P, P, P, I, P, P, P, I, I,
                                          P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.oracle_render.restype = I
            lib.oracle_log_og_bound.argtypes = [I, I, P, P, P, P, P, I, P, P, I, P, P]
            lib.oracle_log_og_bound.restype = None
            lib.oracle_set_dense_limit.argtypes = [ctypes.c_double]
            lib.oracle_set_dense_limit.restype = None
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cam_array(cameras) -> np.ndarray:
    out = np.zeros((len(cameras), 18), dtype=np.float64)
    for v, c in enumerate(cameras):
        out[v, 0] = c["width"]
        out[v, 1] = c["height"]
        out[v, 2:6] = [c["fx"], c["fy"], c["cx"], c["cy"]]
        out[v, 6:15] = np.asarray(c["R"], dtype=np.float64).reshape(9)
        out[v, 15:18] = np.asarray(c["t"], dtype=np.float64).reshape(3)
    return out


def _cfg_array(config) -> np.ndarray:
    c = dict(DEFAULT_CONFIG)
    if config:
        c.update(config)
    bg = tuple(c["bg"])
    return np.array([c["alpha_min"], c["alpha_max"], c["t_min"], c["znear"], c["eps2d"],
                     c["jac_clamp"], bg[0], bg[1], bg[2], c["margin_alpha"], c["margin_t"],
                     c["margin_z"], c["margin_g"], c["margin_effect"], c["margin_cont"]],
                    dtype=np.float64)


def _degree_of(sh) -> int:
    K = sh.shape[1]
    deg = int(round(K ** 0.5)) - 1
    if (deg + 1) ** 2 != K or not 0 <= deg <= 3:
        raise ValueError(f"sh must be [N, (d+1)^2, 3] with d <= 3, got {sh.shape}")
    return deg


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def set_dense_limit(nbytes: float) -> None:
    """Byte limit of the dense per-thread gradient accumulators (above it: hash maps)."""
    _load().oracle_set_dense_limit(float(nbytes))


def sh_basis(degree: int, dirs) -> np.ndarray:
    """Real SH basis (Eq. app-sh) of unit directions dirs [n,3] -> [n,16]."""
    lib = _load()
    d = _f64(dirs, (-1, 3))
    out = np.zeros((d.shape[0], 16), dtype=np.float64)
    lib.oracle_sh_basis(int(degree), d.shape[0], _ptr(d), _ptr(out))
    return out


def quat_to_rotmat(quats) -> np.ndarray:
    lib = _load()
    q = _f64(quats, (-1, 4))
    out = np.zeros((q.shape[0], 3, 3), dtype=np.float64)
    lib.oracle_quat_to_rotmat(q.shape[0], _ptr(q), _ptr(out))
    return out


def project(g: dict, cameras, config=None) -> dict:
    """Per-(view, Gaussian) screen-space quantities of Eq. proj, [V, N] leading dims."""
    lib = _load()
    means = _f64(g["means"], (-1, 3))
    n = means.shape[0]
    sh = _f64(g["sh"])
    deg = _degree_of(sh)
    cams = _cam_array(cameras)
    V = cams.shape[0]
    out = np.zeros((V, n, 16), dtype=np.float64)
    lib.oracle_project(n, deg, _ptr(means), _ptr(_f64(g["log_scales"], (n, 3))),
                       _ptr(_f64(g["quats"], (n, 4))), _ptr(_f64(g["opacity_logits"], (n,))),
                       _ptr(sh), V, _ptr(cams), _ptr(_cfg_array(config)), _ptr(out))
    return dict(valid=out[..., 0] > 0.5, mean2d=out[..., 1:3], cov2d=out[..., 3:6],
                conic=out[..., 6:9], depth=out[..., 9], opacity=out[..., 10], rgb=out[..., 11:14],
                kappa=out[..., 14], flags=out[..., 15].astype(np.int32))


def log_og_bound(g: dict, cameras, items, config=None) -> tuple[np.ndarray, np.ndarray]:
    """ln(o G) in double precision at (view, Gaussian, x, y) items [m, 4], and the float32 error
    bound the oracle's ambiguity flags use there; (-inf, 0) for a Gaussian culled in the view."""
    lib = _load()
    means = _f64(g["means"], (-1, 3))
    n = means.shape[0]
    sh = _f64(g["sh"])
    deg = _degree_of(sh)
    cams = _cam_array(cameras)
    it = _f64(items, (-1, 4))
    out = np.zeros((it.shape[0], 2), dtype=np.float64)
    lib.oracle_log_og_bound(n, deg, _ptr(means), _ptr(_f64(g["log_scales"], (n, 3))),
                            _ptr(_f64(g["quats"], (n, 4))), _ptr(_f64(g["opacity_logits"], (n,))),
                            _ptr(sh), cams.shape[0], _ptr(cams), _ptr(_cfg_array(config)),
                            it.shape[0], _ptr(it), _ptr(out))
    return out[:, 0], out[:, 1]


def render(g: dict, cameras, config=None, *, d_color=None, d_depth=None, d_alpha=None,
           pixel_mask=None, brute_force=False, threads=None, want_2d=False) -> dict:
    """Renders all views (Eq. alpha) and, if any upstream gradient is given, back-propagates it.

    Returns color [P,3], depth [P], alpha [P], t_final [P], n_contrib [P] (int32), ambiguous [P]
    (uint8 bit mask) with P = sum_v W_v H_v, views concatenated row-major; and with a backward:
    g_means, g_log_scales, g_quats, g_opacity_logits, g_sh, g_pose [V,6] = (rho, omega), and
    g_2d [V,N,10] if want_2d.
    """
    lib = _load()
    means = _f64(g["means"], (-1, 3))
    n = means.shape[0]
    sh = _f64(g["sh"])
    deg = _degree_of(sh)
    K = (deg + 1) ** 2
    cams = _cam_array(cameras)
    V = cams.shape[0]
    P = int(sum(int(c["width"]) * int(c["height"]) for c in cameras))
    color = np.zeros((P, 3))
    depth = np.zeros(P)
    alpha = np.zeros(P)
    t_final = np.ones(P)
    n_contrib = np.zeros(P, dtype=np.int32)
    amb = np.zeros(P, dtype=np.uint8)
    mask = None
    if pixel_mask is not None:
        mask = np.ascontiguousarray(np.asarray(pixel_mask).reshape(P).astype(np.uint8))
    backward = d_color is not None or d_depth is not None or d_alpha is not None
    dc = _f64(d_color, (P, 3)) if d_color is not None else None
    dd = _f64(d_depth, (P,)) if d_depth is not None else None
    da = _f64(d_alpha, (P,)) if d_alpha is not None else None
    out = {}
    if backward:
        out["g_means"] = np.zeros((n, 3))
        out["g_log_scales"] = np.zeros((n, 3))
        out["g_quats"] = np.zeros((n, 4))
        out["g_opacity_logits"] = np.zeros(n)
        out["g_sh"] = np.zeros((n, K, 3))
        out["g_pose"] = np.zeros((V, 6))
        if want_2d:
            out["g_2d"] = np.zeros((V, n, 10))
    rc = lib.oracle_render(
        n, deg, _ptr(means), _ptr(_f64(g["log_scales"], (n, 3))), _ptr(_f64(g["quats"], (n, 4))),
        _ptr(_f64(g["opacity_logits"], (n,))), _ptr(sh), V, _ptr(cams),
        _ptr(_cfg_array(config)), _ptr(mask), int(bool(brute_force)),
        int(threads or default_threads()), _ptr(color), _ptr(depth), _ptr(alpha), _ptr(t_final),
        _ptr(n_contrib), _ptr(amb), _ptr(dc), _ptr(dd), _ptr(da),
        _ptr(out.get("g_means")), _ptr(out.get("g_log_scales")), _ptr(out.get("g_quats")),
        _ptr(out.get("g_opacity_logits")), _ptr(out.get("g_sh")), _ptr(out.get("g_pose")),
        _ptr(out.get("g_2d")))
    if rc != 0:
        raise ValueError(f"oracle_render rejected its arguments (code {rc})")
    out.update(color=color, depth=depth, alpha=alpha, t_final=t_final, n_contrib=n_contrib,
               ambiguous=amb)
    return out
