"""FP64 CPU oracle of the NeDF composition render path (arXiv 2308.04669).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import this package.  It shares no code with the CUDA
library and never imports it; both sides consume the same seeded inputs from
``paper_2308_04669_gb300.scenegen``.

The arithmetic lives in ``nedf_oracle.c`` (plain C, double precision); this module compiles it
with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEPTH_MLP, DEPTH_EXACT, DEPTH_MARCH = 0, 1, 2
QUANT_NONE, QUANT_BF16, QUANT_FP8 = 0, 1, 2
ARCH_REGRESSION, ARCH_CLASSIFIER = 0, 1
CLS_IN, CLS_OUT, CLS_NC, CLS_NF = 1008, 1 + 64 + 128, 64, 128


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: the same source runs on x86_64 and aarch64)."""
    src = os.path.join(_HERE, "nedf_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "nedf_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC", "-o",
                               tmp, src, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcType(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.c_double * 8), ("rb", C.c_double),
                ("albedo", C.c_double * 3), ("nedf_hidden", C.c_int), ("nedf_width", C.c_int),
                ("nedf_w", C.POINTER(C.c_double)), ("nerf_hidden", C.c_int), ("nerf_width", C.c_int),
                ("nerf_w", C.POINTER(C.c_double)), ("nedf_arch", C.c_int),
                ("nedf_wq", C.POINTER(C.c_double))]


class OrcScene(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("fov_deg", C.c_double), ("n_lights", C.c_int), ("lights", C.POINTER(C.c_double)),
                ("n_types", C.c_int), ("types", C.POINTER(OrcType)), ("n_inst", C.c_int),
                ("inst_type", C.POINTER(C.c_int)), ("inst_R", C.POINTER(C.c_double)),
                ("inst_T", C.POINTER(C.c_double)), ("inst_s", C.POINTER(C.c_double)),
                ("n_shade", C.c_int), ("shade_half", C.c_double), ("beta", C.c_double),
                ("eps", C.c_double), ("sigma_max", C.c_double), ("sdf_width", C.c_double),
                ("light_parallel", C.POINTER(C.c_int))]


class OrcOpts(C.Structure):
    _fields_ = [("depth_mode", C.c_int), ("march_n", C.c_int), ("march_b", C.c_int),
                ("quant", C.c_int), ("fallback_conf", C.c_double), ("refine_steps", C.c_int),
                ("n_threads", C.c_int), ("outlier_resample", C.c_int), ("shade_resample", C.c_int),
                ("shade_sigma_min", C.c_double), ("miss_check", C.c_int)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            d, i, i64, u32 = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
            sp, op = C.POINTER(OrcScene), C.POINTER(OrcOpts)
            l.orc_sdf.argtypes = [C.c_int, d, d]; l.orc_sdf.restype = C.c_double
            l.orc_density.argtypes = [sp, C.c_int, d]; l.orc_density.restype = C.c_double
            l.orc_camera_ray.argtypes = [sp, C.c_int, C.c_int, d, d]
            l.orc_to_local.argtypes = [sp, C.c_int, d, d, d, d]
            l.orc_bound.argtypes = [d, d, C.c_double, d]; l.orc_bound.restype = C.c_int
            l.orc_posenc.argtypes = [d, C.c_int, C.c_int, d]; l.orc_posenc.restype = C.c_int
            l.orc_nedf_features.argtypes = [d, d, C.c_double, d, d]; l.orc_nedf_features.restype = C.c_int
            l.orc_mlp.argtypes = [d, C.c_int, i, d, d, C.c_int]
            l.orc_mlp_qmargin.argtypes = [d, C.c_int, i, d, d, C.c_int]; l.orc_mlp_qmargin.restype = C.c_double
            l.orc_round_bf16.argtypes = [C.c_double]; l.orc_round_bf16.restype = C.c_double
            l.orc_round_margin.argtypes = [C.c_double, C.c_int]; l.orc_round_margin.restype = C.c_double
            l.orc_round_e4m3.argtypes = [C.c_double]; l.orc_round_e4m3.restype = C.c_double
            l.orc_fp8_scale.argtypes = [C.c_double]; l.orc_fp8_scale.restype = C.c_double
            l.orc_query.argtypes = [sp, op, C.c_int, d, d, d, d]; l.orc_query.restype = C.c_int
            l.orc_exact_depth.argtypes = [C.c_int, d, d, d, C.c_double, C.c_double, i]
            l.orc_exact_depth.restype = C.c_double
            l.orc_march_depth.argtypes = [sp, C.c_int, d, d, C.c_double, C.c_double, C.c_int, C.c_int, i]
            l.orc_march_depth.restype = C.c_double
            l.orc_composite_samples.argtypes = [C.c_int, d, d, C.c_double, d]
            l.orc_render.argtypes = [sp, op, C.c_int64, i64, d, u32, d, d, d, d, d, d, d, d, d]
            l.orc_steps23.argtypes = [sp, op, C.c_int64, i64, u32, d, d, d, d, d]
            l.orc_query_diag.argtypes = [sp, op, C.c_int, d, d, d, d, C.c_double]; l.orc_query_diag.restype = C.c_int
            l.orc_mlp_flip.argtypes = [d, C.c_int, i, d, d, C.c_int, C.c_int, C.c_int, i, d]
            l.orc_mlp_flip2.argtypes = [d, C.c_int, i, d, d, C.c_int, C.c_int, C.c_int]
            l.orc_mlp_flipset.argtypes = [d, C.c_int, i, d, d, C.c_int, C.c_int, i]
            l.orc_volume_render.argtypes = [sp, op, C.c_int, C.c_int64, i64, d, d]
            l.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]; l.orc_splitmix64.restype = C.c_uint64
            l.orc_train_rays.argtypes = [C.c_double, C.c_uint64, C.c_int64, C.c_int, d, d]
            l.orc_train_labels.argtypes = [sp, C.c_int, C.c_int, d, d, C.c_int, C.c_int, d, i]
            l.orc_nedf_loss_grad.argtypes = [sp, C.c_int, C.c_int, d, d, d, i, d, C.c_int]
            l.orc_nedf_loss_grad.restype = C.c_double
            l.orc_adam.argtypes = [C.c_int64, d, d, d, d, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
            l.orc_density_net.argtypes = [d, C.c_int, C.c_int, d]; l.orc_density_net.restype = C.c_double
            l.orc_density_labels.argtypes = [d, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, d, d, d, i, d]
            l.orc_cls_param_count.argtypes = []; l.orc_cls_param_count.restype = C.c_int64
            l.orc_cls_features.argtypes = [d, d, C.c_double, d, d]; l.orc_cls_features.restype = C.c_int
            l.orc_cls_round_bf16.argtypes = [d, d]
            l.orc_cls_forward.argtypes = [d, d, d, C.c_int]
            l.orc_cls_segment.argtypes = [C.c_double, i, i]
            l.orc_cls_decode.argtypes = [d, d, d, i, i]; l.orc_cls_decode.restype = C.c_double
            l.orc_cls_loss_grad.argtypes = [d, C.c_int, d, d, i, d]; l.orc_cls_loss_grad.restype = C.c_double
            _lib = l
    return _lib


class OracleScene:
    """A scenegen.Scene widened to double and laid out for the C oracle (keeps arrays alive)."""

    def __init__(self, scene, nedf_override: dict | None = None):
        self.scene = scene
        self._keep = []
        nt = len(scene.types)
        self.types = (OrcType * nt)()
        for k, t in enumerate(scene.types):
            ct = self.types[k]
            ct.kind = int(t.kind)
            for c in range(8):
                ct.params[c] = float(t.params[c])
            ct.rb = float(t.rb)
            for c in range(3):
                ct.albedo[c] = float(t.albedo[c])
            w = np.ascontiguousarray(
                (nedf_override[k] if nedf_override and k in nedf_override else t.nedf_w), np.float64)
            self._keep.append(w)
            ct.nedf_hidden, ct.nedf_width, ct.nedf_w = t.nedf_hidden, t.nedf_width, _dp(w)
            ct.nedf_arch = int(getattr(t, "nedf_arch", 0))
            if ct.nedf_arch == ARCH_CLASSIFIER:
                wq = cls_round_bf16(w)
                self._keep.append(wq)
                ct.nedf_wq = _dp(wq)
            else:
                ct.nedf_wq = C.POINTER(C.c_double)()
            if t.nerf_hidden:
                wn = np.ascontiguousarray(t.nerf_w, np.float64)
                self._keep.append(wn)
                ct.nerf_hidden, ct.nerf_width, ct.nerf_w = t.nerf_hidden, t.nerf_width, _dp(wn)
            else:
                ct.nerf_hidden, ct.nerf_width = 0, 0
                ct.nerf_w = C.POINTER(C.c_double)()
        self.lights = np.ascontiguousarray(scene.lights, np.float64).reshape(-1)
        self.itype = np.ascontiguousarray(scene.inst_type, np.int32)
        self.R = np.ascontiguousarray(scene.inst_R, np.float64).reshape(-1)
        self.T = np.ascontiguousarray(scene.inst_T, np.float64).reshape(-1)
        self.s = np.ascontiguousarray(scene.inst_s, np.float64)
        sc = OrcScene()
        sc.W, sc.H = scene.W, scene.H
        for c in range(3):
            sc.eye[c] = float(scene.eye[c])
            sc.target[c] = float(scene.target[c])
        sc.fov_deg = float(scene.fov_deg)
        sc.n_lights, sc.lights = scene.lights.shape[0], _dp(self.lights)
        sc.n_types, sc.types = nt, self.types
        sc.n_inst = scene.n_inst
        sc.inst_type = self.itype.ctypes.data_as(C.POINTER(C.c_int))
        sc.inst_R, sc.inst_T, sc.inst_s = _dp(self.R), _dp(self.T), _dp(self.s)
        sc.n_shade, sc.shade_half = scene.n_shade, float(np.float32(scene.shade_half))
        sc.beta, sc.eps = float(np.float32(scene.shadow_beta)), float(np.float32(scene.shadow_eps))
        sc.sigma_max, sc.sdf_width = float(np.float32(scene.sigma_max)), float(np.float32(scene.sdf_width))
        lp = getattr(scene, "light_parallel", None)
        if lp is not None:
            self.lpar = np.ascontiguousarray(np.asarray(lp).reshape(-1) != 0, np.int32)
            sc.light_parallel = self.lpar.ctypes.data_as(C.POINTER(C.c_int))
        else:
            sc.light_parallel = C.POINTER(C.c_int)()
        self.c = sc

    @property
    def ptr(self):
        return C.byref(self.c)


def opts(depth_mode=DEPTH_MLP, march_n=128, march_b=4, quant=QUANT_NONE, fallback_conf=0.0,
         refine_steps=0, n_threads=1, outlier_resample=0, shade_resample=0, shade_sigma_min=1.0,
         miss_check=0) -> OrcOpts:
    return OrcOpts(depth_mode, march_n, march_b, quant, fallback_conf, refine_steps, n_threads, outlier_resample,
                   shade_resample, shade_sigma_min, miss_check)


def render(osc: OracleScene, px=None, alt=True, **kw):
    """Steps 1-3 for the pixels `px` (default: all).  Returns a dict of arrays; with alt=True the
    pixels near a depth decision also carry the alternative outcome (see orc_render): alt_depth,
    alt_id, alt_rgba, alt_shadow, alt_out, has_alt."""
    s = osc.scene
    if px is None:
        px = np.arange(s.W * s.H, dtype=np.int64)
    px = np.ascontiguousarray(px, np.int64)
    n = px.shape[0]
    out = dict(depth=np.empty(n), id=np.empty(n, np.uint32), gap=np.empty(n), pmargin=np.empty(n),
               rgba=np.empty((n, 4)), shadow=np.empty(n), smargin=np.empty(n), out=np.empty((n, 4)),
               shade_smax=np.empty(n), dmargin=np.empty(n))
    a = np.empty((n, 12)) if alt else None
    o = opts(**kw)
    lib().orc_render(osc.ptr, C.byref(o), n, px.ctypes.data_as(C.POINTER(C.c_int64)),
                     _dp(out["depth"]), out["id"].ctypes.data_as(C.POINTER(C.c_uint32)),
                     _dp(out["gap"]), _dp(out["pmargin"]), _dp(out["rgba"]), _dp(out["shadow"]),
                     _dp(out["smargin"]), _dp(out["out"]), _dp(out["shade_smax"]), _dp(out["dmargin"]),
                     _dp(a) if alt else C.POINTER(C.c_double)())
    out["px"] = px
    if alt:
        out["has_alt"] = a[:, 11] == 1.0
        out["alt_depth"] = a[:, 0]
        out["alt_id"] = np.where(a[:, 1] < 0, 0xFFFFFFFF, np.nan_to_num(a[:, 1])).astype(np.uint32)
        out["alt_rgba"] = a[:, 2:6]
        out["alt_shadow"] = a[:, 6]
        out["alt_out"] = a[:, 7:11]
    return out


def steps23(osc: OracleScene, px, ids, depth, **kw):
    """Steps 2-3 of pixels px given each pixel's winner id (uint32, 0xFFFFFFFF none) and world depth:
    dict(rgba, shadow, smargin, out)."""
    px = np.ascontiguousarray(px, np.int64)
    ids = np.ascontiguousarray(ids, np.uint32)
    depth = np.ascontiguousarray(depth, np.float64)
    n = px.shape[0]
    out = dict(rgba=np.empty((n, 4)), shadow=np.empty(n), smargin=np.empty(n), out=np.empty((n, 4)))
    o = opts(**kw)
    lib().orc_steps23(osc.ptr, C.byref(o), n, px.ctypes.data_as(C.POINTER(C.c_int64)),
                      ids.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(depth), _dp(out["rgba"]), _dp(out["shadow"]),
                      _dp(out["smargin"]), _dp(out["out"]))
    return out


def volume_render(osc: OracleScene, n_samples=128, px=None, n_threads=1, quant=QUANT_NONE, margins=False):
    """Plain-method colour of pixels px; with margins=True returns (rgba, vmargin)."""
    s = osc.scene
    if px is None:
        px = np.arange(s.W * s.H, dtype=np.int64)
    px = np.ascontiguousarray(px, np.int64)
    rgba = np.empty((px.shape[0], 4))
    vm = np.empty(px.shape[0])
    o = opts(n_threads=n_threads, quant=quant)
    lib().orc_volume_render(osc.ptr, C.byref(o), n_samples, px.shape[0],
                            px.ctypes.data_as(C.POINTER(C.c_int64)), _dp(rgba), _dp(vm))
    return (rgba, vm) if margins else rgba


def sdf(kind, params, x):
    p = np.ascontiguousarray(np.asarray(params, np.float64).reshape(-1)[:8].tolist() + [0.0] * (8 - min(8, len(params))), np.float64)
    xx = np.ascontiguousarray(x, np.float64)
    return lib().orc_sdf(int(kind), _dp(p), _dp(xx))


def camera_ray(osc: OracleScene, i, j):
    o, d = np.empty(3), np.empty(3)
    lib().orc_camera_ray(osc.ptr, i, j, _dp(o), _dp(d))
    return o, d


def to_local(osc: OracleScene, inst, o, d):
    o = np.ascontiguousarray(o, np.float64); d = np.ascontiguousarray(d, np.float64)
    ol, dl = np.empty(3), np.empty(3)
    lib().orc_to_local(osc.ptr, inst, _dp(o), _dp(d), _dp(ol), _dp(dl))
    return ol, dl


def bound(ol, dl, rb):
    ol = np.ascontiguousarray(ol, np.float64); dl = np.ascontiguousarray(dl, np.float64)
    out = np.empty(4)
    kept = lib().orc_bound(_dp(ol), _dp(dl), float(rb), _dp(out))
    return bool(kept), out


def posenc(x, n_freq):
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty(x.shape[0] * (1 + 2 * n_freq))
    lib().orc_posenc(_dp(x), x.shape[0], n_freq, _dp(out))
    return out


def nedf_features(ol, dl, rb):
    ol = np.ascontiguousarray(ol, np.float64); dl = np.ascontiguousarray(dl, np.float64)
    f, b = np.empty(78), np.empty(4)
    kept = lib().orc_nedf_features(_dp(ol), _dp(dl), float(rb), _dp(f), _dp(b))
    return bool(kept), f, b


def mlp(w, dims, x, quant=QUANT_NONE):
    w = np.ascontiguousarray(w, np.float64)
    dims_c = (C.c_int * len(dims))(*dims)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(dims[-1])
    lib().orc_mlp(_dp(w), len(dims) - 1, dims_c, _dp(x), _dp(y), quant)
    return y


def mlp_qmargin(w, dims, x, quant):
    """(y, margin): the MLP output and the row's rounding knife edge (see orc_mlp_qmargin)."""
    w = np.ascontiguousarray(w, np.float64)
    dims_c = (C.c_int * len(dims))(*dims)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(dims[-1])
    m = lib().orc_mlp_qmargin(_dp(w), len(dims) - 1, dims_c, _dp(x), _dp(y), quant)
    return y, m


def mlp_flip(w, dims, x, quant, flip_idx=-1, n_cand=0):
    """(y, cand_idx, cand_margin): the MLP with value flip_idx rounded the other way, and the
    n_cand values nearest to a rounding boundary (see orc_mlp_flip)."""
    w = np.ascontiguousarray(w, np.float64)
    dims_c = (C.c_int * len(dims))(*dims)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(dims[-1])
    ci = np.full(max(n_cand, 1), -1, np.int32)
    cm = np.empty(max(n_cand, 1))
    lib().orc_mlp_flip(_dp(w), len(dims) - 1, dims_c, _dp(x), _dp(y), int(quant), int(flip_idx), int(n_cand),
                       ci.ctypes.data_as(C.POINTER(C.c_int)), _dp(cm))
    return y, ci[:n_cand], cm[:n_cand]


def mlp_flip2(w, dims, x, quant, flip_a, flip_b):
    """The MLP with two rounded values taken the other way (see orc_mlp_flip2)."""
    w = np.ascontiguousarray(w, np.float64)
    dims_c = (C.c_int * len(dims))(*dims)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(dims[-1])
    lib().orc_mlp_flip2(_dp(w), len(dims) - 1, dims_c, _dp(x), _dp(y), int(quant), int(flip_a), int(flip_b))
    return y


def mlp_flipset(w, dims, x, quant, flips):
    """The MLP with every rounded value listed in flips taken the other way (see orc_mlp_flipset)."""
    w = np.ascontiguousarray(w, np.float64)
    dims_c = (C.c_int * len(dims))(*dims)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(dims[-1])
    f = (C.c_int * max(len(flips), 1))(*[int(v) for v in flips])
    lib().orc_mlp_flipset(_dp(w), len(dims) - 1, dims_c, _dp(x), _dp(y), int(quant), len(flips), f)
    return y


def round_bf16(x):
    return lib().orc_round_bf16(float(x))


def round_margin(x, fmt):
    """Distance of x to its nearest BF16 (fmt 0) / E4M3 (fmt 1) rounding boundary."""
    return lib().orc_round_margin(float(x), int(fmt))


def round_e4m3(x):
    return lib().orc_round_e4m3(float(x))


def fp8_scale(max_abs):
    return lib().orc_fp8_scale(float(max_abs))


def query(osc: OracleScene, inst, o, d, **kw):
    o = np.ascontiguousarray(o, np.float64); d = np.ascontiguousarray(d, np.float64)
    out, mg = np.empty(6), C.c_double()
    op = opts(**kw)
    hit = lib().orc_query(osc.ptr, C.byref(op), inst, _dp(o), _dp(d), _dp(out), C.byref(mg))
    return bool(hit), out, mg.value


def query_diag(osc: OracleScene, inst, o, d, need=0.0, **kw):
    """(hit, out6, (margin, dmargin, dspread)) of one query (see orc_query_diag)."""
    o = np.ascontiguousarray(o, np.float64); d = np.ascontiguousarray(d, np.float64)
    out, dg = np.empty(6), np.empty(3)
    op = opts(**kw)
    hit = lib().orc_query_diag(osc.ptr, C.byref(op), inst, _dp(o), _dp(d), _dp(out), _dp(dg), float(need))
    return bool(hit), out, tuple(dg)


def exact_depth(kind, params, ol, dl, te, tx):
    p = np.zeros(8); p[: len(params)] = params
    ol = np.ascontiguousarray(ol, np.float64); dl = np.ascontiguousarray(dl, np.float64)
    hit = C.c_int()
    D = lib().orc_exact_depth(int(kind), _dp(p), _dp(ol), _dp(dl), te, tx, C.byref(hit))
    return bool(hit.value), D


def march_depth(osc: OracleScene, type_, ol, dl, te, tx, n, b):
    ol = np.ascontiguousarray(ol, np.float64); dl = np.ascontiguousarray(dl, np.float64)
    hit = C.c_int()
    D = lib().orc_march_depth(osc.ptr, type_, _dp(ol), _dp(dl), te, tx, n, b, C.byref(hit))
    return bool(hit.value), D


def composite_samples(sigma, rgb, world_delta):
    sigma = np.ascontiguousarray(sigma, np.float64)
    rgb = np.ascontiguousarray(rgb, np.float64).reshape(-1)
    out = np.empty(4)
    lib().orc_composite_samples(sigma.shape[0], _dp(sigma), _dp(rgb), float(world_delta), _dp(out))
    return out


def splitmix64(seed, index):
    return lib().orc_splitmix64(seed, index)


def train_rays(rb, seed, first, n):
    o, d = np.empty((n, 3)), np.empty((n, 3))
    lib().orc_train_rays(float(rb), seed, first, n, _dp(o), _dp(d))
    return o, d


def train_labels(osc: OracleScene, type_, o, d, march_n=256, march_b=8):
    o = np.ascontiguousarray(o, np.float64); d = np.ascontiguousarray(d, np.float64)
    n = o.shape[0]
    m, h = np.empty(n), np.empty(n, np.int32)
    lib().orc_train_labels(osc.ptr, type_, n, _dp(o), _dp(d), march_n, march_b, _dp(m),
                           h.ctypes.data_as(C.POINTER(C.c_int)))
    return m, h


def nedf_loss_grad(osc: OracleScene, type_, o, d, m_star, hit_star, quant=QUANT_NONE):
    o = np.ascontiguousarray(o, np.float64); d = np.ascontiguousarray(d, np.float64)
    m_star = np.ascontiguousarray(m_star, np.float64)
    hit_star = np.ascontiguousarray(hit_star, np.int32)
    t = osc.scene.types[type_]
    g = np.empty(t.nedf_w.shape[0])
    loss = lib().orc_nedf_loss_grad(osc.ptr, type_, o.shape[0], _dp(o), _dp(d), _dp(m_star),
                                    hit_star.ctypes.data_as(C.POINTER(C.c_int)), _dp(g), quant)
    return loss, g


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    lib().orc_adam(theta.shape[0], _dp(theta), _dp(np.ascontiguousarray(g, np.float64)), _dp(m), _dp(v),
                   t, lr, b1, b2, eps)


# ---- the paper's intersection network (two-level classifier) ---------------------------------
def cls_param_count() -> int:
    return int(lib().orc_cls_param_count())


def cls_features(ol, dl, rb):
    """16 encoded points on the chord through the bound: (feat[1008], (te, tx, tperp, disc)) or
    (None, bound) when the ray misses the bound."""
    ol = np.ascontiguousarray(ol, np.float64); dl = np.ascontiguousarray(dl, np.float64)
    feat, bd = np.zeros(CLS_IN), np.zeros(4)
    ok = lib().orc_cls_features(_dp(ol), _dp(dl), float(rb), _dp(feat), _dp(bd))
    return (feat if ok else None), bd


def cls_round_bf16(w):
    w = np.ascontiguousarray(w, np.float64)
    wq = np.empty_like(w)
    lib().orc_cls_round_bf16(_dp(w), _dp(wq))
    return wq


def cls_forward(w, x, quant=QUANT_NONE):
    """Logits [hit, 64 coarse, 128 fine] for one input x[1008]; BF16 mode rounds w itself."""
    w = np.ascontiguousarray(w, np.float64)
    if quant != QUANT_NONE:
        w = cls_round_bf16(w)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(CLS_OUT)
    lib().orc_cls_forward(_dp(w), _dp(x), _dp(y), int(quant))
    return y


def cls_logits(w_used, X, quant=QUANT_NONE):
    """Logits of every row of X[n][1008] with the weights as given (pass cls_round_bf16(w) for
    the BF16 mode: no rounding per call)."""
    w_used = np.ascontiguousarray(w_used, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, CLS_IN)
    Y = np.empty((X.shape[0], CLS_OUT))
    for i in range(X.shape[0]):
        lib().orc_cls_forward(_dp(w_used), _dp(X[i]), _dp(Y[i]), int(quant))
    return Y


def cls_segment(m):
    c, f = C.c_int(), C.c_int()
    lib().orc_cls_segment(float(m), C.byref(c), C.byref(f))
    return c.value, f.value


def cls_decode(logits):
    """(m = mu / l, hit logit, coarse bin, fine bin, smaller top-2 gap)"""
    logits = np.ascontiguousarray(logits, np.float64)
    m, a, c, f = C.c_double(), C.c_double(), C.c_int(), C.c_int()
    gap = lib().orc_cls_decode(_dp(logits), C.byref(m), C.byref(a), C.byref(c), C.byref(f))
    return m.value, a.value, c.value, f.value, gap


def cls_loss_grad(w, x, m_star, hit_star):
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, CLS_IN)
    m_star = np.ascontiguousarray(m_star, np.float64)
    hit_star = np.ascontiguousarray(hit_star, np.int32)
    g = np.empty_like(w)
    L = lib().orc_cls_loss_grad(_dp(w), x.shape[0], _dp(x), _dp(m_star),
                                hit_star.ctypes.data_as(C.POINTER(C.c_int)), _dp(g))
    return L, g


# ---- supervision by a density network (plugin mode) -------------------------------------------
def density_net(w, hidden, width, x):
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    return float(lib().orc_density_net(_dp(w), int(hidden), int(width), _dp(x)))


def density_labels(w, hidden, width, rb, n_samples, o, d):
    """(m*, hit*, opacity) of rays (o, d) in the object frame, from Eq. 5 on the density net."""
    w = np.ascontiguousarray(w, np.float64)
    o = np.ascontiguousarray(o, np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
    n = o.shape[0]
    m, h, a = np.empty(n), np.empty(n, np.int32), np.empty(n)
    lib().orc_density_labels(_dp(w), int(hidden), int(width), float(rb), int(n_samples), n, _dp(o), _dp(d), _dp(m),
                             h.ctypes.data_as(C.POINTER(C.c_int)), _dp(a))
    return m, h, a
