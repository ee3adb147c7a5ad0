"""ctypes binding of libnedf_compose (include/nedf_compose.h).

Argument marshalling only: every step of the render and training path runs in the CUDA
library.  Importing this module loads the library and raises if it has not been built; there
is no fallback.  Device buffers are passed as torch CUDA tensors (their data_ptr) or raw ints.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnedf_compose.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libnedf_compose.so is not built ({LIB_PATH}); run "
                      "paper_2308_04669_gb300.build.build() or __graft_entry__.build()")

_lib = C.CDLL(LIB_PATH)

NEDF_OK, NEDF_ERR_ARG, NEDF_ERR_CUDA, NEDF_ERR_OOM = 0, -1, -2, -3
NEDF_ERR_UNSUPPORTED, NEDF_ERR_CAPACITY, NEDF_ERR_TIMEOUT, NEDF_ERR_STATE = -4, -5, -6, -7
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
DEPTH_NEDF, DEPTH_MARCH = 0, 1
ARCH_REGRESSION, ARCH_CLASSIFIER = 0, 1
MAX_LIGHTS = 32
N_STAGES = 8


class Config(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("max_instances", C.c_int), ("max_types", C.c_int),
                ("nedf_hidden", C.c_int), ("nedf_width", C.c_int), ("nerf_hidden", C.c_int),
                ("nerf_width", C.c_int), ("precision", C.c_int), ("primary_pair_capacity", C.c_int64),
                ("shadow_pair_capacity", C.c_int64), ("nedf_arch", C.c_int)]


class Options(C.Structure):
    _fields_ = [("n_shade", C.c_int), ("shade_half", C.c_float), ("shadow_beta", C.c_float),
                ("shadow_eps", C.c_float), ("sigma_max", C.c_float), ("sdf_width", C.c_float),
                ("depth_source", C.c_int), ("march_steps", C.c_int), ("march_bisect", C.c_int),
                ("fallback_conf", C.c_float), ("refine_steps", C.c_int), ("outlier_resample", C.c_int),
                ("shade_resample", C.c_int), ("shade_sigma_min", C.c_float), ("miss_check", C.c_int)]


class TypeDesc(C.Structure):
    _fields_ = [("sdf_kind", C.c_int), ("sdf_params", C.c_float * 8), ("rb", C.c_float),
                ("albedo", C.c_float * 3), ("nedf_weights", C.POINTER(C.c_float)),
                ("nerf_weights", C.POINTER(C.c_float))]


class Instance(C.Structure):
    _fields_ = [("type", C.c_uint32), ("R", C.c_float * 9), ("T", C.c_float * 3), ("s", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("fov_y_deg", C.c_float)]


class Light(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("parallel", C.c_int)]


N_SCHEDULE = 5
SCHEDULE_KERNELS = ("step2_shade", "march_colour", "step1_nedf", "step3_nedf", "nedf_query")


class Schedule(C.Structure):
    _fields_ = [("stage_bytes", C.c_int * N_SCHEDULE), ("tuned_ms", C.c_float * N_SCHEDULE),
                ("operand_order", C.c_int * N_SCHEDULE)]


class FrameStats(C.Structure):
    _fields_ = [("primary_pairs", C.c_int64), ("shadow_pairs", C.c_int64), ("hit_pixels", C.c_int64),
                ("fallback_pairs", C.c_int64), ("kernel_launches", C.c_int64), ("status", C.c_uint32),
                ("resampled_pixels", C.c_int64)]


_H = C.c_void_p
_vp = C.c_void_p
_fp = C.POINTER(C.c_float)

EXPORTS = {
    "nedf_compose_create": ([C.POINTER(Config), _vp, C.POINTER(_H)], C.c_int),
    "nedf_compose_destroy": ([_H], None),
    "nedf_compose_last_error": ([_H], C.c_char_p),
    "nedf_compose_set_options": ([_H, C.POINTER(Options)], C.c_int),
    "nedf_compose_get_options": ([_H, C.POINTER(Options)], C.c_int),
    "nedf_compose_sync": ([_H], C.c_int),
    "nedf_compose_set_types": ([_H, C.c_int, C.POINTER(TypeDesc)], C.c_int),
    "nedf_compose_set_instances": ([_H, C.c_int, C.POINTER(Instance)], C.c_int),
    "nedf_compose_render": ([_H, C.POINTER(Camera), C.POINTER(Light), C.c_int, _vp, _vp, _vp, _vp, _vp,
                             C.POINTER(FrameStats)], C.c_int),
    "nedf_compose_render_host": ([_H, C.POINTER(Camera), C.POINTER(Light), C.c_int, _vp, _vp, _vp, _vp, _vp,
                                  C.POINTER(FrameStats)], C.c_int),
    "nedf_compose_render_march": ([_H, C.POINTER(Camera), C.c_int, C.c_int, _vp], C.c_int),
    "nedf_compose_begin_edit": ([_H, C.POINTER(Camera), C.POINTER(Light), C.c_int, C.c_int], C.c_int),
    "nedf_compose_render_edit": ([_H, _vp, _vp, _vp, _vp, _vp, C.POINTER(FrameStats)], C.c_int),
    "nedf_compose_end_edit": ([_H], C.c_int),
    "nedf_compose_stage_name": ([C.c_int], C.c_char_p),
    "nedf_compose_set_profiling": ([_H, C.c_int], C.c_int),
    "nedf_compose_get_stage_times": ([_H, _fp, C.c_int], C.c_int),
    "nedf_compose_get_engine_times": ([_H, _fp, C.c_int], C.c_int),
    "nedf_compose_validate": ([_H], C.c_int),
    "nedf_compose_inject_status": ([_H, C.c_uint32], C.c_int),
    "nedf_compose_check_wait_limit": ([_H], C.c_int),
    "nedf_compose_set_schedule": ([_H, C.POINTER(Schedule)], C.c_int),
    "nedf_compose_get_schedule": ([_H, C.POINTER(Schedule)], C.c_int),
    "nedf_compose_autotune": ([_H, C.POINTER(Camera), C.POINTER(Light), C.c_int, C.c_int, C.POINTER(Schedule)],
                              C.c_int),
    "nedf_compose_nedf_query": ([_H, C.c_int, C.c_int, _vp, _vp, _vp], C.c_int),
    "nedf_compose_depth_noalloc": ([C.c_int, C.c_int, C.POINTER(Camera), C.c_int, _vp, C.c_int, _fp, C.c_int, C.c_int,
                                    _vp, _vp, _vp, _vp], C.c_int),
    "nedf_compose_make_labels": ([_H, C.c_int, C.c_int64, C.c_uint64, C.c_int, C.c_int, _vp, _vp, _vp, _vp],
                                 C.c_int),
    "nedf_compose_make_labels_density": ([_H, C.c_int, C.c_int64, C.c_uint64, C.c_int, C.c_int, C.c_int, _fp, _vp,
                                          _vp, _vp, _vp], C.c_int),
    "nedf_compose_train_step": ([_H, C.c_int, C.c_int, C.c_float, _fp], C.c_int),
    "nedf_compose_loss_grad": ([_H, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _fp], C.c_int),
    "nedf_compose_get_nedf_weights": ([_H, C.c_int, _fp, C.c_int64], C.c_int),
    "nedf_compose_save_state": ([_H, _vp, C.POINTER(C.c_size_t)], C.c_int),
    "nedf_compose_load_state": ([_H, _vp, C.c_size_t], C.c_int),
}

for _name, (_args, _res) in EXPORTS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class NedfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def default_options(**kw) -> Options:
    o = Options(8, 0.05, 0.5, 0.02, 50.0, 0.01, DEPTH_NEDF, 128, 4, 0.0, 0, 0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Renderer:
    """One library handle.  Mirrors the C calls one to one."""

    def __init__(self, width, height, max_instances, max_types, nedf_hidden, nedf_width, nerf_hidden=0,
                 nerf_width=0, precision=PREC_FP32, primary_pair_capacity=0, shadow_pair_capacity=0,
                 stream=None, nedf_arch=0):
        cfg = Config(width, height, max_instances, max_types, nedf_hidden, nedf_width, nerf_hidden, nerf_width,
                     precision, primary_pair_capacity, shadow_pair_capacity, nedf_arch)
        h = _H()
        st = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else None)
        rc = _lib.nedf_compose_create(C.byref(cfg), st, C.byref(h))
        if rc != NEDF_OK:
            raise NedfError(rc, _lib.nedf_compose_last_error(None).decode())
        self.h = h
        self.cfg = cfg
        self._keep = []

    def _check(self, rc):
        if rc != NEDF_OK:
            raise NedfError(rc, _lib.nedf_compose_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            _lib.nedf_compose_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- options / scene ---------------------------------------------------------------------
    def set_options(self, opt: Options):
        return self._check(_lib.nedf_compose_set_options(self.h, C.byref(opt)))

    def get_options(self) -> Options:
        o = Options()
        self._check(_lib.nedf_compose_get_options(self.h, C.byref(o)))
        return o

    def sync(self):
        return self._check(_lib.nedf_compose_sync(self.h))

    def set_types(self, types):
        """types: list of scenegen.ObjType (weights are copied by the library)."""
        arr = (TypeDesc * len(types))()
        keep = []
        for k, t in enumerate(types):
            d = arr[k]
            d.sdf_kind = int(t.kind)
            for c in range(8):
                d.sdf_params[c] = float(t.params[c])
            d.rb = float(t.rb)
            for c in range(3):
                d.albedo[c] = float(t.albedo[c])
            w = np.ascontiguousarray(t.nedf_w, np.float32)
            keep.append(w)
            d.nedf_weights = _fptr(w)
            if t.nerf_w is not None and self.cfg.nerf_hidden > 0:
                wn = np.ascontiguousarray(t.nerf_w, np.float32)
                keep.append(wn)
                d.nerf_weights = _fptr(wn)
        return self._check(_lib.nedf_compose_set_types(self.h, len(types), arr))

    def set_instances(self, inst_type, R, T, s):
        n = int(len(inst_type))
        arr = (Instance * max(n, 1))()
        R = np.asarray(R, np.float32).reshape(n, 9)
        T = np.asarray(T, np.float32).reshape(n, 3)
        s = np.asarray(s, np.float32).reshape(n)
        for i in range(n):
            arr[i].type = int(inst_type[i])
            for c in range(9):
                arr[i].R[c] = float(R[i, c])
            for c in range(3):
                arr[i].T[c] = float(T[i, c])
            arr[i].s = float(s[i])
        return self._check(_lib.nedf_compose_set_instances(self.h, n, arr))

    def load_scene(self, scene):
        self.set_types(scene.types)
        self.set_instances(scene.inst_type, scene.inst_R, scene.inst_T, scene.inst_s)
        o = self.get_options()
        o.n_shade, o.shade_half = scene.n_shade, scene.shade_half
        o.shadow_beta, o.shadow_eps = scene.shadow_beta, scene.shadow_eps
        o.sigma_max, o.sdf_width = scene.sigma_max, scene.sdf_width
        self.set_options(o)

    # ---- render ------------------------------------------------------------------------------
    @staticmethod
    def camera(eye, target, fov):
        c = Camera()
        for k in range(3):
            c.eye[k] = float(eye[k])
            c.target[k] = float(target[k])
        c.fov_y_deg = float(fov)
        return c

    @staticmethod
    def lights(pos, parallel=None):
        """Point lights at the rows of pos; with parallel[i] non-zero, row i is instead the travel
        direction of a parallel light."""
        pos = np.asarray(pos, np.float32).reshape(-1, 3)
        arr = (Light * len(pos))()
        for i in range(len(pos)):
            for k in range(3):
                arr[i].pos[k] = float(pos[i, k])
            arr[i].parallel = int(parallel[i] != 0) if parallel is not None else 0
        return arr, len(pos)

    def render(self, cam, lights, depth=None, id=None, rgba=None, shadow=None, out=None, stats=False):
        la, nl = lights
        st = FrameStats() if stats else None
        self._check(_lib.nedf_compose_render(self.h, C.byref(cam), la, nl, _ptr(depth), _ptr(id), _ptr(rgba),
                                             _ptr(shadow), _ptr(out), C.byref(st) if st is not None else None))
        return st

    def begin_edit(self, cam, lights, inst):
        """Buffer reuse: renders the frozen part (every instance but `inst`) for this camera and
        these lights; later render_edit calls redo only what `inst` changes."""
        la, nl = lights
        self._check(_lib.nedf_compose_begin_edit(self.h, C.byref(cam), la, nl, int(inst)))

    def render_edit(self, depth=None, id=None, rgba=None, shadow=None, out=None, stats=False):
        st = FrameStats() if stats else None
        self._check(_lib.nedf_compose_render_edit(self.h, _ptr(depth), _ptr(id), _ptr(rgba), _ptr(shadow), _ptr(out),
                                                  C.byref(st) if st is not None else None))
        return st

    def end_edit(self):
        self._check(_lib.nedf_compose_end_edit(self.h))

    def render_host(self, cam, lights, depth=None, id=None, rgba=None, shadow=None, out=None, stats=False):
        """Host numpy outputs (pinned torch tensors also work through their data_ptr)."""
        la, nl = lights
        st = FrameStats() if stats else None
        hp = lambda a: None if a is None else (a.ctypes.data if isinstance(a, np.ndarray) else _ptr(a))
        self._check(_lib.nedf_compose_render_host(self.h, C.byref(cam), la, nl, hp(depth), hp(id), hp(rgba),
                                                  hp(shadow), hp(out), C.byref(st) if st is not None else None))
        return st

    def set_profiling(self, on=True):
        return self._check(_lib.nedf_compose_set_profiling(self.h, 1 if on else 0))

    def stage_times(self) -> dict:
        ms = np.zeros(N_STAGES, np.float32)
        self._check(_lib.nedf_compose_get_stage_times(self.h, _fptr(ms), N_STAGES))
        return {_lib.nedf_compose_stage_name(i).decode(): float(ms[i]) for i in range(N_STAGES)}

    def engine_times(self) -> dict:
        """Milliseconds of the Step-1 and Step-3 tensor-core NeDF engine launches alone (last
        profiled render; 0 where the frame ran none)."""
        ms = np.zeros(2, np.float32)
        self._check(_lib.nedf_compose_get_engine_times(self.h, _fptr(ms), 2))
        return {"step1_nedf": float(ms[0]), "step3_nedf": float(ms[1])}

    def render_march(self, cam, n_samples, early_stop, rgba):
        return self._check(_lib.nedf_compose_render_march(self.h, C.byref(cam), n_samples, early_stop, _ptr(rgba)))

    def validate(self):
        return self._check(_lib.nedf_compose_validate(self.h))

    def inject_status(self, bits):
        return self._check(_lib.nedf_compose_inject_status(self.h, bits))

    def check_wait_limit(self):
        return self._check(_lib.nedf_compose_check_wait_limit(self.h))

    def set_schedule(self, stage_bytes, operand_order=None):
        """stage_bytes and operand_order per kernel index (NeDF kernels: 0 default, 1 swapped, 2
        unswapped; NeRF kernels at width 256: 1 the SM-pair engine, 0 default and 2 the one-SM
        engine)."""
        s = Schedule()
        for k, b in enumerate(stage_bytes):
            s.stage_bytes[k] = int(b)
        for k, o in enumerate(operand_order or []):
            s.operand_order[k] = int(o)
        return self._check(_lib.nedf_compose_set_schedule(self.h, C.byref(s)))

    def get_schedule(self) -> dict:
        s = Schedule()
        self._check(_lib.nedf_compose_get_schedule(self.h, C.byref(s)))
        return {k: s.stage_bytes[i] for i, k in enumerate(SCHEDULE_KERNELS)}

    def get_operand_order(self) -> dict:
        s = Schedule()
        self._check(_lib.nedf_compose_get_schedule(self.h, C.byref(s)))
        return {k: s.operand_order[i] for i, k in enumerate(SCHEDULE_KERNELS)}

    def autotune(self, cam, lights, reps=3) -> dict:
        """Picks the stage size of every tensor-core kernel (and the NeDF engines' operand order at
        BF16 width 128) by timing this frame; returns {kernel: {"stage_bytes": b, "operand_order":
        "swapped" | "unswapped" | "fixed" | "sm_pair" | "one_sm", "ms": best time (0 if not
        timed)}}.  The NeRF kernels keep the engine they were set to."""
        s = Schedule()
        la, nl = lights
        self._check(_lib.nedf_compose_autotune(self.h, C.byref(cam), la, nl, reps, C.byref(s)))
        names = {0: "fixed", 1: "swapped", 2: "unswapped"}
        nerf = {0: "one_sm", 1: "sm_pair", 2: "one_sm"} if self.cfg.nerf_width == 256 and \
            self.cfg.precision != PREC_FP32 else None

        def order(i):
            return nerf[s.operand_order[i]] if nerf and i < 2 else names[s.operand_order[i]]
        return {k: {"stage_bytes": s.stage_bytes[i], "operand_order": order(i),
                    "ms": round(float(s.tuned_ms[i]), 4)} for i, k in enumerate(SCHEDULE_KERNELS)}

    def nedf_query(self, type_, o, d, out):
        return self._check(_lib.nedf_compose_nedf_query(self.h, type_, int(o.shape[0]), _ptr(o), _ptr(d), _ptr(out)))

    # ---- learned part ------------------------------------------------------------------------
    def make_labels(self, type_, n_rays, seed, march_steps=256, march_bisect=8, o=None, d=None, m_star=None,
                    hit_star=None):
        return self._check(_lib.nedf_compose_make_labels(self.h, type_, n_rays, seed, march_steps, march_bisect,
                                                         _ptr(o), _ptr(d), _ptr(m_star), _ptr(hit_star)))

    def make_labels_density(self, type_, n_rays, seed, n_samples, dens_hidden, dens_width, dens_w, o=None, d=None,
                            m_star=None, hit_star=None):
        w = np.ascontiguousarray(dens_w, np.float32)
        return self._check(_lib.nedf_compose_make_labels_density(self.h, type_, n_rays, seed, n_samples, dens_hidden,
                                                                 dens_width, _fptr(w), _ptr(o), _ptr(d), _ptr(m_star),
                                                                 _ptr(hit_star)))

    def train_step(self, type_, batch, lr, want_loss=False):
        loss = C.c_float(0.0)
        self._check(_lib.nedf_compose_train_step(self.h, type_, batch, lr, C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def loss_grad(self, type_, o, d, m_star, hit_star, grad):
        loss = C.c_float(0.0)
        self._check(_lib.nedf_compose_loss_grad(self.h, type_, int(o.shape[0]), _ptr(o), _ptr(d), _ptr(m_star),
                                                _ptr(hit_star), _ptr(grad), C.byref(loss)))
        return loss.value

    def get_nedf_weights(self, type_, n):
        out = np.empty(n, np.float32)
        self._check(_lib.nedf_compose_get_nedf_weights(self.h, type_, _fptr(out), n))
        return out

    def save_state(self) -> bytes:
        sz = C.c_size_t(0)
        self._check(_lib.nedf_compose_save_state(self.h, None, C.byref(sz)))
        buf = C.create_string_buffer(sz.value)
        self._check(_lib.nedf_compose_save_state(self.h, buf, C.byref(sz)))
        return buf.raw[: sz.value]

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        return self._check(_lib.nedf_compose_load_state(self.h, buf, len(blob)))


def renderer_for(scene, precision=PREC_FP32, stream=None, **kw) -> Renderer:
    """A Renderer sized for a scenegen.Scene with its types and instances loaded."""
    t0 = scene.types[0]
    kw.setdefault("nedf_arch", getattr(t0, "nedf_arch", 0))
    r = Renderer(scene.W, scene.H, max(scene.n_inst, 1), len(scene.types), t0.nedf_hidden, t0.nedf_width,
                 t0.nerf_hidden, t0.nerf_width, precision, stream=stream, **kw)
    r.load_scene(scene)
    return r
