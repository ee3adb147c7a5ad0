"""Seeded synthetic inputs for the NeDF composition render path.

This module is the one piece that both the CUDA path and the CPU oracle consume.  It draws
numbers and lays out scene records; it holds none of the method's arithmetic (no ray
transform, cull, encoding, network, depth decode, shading or shadow test).

Random streams.  The paper gives seeds for its workloads but no generator, so every draw comes
from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): output i of the stream seeded with `s` is mix(s + (i+1) * 0x9E3779B97F4A7C15).
Uniform rotations use Shoemake's uniform-quaternion method (Graphics Gems III, 1992).
Network weights are Xavier-uniform (Glorot & Bengio 2010), drawn layer by layer in row-major
W[out][in] order, biases zero.  Every value handed to either side is rounded to float32 first,
so the oracle (FP64) and the kernels (FP32 and lower) start from identical numbers.

Scene shapes follow the paper's workloads (few object types, many repeated instances, point
lights; Section "Capability evaluation", Table 2) with analytic signed-distance densities
standing in for the pre-trained NeRFs that are not available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# Signed-distance kinds of the object types (object-local coordinates, bound radius r_b = 1).
SDF_SPHERE, SDF_TORUS, SDF_BOX, SDF_CAPSULE, SDF_ROUNDCONE, SDF_TWOSPHERE, SDF_TWISTTORUS, SDF_OCTA = range(8)

# Shape parameters per kind (padded to 8 floats when stored).
#   sphere: radius | torus (axis y): R, r | box: half extents x,y,z | capsule (axis y): half length, r
#   rounded cone (axis y): r1, y1, r2, y2 | two-sphere union: centre offset along x, r
#   twisted torus (ring in the xy plane, twisted about y): R, r, twist rad per unit y
#   octahedron |x|+|y|+|z| = a: a
DEFAULT_PARAMS = {
    SDF_SPHERE: [0.5],
    SDF_TORUS: [0.4, 0.15],
    SDF_BOX: [0.35, 0.35, 0.35],
    SDF_CAPSULE: [0.3, 0.2],
    SDF_ROUNDCONE: [0.3, -0.25, 0.1, 0.35],
    SDF_TWOSPHERE: [0.25, 0.3],
    SDF_TWISTTORUS: [0.4, 0.12, 2.0],
    SDF_OCTA: [0.55],
}

PE_NEDF_FREQS = 6          # NeDF input encoding: 6 frequencies + identity on 6-D input -> 78
PE_NERF_POS_FREQS = 10     # NeRF position encoding -> 63
PE_NERF_DIR_FREQS = 4      # NeRF direction encoding -> 27
NEDF_IN = 6 * (1 + 2 * PE_NEDF_FREQS)
NERF_IN = 3 * (1 + 2 * PE_NERF_POS_FREQS) + 3 * (1 + 2 * PE_NERF_DIR_FREQS)
# the paper's intersection network (Appendix A): 16 points x 10-frequency encoding = 1008 inputs,
# 256 features, 16 residual blocks, 64 coarse and 128 fine bins plus the hit logit
CLS_PTS, CLS_FREQ, CLS_W, CLS_BLOCKS, CLS_NC, CLS_NF = 16, 10, 256, 16, 64, 128
CLS_IN = CLS_PTS * 3 * (1 + 2 * CLS_FREQ)
CLS_OUT = 1 + CLS_NC + CLS_NF
ARCH_REGRESSION, ARCH_CLASSIFIER = 0, 1


# ----------------------------------------------------------------------------------------------
# SplitMix64
# ----------------------------------------------------------------------------------------------
def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 sequence that starts from state `seed`."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + idx * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def substream(seed: int, tag: int, index: int = 0) -> int:
    """Seed of an independent sub-stream, itself a SplitMix64 draw."""
    return int(splitmix64((seed ^ (tag << 40) ^ (index << 8)) & MASK64, 1)[0])


TAG_NEDF, TAG_NERF, TAG_INST, TAG_MISC = 1, 2, 3, 4


# ----------------------------------------------------------------------------------------------
# Network weights
# ----------------------------------------------------------------------------------------------
def mlp_dims(n_in: int, hidden: int, width: int, n_out: int) -> list[int]:
    """Layer widths of a ReLU MLP with `hidden` hidden layers of `width` units."""
    return [n_in] + [width] * hidden + [n_out]


def mlp_param_count(dims: list[int]) -> int:
    return sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))


def xavier_mlp(seed: int, dims: list[int]) -> np.ndarray:
    """Packed float32 weights: for each layer W[out][in] row-major, then b[out] (zeros)."""
    parts = []
    off = 0
    for i in range(len(dims) - 1):
        fi, fo = dims[i], dims[i + 1]
        a = math.sqrt(6.0 / (fi + fo))
        u = uniform(seed, fi * fo, off)
        off += fi * fo
        parts.append(((2.0 * u - 1.0) * a).astype(np.float32))
        parts.append(np.zeros(fo, np.float32))
    return np.concatenate(parts)


def cls_layers() -> list[tuple[int, int]]:
    """(in, out) of the classifier's packed layers: head, W1 and W2 of each block, tails A and B."""
    return ([(CLS_IN, CLS_W)] + [(CLS_W, CLS_W)] * (2 * CLS_BLOCKS) +
            [(CLS_W, 1 + CLS_NC), (CLS_W, CLS_NF)])


def cls_param_count() -> int:
    return sum(fi * fo + fo for fi, fo in cls_layers())


def cls_weights(seed: int, residual_gain: float = 0.5, bias: float = 0.05) -> np.ndarray:
    """Packed float32 classifier weights (W[out][in] then b[out] per layer): Xavier-uniform
    matrices, the second layer of every residual block scaled by residual_gain, biases uniform in
    [-bias, bias]."""
    parts = []
    off = 0
    for i, (fi, fo) in enumerate(cls_layers()):
        a = math.sqrt(6.0 / (fi + fo)) * (residual_gain if 1 <= i <= 2 * CLS_BLOCKS and i % 2 == 0 else 1.0)
        u = uniform(seed, fi * fo + fo, off)
        off += fi * fo + fo
        parts.append(((2.0 * u[: fi * fo] - 1.0) * a).astype(np.float32))
        parts.append(((2.0 * u[fi * fo:] - 1.0) * bias).astype(np.float32))
    return np.concatenate(parts)


DENS_IN = 3 * (1 + 2 * 10)        # a radiance field's density input: position, 10 frequencies


def density_weights(seed: int, hidden: int = 2, width: int = 64, gain: float = 24.0,
                    shift: float = -10.0) -> np.ndarray:
    """A generic radiance field's density network, packed like xavier_mlp with dims
    [63, width x hidden, 1]: Xavier-uniform matrices, zero hidden biases, the output layer scaled
    by gain and biased by shift so that sigma = ReLU(output) is zero over part of the bound and
    reaches tens elsewhere (seeded blobs with sharp edges)."""
    w = xavier_mlp(seed, mlp_dims(DENS_IN, hidden, width, 1)).astype(np.float64)
    n_out = width + 1
    w[-n_out:-1] *= gain
    w[-1] = shift
    return w.astype(np.float32)


# ----------------------------------------------------------------------------------------------
# Scene records
# ----------------------------------------------------------------------------------------------
@dataclass
class ObjType:
    kind: int
    params: np.ndarray            # float32[8]
    rb: float                     # bound-sphere radius (object-local)
    albedo: np.ndarray            # float32[3], used when there is no NeRF colour network
    nedf_hidden: int
    nedf_width: int
    nedf_w: np.ndarray            # packed float32, dims [78, w * hidden, 2]
    nerf_hidden: int = 0
    nerf_width: int = 0
    nerf_w: np.ndarray | None = None   # packed float32, dims [90, w * hidden, 3] or None
    nedf_arch: int = ARCH_REGRESSION   # ARCH_CLASSIFIER: nedf_w holds the classifier (cls_layers)

    @property
    def nedf_dims(self):
        return mlp_dims(NEDF_IN, self.nedf_hidden, self.nedf_width, 2)

    @property
    def nerf_dims(self):
        return mlp_dims(NERF_IN, self.nerf_hidden, self.nerf_width, 3) if self.nerf_hidden else None


@dataclass
class Scene:
    name: str
    W: int
    H: int
    eye: np.ndarray               # float32[3]
    target: np.ndarray            # float32[3]
    fov_deg: float                # vertical field of view
    lights: np.ndarray            # float32[n, 3] point-light positions
    types: list
    inst_type: np.ndarray         # uint32[n]
    inst_R: np.ndarray            # float32[n, 9] row-major, world = s * R * local + T
    inst_T: np.ndarray            # float32[n, 3]
    inst_s: np.ndarray            # float32[n]
    n_shade: int = 8
    shade_half: float = 0.05
    shadow_beta: float = 0.5
    shadow_eps: float = 0.02
    sigma_max: float = 50.0
    sdf_width: float = 0.01
    half_extent: float = 1.0
    extra: dict = field(default_factory=dict)
    # per light: nonzero = a parallel light whose `lights` row is the direction it travels
    # (None: every light is a point light at its `lights` row)
    light_parallel: np.ndarray = None

    @property
    def n_inst(self):
        return int(self.inst_type.shape[0])

    def permuted(self, perm: np.ndarray) -> "Scene":
        """Same scene with instance i of the result = instance perm[i] of this one."""
        import copy
        s = copy.copy(self)
        s.inst_type = self.inst_type[perm].copy()
        s.inst_R = self.inst_R[perm].copy()
        s.inst_T = self.inst_T[perm].copy()
        s.inst_s = self.inst_s[perm].copy()
        return s


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def make_type(kind: int, seed: int, type_index: int, nedf_hidden: int, nedf_width: int,
              nerf_hidden: int = 0, nerf_width: int = 0, albedo=(0.7, 0.7, 0.7), rb: float = 1.0,
              params=None, nedf_seed: int | None = None, nedf_arch: int = ARCH_REGRESSION) -> ObjType:
    p = np.zeros(8, np.float32)
    vals = DEFAULT_PARAMS[kind] if params is None else params
    p[: len(vals)] = f32(vals)
    ns = substream(seed, TAG_NEDF, type_index) if nedf_seed is None else nedf_seed
    if nedf_arch == ARCH_CLASSIFIER:
        nedf, nedf_hidden, nedf_width = cls_weights(ns), 2 * CLS_BLOCKS, CLS_W
    else:
        nedf = xavier_mlp(ns, mlp_dims(NEDF_IN, nedf_hidden, nedf_width, 2))
    nerf = None
    if nerf_hidden:
        nerf = xavier_mlp(substream(seed, TAG_NERF, type_index),
                          mlp_dims(NERF_IN, nerf_hidden, nerf_width, 3))
    return ObjType(kind, p, float(np.float32(rb)), f32(albedo), nedf_hidden, nedf_width, nedf,
                   nerf_hidden, nerf_width, nerf, nedf_arch)


def uniform_rotations(seed: int, n: int) -> np.ndarray:
    """n rotation matrices (row-major float32[n, 9]) by Shoemake's uniform quaternions."""
    u = uniform(seed, 3 * n).reshape(n, 3)
    u1, u2, u3 = u[:, 0], u[:, 1], u[:, 2]
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    R = np.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
        2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
        2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y),
    ], axis=1)
    return f32(R)


def random_instances(seed: int, n: int, n_types: int, half_extent: float, scale: float = 1.0):
    """Types cycle 0,1,..; rotations uniform; translations uniform in [-E, E]^3."""
    inst_type = (np.arange(n) % n_types).astype(np.uint32)
    R = uniform_rotations(substream(seed, TAG_INST, 0), n)
    T = f32((2.0 * uniform(substream(seed, TAG_INST, 1), 3 * n) - 1.0).reshape(n, 3) * half_extent)
    s = np.full(n, scale, np.float32)
    return inst_type, R, T, s


def orbit_camera(half_extent: float):
    """Eye on a sphere of radius 3E in direction (1, 0.6, 1), looking at the origin."""
    d = np.array([1.0, 0.6, 1.0])
    d /= np.linalg.norm(d)
    return f32(3.0 * half_extent * d), f32([0, 0, 0])


def ring_lights(half_extent: float, n: int) -> np.ndarray:
    """L_k = (1.5E cos 2pi k/n, 2E, 1.5E sin 2pi k/n)."""
    k = np.arange(n)
    return f32(np.stack([1.5 * half_extent * np.cos(2 * np.pi * k / n),
                         np.full(n, 2.0 * half_extent),
                         1.5 * half_extent * np.sin(2 * np.pi * k / n)], axis=1))


# ----------------------------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------------------------
def tiny_sphere_scene(W: int = 64, H: int = 64) -> Scene:
    """1 sphere (r 0.5) at the origin, 64x64 camera at (0,0,3), fov 40, light (2,3,2),
    NeDF 4x64 Xavier seed 0, constant albedo 0.7, no colour network."""
    t = make_type(SDF_SPHERE, 0, 0, 4, 64, nedf_seed=0)
    return Scene("sphere-64", W, H, f32([0, 0, 3]), f32([0, 0, 0]), 40.0, f32([[2, 3, 2]]), [t],
                 np.zeros(1, np.uint32), f32(np.eye(3).reshape(1, 9)), f32([[0, 0, 0]]),
                 f32([1.0]), half_extent=1.0)


def _many_scene(name, kinds, n_inst, seed, W, H, E, n_lights, nerf=True) -> Scene:
    types = [make_type(k, seed, i, 6, 128, 8 if nerf else 0, 256 if nerf else 0)
             for i, k in enumerate(kinds)]
    it, R, T, s = random_instances(seed, n_inst, len(kinds), E)
    eye, target = orbit_camera(E)
    return Scene(name, W, H, eye, target, 40.0, ring_lights(E, n_lights), types, it, R, T, s,
                 half_extent=E)


def three_types_scene(W: int = 512, H: int = 512, nerf: bool = True) -> Scene:
    """Sphere / torus / box x 16 instances each, translations in [-4,4]^3, seed 1, 2 lights."""
    return _many_scene("3x16-512", [SDF_SPHERE, SDF_TORUS, SDF_BOX], 48, 1, W, H, 4.0, 2, nerf)


def classifier_scene(W: int = 64, H: int = 64, n_inst: int = 12, seed: int = 5, E: float = 2.5) -> Scene:
    """Sphere / torus / box types carrying the paper's classifier intersection network (seeded
    random weights), n_inst instances in [-E, E]^3, 2 lights, constant albedo."""
    kinds = [SDF_SPHERE, SDF_TORUS, SDF_BOX]
    types = [make_type(k, seed, i, 0, 0, nedf_arch=ARCH_CLASSIFIER) for i, k in enumerate(kinds)]
    it, R, T, s = random_instances(seed, n_inst, len(kinds), E)
    eye, target = orbit_camera(E)
    return Scene(f"cls{len(kinds)}x{n_inst}-{W}", W, H, eye, target, 40.0, ring_lights(E, 2), types, it, R, T, s,
                 half_extent=E)


def thousand_scene(W: int = 1024, H: int = 1024, nerf: bool = True) -> Scene:
    """1024 sphere/torus/box instances in [-20,20]^3, seed 3, 1024^2, 4 lights."""
    return _many_scene("1024inst-1024", [SDF_SPHERE, SDF_TORUS, SDF_BOX], 1024, 3, W, H, 20.0, 4, nerf)


def stress_scene(W: int = 2048, H: int = 2048, nerf: bool = True, n_inst: int = 4096) -> Scene:
    """8 types x 512 instances in [-40,40]^3, seed 4, 2048^2, 8 lights.  A smaller n_inst keeps the
    instance density: the cube's half extent shrinks as the cube root of the count."""
    kinds = [SDF_SPHERE, SDF_TORUS, SDF_BOX, SDF_CAPSULE, SDF_ROUNDCONE, SDF_TWOSPHERE,
             SDF_TWISTTORUS, SDF_OCTA]
    E = 40.0 * (n_inst / 4096.0) ** (1.0 / 3.0)
    return _many_scene(f"{n_inst}inst-{W}", kinds, n_inst, 4, W, H, E, 8, nerf)


def pixel_subset(W: int, H: int, n: int, seed: int) -> np.ndarray:
    """n distinct pixel indices (row-major j*W+i), sorted."""
    n = min(n, W * H)
    keys = splitmix64(substream(seed, TAG_MISC, 7), W * H)
    return np.sort(np.argsort(keys, kind="stable")[:n]).astype(np.int64)
