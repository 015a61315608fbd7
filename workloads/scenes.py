"""Seeded synthetic channel-flow scenes shaped like the paper's blood-flow runs.

A scene is pure input data: box size, fluid parameters, templates (mesh +
stretch + moduli) and objects (template id, origin, Euler angles, mass).
Nothing here evaluates the method.  The same scene is fed to the FP64
oracle and to the CUDA library.

Recipes (stand-ins for the paper's red-blood-cell channel, Sec. 6-7, whose
mesh and geometry files are not available):

  * ``channel_sphere``  40x20x20 channel, walls at y=0 and y=19, tau=1,
    rho0=1, body force 1e-5 along x, drag 0.05 per step, node mass 1, one
    level-2 icosphere of radius 4 at the box centre, ks=0.1 kb=0.03 kal=0.1 kag=0.4 kv=1.0 (the moduli of the
    paper's feature table), nonlinear stretching; 1000 steps.
  * ``channel_rbc``     256x128x128 channel, same fluid, 200 Evans-Fung red
    blood cells (level-3 icosphere mapped to the biconcave profile, radius 8)
    at seeded non-overlapping positions with uniform random orientation.
  * ``channel_rbc_large`` 512x256x256 with 2000 such cells.
  * ``batch_mix``       64 independent channels of random size and load.
  * ``serving_trace``   a seeded Poisson stream of channel requests.

Placement: centres by rejection sampling; bounding spheres at least
2R+2 apart (minimum image in the periodic x and z directions) and at least
R+2 from the wall planes y=1 and y=ny-1.  Orientation: a uniform random
unit quaternion (Shoemake's method) converted to Euler angles (rx, ry, rz)
with R = Rz(rz) Ry(ry) Rx(rx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import mesh as _mesh

PAPER_MODULI = dict(ks=0.1, kb=0.03, kal=0.1, kag=0.4, kv=1.0)

# The soft-sphere interactions of the paper's blood-cell example (Sec. 6):
# object-object (a 0.005, n 2, cutoff 0.3) and object-wall (a 0.0001, n 1.2,
# cutoff 0.1), set at an MD time step of 0.1 with the lattice spacing as the
# length unit.  A force integrated over one lattice step (the unit time step
# here) scales with the time step squared, so in lattice units a becomes
# a x 0.1^2; n and the cutoffs are lengths' exponents and lengths and stay.
PAPER_REPULSION = ((0.005 * 0.1 ** 2, 2.0, 0.3), (0.0001 * 0.1 ** 2, 1.2, 0.1))


@dataclass
class Template:
    nodes: np.ndarray           # float64 [N,3], unit-size, centred
    tris: np.ndarray            # int32 [T,3], inward-oriented
    stretch: tuple = (1.0, 1.0, 1.0)
    ks: float = 0.0
    kb: float = 0.0
    kal: float = 0.0
    kag: float = 0.0
    kv: float = 0.0
    nonlinear: int = 1


@dataclass
class Obj:
    tid: int
    origin: tuple
    rotate: tuple = (0.0, 0.0, 0.0)
    mass: float = 1.0
    force: tuple = (0.0, 0.0, 0.0)


@dataclass
class Scene:
    name: str
    nx: int
    ny: int
    nz: int
    walls: int = 1
    tau: float = 1.0
    rho0: float = 1.0
    body_force: tuple = (1e-5, 0.0, 0.0)
    # drag coefficient per lattice step: the paper's example pairs friction
    # 0.5 with an integration time step of 0.1 (Sec. 6), i.e. a momentum
    # exchange of 0.05 of the relative velocity per step for unit node mass
    friction: float = 0.05
    steps: int = 1000
    # soft-sphere repulsion ((a, n, cutoff) object-object, (a, n, cutoff)
    # object-wall), or None for none
    repulsion: tuple = None
    # velocity inlet ((x0, x1, y0, y1, z0, z1) cell box, (ux, uy, uz)), or None
    inlet: tuple = None
    # obstacle cells: bool [nz][ny][nx] (see geometry.rhomboid_mask), or None
    solid: object = None
    templates: list = field(default_factory=list)
    objects: list = field(default_factory=list)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_fluid_cells(self) -> int:
        return self.nx * (self.ny - 2 if self.walls else self.ny) * self.nz

    @property
    def n_nodes(self) -> int:
        return sum(len(self.templates[o.tid].nodes) for o in self.objects)


def quaternion_to_euler_zyx(q: np.ndarray) -> tuple:
    """Euler angles (rx, ry, rz) with R = Rz(rz) Ry(ry) Rx(rx) for unit q=(w,x,y,z)."""
    w, x, y, z = q
    r00 = 1 - 2 * (y * y + z * z)
    r10 = 2 * (x * y + w * z)
    r20 = 2 * (x * z - w * y)
    r21 = 2 * (y * z + w * x)
    r22 = 1 - 2 * (x * x + y * y)
    ry = math.asin(max(-1.0, min(1.0, -r20)))
    rx = math.atan2(r21, r22)
    rz = math.atan2(r10, r00)
    return (rx, ry, rz)


def random_rotation(rng: np.random.Generator) -> tuple:
    """Uniformly distributed rotation (Shoemake 1992) as ZYX Euler angles."""
    u1, u2, u3 = rng.random(3)
    q = np.array([
        math.sqrt(u1) * math.cos(2 * math.pi * u3),
        math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
        math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
        math.sqrt(u1) * math.sin(2 * math.pi * u3),
    ])
    return quaternion_to_euler_zyx(q)


def place_spheres(rng, nx, ny, nz, radius, count, walls=True, max_tries=200000):
    """Seeded rejection sampling of non-overlapping bounding spheres."""
    sep = 2.0 * radius + 2.0
    ylo, yhi = (1.0 + radius + 2.0, ny - 1.0 - radius - 2.0) if walls else (0.0, float(ny))
    if yhi < ylo:
        return np.zeros((0, 3))
    box = np.array([nx, ny, nz], dtype=np.float64)
    centres = np.zeros((0, 3))
    tries = 0
    while len(centres) < count and tries < max_tries:
        tries += 1
        c = np.array([rng.random() * nx, ylo + rng.random() * (yhi - ylo), rng.random() * nz])
        if len(centres):
            d = centres - c
            for ax in (0, 2):
                d[:, ax] -= box[ax] * np.round(d[:, ax] / box[ax])
            if not walls:
                d[:, 1] -= box[1] * np.round(d[:, 1] / box[1])
            if np.min(np.einsum("ij,ij->i", d, d)) < sep * sep:
                continue
        centres = np.vstack([centres, c])
    return centres


def channel_sphere(steps: int = 1000, with_object: bool = True) -> Scene:
    s = Scene("channel_sphere_40x20x20", 40, 20, 20, steps=steps)
    if with_object:
        nodes, tris = _mesh.icosphere(2)
        s.templates.append(Template(nodes, tris, (4.0, 4.0, 4.0), **PAPER_MODULI))
        s.objects.append(Obj(0, (20.0, 10.0, 10.0)))
    return s


def _rbc_channel(name, nx, ny, nz, count, seed, level=3, radius=8.0, steps=10000):
    rng = np.random.default_rng(seed)
    s = Scene(name, nx, ny, nz, steps=steps)
    nodes, tris = _mesh.biconcave(level)
    s.templates.append(Template(nodes, tris, (radius, radius, radius), **PAPER_MODULI))
    centres = place_spheres(rng, nx, ny, nz, radius, count)
    for c in centres:
        s.objects.append(Obj(0, tuple(float(v) for v in c), random_rotation(rng)))
    return s


def channel_rbc(count: int = 200, seed: int = 1, steps: int = 10000) -> Scene:
    return _rbc_channel("channel_rbc_256x128x128", 256, 128, 128, count, seed, steps=steps)


def channel_rbc_large(count: int = 2000, seed: int = 2, steps: int = 20000) -> Scene:
    return _rbc_channel("channel_rbc_512x256x256", 512, 256, 256, count, seed, steps=steps)


def _log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def _min_radius(level: int) -> float:
    """Smallest radius at which a level-`level` mesh keeps its mean edge at
    0.5 lu or more (edge ~ 1.05 R / 2^level): finer meshes make the explicit
    membrane update unstable at the paper's moduli with unit node mass."""
    return 0.5 * 2 ** level / 1.05


def batch_mix(n_sims: int = 64, seed: int = 3, steps: int = 100) -> list:
    """Independent channels: box log-uniform per axis in [32, (128,64,64)],
    0-40 biconcave cells of level 2, 3 or 4, radius scaled to the box (at
    least the level's stable minimum; a level that does not fit the box at
    that radius drops to the next lower one)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_sims):
        nx = _log_uniform_int(rng, 32, 128)
        ny = _log_uniform_int(rng, 32, 64)
        nz = _log_uniform_int(rng, 32, 64)
        count = int(rng.integers(0, 41))
        level = int(rng.choice([2, 3, 4]))
        radius = float(min(8.0, max(3.0, 0.2 * min(nx, ny - 2, nz))))
        while level > 2 and 2.0 * max(radius, _min_radius(level)) + 4.0 > min(nx, ny - 2, nz):
            level -= 1
        radius = max(radius, _min_radius(level))
        s = Scene(f"batch{i}_{nx}x{ny}x{nz}", nx, ny, nz, steps=steps)
        nodes, tris = _mesh.biconcave(level)
        s.templates.append(Template(nodes, tris, (radius,) * 3, **PAPER_MODULI))
        for c in place_spheres(rng, nx, ny, nz, radius, count, max_tries=5000):
            s.objects.append(Obj(0, tuple(float(v) for v in c), random_rotation(rng)))
        out.append(s)
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    scene: Scene
    steps: int


def serving_trace(n_requests: int = 256, seed: int = 4, rate_per_s: float = 1.0,
                  max_box=(192, 96, 96), max_rbc: int = 100,
                  steps_range=(1000, 20000)) -> list:
    """Poisson arrivals of channel requests: box log-uniform per axis between
    32^3 and max_box, 1..max_rbc level-3 cells (as many as fit), steps
    log-uniform in steps_range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    nodes, tris = _mesh.biconcave(3)
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        nx = _log_uniform_int(rng, 32, max_box[0])
        ny = _log_uniform_int(rng, 32, max_box[1])
        nz = _log_uniform_int(rng, 32, max_box[2])
        want = int(rng.integers(1, max_rbc + 1))
        steps = _log_uniform_int(rng, *steps_range)
        s = Scene(f"req{i}_{nx}x{ny}x{nz}", nx, ny, nz, steps=steps)
        s.templates.append(Template(nodes, tris, (8.0, 8.0, 8.0), **PAPER_MODULI))
        for c in place_spheres(rng, nx, ny, nz, 8.0, want, max_tries=3000):
            s.objects.append(Obj(0, tuple(float(v) for v in c), random_rotation(rng)))
        out.append(Request(i, t, s, steps))
    return out
