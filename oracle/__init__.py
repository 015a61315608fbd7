"""FP64 CPU oracle of the LB-IB step — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its binding) never imports, links or runs it.  It shares no code with
that path; the two meet only in the seeded inputs of ``workloads``.

``build()`` compiles ``lbib_oracle.c`` with the host C compiler (OpenMP when
the compiler supports it) into ``_lbib_oracle.so`` next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbib_oracle.c")
_LIB = os.path.join(_HERE, "_lbib_oracle.so")
_lib = None

NQ = 19


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, no CUDA)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-D_DEFAULT_SOURCE",
            "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    P = C.c_void_p
    dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    sig = {
        "oracle_create": (P, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp, C.c_double]),
        "oracle_destroy": (None, [P]),
        "oracle_threads": (C.c_int, []),
        "oracle_lattice": (None, [P, ip, dp]),
        "oracle_template_create": (C.c_int, [P, dp, C.c_int, ip, C.c_int, dp, C.c_double, C.c_double,
                                             C.c_double, C.c_double, C.c_double, C.c_int]),
        "oracle_template_topology": (C.c_int, [P, C.c_int, P, P, P, P, P, P]),
        "oracle_object_add": (C.c_int, [P, C.c_int, dp, dp, C.c_double]),
        "oracle_object_nodes": (C.c_int, [P, C.c_int]),
        "oracle_object_set_force": (C.c_int, [P, C.c_int, dp]),
        "oracle_object_set_nodes": (C.c_int, [P, C.c_int, dp]),
        "oracle_object_set_velocities": (C.c_int, [P, C.c_int, dp]),
        "oracle_read_nodes": (C.c_int, [P, C.c_int, P, P]),
        "oracle_object_measures": (C.c_int, [P, C.c_int, dp]),
        "oracle_membrane_forces": (C.c_int, [P, C.c_int, C.c_int, dp]),
        "oracle_fluid_init": (None, [P]),
        "oracle_step": (None, [P, C.c_int]),
        "oracle_step_nodes_only": (None, [P, C.c_int]),
        "oracle_set_repulsion": (C.c_int, [P, dp, dp]),
        "oracle_set_inlet": (C.c_int, [P, ip, dp]),
        "oracle_set_solid": (C.c_int, [P, P]),
        "oracle_template_set_kal_direction": (C.c_int, [P, C.c_int, C.c_int]),
        "oracle_repulsion_forces": (None, [P, dp]),
        "oracle_read_velocity": (None, [P, dp]),
        "oracle_set_velocity": (None, [P, dp]),
        "oracle_read_density": (None, [P, dp]),
        "oracle_read_populations": (None, [P, dp]),
        "oracle_set_populations": (None, [P, dp]),
        "oracle_read_ib_force": (None, [P, dp]),
        "oracle_read_dropped": (None, [P, dp]),
        "oracle_fluid_totals": (None, [P, dp]),
        "oracle_interpolate": (None, [P, dp, dp]),
        "oracle_object_edge_angles": (C.c_int, [P, C.c_int, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def threads() -> int:
    return int(_load().oracle_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One FP64 simulation: fluid box, templates, objects (see lbib_oracle.c)."""

    def __init__(self, nx, ny, nz, walls=True, tau=1.0, rho0=1.0, body_force=(0, 0, 0), friction=0.5):
        self._lib = _load()
        g = np.ascontiguousarray(body_force, dtype=np.float64)
        self._h = self._lib.oracle_create(nx, ny, nz, int(bool(walls)), tau, rho0, g, friction)
        if not self._h:
            raise ValueError("oracle_create rejected the fluid parameters")
        self.nx, self.ny, self.nz, self.walls = nx, ny, nz, bool(walls)
        self.n_templates = 0
        self.n_objects = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    @classmethod
    def from_scene(cls, scene, with_objects=True):
        o = cls(scene.nx, scene.ny, scene.nz, scene.walls, scene.tau, scene.rho0,
                scene.body_force, scene.friction)
        if with_objects:
            for t in scene.templates:
                o.template_create(t.nodes, t.tris, t.stretch, t.ks, t.kb, t.kal, t.kag, t.kv, t.nonlinear)
            for ob in scene.objects:
                oid = o.object_add(ob.tid, ob.origin, ob.rotate, ob.mass)
                if any(ob.force):
                    o.object_set_force(oid, ob.force)
        rep = getattr(scene, "repulsion", None)
        if rep is not None:
            o.set_repulsion(*rep)
        inlet = getattr(scene, "inlet", None)
        if inlet is not None:
            o.set_inlet(*inlet)
        solid = getattr(scene, "solid", None)
        if solid is not None:
            o.set_solid(solid)
        o.fluid_init()
        return o

    # lattice -----------------------------------------------------------
    def lattice(self):
        e = np.zeros((NQ, 3), np.int32)
        w = np.zeros(NQ, np.float64)
        self._lib.oracle_lattice(self._h, e, w)
        return e, w

    # templates / objects ----------------------------------------------
    def template_create(self, nodes, tris, stretch=(1, 1, 1), ks=0.0, kb=0.0, kal=0.0, kag=0.0, kv=0.0,
                        nonlinear=1):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        tris = np.ascontiguousarray(tris, dtype=np.int32)
        rc = self._lib.oracle_template_create(self._h, nodes, len(nodes), tris, len(tris),
                                              np.ascontiguousarray(stretch, dtype=np.float64),
                                              ks, kb, kal, kag, kv, int(nonlinear))
        if rc < 0:
            raise ValueError(f"oracle_template_create failed ({rc})")
        self.n_templates += 1
        return rc

    def topology(self, tid, n_tris):
        ne = self._lib.oracle_template_topology(self._h, tid, None, None, None, None, None, None)
        edges = np.zeros((ne, 2), np.int32)
        quads = np.zeros((ne, 4), np.int32)
        L0 = np.zeros(ne)
        th0 = np.zeros(ne)
        S0 = np.zeros(n_tris)
        glob = np.zeros(2)
        self._lib.oracle_template_topology(self._h, tid, _ptr(edges), _ptr(quads), _ptr(L0), _ptr(th0),
                                           _ptr(S0), _ptr(glob))
        return dict(edges=edges, quads=quads, L0=L0, theta0=th0, S0=S0, Sg0=glob[0], V0=glob[1])

    def object_add(self, tid, origin, rotate=(0, 0, 0), mass=1.0):
        rc = self._lib.oracle_object_add(self._h, tid, np.ascontiguousarray(origin, dtype=np.float64),
                                         np.ascontiguousarray(rotate, dtype=np.float64), mass)
        if rc < 0:
            raise ValueError("oracle_object_add failed")
        self.n_objects += 1
        return rc

    def object_set_force(self, oid, f):
        self._lib.oracle_object_set_force(self._h, oid, np.ascontiguousarray(f, dtype=np.float64))

    def object_set_nodes(self, oid, xyz):
        self._lib.oracle_object_set_nodes(self._h, oid, np.ascontiguousarray(xyz, dtype=np.float64))

    def object_set_velocities(self, oid, v):
        self._lib.oracle_object_set_velocities(self._h, oid, np.ascontiguousarray(v, dtype=np.float64))

    def read_nodes(self, oid):
        n = self._lib.oracle_object_nodes(self._h, oid)
        x = np.zeros((n, 3))
        v = np.zeros((n, 3))
        self._lib.oracle_read_nodes(self._h, oid, _ptr(x), _ptr(v))
        return x, v

    def object_measures(self, oid):
        out = np.zeros(2)
        self._lib.oracle_object_measures(self._h, oid, out)
        return out[0], out[1]

    def membrane_forces(self, oid, mask=31):
        n = self._lib.oracle_object_nodes(self._h, oid)
        F = np.zeros((n, 3))
        self._lib.oracle_membrane_forces(self._h, oid, mask, F)
        return F

    # fluid --------------------------------------------------------------
    def set_repulsion(self, obj=(0.0, 1.0, 0.0), wall=(0.0, 1.0, 0.0)):
        """Soft-sphere repulsion (a, n, cutoff) between objects and against the walls."""
        rc = self._lib.oracle_set_repulsion(self._h, np.ascontiguousarray(obj, dtype=np.float64),
                                            np.ascontiguousarray(wall, dtype=np.float64))
        if rc != 0:
            raise ValueError("invalid repulsion parameters")

    def set_inlet(self, box, u):
        """Velocity inlet over cells box = (x0, x1, y0, y1, z0, z1) (half-open)."""
        self._lib.oracle_set_inlet(self._h, np.ascontiguousarray(box, dtype=np.int32),
                                   np.ascontiguousarray(u, dtype=np.float64))

    def template_set_kal_direction(self, tid, altitude):
        if self._lib.oracle_template_set_kal_direction(self._h, tid, int(bool(altitude))) != 0:
            raise ValueError("unknown template")

    def set_solid(self, mask):
        """Obstacle cells from a [nz][ny][nx] boolean mask (None: none)."""
        if mask is None:
            self._lib.oracle_set_solid(self._h, None)
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.nz, self.ny, self.nx)
        self._solid = m
        self._lib.oracle_set_solid(self._h, m.ctypes.data_as(C.c_void_p))

    def n_nodes(self):
        return sum(self._lib.oracle_object_nodes(self._h, o) for o in range(self.n_objects))

    def repulsion_forces(self):
        F = np.zeros(3 * self.n_nodes())
        self._lib.oracle_repulsion_forces(self._h, F)
        return F.reshape(-1, 3)

    def fluid_init(self):
        self._lib.oracle_fluid_init(self._h)

    def step(self, n=1):
        self._lib.oracle_step(self._h, int(n))

    def step_nodes_only(self, n=1):
        self._lib.oracle_step_nodes_only(self._h, int(n))

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def velocity(self):
        u = np.zeros(3 * self.ncell)
        self._lib.oracle_read_velocity(self._h, u)
        return u.reshape(3, self.nz, self.ny, self.nx)

    def set_velocity(self, u):
        self._lib.oracle_set_velocity(self._h, np.ascontiguousarray(u, dtype=np.float64).ravel())

    def density(self):
        r = np.zeros(self.ncell)
        self._lib.oracle_read_density(self._h, r)
        return r.reshape(self.nz, self.ny, self.nx)

    def populations(self):
        f = np.zeros(self.ncell * NQ)
        self._lib.oracle_read_populations(self._h, f)
        return f.reshape(self.nz, self.ny, self.nx, NQ)

    def set_populations(self, f):
        self._lib.oracle_set_populations(self._h, np.ascontiguousarray(f, dtype=np.float64).ravel())

    def ib_force(self):
        g = np.zeros(3 * self.ncell)
        self._lib.oracle_read_ib_force(self._h, g)
        return g.reshape(3, self.nz, self.ny, self.nx)

    def dropped(self):
        d = np.zeros(3)
        self._lib.oracle_read_dropped(self._h, d)
        return d

    def fluid_totals(self):
        out = np.zeros(4)
        self._lib.oracle_fluid_totals(self._h, out)
        return out[0], out[1:].copy()

    def edge_angles(self, oid, n_edges):
        th = np.zeros(n_edges)
        self._lib.oracle_object_edge_angles(self._h, oid, _ptr(th))
        return th

    def interpolate(self, X):
        u = np.zeros(3)
        self._lib.oracle_interpolate(self._h, np.ascontiguousarray(X, dtype=np.float64), u)
        return u
