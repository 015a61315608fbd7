"""Thin ctypes binding of the C ABI in ``include/lbib.h``.

Every function here has the name of the C entry point it calls and only
marshals arguments (numpy arrays in, numpy arrays out); all computation runs
in the CUDA library ``_lbib.so``.  There is no fallback: if the library is
missing or fails to load, :func:`load` raises.

The :class:`Sim` class bundles the calls for one simulation handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lbib.so")
_lib = None

LBIB_OK = 0
LBIB_ERR_ARG = -1
LBIB_ERR_NOMEM = -4
STATUS_NAMES = {
    0: "LBIB_OK", -1: "LBIB_ERR_ARG", -2: "LBIB_ERR_ID", -3: "LBIB_ERR_MESH", -4: "LBIB_ERR_NOMEM",
    -5: "LBIB_ERR_UNSTABLE", -6: "LBIB_ERR_TIMEOUT", -7: "LBIB_ERR_CUDA", -8: "LBIB_ERR_STATE",
}
LBIB_POP_F32, LBIB_POP_F16S, LBIB_POP_BF16S = 0, 1, 2
PRECISIONS = {"f32": LBIB_POP_F32, "f16s": LBIB_POP_F16S, "bf16s": LBIB_POP_BF16S}


class LbibError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


class lbib_fluid_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("walls_y", C.c_int),
        ("tau", C.c_double), ("rho0", C.c_double), ("body_force", C.c_double * 3),
        ("friction", C.c_double), ("precision", C.c_int), ("pop_scale_log2", C.c_int),
    ]


def load(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run paper_1312_3426_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    st = C.c_int
    pp = C.POINTER(lbib_fluid_params)
    sig = {
        "lbib_create": (st, [pp, P, C.POINTER(P)]),
        "lbib_destroy": (None, [P]),
        "lbib_last_error": (C.c_char_p, [P]),
        "lbib_template_create": (st, [P, C.c_int, P, C.c_int, P, C.c_int, P, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.c_int]),
        "lbib_template_topology": (st, [P, C.c_int, P, P, P, P, P, P, C.POINTER(C.c_int)]),
        "lbib_mesh_check": (st, [P, C.c_int, P, C.c_int, P, P, P, P, P, P, P, C.POINTER(C.c_int), C.c_char_p,
                                 C.c_int]),
        "lbib_object_add": (st, [P, C.c_int, C.c_int, P, P, C.c_double]),
        "lbib_object_set_force": (st, [P, C.c_int, P]),
        "lbib_set_repulsion": (st, [P, P, P]),
        "lbib_set_inlet": (st, [P, P, P]),
        "lbib_set_solid": (st, [P, P, C.c_int64]),
        "lbib_template_set_kal_direction": (st, [P, C.c_int, C.c_int]),
        "lbib_mesh_orient": (st, [P, C.c_int, P, C.c_int, C.c_int, P, C.POINTER(C.c_int)]),
        "lbib_object_set_nodes": (st, [P, C.c_int, P, C.c_int]),
        "lbib_object_set_velocities": (st, [P, C.c_int, P, C.c_int]),
        "lbib_fluid_init": (st, [P]),
        "lbib_step": (st, [P, C.c_int]),
        "lbib_sync": (st, [P]),
        "lbib_read_nodes": (st, [P, C.c_int, P, P, C.c_int64]),
        "lbib_read_velocity": (st, [P, P, C.c_int64]),
        "lbib_read_density": (st, [P, P, C.c_int64]),
        "lbib_read_populations": (st, [P, P, C.c_int64]),
        "lbib_read_coupling_force": (st, [P, P, C.c_int64]),
        "lbib_set_coupling_force": (st, [P, P, C.c_int64]),
        "lbib_set_populations": (st, [P, P, C.c_int64]),
        "lbib_object_analyze": (st, [P, C.c_int, P]),
        "lbib_fluid_mass": (st, [P, P]),
        "lbib_fluid_mass_noalloc": (st, [P, P]),
        "lbib_info": (st, [P, P]),
        "lbib_dropped_momentum": (st, [P, P]),
        "lbib_lattice": (C.c_int, [P, P]),
        "lbib_footprint_bytes": (C.c_int64, [pp, C.c_int64, C.c_int64]),
        "lbib_batch_step": (st, [P, C.c_int, C.c_int]),
        "lbib_objects_set_force": (st, [P, P, C.c_int]),
        "lbib_objects_analyze": (st, [P, P, C.c_int64]),
        "lbib_objects_analyze_async": (st, [P, C.c_int]),
        "lbib_objects_analyze_wait": (st, [P, C.c_int, P, C.c_int64]),
        "lbib_profile_enable": (st, [P, C.c_int]),
        "lbib_set_tuning": (st, [P, C.c_int, C.c_int]),
        "lbib_get_tuning": (st, [P, C.c_int, C.POINTER(C.c_int)]),
        "lbib_profile_read": (st, [P, P]),
        "lbib_abi_version": (C.c_int, []),
        "lbib_check_bounded_wait": (st, [C.c_double, C.c_int, C.POINTER(C.c_int)]),
        "lbib_server_create": (st, [C.c_int64, C.c_int, C.c_int, C.POINTER(P)]),
        "lbib_server_destroy": (None, [P]),
        "lbib_server_admit": (st, [P, P, C.c_int64, C.c_int64]),
        "lbib_server_advance": (st, [P, P, C.c_int, C.POINTER(C.c_int)]),
        "lbib_server_stats": (st, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(h, status):
    if status != LBIB_OK:
        msg = _lib.lbib_last_error(h).decode() if h else ""
        raise LbibError(status, msg)


def fluid_params(nx, ny, nz, walls=True, tau=1.0, rho0=1.0, body_force=(0.0, 0.0, 0.0), friction=0.5,
                 precision="f32", pop_scale_log2=0) -> lbib_fluid_params:
    p = lbib_fluid_params()
    p.nx, p.ny, p.nz, p.walls_y = int(nx), int(ny), int(nz), int(bool(walls))
    p.tau, p.rho0, p.friction = float(tau), float(rho0), float(friction)
    for k in range(3):
        p.body_force[k] = float(body_force[k])
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.pop_scale_log2 = int(pop_scale_log2)
    return p


# ----------------------------------------------------------------- C entry points

def lbib_create(params: lbib_fluid_params, stream: int | None = None):
    load()
    h = C.c_void_p()
    _check(None, _lib.lbib_create(C.byref(params), C.c_void_p(stream or 0), C.byref(h)))
    return h


def lbib_destroy(h):
    load().lbib_destroy(h)


def lbib_last_error(h) -> str:
    return load().lbib_last_error(h).decode()


def lbib_template_create(h, tid, nodes, tris, stretch=(1.0, 1.0, 1.0), ks=0.0, kb=0.0, kal=0.0, kag=0.0, kv=0.0,
                         nonlinear_ks=1):
    nodes = _f64(nodes)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    st = _f64(stretch)
    _check(h, _lib.lbib_template_create(h, int(tid), _p(nodes), len(nodes), _p(tris), len(tris), _p(st),
                                        ks, kb, kal, kag, kv, int(nonlinear_ks)))


def lbib_template_topology(h, tid, n_tris):
    ne = C.c_int()
    _check(h, _lib.lbib_template_topology(h, int(tid), None, None, None, None, None, None, C.byref(ne)))
    n = ne.value
    edges = np.zeros((n, 2), np.int32)
    quads = np.zeros((n, 4), np.int32)
    L0, th0, S0, glob = np.zeros(n), np.zeros(n), np.zeros(n_tris), np.zeros(2)
    _check(h, _lib.lbib_template_topology(h, int(tid), _p(edges), _p(quads), _p(L0), _p(th0), _p(S0), _p(glob),
                                          C.byref(ne)))
    return dict(edges=edges, quads=quads, L0=L0, theta0=th0, S0=S0, Sg0=glob[0], V0=glob[1])


def lbib_mesh_check(nodes, tris, stretch=(1.0, 1.0, 1.0)):
    """Validates a mesh on the host; returns the topology dict or raises LbibError."""
    load()
    nodes = _f64(nodes)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    st = _f64(stretch)
    ne_max = (3 * len(tris)) // 2 + 1
    edges = np.zeros((ne_max, 2), np.int32)
    quads = np.zeros((ne_max, 4), np.int32)
    L0, th0, S0, glob = np.zeros(ne_max), np.zeros(ne_max), np.zeros(len(tris)), np.zeros(2)
    ne = C.c_int()
    msg = C.create_string_buffer(256)
    status = _lib.lbib_mesh_check(_p(nodes), len(nodes), _p(tris), len(tris), _p(st), _p(edges), _p(quads), _p(L0),
                                  _p(th0), _p(S0), _p(glob), C.byref(ne), msg, 256)
    if status != LBIB_OK:
        raise LbibError(status, msg.value.decode())
    n = ne.value
    return dict(edges=edges[:n], quads=quads[:n], L0=L0[:n], theta0=th0[:n], S0=S0, Sg0=glob[0], V0=glob[1])


def lbib_object_add(h, oid, tid, origin, rotate=(0.0, 0.0, 0.0), mass=1.0):
    o, r = _f64(origin), _f64(rotate)
    _check(h, _lib.lbib_object_add(h, int(oid), int(tid), _p(o), _p(r), float(mass)))


def lbib_object_set_force(h, oid, f):
    f = _f64(f)
    _check(h, _lib.lbib_object_set_force(h, int(oid), _p(f)))


def lbib_object_set_nodes(h, oid, xyz):
    xyz = _f64(xyz)
    _check(h, _lib.lbib_object_set_nodes(h, int(oid), _p(xyz), len(xyz)))


def lbib_object_set_velocities(h, oid, v):
    v = _f64(v)
    _check(h, _lib.lbib_object_set_velocities(h, int(oid), _p(v), len(v)))


def lbib_fluid_init(h):
    _check(h, _lib.lbib_fluid_init(h))


def lbib_step(h, n=1):
    _check(h, _lib.lbib_step(h, int(n)))


def lbib_sync(h):
    _check(h, _lib.lbib_sync(h))


def lbib_read_nodes(h, oid, n_nodes, xyz_out=None, v_out=None, velocities=True):
    """Positions (and velocities) [n][3]; writes into the given arrays when provided."""
    xyz = xyz_out if xyz_out is not None else np.empty((n_nodes, 3))
    v = v_out if v_out is not None else (np.empty((n_nodes, 3)) if velocities else None)
    _check(h, _lib.lbib_read_nodes(h, int(oid), _p(xyz), _p(v), int(n_nodes)))
    return xyz, v


def lbib_read_velocity(h, nx, ny, nz):
    u = np.empty((3, nz, ny, nx), np.float32)
    _check(h, _lib.lbib_read_velocity(h, _p(u), u.size))
    return u


def lbib_read_density(h, nx, ny, nz):
    r = np.empty((nz, ny, nx), np.float32)
    _check(h, _lib.lbib_read_density(h, _p(r), r.size))
    return r


def lbib_read_coupling_force(h, nx, ny, nz):
    g = np.zeros((3, nz, ny, nx), np.float32)
    _check(h, _lib.lbib_read_coupling_force(h, _p(g), g.size))
    return g


def lbib_set_coupling_force(h, g):
    g = np.ascontiguousarray(g, dtype=np.float32)
    _check(h, _lib.lbib_set_coupling_force(h, _p(g), g.size))


def lbib_read_populations(h, nx, ny, nz):
    f = np.empty((19, nz, ny, nx), np.float64)
    _check(h, _lib.lbib_read_populations(h, _p(f), f.size))
    return f


def lbib_set_populations(h, hpop):
    hpop = _f64(hpop)
    _check(h, _lib.lbib_set_populations(h, _p(hpop), hpop.size))


def lbib_object_analyze(h, oid):
    out = np.zeros(14)
    _check(h, _lib.lbib_object_analyze(h, int(oid), _p(out)))
    return out


def lbib_objects_set_force(h, f):
    f = _f64(f)
    _check(h, _lib.lbib_objects_set_force(h, _p(f), len(f)))


def lbib_objects_analyze(h, n_obj, out=None):
    out = out if out is not None else np.zeros((n_obj, 14))
    _check(h, _lib.lbib_objects_analyze(h, _p(out), int(n_obj)))
    return out


def lbib_objects_analyze_async(h, slot):
    _check(h, _lib.lbib_objects_analyze_async(h, int(slot)))


def lbib_objects_analyze_wait(h, slot, n_obj, out=None):
    out = out if out is not None else np.zeros((max(n_obj, 1), 14))
    _check(h, _lib.lbib_objects_analyze_wait(h, int(slot), _p(out), int(n_obj)))
    return out


LBIB_TUNE_IB_CLUSTER = 0
LBIB_TUNE_OVERLAP = 1
LBIB_TUNE_MEMBRANE_CLUSTERS = 2
LBIB_TUNE_MEMBRANE_THREADS = 3
LBIB_TUNE_FLUID_KERNEL = 4
LBIB_TUNE_NODE_THREADS = 5
LBIB_TUNE_MEMBRANE_GROUP = 6
LBIB_TUNE_EARLY_LAUNCH = 7


def lbib_set_tuning(h, key, value):
    _check(h, _lib.lbib_set_tuning(h, int(key), int(value)))


def lbib_get_tuning(h, key):
    v = C.c_int()
    _check(h, _lib.lbib_get_tuning(h, int(key), C.byref(v)))
    return v.value


def lbib_profile_enable(h, on=True):
    """on: False/0 off, True/1 every step, n > 1 every n-th step."""
    _check(h, _lib.lbib_profile_enable(h, int(on)))


def lbib_profile_read(h):
    out = np.zeros(6)
    _check(h, _lib.lbib_profile_read(h, _p(out)))
    return dict(fluid_ms=out[0], fluid_launches=int(out[1]), nodes_ms=out[2], nodes_launches=int(out[3]),
                membrane_ms=out[4], membrane_launches=int(out[5]))


def lbib_set_repulsion(h, obj=(0.0, 1.0, 0.0), wall=(0.0, 1.0, 0.0)):
    a = _f64(obj, (3,))
    b = _f64(wall, (3,))
    _check(h, _lib.lbib_set_repulsion(h, _p(a), _p(b)))


MESH_CHECK, MESH_REPAIR, MESH_FLIP = 0, 1, 2


def lbib_mesh_orient(nodes, tris, mode=MESH_REPAIR):
    """(triangles after the operation, number of triangles turned)."""
    load()
    x = _f64(nodes).reshape(-1, 3)
    t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    out = np.zeros_like(t)
    n = C.c_int(0)
    st = _lib.lbib_mesh_orient(_p(x), len(x), _p(t), len(t), int(mode), _p(out), C.byref(n))
    if st != LBIB_OK:
        raise LbibError(st, "lbib_mesh_orient")
    return out, n.value


def lbib_template_set_kal_direction(h, tid, altitude):
    _check(h, _lib.lbib_template_set_kal_direction(h, int(tid), int(bool(altitude))))


def lbib_set_solid(h, mask):
    """Obstacle cells from a [nz][ny][nx] boolean mask (None: none)."""
    if mask is None:
        _check(h, _lib.lbib_set_solid(h, None, 0))
        return
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    _check(h, _lib.lbib_set_solid(h, _p(m), int(m.size)))


def lbib_set_inlet(h, box, u):
    b = np.ascontiguousarray(box, dtype=np.int32).reshape(6)
    v = _f64(u, (3,))
    _check(h, _lib.lbib_set_inlet(h, _p(b), _p(v)))


def lbib_fluid_mass_noalloc(h):
    out = np.zeros(1)
    _check(h, _lib.lbib_fluid_mass_noalloc(h, _p(out)))
    return float(out[0])


def lbib_fluid_mass(h):
    out = np.zeros(1)
    _check(h, _lib.lbib_fluid_mass(h, _p(out)))
    return float(out[0])


def lbib_info(h):
    out = np.zeros(8, np.int64)
    _check(h, _lib.lbib_info(h, _p(out)))
    return out


def lbib_dropped_momentum(h):
    out = np.zeros(3)
    _check(h, _lib.lbib_dropped_momentum(h, _p(out)))
    return out


def lbib_lattice():
    load()
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    _lib.lbib_lattice(_p(e), _p(w))
    return e, w


def lbib_footprint_bytes(params, n_nodes, n_tri_total):
    load()
    return int(_lib.lbib_footprint_bytes(C.byref(params), int(n_nodes), int(n_tri_total)))


def lbib_batch_step(handles, n_steps=1):
    arr = (C.c_void_p * len(handles))(*[h.value for h in handles])
    st = _lib.lbib_batch_step(arr, len(handles), int(n_steps))
    if st != LBIB_OK:
        raise LbibError(st, _lib.lbib_last_error(handles[0]).decode())


def lbib_abi_version():
    return int(load().lbib_abi_version())


def lbib_check_bounded_wait(seconds, arrive=False):
    """True when a device wait on a barrier bounded by `seconds` gave up."""
    load()
    out = C.c_int(-1)
    st = _lib.lbib_check_bounded_wait(float(seconds), int(bool(arrive)), C.byref(out))
    if st != LBIB_OK:
        raise LbibError(st, "")
    return bool(out.value)


def lbib_server_create(budget_bytes, max_resident, chunk_steps):
    load()
    out = C.c_void_p()
    st = _lib.lbib_server_create(int(budget_bytes), int(max_resident), int(chunk_steps), C.byref(out))
    if st != LBIB_OK:
        raise LbibError(st, "lbib_server_create")
    return out


def lbib_server_destroy(srv):
    _lib.lbib_server_destroy(srv)


def lbib_server_admit(srv, h, n_steps, tag):
    """True when admitted, False when the budget or the slots are full."""
    st = _lib.lbib_server_admit(srv, h, int(n_steps), int(tag))
    if st == LBIB_ERR_NOMEM:
        return False
    if st != LBIB_OK:
        raise LbibError(st, _lib.lbib_last_error(h).decode() if st != LBIB_ERR_ARG else "lbib_server_admit")
    return True


def lbib_server_advance(srv, cap=1024):
    done = np.zeros(max(1, cap), np.int64)
    n = C.c_int(0)
    st = _lib.lbib_server_advance(srv, _p(done), int(cap), C.byref(n))
    if st != LBIB_OK:
        raise LbibError(st, "lbib_server_advance")
    return [int(t) for t in done[:n.value]]


def lbib_server_stats(srv):
    out = np.zeros(4, np.int64)
    st = _lib.lbib_server_stats(srv, _p(out))
    if st != LBIB_OK:
        raise LbibError(st, "lbib_server_stats")
    return dict(resident=int(out[0]), resident_bytes=int(out[1]), advances=int(out[2]), updates=int(out[3]))


# ----------------------------------------------------------------- convenience

class Sim:
    """One simulation handle with the calls above as methods."""

    def __init__(self, nx, ny, nz, walls=True, tau=1.0, rho0=1.0, body_force=(0, 0, 0), friction=0.5,
                 precision="f32", pop_scale_log2=0, stream=None):
        self.params = fluid_params(nx, ny, nz, walls, tau, rho0, body_force, friction, precision, pop_scale_log2)
        self.h = lbib_create(self.params, stream)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.walls = bool(walls)
        self.n_nodes = []
        self.n_tris = []
        self.obj_tid = []

    @classmethod
    def from_scene(cls, scene, precision="f32", pop_scale_log2=0, stream=None, init=True):
        s = cls(scene.nx, scene.ny, scene.nz, scene.walls, scene.tau, scene.rho0, scene.body_force,
                scene.friction, precision, pop_scale_log2, stream)
        for t in scene.templates:
            s.template_create(t.nodes, t.tris, t.stretch, t.ks, t.kb, t.kal, t.kag, t.kv, t.nonlinear)
        for o in scene.objects:
            oid = s.object_add(o.tid, o.origin, o.rotate, o.mass)
            if any(o.force):
                s.object_set_force(oid, o.force)
        rep = getattr(scene, "repulsion", None)
        if rep is not None:
            lbib_set_repulsion(s.h, *rep)
        inlet = getattr(scene, "inlet", None)
        if inlet is not None:
            lbib_set_inlet(s.h, *inlet)
        solid = getattr(scene, "solid", None)
        if solid is not None:
            lbib_set_solid(s.h, solid)
        if init:
            s.fluid_init()
        return s

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lbib_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def total_nodes(self):
        return sum(self.n_nodes[t] for t in self.obj_tid)

    def template_create(self, nodes, tris, stretch=(1, 1, 1), ks=0.0, kb=0.0, kal=0.0, kag=0.0, kv=0.0,
                        nonlinear=1):
        tid = len(self.n_nodes)
        lbib_template_create(self.h, tid, nodes, tris, stretch, ks, kb, kal, kag, kv, nonlinear)
        self.n_nodes.append(len(nodes))
        self.n_tris.append(len(tris))
        return tid

    def topology(self, tid):
        return lbib_template_topology(self.h, tid, self.n_tris[tid])

    def object_add(self, tid, origin, rotate=(0, 0, 0), mass=1.0):
        oid = len(self.obj_tid)
        lbib_object_add(self.h, oid, tid, origin, rotate, mass)
        self.obj_tid.append(tid)
        return oid

    def object_set_force(self, oid, f):
        lbib_object_set_force(self.h, oid, f)

    def object_set_nodes(self, oid, xyz):
        lbib_object_set_nodes(self.h, oid, xyz)

    def object_set_velocities(self, oid, v):
        lbib_object_set_velocities(self.h, oid, v)

    def fluid_init(self):
        lbib_fluid_init(self.h)

    def step(self, n=1):
        lbib_step(self.h, n)

    def sync(self):
        lbib_sync(self.h)

    def read_nodes(self, oid=-1):
        n = self.total_nodes if oid < 0 else self.n_nodes[self.obj_tid[oid]]
        return lbib_read_nodes(self.h, oid, n)

    def velocity(self):
        return lbib_read_velocity(self.h, self.nx, self.ny, self.nz)

    def density(self):
        return lbib_read_density(self.h, self.nx, self.ny, self.nz)

    def coupling_force(self):
        return lbib_read_coupling_force(self.h, self.nx, self.ny, self.nz)

    def set_coupling_force(self, g):
        lbib_set_coupling_force(self.h, g)

    def populations(self):
        return lbib_read_populations(self.h, self.nx, self.ny, self.nz)

    def set_populations(self, hpop):
        lbib_set_populations(self.h, hpop)

    def analyze(self, oid):
        return lbib_object_analyze(self.h, oid)

    def mass(self):
        return lbib_fluid_mass(self.h)

    def objects_set_force(self, f):
        lbib_objects_set_force(self.h, f)

    def objects_analyze(self, out=None):
        return lbib_objects_analyze(self.h, len(self.obj_tid), out)

    def info(self):
        return lbib_info(self.h)

    def dropped(self):
        return lbib_dropped_momentum(self.h)
