"""The evaluation order of the membrane elements (csrc/topology.cpp), on the
host: a permutation of the elements in which the 32 elements a warp takes
together touch distinct nodes where the mesh is large enough, and whose staged
position loads (16 bytes per node, 8 lanes per shared-memory wavefront) and
force atomics (32 banks) meet fewer bank conflicts than the mesh's own
order or a plain disjoint-nodes packing.  The order changes no result beyond
the order of FP32 additions; this pins what it is for."""
import os
import subprocess

import numpy as np
import pytest

from paper_1312_3426_gb300 import lbib
from workloads import mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1312_3426_gb300", "csrc")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("topology_order") / "topology_order")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Werror", "-I", CSRC, os.path.join(HERE, "topology_order.cpp"),
                    os.path.join(CSRC, "topology.cpp"), "-o", exe], check=True)
    return exe


def order_of(driver, elems):
    elems = np.asarray(elems, np.int64)
    text = f"{elems.shape[1]} {elems.shape[0]}\n" + " ".join(map(str, elems.reshape(-1)))
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout
    return np.array(out.split(), np.int64)


def disjoint_packing(elems, width=32):
    """The plain greedy: fill each group with the next elements whose nodes
    are not yet in it."""
    remaining, order = list(range(len(elems))), []
    while remaining:
        used, rest = set(), []
        for e in remaining:
            if len(order) % width < width and not used & set(elems[e]) and \
                    len(used) // elems.shape[1] < width:
                used |= set(elems[e])
                order.append(e)
            else:
                rest.append(e)
        remaining = rest
    return np.array(order)


def wavefronts(elems, order, width=32):
    """Shared-memory wavefronts of the position loads (per slot, per 8-lane
    phase: the largest count of distinct nodes sharing a 16-byte bank group)
    and of the force atomics (per slot: the largest count sharing a bank)."""
    ld = at = 0
    for g0 in range(0, len(order), width):
        grp = elems[order[g0:g0 + width]]
        for k in range(elems.shape[1]):
            p = grp[:, k]
            for q0 in range(0, len(p), 8):
                ld += np.bincount(np.unique(p[q0:q0 + 8]) % 8, minlength=8).max()
            at += np.bincount(p % 32, minlength=32).max()
    return ld, at


def meshes():
    for level in (2, 3, 4):
        yield f"icosphere{level}", mesh.icosphere(level)
    yield "biconcave3", mesh.biconcave(3)


@pytest.mark.parametrize("name,m", list(meshes()))
def test_element_order_is_a_permutation_with_fewer_bank_conflicts(driver, name, m):
    nodes, tris = m
    topo = lbib.lbib_mesh_check(nodes, tris)
    for elems in (np.asarray(topo["quads"]).reshape(-1, 4), np.asarray(tris).reshape(-1, 3)):
        order = order_of(driver, elems)
        assert np.array_equal(np.sort(order), np.arange(len(elems)))
        # full groups touch distinct nodes
        full = 0
        for g0 in range(0, len(order) - 31, 32):
            grp = elems[order[g0:g0 + 32]].reshape(-1)
            full += len(np.unique(grp)) == grp.size
        if len(nodes) >= 4 * 32 * elems.shape[1]:  # small meshes cannot fill a group with distinct nodes
            assert full >= 0.9 * (len(order) // 32), (name, full)
        ld, at = wavefronts(elems, order)
        ld0, at0 = wavefronts(elems, np.arange(len(elems)))
        ld1, at1 = wavefronts(elems, disjoint_packing(elems))
        print(f"\n{name} arity {elems.shape[1]}: loads {ld} (mesh order {ld0}, disjoint {ld1}), "
              f"atomics {at} (mesh order {at0}, disjoint {at1})")
        assert ld < min(ld0, 0.9 * ld1) and at < 0.8 * min(at0, at1)
