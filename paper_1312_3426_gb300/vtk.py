"""VTK output of object meshes (Sec. 5, visualization and data output: the
mesh of an object written as a legacy-format VTK file that visualisation
tools such as ParaView read).  Host-side only."""
from __future__ import annotations

import numpy as np


def write_vtk(path, nodes, tris, point_data=None):
    """Writes an ASCII legacy VTK POLYDATA file: nodes [n][3], triangles
    [m][3] (node ids from 0), optional point_data {name: [n] or [n][3]}."""
    X = np.asarray(nodes, dtype=np.float64).reshape(-1, 3)
    T = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    with open(path, "w") as f:
        f.write("# vtk DataFile Version 3.0\nlbib object mesh\nASCII\nDATASET POLYDATA\n")
        f.write(f"POINTS {len(X)} double\n")
        for p in X:
            f.write(f"{p[0]:.17g} {p[1]:.17g} {p[2]:.17g}\n")
        f.write(f"POLYGONS {len(T)} {4 * len(T)}\n")
        for t in T:
            f.write(f"3 {t[0]} {t[1]} {t[2]}\n")
        if point_data:
            f.write(f"POINT_DATA {len(X)}\n")
            for name, val in point_data.items():
                v = np.asarray(val, dtype=np.float64)
                if v.ndim == 2:
                    f.write(f"VECTORS {name} double\n")
                    for r in v:
                        f.write(f"{r[0]:.17g} {r[1]:.17g} {r[2]:.17g}\n")
                else:
                    f.write(f"SCALARS {name} double 1\nLOOKUP_TABLE default\n")
                    for r in v:
                        f.write(f"{r:.17g}\n")


def read_vtk(path):
    """Reads back the points and triangles of a file written by write_vtk."""
    with open(path) as f:
        tok = f.read().split("\n")
    i = tok.index(next(t for t in tok if t.startswith("POINTS")))
    n = int(tok[i].split()[1])
    X = np.array([[float(v) for v in tok[i + 1 + k].split()] for k in range(n)])
    j = tok.index(next(t for t in tok if t.startswith("POLYGONS")))
    m = int(tok[j].split()[1])
    T = np.array([[int(v) for v in tok[j + 1 + k].split()[1:]] for k in range(m)])
    return X, T
