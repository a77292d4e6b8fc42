import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def homogeneous(o, lam=1.6e8, mu=0.8e8):
    shape = o.mat_shape()
    return np.full(shape, lam), np.full(shape, mu)


def node_coords(o):
    """(x, y, z) of every node, in m, z positive downwards, origin at node (0,0,0)."""
    n = np.arange(o.nnode)
    i = n % o.nn[0]
    j = (n // o.nn[0]) % o.nn[1]
    k = n // (o.nn[0] * o.nn[1])
    return i * 0.5 * o.h, j * 0.5 * o.h, k * 0.5 * o.h


def node_classes(o):
    """Boolean masks over the oracle's nodes for the four node sets the CUDA stage kernels
    split a stage into: 'interior' (every element around the node is interior), 'shell'
    (interior and PML elements), 'face' (PML only, on an outer face of the grid: the fixed
    faces, and the free top outside the interior) and 'deep' (PML only, elsewhere)."""
    n = np.arange(o.nnode)
    c = (n % o.nn[0], (n // o.nn[0]) % o.nn[1], n // (o.nn[0] * o.nn[1]))
    touch_int = np.zeros(o.nnode, bool)
    touch_pml = np.zeros(o.nnode, bool)
    for dx in (-1, 0):
        for dy in (-1, 0):
            for dz in (-1, 0):
                e, ok = [], np.ones(o.nnode, bool)
                for a, d in enumerate((dx, dy, dz)):
                    # element index along axis a on side d of the node (an odd coordinate
                    # lies inside one element: both sides are that element)
                    ea = np.where(c[a] % 2 == 1, (c[a] - 1) // 2, c[a] // 2 + d)
                    ok &= (ea >= 0) & (ea < o.N[a])
                    e.append(ea)
                inside = ok.copy()
                for a in range(3):
                    inside &= (e[a] >= o.lo[a]) & (e[a] < o.hi[a])
                touch_int |= inside
                touch_pml |= ok & ~inside
    outer = (c[0] == 0) | (c[0] == o.nn[0] - 1) | (c[1] == 0) | (c[1] == o.nn[1] - 1) | (c[2] == o.nn[2] - 1) | (c[2] == 0)
    pml_only = touch_pml & ~touch_int
    return {"interior": touch_int & ~touch_pml, "shell": touch_int & touch_pml,
            "face": pml_only & outer, "deep": pml_only & ~outer}
