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
