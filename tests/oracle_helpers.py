"""Small helpers shared by the oracle tests (no method arithmetic here)."""
import numpy as np


def global_node_coords(mesh, eta, h):
    """Physical (x, y, z) at every global node, taken from the oracle's
    element-local coordinates (the first element writing a node wins)."""
    xe, ye, ze = mesh.element_coords(eta, h)
    x = np.zeros(mesh.N)
    y = np.zeros(mesh.N)
    z = np.zeros(mesh.N)
    g = mesh.glob.ravel()[::-1]
    x[g] = xe.ravel()[::-1]
    y[g] = ye.ravel()[::-1]
    z[g] = ze.ravel()[::-1]
    return x, y, z
