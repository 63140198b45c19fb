"""DFT symbols of the P1 operators on the torus (test helper).

On the m x m torus with mesh width h the lumped mass is h^2, the P1
stiffness is the 5-point stencil (4; -1 at the axis neighbours; the diagonal
couplings vanish on right triangles), with symbol
s(w) = 4 sin^2(w_x / 2) + 4 sin^2(w_y / 2), and the x-advection matrix
int phi_i c d/dx phi_j is the antisymmetric stencil (c h / 6)[x+1: 2,
x-1: -2, (+1,+1): 1, (-1,-1): -1, y+1: -1, y-1: 1], with symbol
i (c h / 3)(2 sin w_x + sin(w_x + w_y) - sin w_y).  So the root
B = tau h^-1 (kappa^2 h^2 + nu S + c Bx) has the symbol returned by
`symbol`, and Q = B^T B has |b(w)|^2.  Written from the element integrals by
hand, independently of the oracle's element loops and of the library.
"""
import numpy as np


def symbol(pr):
    """(b, m): the symbol of B on the [m, m] frequency grid (array index
    [k_y, k_x], matching the node index j * m + i) and the torus size."""
    m = pr["n"][0] - 1
    h = (pr["hi"][0] - pr["lo"][0]) / m
    w = 2.0 * np.pi * np.fft.fftfreq(m)
    wy, wx = np.meshgrid(w, w, indexing="ij")
    s = 4.0 * np.sin(wx / 2) ** 2 + 4.0 * np.sin(wy / 2) ** 2
    nu = 1.0 if pr["kind"] == "matern2d" else pr["nu"]
    c = 0.0 if pr["kind"] == "matern2d" else pr["cx"]
    adv = 1j * (c * h / 3.0) * (2.0 * np.sin(wx) + np.sin(wx + wy) - np.sin(wy))
    return (pr["tau"] / h) * (pr["kappa"] ** 2 * h * h + nu * s + adv), m


def apply_symbol(sym, v, m):
    """(C v) for the circulant C with (C v)_n = sum_d c_d v_(n+d), given its
    symbol sum_d c_d exp(i w.d): in numpy's DFT convention a shift by +d
    multiplies the transform by exp(+i w.d)."""
    V = np.fft.fft2(v.reshape(m, m))
    return np.real(np.fft.ifft2(sym * V)).ravel()


def all_nodes_mean(pr, y, sigma):
    """Posterior mean with every torus node observed once with noise sigma:
    Q_u|y = Q + sigma^-2 I is circulant, mu = (|b|^2 + sigma^-2)^-1 sigma^-2 y."""
    b, m = symbol(pr)
    rinv = 1.0 / sigma ** 2
    Y = np.fft.fft2((rinv * np.asarray(y)).reshape(m, m))
    return np.real(np.fft.ifft2(Y / (np.abs(b) ** 2 + rinv))).ravel()
