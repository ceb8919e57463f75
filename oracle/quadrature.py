"""Quadrature rules of the fast spectral method (Sec. 4).

* Radial direction: Gauss-Legendre with N_rho points on [0, R] (Sec. 4, the
  quadrature approximation of Eq. GG).
* Sphere: an M-point spherical design with equal weights 4*pi/M (Sec. 4).  The paper
  takes Womersley's designs; their point files are not available here, so the built-in
  designs are the Platonic-solid designs listed below, in the orientation written here:

  - M = 6  : octahedron vertices +-e_d (a spherical 3-design),
  - M = 12 : icosahedron vertices (0, +-1, +-phi) and cyclic permutations (5-design),
  - M = 32 : icosahedron U dodecahedron vertices, equal weights (5-design).
"""

import numpy as np

GOLDEN = (1.0 + np.sqrt(5.0)) / 2.0


def gauss_legendre_radial(n, R):
    """Gauss-Legendre nodes and weights on [0, R] (Sec. 4, radial rule)."""
    x, w = np.polynomial.legendre.leggauss(int(n))
    rho = 0.5 * R * (x + 1.0)
    return rho, 0.5 * R * w


def _normalise(p):
    p = np.asarray(p, dtype=np.float64)
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def octahedron():
    pts = []
    for d in range(3):
        for s in (1.0, -1.0):
            e = [0.0, 0.0, 0.0]
            e[d] = s
            pts.append(e)
    return _normalise(pts)


def icosahedron():
    pts = []
    for a in (1.0, -1.0):
        for b in (GOLDEN, -GOLDEN):
            pts.append([0.0, a, b])
            pts.append([a, b, 0.0])
            pts.append([b, 0.0, a])
    return _normalise(pts)


def dodecahedron():
    pts = []
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            for c in (1.0, -1.0):
                pts.append([a, b, c])
    ig = 1.0 / GOLDEN
    for a in (ig, -ig):
        for b in (GOLDEN, -GOLDEN):
            pts.append([0.0, a, b])
            pts.append([a, b, 0.0])
            pts.append([b, 0.0, a])
    return _normalise(pts)


def spherical_design(M):
    """Built-in M-point design with equal weights 4*pi/M (Sec. 4)."""
    if M == 6:
        pts = octahedron()
    elif M == 12:
        pts = icosahedron()
    elif M == 32:
        pts = np.concatenate([icosahedron(), dodecahedron()], axis=0)
    else:
        raise ValueError("no built-in spherical design with M=%d (use 6, 12 or 32)" % M)
    w = np.full(len(pts), 4.0 * np.pi / len(pts))
    return pts, w
