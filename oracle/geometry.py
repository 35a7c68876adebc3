"""Oracle: plane-wave spheres, k/q meshes and e-h pair bookkeeping (step A0).

Test infrastructure only (see package docstring).

Definitions followed:
- k and q meshes are Gamma-centred and share one form; a k-point difference
  k' - k is folded back onto the q mesh with a reciprocal lattice vector G0
  (Sec. III A: the q mesh is the k mesh of differences, always containing
  Gamma; q = T q_IBZ + G0 with T = identity).
- Plane-wave spheres: |k+G|^2/2 <= Ecut for wavefunctions and |q+G|^2/2 <= Ecut
  for pair densities and W (Sec. II C, plane-wave representation).
- Canonical order inside a sphere: ascending exact key, then g1, g2, g3.  The
  key is an integer for the fcc lattice (Gram matrix of the reciprocal basis in
  units of (2 pi/a)^2, times nk^2) and a double evaluated in a fixed order for
  the hexagonal sheet.
- e-h pair index S = (ik*Nv + iv)*Nc + ic (basis psi_S of Eq. bse_eig).

Pinned by tests/test_oracle_geometry.py (closed-form shell counts, symmetry
of the spheres under G -> -G, agreement with the input generator's layout).
"""
from __future__ import annotations

import math

import numpy as np

PI = 3.141592653589793

# integer Gram matrix of the fcc reciprocal basis b_i = (2 pi/a)(-1,1,1),(1,-1,1),(1,1,-1)
_FCC_GRAM = ((3, -1, -1), (-1, 3, -1), (-1, -1, 3))


def cell_volume(spec) -> float:
    if spec.lattice == "fcc":
        return spec.a ** 3 / 4.0
    return spec.a * spec.a * math.sqrt(3.0) / 2.0 * spec.c


def reciprocal_basis(spec) -> np.ndarray:
    """Rows b_1, b_2, b_3 (bohr^-1) written out for the two lattices used."""
    if spec.lattice == "fcc":
        s = 2.0 * PI / spec.a
        return s * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])
    s = 2.0 * PI / spec.a
    return np.array([[s, s / math.sqrt(3.0), 0.0], [0.0, 2.0 * s / math.sqrt(3.0), 0.0],
                     [0.0, 0.0, 2.0 * PI / spec.c]])


def mesh_offsets(spec) -> np.ndarray:
    n1, n2, n3 = spec.nk
    out = np.zeros((n1 * n2 * n3, 3), dtype=np.int64)
    for i1 in range(n1):
        for i2 in range(n2):
            for i3 in range(n3):
                out[(i1 * n2 + i2) * n3 + i3] = (i1, i2, i3)
    return out


def mesh_index(spec, off) -> int:
    n1, n2, n3 = spec.nk
    return (int(off[0]) * n2 + int(off[1])) * n3 + int(off[2])


def fold(spec, i_from, i_to):
    """q index and G0 with (k_to - k_from) = q + G0, q on the Gamma-centred mesh."""
    n = np.asarray(spec.nk, dtype=np.int64)
    d = np.asarray(i_to, dtype=np.int64) - np.asarray(i_from, dtype=np.int64)
    iq = np.mod(d, n)
    g0 = (d - iq) // n
    return mesh_index(spec, iq), iq, g0


def _sphere_key(spec, g, off):
    n = spec.nk[0]
    if spec.lattice == "fcc":
        x = [n * int(g[j]) + int(off[j]) for j in range(3)]
        q = 0
        for i in range(3):
            for j in range(3):
                q += _FCC_GRAM[i][j] * x[i] * x[j]
        t = spec.a / (2.0 * PI)
        rhs = 2.0 * spec.ecut * (t * t) * float(n * n)
        return float(q), float(q) <= rhs
    x1 = n * int(g[0]) + int(off[0])
    x2 = n * int(g[1]) + int(off[1])
    s = 2.0 * PI / spec.a
    u = 2.0 * PI / spec.c
    c1 = (4.0 / 3.0) * (s * s)
    c3 = u * u
    z = float(n * int(g[2]))
    key = c1 * float(x1 * x1 + x1 * x2 + x2 * x2) + c3 * (z * z)
    return key, key <= 2.0 * spec.ecut * float(n * n)


def _bound(spec, j):
    """Largest |g_j| that can lie inside any sphere: |g_j| <= |p| |a_j| / (2 pi) + 1."""
    if spec.lattice == "fcc":
        alen = spec.a / math.sqrt(2.0)
    else:
        alen = spec.a if j < 2 else spec.c
    return int(math.sqrt(2.0 * spec.ecut) * alen / (2.0 * PI)) + 2


_cache: dict = {}


def sphere(spec, off) -> np.ndarray:
    """Sorted G list (int64 [n,3]) with |off/nk + G|^2/2 <= ecut (scalar loops, exact keys)."""
    ck = (spec.lattice, spec.a, spec.c, spec.nk, spec.ecut, tuple(int(o) for o in off))
    if ck in _cache:
        return _cache[ck]
    rows = []
    b = [_bound(spec, j) for j in range(3)]
    for g1 in range(-b[0], b[0] + 1):
        for g2 in range(-b[1], b[1] + 1):
            for g3 in range(-b[2], b[2] + 1):
                key, inside = _sphere_key(spec, (g1, g2, g3), off)
                if inside:
                    rows.append((key, g1, g2, g3))
    rows.sort()
    out = np.array([r[1:] for r in rows], dtype=np.int64).reshape(-1, 3)
    _cache[ck] = out
    return out


def cart(spec, off, g) -> np.ndarray:
    """Cartesian k+G (bohr^-1) for mesh offset off and reduced G rows g."""
    red = np.asarray(g, dtype=np.float64) + np.asarray(off, dtype=np.float64) / np.asarray(spec.nk, dtype=np.float64)
    return red @ reciprocal_basis(spec)


def pair_index(spec, ik, iv, ic) -> int:
    return (ik * spec.nv + iv) * spec.nc + ic


def upper_blocks(spec) -> list:
    """(ik, ik') with ik <= ik', row-major: the blocks the direct term is evaluated on."""
    nk = spec.nkpt
    return [(i, j) for i in range(nk) for j in range(i, nk)]
