"""Synthetic BSE systems: lattices, plane-wave coefficients, energies and model W.

Everything here is input construction, seeded through ``numpy.random.default_rng``
and drawn in a fixed, documented order, so the CUDA path and the oracle see the
same numbers.  Units are Hartree atomic units (bohr, Ha).

Workload shapes follow the paper's BSE calculations: 8x8x8 and 12x12x12 k
meshes with three or four valence and conduction bands (Sec. IV C), and 2D
hexagonal sheets on dense in-plane meshes with a truncated Coulomb interaction
(Sec. V).  Real-material DFT inputs do not exist here; random orthonormal
plane-wave states, random band energies and a model inverse dielectric matrix
stand in for them.

Plane-wave spheres are enumerated here only to lay out the coefficients and W
in the canonical order (sorted by |k+G|^2 key, then g1, g2, g3); the oracle and
the CUDA host planner each enumerate them independently and the tests check
that all three agree bit for bit.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np

HARTREE_EV = 27.211386245988
PI = 3.141592653589793
EV = 1.0 / HARTREE_EV


@dataclass(frozen=True)
class SystemSpec:
    name: str
    lattice: str              # "fcc" (conventional cubic constant a) or "hex" (a, c)
    a: float                  # bohr
    c: float                  # bohr, hex out-of-plane period (ignored for fcc)
    nk: tuple                 # Gamma-centred k mesh (n1, n2, n3)
    nv: int
    nc: int
    ecut: float               # Ha, for |k+G|^2/2 and |q+G|^2/2
    fft: tuple                # real-space grid (N1, N2, N3)
    coulomb: str              # "3d" or "slab"
    eps_inf: float = 11.0     # bulk model screening
    r0: float = 0.0           # slab model screening length (bohr)
    delta: float = 0.8 * EV   # scissor shift (Ha)
    eta: float = 0.1 * EV     # Lorentzian broadening (Ha)
    nsteps: int = 100         # Haydock steps
    nw: int = 1000            # frequency points
    omega_max: float = 10.0 * EV
    seed: int = 0
    eg: float = 0.0           # slab: gap of the drawn conduction window (Ha)
    dirac: bool = False       # slab: Dirac-like top valence / bottom conduction pair
    ev_range: tuple = (-6.0 * EV, 0.0)
    ec_range: tuple = (1.5 * EV, 10.0 * EV)
    w_offdiag: float = 0.02   # scale of the random off-diagonal part of the model eps^-1
    symmetric: bool = False   # states and energies carry the point group of the lattice (see below)

    @property
    def nb(self):
        return self.nv + self.nc

    @property
    def nkpt(self):
        return self.nk[0] * self.nk[1] * self.nk[2]

    @property
    def dim(self):
        return self.nkpt * self.nv * self.nc

    def replace(self, **kw):
        return dataclasses.replace(self, **kw)


def config_spec(name: str) -> SystemSpec:
    """Named bulk workloads.

    fcc_4x4x4_3v3c    : dim 576,   ~97 G (max 113), grid 24^3, 100 steps, 1000 w, eta 0.1 eV
    fcc_8x8x8_3v4c    : dim 6144,  ~301 G (max 314), grid 32^3, 300 steps, 2000 w, eta 0.05 eV
    fcc_12x12x12_4v4c : dim 27648, ~496 G (max 531), grid 48^3, 300 steps, 2000 w, eta 0.05 eV
    """
    if name == "fcc_4x4x4_3v3c":
        return SystemSpec(name, "fcc", 10.0, 0.0, (4, 4, 4), 3, 3, 4.0, (24, 24, 24), "3d",
                          eps_inf=11.0, eta=0.1 * EV, nsteps=100, nw=1000)
    if name == "fcc_8x8x8_3v4c":
        return SystemSpec(name, "fcc", 10.0, 0.0, (8, 8, 8), 3, 4, 8.6, (32, 32, 32), "3d",
                          eps_inf=11.0, eta=0.05 * EV, nsteps=300, nw=2000)
    if name == "fcc_12x12x12_4v4c":
        return SystemSpec(name, "fcc", 10.0, 0.0, (12, 12, 12), 4, 4, 12.0, (48, 48, 48), "3d",
                          eps_inf=11.0, eta=0.05 * EV, nsteps=300, nw=2000)
    raise KeyError(name)


def omega_grid(spec: SystemSpec) -> np.ndarray:
    """Inclusive linear frequency grid 0..omega_max with nw points (Ha)."""
    return np.linspace(0.0, spec.omega_max, spec.nw)


# --------------------------------------------------------------------------
# lattice geometry (input layout only)
# --------------------------------------------------------------------------

def real_lattice(spec: SystemSpec) -> np.ndarray:
    """Rows are a_1, a_2, a_3 in bohr."""
    a = spec.a
    if spec.lattice == "fcc":
        return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    if spec.lattice == "hex":
        return np.array([[a, 0.0, 0.0], [-0.5 * a, 0.5 * np.sqrt(3.0) * a, 0.0], [0.0, 0.0, spec.c]])
    raise ValueError(spec.lattice)


def recip_lattice(spec: SystemSpec) -> np.ndarray:
    """Rows are b_1, b_2, b_3 with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * PI * np.linalg.inv(real_lattice(spec)).T


def _box(spec: SystemSpec) -> list:
    amat = real_lattice(spec)
    r = np.sqrt(2.0 * spec.ecut)
    out = []
    for j in range(3):
        m = int(np.ceil(r * np.linalg.norm(amat[j]) / (2.0 * PI))) + 2
        out.append(np.arange(-m, m + 1))
    return out


def _keys(spec: SystemSpec, g: np.ndarray, off: tuple):
    """Integer/float sphere key for k (or q) = off/nk and G = g (reduced)."""
    n = spec.nk
    if spec.lattice == "fcc":
        assert n[0] == n[1] == n[2]
        nn = n[0]
        x = nn * g + np.asarray(off, dtype=np.int64)[None, :]
        q = (3 * x[:, 0] * x[:, 0] + 3 * x[:, 1] * x[:, 1] + 3 * x[:, 2] * x[:, 2]
             - 2 * x[:, 0] * x[:, 1] - 2 * x[:, 0] * x[:, 2] - 2 * x[:, 1] * x[:, 2])
        t = spec.a / (2.0 * PI)
        rhs = 2.0 * spec.ecut * (t * t) * float(nn * nn)
        keyf = q.astype(np.float64)
        p2 = keyf * ((2.0 * PI / spec.a) ** 2) / float(nn * nn)
        return keyf, keyf <= rhs, p2
    if spec.lattice == "hex":
        assert n[0] == n[1] and n[2] == 1
        nn = n[0]
        x1 = nn * g[:, 0] + off[0]
        x2 = nn * g[:, 1] + off[1]
        qpar = (x1 * x1 + x1 * x2 + x2 * x2).astype(np.float64)
        s = 2.0 * PI / spec.a
        u = 2.0 * PI / spec.c
        c1 = (4.0 / 3.0) * (s * s)
        c3 = u * u
        z = (nn * g[:, 2]).astype(np.float64)
        keyf = c1 * qpar + c3 * (z * z)
        rhs = 2.0 * spec.ecut * float(nn * nn)
        return keyf, keyf <= rhs, keyf / float(nn * nn)
    raise ValueError(spec.lattice)


def sphere(spec: SystemSpec, off: tuple):
    """G vectors (int32 [n,3]) with |off/nk + G|^2/2 <= ecut in canonical order, and |p|^2."""
    b = _box(spec)
    g = np.stack(np.meshgrid(*b, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.int64)
    keyf, inside, p2 = _keys(spec, g, off)
    g, keyf, p2 = g[inside], keyf[inside], p2[inside]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], keyf))
    return g[order].astype(np.int32), p2[order]


def kpoint_offsets(spec: SystemSpec) -> np.ndarray:
    """Integer k (and q) offsets i with k_red = i / nk, ik = (i1*n2 + i2)*n3 + i3."""
    n1, n2, n3 = spec.nk
    i = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), axis=-1)
    return i.reshape(-1, 3)


def _cart(spec: SystemSpec, off: tuple, g: np.ndarray) -> np.ndarray:
    bm = recip_lattice(spec)
    red = g.astype(np.float64) + np.asarray(off, dtype=np.float64)[None, :] / np.asarray(spec.nk, dtype=np.float64)
    return red @ bm


# --------------------------------------------------------------------------
# the generated system
# --------------------------------------------------------------------------

@dataclass
class BulkSystem:
    spec: SystemSpec
    kred: np.ndarray          # [Nk,3] int offsets
    gk: list                  # per k: int32 [npw_k,3]
    npw: np.ndarray           # [Nk]
    coef: np.ndarray          # complex [Nk][Nb][NPWmax], zero padded, orthonormal rows on npw_k
    energies: np.ndarray      # float64 [Nk][Nb] (Ha), valence ascending then conduction ascending
    gq: list                  # per q: int32 [ng_q,3]
    ngq: np.ndarray           # [Nq]
    W: np.ndarray             # complex [Nq][NGmax][NGmax], zero padded
    omega: np.ndarray         # [nw] Ha

    @property
    def npwmax(self):
        return int(self.coef.shape[2])

    @property
    def ngmax(self):
        return int(self.W.shape[1]) if self.W is not None else int(self.ngq.max())


def _coefficients(spec: SystemSpec, rng, kred):
    gk, npw, cols = [], [], []
    for ik in range(len(kred)):
        g, p2 = sphere(spec, tuple(kred[ik]))
        gk.append(g)
        npw.append(len(g))
        z = (rng.standard_normal((len(g), spec.nb)) + 1j * rng.standard_normal((len(g), spec.nb))) / np.sqrt(2.0)
        z *= np.exp(-p2 / 8.0)[:, None]
        qm, rm = np.linalg.qr(z)
        d = np.diag(rm)
        qm = qm * (d / np.abs(d))[None, :]
        cols.append(qm.T.copy())
    npw = np.array(npw, dtype=np.int64)
    coef = np.zeros((len(kred), spec.nb, npw.max()), dtype=np.complex128)
    for ik, c in enumerate(cols):
        coef[ik, :, : c.shape[1]] = c
    return gk, npw, coef


def _energies(spec: SystemSpec, rng, nkpt):
    e = np.zeros((nkpt, spec.nb))
    for ik in range(nkpt):
        e[ik, : spec.nv] = np.sort(rng.uniform(spec.ev_range[0], spec.ev_range[1], spec.nv))
        e[ik, spec.nv:] = np.sort(rng.uniform(spec.ec_range[0], spec.ec_range[1], spec.nc))
    return e


def _gl_head_slab(spec: SystemSpec, qc: float) -> float:
    """Disc average of the truncated, screened 2D Coulomb head (64-point Gauss-Legendre)."""
    x, w = np.polynomial.legendre.leggauss(64)
    q = 0.5 * qc * (x + 1.0)
    zc = 0.5 * spec.c
    f = 2.0 * PI * q * (4.0 * PI * (1.0 - np.exp(-q * zc)) / (q * q)) / (1.0 + spec.r0 * q)
    return float(0.5 * qc * np.sum(w * f) / (PI * qc * qc))


def _w_model(spec: SystemSpec, rng, kred, wdtype):
    """Model W_GG'(q) = v^1/2(q+G) eps^-1_GG'(q) v^1/2(q+G') on every q of the mesh.

    eps^-1 = diag(d) + B with B Hermitian, zero diagonal, 0.02*sqrt(d d') h / sqrt(NG);
    reciprocity W_GG'(q) = conj(W_{-G-G0',-G'-G0'}(qbar)) (qbar = fold(-q)) is imposed by
    drawing h only for q <= qbar (linear index) and symmetrising self-partner q.
    """
    n = np.asarray(spec.nk)
    nq = len(kred)
    gq, p2q, ngq = [], [], []
    for iq in range(nq):
        g, p2 = sphere(spec, tuple(kred[iq]))
        gq.append(g)
        p2q.append(p2)
        ngq.append(len(g))
    ngq = np.array(ngq, dtype=np.int64)
    ngmax = int(ngq.max())
    W = np.zeros((nq, ngmax, ngmax), dtype=wdtype)

    def lin(i):
        return (int(i[0]) * n[1] + int(i[1])) * n[2] + int(i[2])

    def keyof(g):
        g = g.astype(np.int64) + 64
        return (g[:, 0] * 128 + g[:, 1]) * 128 + g[:, 2]

    keys = [keyof(g) for g in gq]
    orders = [np.argsort(k) for k in keys]

    def partner_index(iq, iqb, g0p):
        """Index in sphere(qbar) of G'' = G0' - G for each G of sphere(q)."""
        tgt = keyof(g0p[None, :] - gq[iq].astype(np.int64))
        kb, ob = keys[iqb], orders[iqb]
        pos = np.searchsorted(kb[ob], tgt)
        idx = ob[np.minimum(pos, len(ob) - 1)]
        assert np.all(kb[idx] == tgt), "reciprocal partner missing from sphere"
        return idx

    cell_area = abs(np.linalg.det(real_lattice(spec)[:2, :2]))
    omega_cell = abs(np.linalg.det(real_lattice(spec)))
    nkpt = nq
    B = [None] * nq
    for iq in range(nq):
        iqv = kred[iq]
        iqb_v = (-iqv) % n
        iqb = lin(iqb_v)
        if iq > iqb:
            continue
        g = gq[iq]
        ng = len(g)
        p2 = p2q[iq]
        if spec.coulomb == "3d":
            d = 1.0 - (1.0 - 1.0 / spec.eps_inf) * np.exp(-p2 / 4.0)
        else:
            ppar = _ppar(spec, iqv, g)
            d = 1.0 / (1.0 + spec.r0 * ppar)
        iu = np.triu_indices(ng, 1)
        draws = rng.standard_normal((len(iu[0]), 2)) * np.sqrt(0.5)
        h = np.zeros((ng, ng), dtype=np.complex128)
        h[iu] = draws[:, 0] + 1j * draws[:, 1]
        h = h + h.conj().T
        if iq == 0:
            h[0, :] = 0.0
            h[:, 0] = 0.0
        b = spec.w_offdiag * np.sqrt(np.outer(d, d)) * h / np.sqrt(ng)
        if iq == iqb:
            g0p = (-iqv - iqb_v) // n
            pi_ = partner_index(iq, iqb, g0p)
            b = 0.5 * (b + b.T[np.ix_(pi_, pi_)])
        B[iq] = (d, b)
    for iq in range(nq):
        iqv = kred[iq]
        iqb_v = (-iqv) % n
        iqb = lin(iqb_v)
        g = gq[iq]
        ng = len(g)
        if iq > iqb:
            g0p = (-iqv - iqb_v) // n
            pi_ = partner_index(iq, iqb, g0p)
            d_b, b_b = B[iqb]
            d = d_b[pi_]
            b = np.conj(b_b[np.ix_(pi_, pi_)])
        else:
            d, b = B[iq]
        eps = np.diag(d).astype(np.complex128) + b
        p2 = p2q[iq]
        if spec.coulomb == "3d":
            with np.errstate(divide="ignore"):
                vh = np.sqrt(4.0 * PI / p2)
        else:
            vh = np.sqrt(_v2d(spec, iqv, g, p2))
        if iq == 0:
            vh[0] = 0.0
        w = np.outer(vh, vh) * eps      # commutative product: exactly Hermitian and reciprocal
        if iq == 0:
            if spec.coulomb == "3d":
                qc = (6.0 * PI * PI / (omega_cell * nkpt)) ** (1.0 / 3.0)
                w[0, 0] = (1.0 / spec.eps_inf) * 12.0 * PI / (qc * qc)
            else:
                qc = np.sqrt(4.0 * PI / (cell_area * nkpt))
                w[0, 0] = _gl_head_slab(spec, qc)
        W[iq, :ng, :ng] = w.astype(wdtype)
    return gq, ngq, W


def _ppar(spec, off, g):
    """|(q+G)_parallel| for the hexagonal sheet (bohr^-1)."""
    nn = spec.nk[0]
    x1 = (nn * g[:, 0] + off[0]).astype(np.float64)
    x2 = (nn * g[:, 1] + off[1]).astype(np.float64)
    s = 2.0 * PI / spec.a
    return np.sqrt((4.0 / 3.0) * s * s * (x1 * x1 + x1 * x2 + x2 * x2)) / nn


def _v2d(spec, off, g, p2):
    """Slab-truncated Coulomb 4 pi/|p|^2 [1 - exp(-|p_par| zc) cos(p_z zc)], zc = c/2."""
    zc = 0.5 * spec.c
    ppar = _ppar(spec, off, g)
    pz = (2.0 * PI / spec.c) * g[:, 2].astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = 4.0 * PI / p2 * (1.0 - np.exp(-ppar * zc) * np.cos(pz * zc))
    return np.where(p2 > 0, v, 0.0)


# --------------------------------------------------------------------------
# symmetric systems: states and energies that carry the point group of the lattice
# --------------------------------------------------------------------------

def point_group(spec: SystemSpec) -> list:
    """Integer 3x3 matrices R acting on reduced reciprocal coordinates (k -> R k) that keep the reciprocal
    metric and map the k mesh onto itself, identity first, the others in ascending row-major order of
    their entries (all entries in {-1, 0, 1})."""
    bm = recip_lattice(spec)
    M = bm @ bm.T
    n = np.asarray(spec.nk)
    ops = []
    for code in range(3 ** 9):
        c = code
        e = np.zeros(9, dtype=np.int64)
        for t in range(8, -1, -1):
            e[t] = c % 3 - 1
            c //= 3
        R = e.reshape(3, 3)
        if abs(round(np.linalg.det(R))) != 1:
            continue
        if np.abs(R.T @ M @ R - M).max() > 1e-9 * np.abs(M).max():
            continue
        if np.any((R * n[:, None]) % n[None, :] != 0):
            continue
        ops.append(R)
    ident = np.eye(3, dtype=np.int64)
    return [ident] + [R for R in ops if not np.array_equal(R, ident)]


def _symmetric_states(spec: SystemSpec, rng, kred):
    """Coefficients and energies with psi_{Rk}(r) = psi_k(R^-1 r) for every operation R of the point group
    (no time reversal): c_{k'}(R G + G0) = c_k(G) where R k = k' + G0 on the mesh.  Random states are
    drawn at the first k of each orbit (ascending index), projected onto the invariants of its little group
    (the average over R with R k = k + G0 of c(R^-1 (G - G0))), orthonormalised (QR, diag(R) > 0: linear
    combinations of invariant columns stay invariant) and copied to the other points of the orbit by the
    first operation (in the order of point_group) that reaches them; energies are shared by the orbit."""
    n = np.asarray(spec.nk, dtype=np.int64)
    ops = point_group(spec)
    inv = [np.rint(np.linalg.inv(R)).astype(np.int64) for R in ops]
    nk = len(kred)

    def lin(i):
        return int((i[0] * n[1] + i[1]) * n[2] + i[2])

    rep, opi = [-1] * nk, [-1] * nk
    for ik in range(nk):
        if rep[ik] >= 0:
            continue
        for io, R in enumerate(ops):
            img = R @ kred[ik]
            j = lin(np.mod(img, n))
            if rep[j] < 0:
                rep[j], opi[j] = ik, io
    spheres = [sphere(spec, tuple(kred[ik])) for ik in range(nk)]

    def index_of(g):
        return {tuple(int(x) for x in v): t for t, v in enumerate(g)}

    cols, energies = {}, np.zeros((nk, spec.nb))
    for ik in range(nk):
        if rep[ik] != ik:
            continue
        g, p2 = spheres[ik]
        g = g.astype(np.int64)
        pos = index_of(g)
        z = (rng.standard_normal((len(g), spec.nb)) + 1j * rng.standard_normal((len(g), spec.nb))) / np.sqrt(2.0)
        z *= np.exp(-p2 / 8.0)[:, None]
        acc = np.zeros_like(z)
        cnt = 0
        for R, Ri in zip(ops, inv):
            img = R @ kred[ik]
            if np.any(np.mod(img, n) != kred[ik]):
                continue
            g0 = (img - kred[ik]) // n
            src = [pos[tuple(int(x) for x in Ri @ (v - g0))] for v in g]
            acc += z[src]
            cnt += 1
        z = acc / cnt
        qm, rm = np.linalg.qr(z)
        d = np.diag(rm)
        qm = qm * (d / np.abs(d))[None, :]
        cols[ik] = qm
        energies[ik, : spec.nv] = np.sort(rng.uniform(spec.ev_range[0], spec.ev_range[1], spec.nv))
        energies[ik, spec.nv:] = np.sort(rng.uniform(spec.ec_range[0], spec.ec_range[1], spec.nc))
    gk, npw = [], []
    coef = np.zeros((nk, spec.nb, max(len(sp[0]) for sp in spheres)), dtype=np.complex128)
    for ik in range(nk):
        r, R, Ri = rep[ik], ops[opi[ik]], inv[opi[ik]]
        g = spheres[ik][0].astype(np.int64)
        g0 = (R @ kred[r] - kred[ik]) // n
        pos = index_of(spheres[r][0].astype(np.int64))
        src = [pos[tuple(int(x) for x in Ri @ (v - g0))] for v in g]
        coef[ik, :, : len(g)] = cols[r][src].T
        energies[ik] = energies[r]
        gk.append(spheres[ik][0])
        npw.append(len(g))
    return gk, np.array(npw, dtype=np.int64), coef, energies


def generate(spec: SystemSpec, wdtype=np.complex128, with_w: bool = True) -> BulkSystem:
    """Draw one system.  Order: coefficients (k ascending), energies (k ascending), W (q ascending).
    A symmetric spec draws its states on the first point of every orbit of the point group (see
    _symmetric_states) and needs a model W without the random off-diagonal part (w_offdiag = 0), whose
    entries depend only on |q + G| and |q + G'| and so carry the point group too."""
    rng = np.random.default_rng(spec.seed if not isinstance(spec.seed, tuple) else list(spec.seed))
    kred = kpoint_offsets(spec)
    if spec.symmetric:
        if spec.w_offdiag != 0.0 or spec.dirac:
            raise ValueError("a symmetric system needs w_offdiag = 0 and no Dirac bands")
        gk, npw, coef, energies = _symmetric_states(spec, rng, kred)
    else:
        gk, npw, coef = _coefficients(spec, rng, kred)
        energies = _energies(spec, rng, len(kred))
    if spec.dirac:
        energies = _dirac_bands(spec, kred, energies)
    if with_w:
        gq, ngq, W = _w_model(spec, rng, kred, wdtype)
    else:
        gq = [sphere(spec, tuple(kred[iq]))[0] for iq in range(len(kred))]
        ngq = np.array([len(g) for g in gq], dtype=np.int64)
        W = None
    return BulkSystem(spec, kred, gk, npw, coef, energies, gq, ngq, W, omega_grid(spec))


def _dirac_bands(spec, kred, energies):
    """Top valence / bottom conduction -> -/+ v_F * min(|k-K|, |k-K'|) (minimum image)."""
    vf = 0.46
    bm = recip_lattice(spec)
    nn = spec.nk[0]
    out = energies.copy()
    kpts = kred[:, :2].astype(np.float64) / nn
    best = np.full(len(kred), np.inf)
    for kk in (np.array([1.0 / 3.0, 1.0 / 3.0]), np.array([2.0 / 3.0, 2.0 / 3.0])):
        for m1 in (-1, 0, 1):
            for m2 in (-1, 0, 1):
                d = kpts - kk[None, :] + np.array([m1, m2])[None, :]
                cart = d[:, 0:1] * bm[0][None, :] + d[:, 1:2] * bm[1][None, :]
                best = np.minimum(best, np.linalg.norm(cart, axis=1))
    out[:, spec.nv - 1] = -vf * best
    out[:, spec.nv] = vf * best
    out[:, : spec.nv] = np.sort(out[:, : spec.nv], axis=1)
    out[:, spec.nv:] = np.sort(out[:, spec.nv:], axis=1)
    return out


# --------------------------------------------------------------------------
# layered 2D batch: 16 hexagonal sheets of uneven size
# --------------------------------------------------------------------------

def slab_batch_specs(seed: int = 0, nsys: int = 16, nmin: int = 24, nmax: int = 48) -> list:
    """Per-system parameters, drawn in order (n, Nv, Nc, Eg, r0) for s = 0..nsys-1.

    Hexagonal a = 4.7, c = 30 bohr; Ecut 2.5 Ha; grid 12x12x48; systems 0..3 carry a
    Dirac-like pair (Delta = 0 for every sheet: the drawn gap is the quasiparticle gap).
    """
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nsys):
        n = int(rng.integers(nmin, nmax + 1))
        nv = int(rng.integers(1, 4))
        nc = int(rng.integers(1, 4))
        eg = float(rng.uniform(0.0, 6.0)) * EV
        r0 = float(rng.uniform(10.0, 40.0))
        out.append(SystemSpec(
            f"hex_{s:02d}_{n}x{n}_{nv}v{nc}c", "hex", 4.7, 30.0, (n, n, 1), nv, nc, 2.5,
            (12, 12, 48), "slab", r0=r0, delta=0.0, eta=0.05 * EV, nsteps=300, nw=2000,
            seed=(seed, s + 1), eg=eg, dirac=(s < 4),
            ec_range=(eg, eg + 8.5 * EV)))
    return out


def generate_slab_batch(seed: int = 0, wdtype=np.complex64, **kw) -> list:
    return [generate(s, wdtype=wdtype) for s in slab_batch_specs(seed, **kw)]
