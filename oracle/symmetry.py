"""Oracle: q-point symmetry reduction of the screened interaction (Sec. III A).

Test infrastructure only (see package docstring).

Sec. III A: for q = T q_IBZ + G0 (T a crystal symmetry, G0 a reciprocal lattice vector)
W_GG'(q) = W_{T^-1(G + G0), T^-1(G' + G0)}(q_IBZ), and for q = -T q_IBZ + G0 (time reversal)
W_GG'(q) = conj W_{-T^-1(G + G0), -T^-1(G' + G0)}(q_IBZ); T must map the k mesh onto itself.

Readings:
- Operations are the lattice's point-group operations written as integer matrices R acting on
  reduced reciprocal coordinates (q_red -> R q_red) that preserve the reciprocal metric
  (R^T M R = M, M_ij = b_i.b_j) and map the Gamma-centred mesh onto itself; no fractional
  translations (symmorphic operations, as the relations above carry no phase).
- Canonical order of the operations: the identity first, then the others ascending in the
  lexicographic order of their row-major entries.  The irreducible points and the map of every
  q are assigned greedily: q points are visited by ascending mesh index; an unassigned q becomes
  irreducible, then each operation in order, image R q before the time-reversed image -R q,
  assigns every still unassigned image q' to it with G0 = q' - (+-R q_IBZ) (integer).
- The sphere of q maps onto the sphere of q_IBZ by G -> G' = s R^-1 (G + G0), s = +-1:
  q + G = s R (q_IBZ + G') keeps |q + G|.

k-point symmetry of the e-h blocks.  When the states carry the point group (psi_{Tk}(r) = psi_k(T^-1 r),
energies shared by the orbit of k) and W carries it too, Sec. III A's relation
n_{nk,n'k+q}(G) = n_{nT^-1k,n'T^-1(k+q)}(T^-1(G0 + G)) makes the pair densities, and with them every
kernel block, of the pair (k, k') equal to those of (Tk, Tk'): H_{Tk,Tk'} = H_{k,k'} block for block
(same band indices; no phases for symmorphic operations).  ``reduce_blocks`` reads this as a reduction
of the upper blocks: they are visited in row-major order (k ascending, then k' >= k); an unassigned
block becomes a representative, then each operation in order maps it to (a, b) = (R k, R k') on the
mesh and assigns the upper block (a, b) to it directly if a <= b, or (b, a) as its Hermitian mirror if
a > b, when that block is still unassigned.  Time reversal is not used for the blocks.

Pinned by tests/test_oracle_symmetry.py: group closure and metric, orbit sizes, invariance of the
integer sphere keys under the map, bijective sphere permutations, and the Sec. III A relation for
every operation of the group once W(q_IBZ) is made invariant under its little group; the block
reduction covers every upper block once and, on a system whose states carry the group, the oracle's
independent full Hamiltonian has every block equal to its representative (or its mirror).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import geometry as geo


def point_group(spec) -> list:
    """Integer matrices R (3x3, reduced reciprocal coordinates) preserving the metric and the mesh."""
    b = geo.reciprocal_basis(spec)
    M = b @ b.T
    nk = np.asarray(spec.nk)
    ops = []
    for e in itertools.product((-1, 0, 1), repeat=9):
        R = np.array(e, dtype=np.int64).reshape(3, 3)
        if round(abs(np.linalg.det(R))) != 1:
            continue
        if np.abs(R.T @ M @ R - M).max() > 1e-9 * np.abs(M).max():
            continue
        # the mesh {i/n} maps onto itself: R (i/n) must be a mesh point mod 1 for every i
        ok = True
        for j in range(3):
            e_j = np.zeros(3)
            e_j[j] = 1.0 / nk[j]
            img = R @ e_j
            if np.abs(img * nk - np.round(img * nk)).max() > 1e-12:
                ok = False
                break
        if ok:
            ops.append(R)
    ident = np.eye(3, dtype=np.int64)
    rest = sorted((R for R in ops if not np.array_equal(R, ident)), key=lambda R: tuple(R.reshape(-1)))
    return [ident] + rest


def reduce_mesh(spec, ops=None):
    """Irreducible q points and, for every q, (iq_ibz, op, tr, G0) with q = s R q_IBZ + G0, s = -1 if tr."""
    if ops is None:
        ops = point_group(spec)
    nk = np.asarray(spec.nk)
    kr = geo.mesh_offsets(spec)
    nq = spec.nkpt
    qmap = [None] * nq
    ibz = []
    for iq in range(nq):
        if qmap[iq] is not None:
            continue
        ibz.append(iq)
        for io, R in enumerate(ops):
            for tr in (0, 1):
                img = (-1 if tr else 1) * (R @ kr[iq])             # in units of 1/nk (integers)
                fold = np.mod(img, nk)
                iq2 = geo.mesh_index(spec, fold)
                if qmap[iq2] is None:
                    g0 = (fold - img) // nk                             # q' = s R q_IBZ + G0 (reduced)
                    qmap[iq2] = (len(ibz) - 1, io, tr, int(g0[0]), int(g0[1]), int(g0[2]))
    return ibz, qmap


def sphere_perm(spec, iq, ibz, qmap, ops):
    """perm[p] = index in the sphere of q_IBZ of G' = s R^-1 (g_p + G0), p over the sphere of q."""
    kr = geo.mesh_offsets(spec)
    ii, io, tr, g0x, g0y, g0z = qmap[iq]
    R = ops[io]
    Rinv = np.round(np.linalg.inv(R)).astype(np.int64)
    s = -1 if tr else 1
    gq = geo.sphere(spec, tuple(kr[iq]))
    gi = geo.sphere(spec, tuple(kr[ibz[ii]]))
    pos = {tuple(int(x) for x in g): j for j, g in enumerate(gi)}
    g0 = np.array([g0x, g0y, g0z], dtype=np.int64)
    return np.array([pos[tuple(int(x) for x in s * (Rinv @ (g + g0)))] for g in gq], dtype=np.int64)


def unfold_w(spec, W_ibz, ibz=None, qmap=None, ops=None):
    """Full-mesh W from W on the irreducible points (W_ibz[i] belongs to ibz[i]), by the Sec. III A rule."""
    if ops is None:
        ops = point_group(spec)
    if ibz is None:
        ibz, qmap = reduce_mesh(spec, ops)
    nq = spec.nkpt
    ng = W_ibz.shape[1]
    W = np.zeros((nq, ng, ng), dtype=W_ibz.dtype)
    for iq in range(nq):
        perm = sphere_perm(spec, iq, ibz, qmap, ops)
        n = len(perm)
        blk = W_ibz[qmap[iq][0]][np.ix_(perm, perm)]
        W[iq, :n, :n] = np.conj(blk) if qmap[iq][2] else blk
    return W


def reduce_blocks(spec, ops=None):
    """For every upper block (ik, ik2), ik <= ik2 in row-major order: (rep, mirrored) with rep the index of
    its representative in the same order; returns (reps, table) with reps the representative indices."""
    if ops is None:
        ops = point_group(spec)
    nk = np.asarray(spec.nk)
    kr = geo.mesh_offsets(spec)
    blocks = geo.upper_blocks(spec)
    index = {b: i for i, b in enumerate(blocks)}
    table = [None] * len(blocks)
    reps = []
    for i, (a0, b0) in enumerate(blocks):
        if table[i] is not None:
            continue
        reps.append(i)
        for R in ops:
            a = geo.mesh_index(spec, np.mod(R @ kr[a0], nk))
            b = geo.mesh_index(spec, np.mod(R @ kr[b0], nk))
            j, mirrored = (index[(a, b)], 0) if a <= b else (index[(b, a)], 1)
            if table[j] is None:
                table[j] = (i, mirrored)
    return reps, table
