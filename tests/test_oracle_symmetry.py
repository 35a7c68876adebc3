"""Pins of oracle/symmetry.py (q-point symmetry reduction of W, Sec. III A)."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import symmetry as sy
from synth import config_spec, slab_batch_specs


def _specs():
    return [config_spec("fcc_4x4x4_3v3c"), slab_batch_specs(0)[5].replace(name="hex6", nk=(6, 6, 1))]


@pytest.mark.parametrize("spec", _specs(), ids=lambda s: s.name)
def test_point_group_is_a_group_preserving_the_metric(spec):
    ops = sy.point_group(spec)
    assert len(ops) == (48 if spec.lattice == "fcc" else 24)        # O_h; D_6h of the sheet
    assert np.array_equal(ops[0], np.eye(3, dtype=np.int64))
    keys = {tuple(R.reshape(-1)) for R in ops}
    b = geo.reciprocal_basis(spec)
    M = b @ b.T
    for R in ops:
        assert np.abs(R.T @ M @ R - M).max() < 1e-9 * np.abs(M).max()
        assert tuple(np.round(np.linalg.inv(R)).astype(np.int64).reshape(-1)) in keys
        for R2 in ops[::5]:
            assert tuple((R @ R2).reshape(-1)) in keys


def test_irreducible_counts_of_the_fcc_gamma_meshes():
    """Textbook counts of irreducible points of Gamma-centred fcc meshes under O_h: 4^3 -> 8, 8^3 -> 29."""
    for n, want in ((4, 8), (8, 29)):
        spec = config_spec("fcc_8x8x8_3v4c").replace(nk=(n, n, n))
        ibz, _ = sy.reduce_mesh(spec)
        assert len(ibz) == want


@pytest.mark.parametrize("spec", _specs(), ids=lambda s: s.name)
def test_map_reconstructs_every_q_and_permutes_spheres(spec):
    ops = sy.point_group(spec)
    ibz, qmap = sy.reduce_mesh(spec, ops)
    kr = geo.mesh_offsets(spec)
    nk = np.asarray(spec.nk)
    b = geo.reciprocal_basis(spec)
    sizes = np.zeros(len(ibz), dtype=int)
    for iq in range(spec.nkpt):
        ii, io, tr, *g0 = qmap[iq]
        s = -1 if tr else 1
        assert np.array_equal(kr[iq], s * (ops[io] @ kr[ibz[ii]]) + np.array(g0) * nk)
        sizes[ii] += 1
        perm = sy.sphere_perm(spec, iq, ibz, qmap, ops)
        gq = geo.sphere(spec, tuple(kr[iq]))
        gi = geo.sphere(spec, tuple(kr[ibz[ii]]))
        assert len(perm) == len(gq) == len(gi) and len(set(perm.tolist())) == len(perm)
        cq = (gq + kr[iq][None, :] / nk) @ b
        ci = (gi[perm] + kr[ibz[ii]][None, :] / nk) @ b
        assert np.abs((cq * cq).sum(1) - (ci * ci).sum(1)).max() < 1e-9     # |q + G| = |q_IBZ + G'|
    assert sizes.sum() == spec.nkpt and sizes.min() >= 1
    assert all(qmap[i][0] == j and qmap[i][1] == 0 and qmap[i][2] == 0 for j, i in enumerate(ibz))


def _image_perm(spec, R, tr, iq_from, iq_to):
    """Sphere map of q_to = s R q_from + G0: p (sphere of q_to) -> index of s R^-1 (g_p + G0) in q_from's."""
    kr = geo.mesh_offsets(spec)
    nk = np.asarray(spec.nk)
    s = -1 if tr else 1
    g0 = (kr[iq_to] - s * (R @ kr[iq_from])) // nk
    Rinv = np.round(np.linalg.inv(R)).astype(np.int64)
    gt = geo.sphere(spec, tuple(kr[iq_to]))
    gf = geo.sphere(spec, tuple(kr[iq_from]))
    pos = {tuple(int(x) for x in g): j for j, g in enumerate(gf)}
    return np.array([pos[tuple(int(x) for x in s * (Rinv @ (g + g0)))] for g in gt])


@pytest.mark.parametrize("spec", _specs(), ids=lambda s: s.name)
def test_unfolded_w_obeys_the_relation_for_every_operation(spec):
    """Make W(q_IBZ) invariant under its little group (average of its images); then the unfolded W
    satisfies the Sec. III A relation for every operation and time reversal, not only the chosen one."""
    ops = sy.point_group(spec)
    ibz, qmap = sy.reduce_mesh(spec, ops)
    kr = geo.mesh_offsets(spec)
    nk = np.asarray(spec.nk)
    ng = max(len(geo.sphere(spec, tuple(k))) for k in kr)
    rng = np.random.default_rng(3)
    W_ibz = np.zeros((len(ibz), ng, ng), dtype=np.complex128)
    for j, iq in enumerate(ibz):
        n = len(geo.sphere(spec, tuple(kr[iq])))
        x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        x = x + x.conj().T
        acc, cnt = np.zeros_like(x), 0
        for R in ops:
            for tr in (0, 1):
                img = np.mod((-1 if tr else 1) * (R @ kr[iq]), nk)
                if geo.mesh_index(spec, img) != iq:
                    continue
                perm = _image_perm(spec, R, tr, iq, iq)
                blk = x[np.ix_(perm, perm)]
                acc += np.conj(blk) if tr else blk
                cnt += 1
        W_ibz[j, :n, :n] = acc / cnt
    W = sy.unfold_w(spec, W_ibz, ibz, qmap, ops)
    for iq in range(spec.nkpt):
        ii = qmap[iq][0]
        src = ibz[ii]
        n = len(geo.sphere(spec, tuple(kr[iq])))
        for R in ops[::3]:
            for tr in (0, 1):
                img = np.mod((-1 if tr else 1) * (R @ kr[src]), nk)
                if geo.mesh_index(spec, img) != iq:
                    continue
                perm = _image_perm(spec, R, tr, src, iq)
                blk = W_ibz[ii][np.ix_(perm, perm)]
                assert np.abs(W[iq, :n, :n] - (np.conj(blk) if tr else blk)).max() < 1e-12
        assert np.abs(W[iq, :n, :n] - W[iq, :n, :n].conj().T).max() < 1e-12
