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


def test_block_reduction_covers_every_upper_block_and_symmetric_h_repeats_it():
    """k-point symmetry of the e-h blocks on a system whose states carry the point group (synthetic
    symmetric states, diagonal model W): the oracle's full Hamiltonian, every block built independently,
    has each upper block equal to its representative (mirrored blocks to its Hermitian conjugate)."""
    from oracle import geometry as geo
    from oracle import kernel as ok
    from oracle import symmetry as sym
    from synth import config_spec, generate
    spec = config_spec("fcc_4x4x4_3v3c").replace(name="sym4", symmetric=True, w_offdiag=0.0, nsteps=20, nw=50)
    s = generate(spec)
    reps, table = sym.reduce_blocks(spec)
    blocks = geo.upper_blocks(spec)
    assert all(t is not None for t in table)
    assert all(table[r] == (r, 0) for r in reps)
    assert len(reps) < len(blocks) / 10                      # O_h: 2080 upper blocks reduce to a few dozen
    H = ok.hamiltonian_full(spec, s.gk, s.coef, s.energies, s.W, spec.delta)
    nvc = spec.nv * spec.nc
    scale = np.abs(H).max()
    worst = 0.0
    for i, (a, b) in enumerate(blocks):
        r, mir = table[i]
        ra, rb = blocks[r]
        ref = H[ra * nvc:(ra + 1) * nvc, rb * nvc:(rb + 1) * nvc]
        if mir:
            ref = ref.conj().T
        worst = max(worst, np.abs(H[a * nvc:(a + 1) * nvc, b * nvc:(b + 1) * nvc] - ref).max())
    assert worst < 1e-12 * scale
    # a system without the symmetry does not repeat its blocks
    s2 = generate(spec.replace(symmetric=False))
    H2 = ok.hamiltonian_full(spec, s2.gk, s2.coef, s2.energies, s2.W, spec.delta)
    i = next(j for j, t in enumerate(table) if t[0] != j)
    r = table[i][0]
    (a, b), (ra, rb) = blocks[i], blocks[r]
    blk = H2[a * nvc:(a + 1) * nvc, b * nvc:(b + 1) * nvc]
    ref = H2[ra * nvc:(ra + 1) * nvc, rb * nvc:(rb + 1) * nvc]
    if table[i][1]:
        ref = ref.conj().T
    assert np.abs(blk - ref).max() > 0.1 * np.abs(ref).max()


def test_symmetric_states_carry_the_group():
    """c_{Rk}(R G + G0) = c_k(G) for every operation (R k = k' + G0 on the mesh) and shared energies."""
    from oracle import geometry as geo
    from oracle import symmetry as sym
    from synth import config_spec, generate
    spec = config_spec("fcc_4x4x4_3v3c").replace(name="sym4", symmetric=True, w_offdiag=0.0)
    s = generate(spec)
    ops = sym.point_group(spec)
    nk = np.asarray(spec.nk)
    kr = geo.mesh_offsets(spec)
    worst = 0.0
    for ik in (0, 1, 5, 21, 42):
        pos = {tuple(int(x) for x in g): t for t, g in enumerate(s.gk[ik])}
        for R in ops:
            img = R @ kr[ik]
            k2 = geo.mesh_index(spec, np.mod(img, nk))
            g0 = (img - np.mod(img, nk)) // nk
            pos2 = {tuple(int(x) for x in g): t for t, g in enumerate(s.gk[k2])}
            for g, t in pos.items():
                t2 = pos2[tuple(int(x) for x in R @ np.array(g) + g0)]
                worst = max(worst, np.abs(s.coef[k2, :, t2] - s.coef[ik, :, t]).max())
            assert np.array_equal(s.energies[k2], s.energies[ik])
    assert worst < 1e-13
