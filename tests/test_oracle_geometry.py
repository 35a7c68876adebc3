"""Pins for the oracle's plane-wave spheres and mesh bookkeeping (step A0)."""
import itertools
import math

import numpy as np
import pytest

from oracle import geometry as geo
from synth import config_spec, slab_batch_specs
from synth import systems as gen


def _fcc_cartesian_count(a, ecut, kcart=(0.0, 0.0, 0.0)):
    """Count G of the fcc reciprocal (bcc) lattice with |k+G|^2/2 <= ecut.

    Written in Cartesian integer coordinates: G = (2 pi/a)(h,k,l) with h, k, l all
    odd or all even - the textbook bcc description, independent of the reduced
    basis and Gram matrix used by the oracle.
    """
    s = 2.0 * math.pi / a
    r = int(math.sqrt(2.0 * ecut) / s) + 3
    n = 0
    for h, k, l in itertools.product(range(-r, r + 1), repeat=3):
        if not (h % 2 == k % 2 == l % 2):
            continue
        p = np.array([h, k, l]) * s + np.asarray(kcart)
        if 0.5 * p @ p <= ecut:
            n += 1
    return n


def test_fcc_gamma_shell_count_closed_form():
    # shells h^2+k^2+l^2 = 0,3,4,8,11,12,16,19,20 with multiplicities 1,8,6,12,24,8,6,24,24 -> 113
    spec = config_spec("fcc_4x4x4_3v3c")
    assert len(geo.sphere(spec, (0, 0, 0))) == 113
    assert _fcc_cartesian_count(10.0, 4.0) == 113


def test_fcc_sphere_counts_off_gamma_match_cartesian():
    spec = config_spec("fcc_4x4x4_3v3c")
    b = geo.reciprocal_basis(spec)
    for off in [(1, 0, 0), (1, 2, 3), (3, 3, 1)]:
        kc = (np.asarray(off) / 4.0) @ b
        assert len(geo.sphere(spec, off)) == _fcc_cartesian_count(10.0, 4.0, kc)


def test_sphere_in_canonical_order_and_inside():
    spec = config_spec("fcc_4x4x4_3v3c")
    for off in [(0, 0, 0), (2, 1, 3)]:
        g = geo.sphere(spec, off)
        kg = geo.cart(spec, off, g)
        e = 0.5 * np.sum(kg * kg, axis=1)
        assert np.all(e <= spec.ecut + 1e-9)
        assert np.all(np.diff(e) >= -1e-9)          # ascending |k+G|^2


def test_gamma_sphere_inversion_symmetric():
    spec = config_spec("fcc_4x4x4_3v3c")
    g = {tuple(x) for x in geo.sphere(spec, (0, 0, 0))}
    assert all(tuple(-np.asarray(x)) in g for x in g)


def test_fold_and_partner():
    spec = config_spec("fcc_4x4x4_3v3c")
    iq, iqv, g0 = geo.fold(spec, (3, 0, 1), (1, 2, 1))
    assert tuple(iqv) == (2, 2, 0) and tuple(g0) == (-1, 0, 0)
    assert iq == geo.mesh_index(spec, iqv)
    # -(q + G) lies on the sphere of fold(-q) at G'' = G0' - G
    for q in [(1, 0, 0), (2, 3, 1), (2, 2, 2)]:
        qb = tuple(np.mod(-np.asarray(q), 4))
        g0p = (-np.asarray(q) - np.asarray(qb)) // 4
        gb = {tuple(x) for x in geo.sphere(spec, qb)}
        assert all(tuple(g0p - x) in gb for x in geo.sphere(spec, q))


@pytest.mark.parametrize("name", ["fcc_4x4x4_3v3c"])
def test_oracle_spheres_equal_generator_layout(name):
    spec = config_spec(name)
    for off in gen.kpoint_offsets(spec)[::7]:
        a = geo.sphere(spec, tuple(off))
        b, _ = gen.sphere(spec, tuple(off))
        assert np.array_equal(a, b)


def test_hex_spheres_equal_generator_and_cartesian():
    spec = slab_batch_specs(0)[0]
    b = geo.reciprocal_basis(spec)
    for off in [(0, 0, 0), (5, 7, 0)]:
        a = geo.sphere(spec, off)
        g, _ = gen.sphere(spec, off)
        assert np.array_equal(a, g)
        kc = (np.asarray(off, dtype=float) / np.asarray(spec.nk)) @ b
        # brute-force Cartesian count
        n = 0
        for g1, g2, g3 in itertools.product(range(-4, 5), range(-4, 5), range(-15, 16)):
            p = np.array([g1, g2, g3]) @ b + kc
            n += 0.5 * p @ p <= spec.ecut
        assert n == len(a)


def test_pair_index_and_blocks():
    spec = config_spec("fcc_4x4x4_3v3c")
    assert geo.pair_index(spec, 1, 2, 0) == (1 * 3 + 2) * 3 + 0
    bl = geo.upper_blocks(spec)
    assert len(bl) == 64 * 65 // 2 and bl[0] == (0, 0) and bl[1] == (0, 1) and bl[64] == (1, 1)
