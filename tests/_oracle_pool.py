"""Worker functions for parity tests that compare many sampled H blocks with the oracle in a process pool.

Test infrastructure only.  Each worker draws the system's coefficients and energies from the seeded
generator (W arrives with each task, one q at a time) and computes the oracle's exchange rows of every k
once; a task then rebuilds the oracle's H blocks of one q point and returns the error statistics of the
GPU's blocks against them.  The pool must be started with the 'spawn' method (never forked from a process
that has touched the GPU).
"""
from __future__ import annotations

import os

import numpy as np

_S = {}


def init(config_name):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import kernel as ok
    from oracle import pair as op
    from synth import config_spec, generate
    spec = config_spec(config_name)
    s = generate(spec, wdtype=np.complex64, with_w=False)
    _S["spec"] = spec
    _S["s"] = s
    _S["vbar"] = ok.coulomb_bar(spec)
    _S["de"] = ok.transition_energies(spec, s.energies, spec.delta)
    _S["op"] = op
    _S["ok"] = ok


def _rows(ik):
    """Exchange rows rho_vc^{kk}(G) of k on the q = 0 sphere (oracle correlation), cached per worker."""
    from oracle import geometry as geo
    spec, s = _S["spec"], _S["s"]
    cache = _S.setdefault("rows", {})
    if ik not in cache:
        g0 = geo.sphere(spec, (0, 0, 0))
        r = _S["op"].rho_corr(spec, ik, ik, list(range(spec.nv)), list(range(spec.nv, spec.nb)), g0, s.gk, s.coef)
        cache[ik] = r.reshape(spec.nv * spec.nc, -1)
    return cache[ik]


def block_errors(task):
    """task = (w_q [ng][ng] complex, [(ik, ik2)], [gpu blocks per build] each [n][nvc][nvc]).
    Returns (per build: max |err|, sum |err|, number of entries), max |ref| over kernel entries."""
    w_q, pairs, gpu = task
    spec, s, ok, op = _S["spec"], _S["s"], _S["ok"], _S["op"]
    nvc = spec.nv * spec.nc
    w = np.asarray(w_q, dtype=np.complex128)
    stats = [[0.0, 0.0, 0] for _ in gpu]
    scale = 0.0
    for i, (ik, ik2) in enumerate(pairs):
        iq, rv, rc = op.direct_rho_block(spec, ik, ik2, s.gk, s.coef)
        ng = rv.shape[-1]
        kd = ok.direct_block(spec, rv, rc, w[:ng, :ng])
        ref = 2.0 * ok.norm_factor(spec) * (np.conj(_rows(ik)) * _S["vbar"][None, :]) @ _rows(ik2).T - kd
        if ik == ik2:
            ref = ref + np.diag(_S["de"][ik * nvc:(ik + 1) * nvc])
            ref = 0.5 * (ref + ref.conj().T)
        off = ~np.eye(nvc, dtype=bool) if ik == ik2 else np.ones((nvc, nvc), bool)
        scale = max(scale, float(np.abs(ref[off]).max()))
        for st, g in zip(stats, gpu):
            e = np.abs(g[i] - ref)[off]
            st[0] = max(st[0], float(e.max()))
            st[1] += float(e.sum())
            st[2] += int(e.size)
    return stats, scale
