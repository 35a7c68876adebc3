"""ctypes binding of the C ABI in include/bse.h (argument marshalling only).

Device buffers are torch CUDA tensors (complex64 for float2 arrays, complex128
for double2, float64, int32); the current torch stream is passed to every call.
Loading fails loudly when the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbse.so")

BSE_OK, BSE_ERR_ARG, BSE_ERR_CUDA, BSE_ERR_NONFINITE, BSE_ERR_TIMEOUT, BSE_ERR_UNSUPPORTED, BSE_ERR_WORKSPACE = range(7)
BSE_ERR_INDEFINITE = 7
BSE_LATTICE_FCC, BSE_LATTICE_HEX = 0, 1
BSE_COULOMB_3D, BSE_COULOMB_SLAB = 0, 1
BSE_PREC_FP32, BSE_PREC_BF16X3 = 0, 1
BSE_WS_PAIR, BSE_WS_KERNEL, BSE_WS_SPECTRUM, BSE_WS_BACKWARD, BSE_WS_SCREEN = 0, 1, 2, 3, 4
BSE_WS_COUPLING, BSE_WS_COUPLED, BSE_WS_RITZ = 5, 6, 7
BSE_WS_CHI0, BSE_WS_ALDA, BSE_WS_EPSM, BSE_WS_STATES = 8, 9, 10, 11
BSE_PD_REALSPACE, BSE_PD_EXCHANGE, BSE_PD_DIRECT, BSE_PD_CHI0, BSE_PD_COUPLING, BSE_PD_TENSOR = 1, 2, 4, 8, 16, 32
BSE_BK_INIT, BSE_BK_DIRECT, BSE_BK_MIRROR, BSE_BK_SYMFILL = 1, 2, 4, 8
BSE_BC_INIT, BSE_BC_DIRECT, BSE_BC_MIRROR = 1, 2, 4

EXPORTED = [
    "bse_last_error", "bse_plan_create", "bse_plan_create_host", "bse_plan_destroy", "bse_plan_info", "bse_gvectors",
    "bse_pair_blocks", "bse_workspace_size", "bse_rho_dir_count", "bse_pair_densities",
    "bse_build_kernel", "bse_apply_H", "bse_spectrum", "bse_spectrum_static", "bse_spectrum_batch", "bse_spectrum_backward", "bse_status_read",
    "bse_pair_variants", "bse_set_pair_variant", "bse_autotune_pair", "bse_set_wait_limit", "bse_screening",
    "bse_rho_cpl_count", "bse_build_coupling", "bse_spectrum_coupled", "bse_ritz", "bse_symmetry", "bse_unfold_w",
    "bse_chi0_optical", "bse_xc_kernel_alda", "bse_epsilon_macro", "bse_exciton_states",
]


class BseSystem(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("a", ctypes.c_double), ("c", ctypes.c_double),
                ("nk", ctypes.c_int * 3), ("nv", ctypes.c_int), ("nc", ctypes.c_int),
                ("ecut", ctypes.c_double), ("fft", ctypes.c_int * 3), ("coulomb", ctypes.c_int),
                ("qhat", ctypes.c_double * 3), ("gap_floor", ctypes.c_double), ("kpoint_symmetry", ctypes.c_int)]


class BseInfo(ctypes.Structure):
    _fields_ = [("nkpt", ctypes.c_int), ("nb", ctypes.c_int), ("dim", ctypes.c_int),
                ("npw_max", ctypes.c_int), ("ng_max", ctypes.c_int), ("ng0", ctypes.c_int),
                ("nq", ctypes.c_int), ("nblocks", ctypes.c_longlong), ("omega_cell", ctypes.c_double),
                ("norm", ctypes.c_double), ("prefactor", ctypes.c_double), ("kpoint_symmetry", ctypes.c_int),
                ("nfill", ctypes.c_longlong), ("tensor_pair", ctypes.c_int), ("tc_region", ctypes.c_int * 3),
                ("tc_kpad", ctypes.c_int)]


class BsePairVariant(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int), ("threads", ctypes.c_int), ("rows", ctypes.c_int),
                ("max_products", ctypes.c_int), ("max_bands", ctypes.c_int), ("points_per_thread", ctypes.c_int),
                ("merged", ctypes.c_int)]


class BseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bse status {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libbse.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, ll, d, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_uint
    sz = ctypes.c_size_t
    lib.bse_last_error.restype = ctypes.c_char_p
    lib.bse_plan_create.argtypes = [ctypes.POINTER(BseSystem), i, ctypes.POINTER(vp)]
    lib.bse_plan_create_host.argtypes = [ctypes.POINTER(BseSystem), i, ctypes.POINTER(vp)]
    lib.bse_plan_destroy.argtypes = [vp]
    lib.bse_plan_info.argtypes = [vp, i, ctypes.POINTER(BseInfo)]
    lib.bse_gvectors.argtypes = [vp, i, i, i, vp, ctypes.POINTER(i)]
    lib.bse_pair_blocks.argtypes = [vp, i, i, vp, vp, ctypes.POINTER(i)]
    lib.bse_workspace_size.argtypes = [vp, i, i, ll, ctypes.POINTER(sz)]
    lib.bse_rho_dir_count.argtypes = [vp, i, i, i, ctypes.POINTER(ll)]
    lib.bse_pair_densities.argtypes = [vp, i, u, vp, vp, vp, vp, vp, i, i, vp, sz, vp]
    lib.bse_build_kernel.argtypes = [vp, i, u, vp, vp, i, i, vp, vp, d, i, vp, vp, sz, vp]
    lib.bse_apply_H.argtypes = [vp, i, vp, vp, vp, i, vp]
    lib.bse_spectrum.argtypes = [vp, i, vp, vp, i, vp, i, d, vp, vp, vp, vp, sz, vp]
    lib.bse_spectrum_static.argtypes = [vp, i, vp, vp, i, vp, i, d, vp, vp, vp, vp]
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.bse_spectrum_batch.argtypes = [vp, i, ctypes.POINTER(i), pp, pp, i, vp, i, d, pp, pp, pp, pp,
                                       ctypes.POINTER(sz), vp]
    lib.bse_spectrum_backward.argtypes = [vp, i, vp, vp, i, vp, i, d, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.bse_status_read.argtypes = [vp, vp]
    lib.bse_pair_variants.argtypes = [vp, i, ctypes.POINTER(BsePairVariant), i, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.bse_set_pair_variant.argtypes = [vp, i, i]
    lib.bse_set_wait_limit.argtypes = [ctypes.c_ulonglong]
    lib.bse_screening.argtypes = [vp, i, vp, vp, vp, i, i, i, vp, vp, vp, sz, vp]
    lib.bse_autotune_pair.argtypes = [vp, i, vp, sz, vp, i, i, i, ctypes.POINTER(ctypes.c_float), i,
                                      ctypes.POINTER(i), vp]
    lib.bse_rho_cpl_count.argtypes = [vp, i, i, i, ctypes.POINTER(ll)]
    lib.bse_build_coupling.argtypes = [vp, i, u, vp, vp, i, i, vp, i, vp, vp, sz, vp]
    lib.bse_spectrum_coupled.argtypes = [vp, i, vp, vp, vp, i, vp, i, d, vp, vp, vp, vp, sz, vp]
    lib.bse_ritz.argtypes = [vp, vp, i, vp, vp, vp, sz, vp]
    lib.bse_symmetry.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), vp, vp, vp]
    lib.bse_unfold_w.argtypes = [vp, i, vp, vp, i, i, vp]
    lib.bse_chi0_optical.argtypes = [vp, i, vp, vp, vp, d, vp, i, d, vp, vp, sz, vp]
    lib.bse_xc_kernel_alda.argtypes = [vp, i, vp, sz, vp, vp, sz, vp]
    lib.bse_epsilon_macro.argtypes = [vp, i, vp, vp, i, vp, vp, sz, vp]
    lib.bse_exciton_states.argtypes = [vp, i, vp, vp, i, vp, vp, vp, vp, vp, sz, vp]
    for name in EXPORTED:
        if name != "bse_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code):
    if code != BSE_OK:
        raise BseError(code, load().bse_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _nbytes(t):
    return 0 if t is None else t.numel() * t.element_size()


def system_struct(spec) -> BseSystem:
    """Fill bse_system from any object with the SystemSpec attribute names."""
    s = BseSystem()
    s.lattice = BSE_LATTICE_FCC if spec.lattice == "fcc" else BSE_LATTICE_HEX
    s.a = float(spec.a)
    s.c = float(spec.c)
    s.nk[:] = [int(x) for x in spec.nk]
    s.nv, s.nc = int(spec.nv), int(spec.nc)
    s.ecut = float(spec.ecut)
    s.fft[:] = [int(x) for x in spec.fft]
    s.coulomb = BSE_COULOMB_3D if spec.coulomb == "3d" else BSE_COULOMB_SLAB
    s.qhat[:] = list(getattr(spec, "qhat", (1.0, 0.0, 0.0)))
    s.gap_floor = float(getattr(spec, "gap_floor", 0.1 / 27.211386245988))
    s.kpoint_symmetry = 1 if getattr(spec, "symmetric", False) else 0
    return s


class Plan:
    """Owns a bse_plan*; systems are addressed by index."""

    def __init__(self, specs, host_only=False):
        lib = load()
        specs = list(specs)
        arr = (BseSystem * len(specs))(*[system_struct(s) for s in specs])
        h = ctypes.c_void_p()
        create = lib.bse_plan_create_host if host_only else lib.bse_plan_create
        _check(create(arr, len(specs), ctypes.byref(h)))
        self.handle = h
        self.nsys = len(specs)

    def close(self):
        if self.handle:
            load().bse_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, s=0) -> dict:
        inf = BseInfo()
        _check(load().bse_plan_info(self.handle, s, ctypes.byref(inf)))
        out = {f: getattr(inf, f) for f, _ in BseInfo._fields_}
        out["tc_region"] = tuple(inf.tc_region)
        return out


def bse_plan_create(specs) -> Plan:
    return Plan(specs)


def bse_plan_create_host(specs) -> Plan:
    return Plan(specs, host_only=True)


def bse_gvectors(plan, s, kq, is_q):
    n = ctypes.c_int()
    _check(load().bse_gvectors(plan.handle, s, kq, int(is_q), None, ctypes.byref(n)))
    out = np.zeros((n.value, 3), dtype=np.int32)
    _check(load().bse_gvectors(plan.handle, s, kq, int(is_q), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return out


def bse_pair_blocks(plan, s, iq):
    n = ctypes.c_int()
    _check(load().bse_pair_blocks(plan.handle, s, iq, None, None, ctypes.byref(n)))
    blk = np.zeros((n.value, 2), dtype=np.int32)
    g0 = np.zeros((n.value, 3), dtype=np.int32)
    _check(load().bse_pair_blocks(plan.handle, s, iq, blk.ctypes.data_as(ctypes.c_void_p),
                                  g0.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return blk, g0


def bse_workspace_size(plan, s, kind, arg=0) -> int:
    b = ctypes.c_size_t()
    _check(load().bse_workspace_size(plan.handle, s, kind, int(arg), ctypes.byref(b)))
    return int(b.value)


def bse_rho_dir_count(plan, s, q_begin, q_end) -> int:
    n = ctypes.c_longlong()
    _check(load().bse_rho_dir_count(plan.handle, s, q_begin, q_end, ctypes.byref(n)))
    return int(n.value)


def bse_pair_densities(plan, s, flags, coef, energies, rho_x, P, rho_dir, q_begin, q_end, ws):
    _check(load().bse_pair_densities(plan.handle, s, flags, _ptr(coef), _ptr(energies), _ptr(rho_x), _ptr(P),
                                     _ptr(rho_dir), q_begin, q_end, _ptr(ws), _nbytes(ws), _stream()))


def bse_build_kernel(plan, s, flags, rho_x, rho_dir, q_begin, q_end, W, energies, delta, prec, H, ws):
    _check(load().bse_build_kernel(plan.handle, s, flags, _ptr(rho_x), _ptr(rho_dir), q_begin, q_end, _ptr(W),
                                   _ptr(energies), float(delta), int(prec), _ptr(H), _ptr(ws), _nbytes(ws),
                                   _stream()))


def bse_apply_H(plan, s, H, X, Y):
    nvec = X.shape[0] if X.dim() == 2 else 1
    _check(load().bse_apply_H(plan.handle, s, _ptr(H), _ptr(X), _ptr(Y), nvec, _stream()))


def bse_spectrum(plan, s, H, P, nsteps, omega, eta, eps2, ab, steps_done, ws):
    _check(load().bse_spectrum(plan.handle, s, _ptr(H), _ptr(P), int(nsteps), _ptr(omega), omega.numel(),
                               float(eta), _ptr(eps2), _ptr(ab), _ptr(steps_done), _ptr(ws), _nbytes(ws),
                               _stream()))


def bse_spectrum_batch(plan, systems, H, P, nsteps, omega, eta, eps2, ab, steps_done, ws):
    """Per-system lists of device tensors; one cooperative launch for all systems."""
    n = len(systems)

    def arr(ts):
        return (ctypes.c_void_p * n)(*[ctypes.c_void_p(t.data_ptr()) for t in ts])
    for t in list(H) + list(P) + list(eps2) + list(ab) + list(steps_done) + list(ws):
        _ptr(t)
    sysa = (ctypes.c_int * n)(*systems)
    wsb = (ctypes.c_size_t * n)(*[_nbytes(w) for w in ws])
    _check(load().bse_spectrum_batch(plan.handle, n, sysa, arr(H), arr(P), int(nsteps), _ptr(omega), omega.numel(),
                                     float(eta), arr(eps2), arr(ab), arr(steps_done), arr(ws), wsb, _stream()))


def bse_spectrum_static(plan, s, H, P, nsteps, omega, eta, eps2, ab, steps_done):
    _check(load().bse_spectrum_static(plan.handle, s, _ptr(H), _ptr(P), int(nsteps), _ptr(omega), omega.numel(),
                                      float(eta), _ptr(eps2), _ptr(ab), _ptr(steps_done), _stream()))


def bse_spectrum_backward(plan, s, H, P, nsteps, omega, eta, dL_deps2, rho_x, rho_dir, W, dL_ddelta, dL_dH,
                          dL_drho_x, dL_drho_dir, dL_dW, ws):
    _check(load().bse_spectrum_backward(plan.handle, s, _ptr(H), _ptr(P), int(nsteps), _ptr(omega), omega.numel(),
                                        float(eta), _ptr(dL_deps2), _ptr(rho_x), _ptr(rho_dir), _ptr(W),
                                        _ptr(dL_ddelta), _ptr(dL_dH), _ptr(dL_drho_x), _ptr(dL_drho_dir),
                                        _ptr(dL_dW), _ptr(ws), _nbytes(ws), _stream()))


def bse_status_read(plan):
    _check(load().bse_status_read(plan.handle, _stream()))


def bse_pair_variants(plan, s):
    """Valid pair-kernel variants of system s (list of dicts) and the index in use."""
    lib = load()
    arr = (BsePairVariant * 64)()
    n, cur = ctypes.c_int(), ctypes.c_int()
    _check(lib.bse_pair_variants(plan.handle, s, arr, 64, ctypes.byref(n), ctypes.byref(cur)))
    out = [{f: getattr(arr[k], f) for f, _ in BsePairVariant._fields_} for k in range(min(n.value, 64))]
    return out, cur.value


def bse_set_pair_variant(plan, s, index):
    _check(load().bse_set_pair_variant(plan.handle, s, int(index)))


def bse_autotune_pair(plan, s, ws, rho_dir, q_begin, q_end, reps=3):
    """Times every valid variant on the direct pair densities of [q_begin, q_end), selects the fastest.

    Returns (ms per launch in bse_pair_variants order, chosen index)."""
    ms = (ctypes.c_float * 64)()
    chosen = ctypes.c_int()
    _check(load().bse_autotune_pair(plan.handle, s, _ptr(ws), _nbytes(ws), _ptr(rho_dir), q_begin, q_end, int(reps),
                                    ms, 64, ctypes.byref(chosen), _stream()))
    n = len(bse_pair_variants(plan, s)[0])
    return [float(ms[k]) for k in range(n)], chosen.value


def bse_set_wait_limit(ns):
    """Limit of each grid-barrier wait of the spectrum kernels on the current device (failure injection)."""
    _check(load().bse_set_wait_limit(int(ns)))


def bse_screening(plan, s, rho_chi, energies, P, q_begin, q_end, iterations, W, residual, ws):
    """Static RPA W of q in [q_begin, q_end) from BSE_PD_CHI0 pair densities (rho_chi is overwritten)."""
    _check(load().bse_screening(plan.handle, s, _ptr(rho_chi), _ptr(energies), _ptr(P), q_begin, q_end,
                                int(iterations), _ptr(W), _ptr(residual), _ptr(ws), _nbytes(ws), _stream()))


def bse_rho_cpl_count(plan, s, q_begin, q_end) -> int:
    n = ctypes.c_longlong()
    _check(load().bse_rho_cpl_count(plan.handle, s, q_begin, q_end, ctypes.byref(n)))
    return int(n.value)


def bse_build_coupling(plan, s, flags, rho_x, rho_cpl, q_begin, q_end, W, prec, Bm, ws):
    """Coupling block B = 2 Bx - Bd of the BSE beyond the Tamm-Dancoff approximation."""
    _check(load().bse_build_coupling(plan.handle, s, flags, _ptr(rho_x), _ptr(rho_cpl), q_begin, q_end, _ptr(W),
                                     int(prec), _ptr(Bm), _ptr(ws), _nbytes(ws), _stream()))


def bse_spectrum_coupled(plan, s, A, Bm, P, nsteps, omega, eta, eps2, b, steps_done, ws):
    """eps_2 of H2 = [[A, B], [-conj B, -conj A]] by Lanczos in the F H2 inner product."""
    _check(load().bse_spectrum_coupled(plan.handle, s, _ptr(A), _ptr(Bm), _ptr(P), int(nsteps), _ptr(omega),
                                       omega.numel(), float(eta), _ptr(eps2), _ptr(b), _ptr(steps_done), _ptr(ws),
                                       _nbytes(ws), _stream()))


def bse_ritz(ab, steps_done, nsteps, theta, weight, ws):
    """Ritz values (exciton energies) and weights (normalised oscillator strengths) of a Haydock recursion."""
    _check(load().bse_ritz(_ptr(ab), _ptr(steps_done), int(nsteps), _ptr(theta), _ptr(weight), _ptr(ws), _nbytes(ws),
                           _stream()))


def bse_symmetry(plan, s):
    """(nops, ibz [nibz], qmap [nq][6], perm [nq][ng_max]) of the plan's q-point symmetry reduction."""
    import numpy as np
    inf = plan.info(s)
    nq, ng = inf["nq"], inf["ng_max"]
    nops, nibz = ctypes.c_int(), ctypes.c_int()
    ibz = np.zeros(nq, dtype=np.int32)
    qmap = np.zeros((nq, 6), dtype=np.int32)
    perm = np.zeros((nq, ng), dtype=np.int32)
    _check(load().bse_symmetry(plan.handle, s, ctypes.byref(nops), ctypes.byref(nibz), ibz.ctypes.data_as(ctypes.c_void_p),
                               qmap.ctypes.data_as(ctypes.c_void_p), perm.ctypes.data_as(ctypes.c_void_p)))
    return int(nops.value), ibz[: nibz.value].copy(), qmap, perm


def bse_unfold_w(plan, s, W_ibz, W, q_begin, q_end):
    """W on the q range from W on the irreducible points (Sec. III A)."""
    _check(load().bse_unfold_w(plan.handle, s, _ptr(W_ibz), _ptr(W), q_begin, q_end, _stream()))


def bse_chi0_optical(plan, s, rho_x, P, energies, delta, omega, eta, chi0, ws):
    """Symmetrised Adler-Wiser response chi~0(w) [nw][ng0][ng0] in the optical limit (TDDFT, Sec. II B)."""
    _check(load().bse_chi0_optical(plan.handle, s, _ptr(rho_x), _ptr(P), _ptr(energies), float(delta), _ptr(omega),
                                   omega.numel(), float(eta), _ptr(chi0), _ptr(ws), _nbytes(ws), _stream()))


def bse_xc_kernel_alda(plan, s, pair_ws, F, ws):
    """F = v^-1/2 f_xc v^-1/2 [ng0][ng0] of the adiabatic local-density kernel (density from the pair workspace)."""
    _check(load().bse_xc_kernel_alda(plan.handle, s, _ptr(pair_ws), _nbytes(pair_ws), _ptr(F), _ptr(ws), _nbytes(ws),
                                     _stream()))


def bse_epsilon_macro(plan, s, chi0, F, eps_m, ws):
    """eps_M(w) = 1/[eps^-1]_00 from the Dyson equation with K = v (F None) or v + f_xc (complex128 [nw])."""
    _check(load().bse_epsilon_macro(plan.handle, s, _ptr(chi0), _ptr(F), eps_m.numel(), _ptr(eps_m), _ptr(ws),
                                    _nbytes(ws), _stream()))


def bse_exciton_states(plan, s, H, X0, n, theta, A, ab, steps_done, ws):
    """Eigenpairs of H (Eq. bse_eig) from a Lanczos tridiagonalisation of Krylov dimension n started at X0:
    theta [n] ascending, A [n][dim] unit eigenvectors (A may be None)."""
    _check(load().bse_exciton_states(plan.handle, s, _ptr(H), _ptr(X0), int(n), _ptr(theta), _ptr(A), _ptr(ab),
                                     _ptr(steps_done), _ptr(ws), _nbytes(ws), _stream()))
