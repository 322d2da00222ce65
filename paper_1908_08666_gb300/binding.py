"""Thin ctypes binding of libhhgs (include/hhg.h): same names, argument marshalling only.

Every numeric step runs in the library's CUDA kernels.  Loading fails loudly when
the shared library has not been built; there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhhgs.so")

HHG_OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_UNSUPPORTED", 5: "ERR_NOT_CONVERGED",
          6: "ERR_NUMERIC", 7: "ERR_TIMEOUT", 8: "ERR_STATE"}
F64, F32, BF16 = 0, 1, 2
ELASTICITY, STOKES = 0, 1
PHYSICAL, UNPHYSICAL, NODAL, STORED = 0, 1, 2, 3
KHAT_PATCH, KHAT_EDGE = 0, 1
IFACE_SYMMETRIC, IFACE_PRACTICAL = 0, 1


class HhgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


SMOOTH_JACOBI, SMOOTH_CHEBYSHEV, SMOOTH_HYBRID_GS = 0, 1, 2
COARSE_INJECT, COARSE_MEAN, COARSE_HARMONIC = 0, 1, 2
SOLVE_PCG_JACOBI, SOLVE_MG_CG, SOLVE_IR_MG_CG, SOLVE_MG, SOLVE_STOKES_MINRES, SOLVE_STOKES_IR_MINRES = 0, 1, 2, 3, 4, 5
SOLVE_IR_FCG_LEARNED, SOLVE_IR_FCG = 6, 7
SOLVE_STOKES_UZAWA, SOLVE_STOKES_IR_UZAWA = 8, 9
SOLVE_STOKES_IR_FGCR_LEARNED, SOLVE_STOKES_IR_FGCR = 10, 11


class hhg_mg_params(C.Structure):
    _fields_ = [("smoother", C.c_int), ("pre", C.c_int), ("post", C.c_int), ("omega", C.c_double),
                ("cheby_lo", C.c_double), ("cheby_hi", C.c_double), ("power_iters", C.c_int),
                ("coarse_coeff", C.c_int), ("uzawa_pre", C.c_int), ("uzawa_post", C.c_int),
                ("uzawa_extra", C.c_int), ("uzawa_vsteps", C.c_int), ("uzawa_omega", C.c_double)]


class hhg_solve_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("level", C.c_int), ("dt", C.c_int), ("rtol", C.c_double),
                ("max_iter", C.c_int), ("inner_rtol", C.c_double), ("inner_max_iter", C.c_int)]


class hhg_solve_report(C.Structure):
    _fields_ = [("iterations", C.c_int), ("inner_iterations", C.c_int), ("residual0", C.c_double),
                ("rel_residual", C.c_double), ("seconds", C.c_double), ("converged", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hhg_carreau(C.Structure):
    _fields_ = [("eta0", C.c_double), ("eta_inf", C.c_double), ("kappa", C.c_double), ("r", C.c_double)]


class hhg_picard_opts(C.Structure):
    _fields_ = [("carreau", hhg_carreau), ("level", C.c_int), ("picard_tol", C.c_double), ("max_picard", C.c_int),
                ("step_rtol", C.c_double), ("step_max_iter", C.c_int), ("final_rtol", C.c_double)]


class hhg_picard_report(C.Structure):
    _fields_ = [("picard_iterations", C.c_int), ("minres_iterations", C.c_int), ("final_rel_residual", C.c_double),
                ("last_change", C.c_double), ("mu_min", C.c_double), ("mu_max", C.c_double),
                ("seconds", C.c_double), ("converged", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hhg_learn_train_opts(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("crop", C.c_int), ("lr", C.c_double), ("seed", C.c_uint64)]


class hhg_learn_train_report(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("pairs", C.c_int64), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hhg_learn_stats_report(C.Structure):
    _fields_ = [("applications", C.c_int64), ("fallbacks", C.c_int64), ("alpha_mean", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("gain_mean", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hhg_problem(C.Structure):
    _fields_ = [("kind", C.c_int), ("nu", C.c_double), ("variant", C.c_int), ("khat", C.c_int), ("iface", C.c_int)]


_lib = None

# name -> argtypes (all return int status unless listed in _RESTYPE)
_SIGS = {
    "hhg_create": [C.POINTER(C.c_void_p), C.c_int, C.c_void_p],
    "hhg_destroy": [C.c_void_p],
    "hhg_last_error": [C.c_void_p],
    "hhg_set_timeout": [C.c_void_p, C.c_int64],
    "hhg_set_macro_mesh": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p],
    "hhg_refine": [C.c_void_p, C.c_int],
    "hhg_set_coarsest_level": [C.c_void_p, C.c_int],
    "hhg_set_strain_fit": [C.c_void_p, C.c_int],
    "hhg_apply_2d": [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                     C.c_void_p],
    "hhg_traction_load": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "hhg_set_problem": [C.c_void_p, C.POINTER(hhg_problem)],
    "hhg_num_nodes": [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "hhg_entry_coords": [C.c_void_p, C.c_int, C.c_void_p],
    "hhg_entry_to_unique": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_gather_unique": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_scatter_unique": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_set_coefficient": [C.c_void_p, C.c_void_p, C.c_int],
    "hhg_apply": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_residual": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)],
    "hhg_apply_host": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_set_mg_params": [C.c_void_p, C.POINTER(hhg_mg_params)],
    "hhg_mg_setup": [C.c_void_p],
    "hhg_get_lambda_max": [C.c_void_p, C.c_int, C.POINTER(C.c_double)],
    "hhg_set_lambda_max": [C.c_void_p, C.c_int, C.c_double],
    "hhg_diagonal": [C.c_void_p, C.c_int, C.c_int, C.c_void_p],
    "hhg_smooth": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_prolongate_add": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_restrict": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_vcycle": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_stokes_apply": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_stokes_residual": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)],
    "hhg_carreau_viscosity": [C.c_void_p, C.c_int, C.POINTER(hhg_carreau), C.c_void_p, C.c_void_p],
    "hhg_picard": [C.c_void_p, C.POINTER(hhg_picard_opts), C.c_void_p, C.c_void_p, C.POINTER(hhg_picard_report)],
    "hhg_solve": [C.c_void_p, C.POINTER(hhg_solve_opts), C.c_void_p, C.c_void_p, C.POINTER(hhg_solve_report)],
    "hhg_profile": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "hhg_set_interior_kernel": [C.c_void_p, C.c_int],
    "hhg_fp32_fma_probe": [C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)],
    "hhg_residual_noalloc": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.POINTER(C.c_double)],
    "hhg_learn_num_params": [],
    "hhg_learn_init": [C.c_void_p, C.c_uint64],
    "hhg_learn_set_conv_kernel": [C.c_void_p, C.c_int],
    "hhg_learn_set_coarsening": [C.c_void_p, C.c_int],
    "hhg_learn_set_conv_wait": [C.c_void_p, C.c_int64],
    "hhg_learn_get_params": [C.c_void_p, C.c_void_p, C.c_int64],
    "hhg_learn_set_params": [C.c_void_p, C.c_void_p, C.c_int64],
    "hhg_learn_grid": [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int64)],
    "hhg_learn_channels": [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "hhg_learn_forward": [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p],
    "hhg_learn_loss_grad": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                            C.POINTER(C.c_double), C.c_void_p],
    "hhg_learn_reserve_pairs": [C.c_void_p, C.c_int, C.c_int64],
    "hhg_learn_collect": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int64)],
    "hhg_learn_collect_cg": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int64)],
    "hhg_learn_get_pair": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
    "hhg_learn_train": [C.c_void_p, C.POINTER(hhg_learn_train_opts), C.POINTER(hhg_learn_train_report)],
    "hhg_learn_precondition": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)],
    "hhg_learn_stats": [C.c_void_p, C.POINTER(hhg_learn_stats_report), C.c_int],
}
_RESTYPE = {"hhg_last_error": C.c_char_p, "hhg_learn_num_params": C.c_int64}


def declared_symbols():
    """Names declared in include/hhg.h (parsed from the header)."""
    import re

    hdr = open(os.path.join(os.path.dirname(HERE), "include", "hhg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(hhg_[a-z0-9_]+)\s*\(", hdr)))


def load(path=None):
    """Load libhhgs.so (raises if it is missing: the library has no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libhhgs.so not built (%s); run __graft_entry__.build()" % p)
    lib = C.CDLL(p)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, C.c_int)
    _lib = lib
    return lib


def _check(ctx, st):
    if st != HHG_OK:
        msg = _lib.hhg_last_error(ctx).decode() if ctx else ""
        raise HhgError(st, msg)


def _ptr(a):
    """Device/host address of a torch tensor, numpy array or int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(type(a))


def hhg_create(device=0, stream=0):
    lib = load()
    h = C.c_void_p()
    _check(None, lib.hhg_create(C.byref(h), device, stream or None))
    return h.value


def hhg_destroy(ctx):
    _check(None, load().hhg_destroy(ctx))


def hhg_last_error(ctx):
    return load().hhg_last_error(ctx).decode()


def hhg_set_timeout(ctx, ms):
    _check(ctx, load().hhg_set_timeout(ctx, int(ms)))


def hhg_set_macro_mesh(ctx, xyz, tets, dirichlet_face_flags=None):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int64)
    fl = None if dirichlet_face_flags is None else np.ascontiguousarray(dirichlet_face_flags, dtype=np.int32)
    _check(ctx, load().hhg_set_macro_mesh(ctx, xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, tets.shape[0],
                                          None if fl is None else fl.ctypes.data))


def hhg_refine(ctx, level_max):
    _check(ctx, load().hhg_refine(ctx, level_max))


def hhg_set_coarsest_level(ctx, level):
    _check(ctx, load().hhg_set_coarsest_level(ctx, int(level)))


def hhg_apply_2d(ctx, tri, level, nu, variant, dt, k, x, y):
    t = np.ascontiguousarray(np.asarray(tri, dtype=np.float64).reshape(6))
    _check(ctx, load().hhg_apply_2d(ctx, t.ctypes.data_as(C.c_void_p), int(level), float(nu), int(variant), int(dt),
                                    _ptr(k), _ptr(x), _ptr(y)))


def hhg_set_strain_fit(ctx, degree):
    _check(ctx, load().hhg_set_strain_fit(ctx, int(degree)))


def hhg_traction_load(ctx, level, dt, face_flags, t, f):
    fl = np.ascontiguousarray(np.asarray(face_flags, dtype=np.int32).reshape(-1))
    _check(ctx, load().hhg_traction_load(ctx, level, dt, fl.ctypes.data_as(C.c_void_p), _ptr(t), _ptr(f)))


def hhg_set_problem(ctx, kind=ELASTICITY, nu=0.3, variant=PHYSICAL, khat=KHAT_PATCH, iface=IFACE_SYMMETRIC):
    p = hhg_problem(kind, nu, variant, khat, iface)
    _check(ctx, load().hhg_set_problem(ctx, C.byref(p)))


def hhg_num_nodes(ctx, level):
    e, u, f = C.c_int64(), C.c_int64(), C.c_int64()
    _check(ctx, load().hhg_num_nodes(ctx, level, C.byref(e), C.byref(u), C.byref(f)))
    return e.value, u.value, f.value


def hhg_entry_coords(ctx, level):
    E, _, _ = hhg_num_nodes(ctx, level)
    out = np.empty((E, 3))
    _check(ctx, load().hhg_entry_coords(ctx, level, out.ctypes.data))
    return out


def hhg_entry_to_unique(ctx, level):
    E, U, _ = hhg_num_nodes(ctx, level)
    m = np.empty(E, dtype=np.int64)
    d = np.empty(U, dtype=np.int8)
    _check(ctx, load().hhg_entry_to_unique(ctx, level, m.ctypes.data, d.ctypes.data))
    return m, d.astype(bool)


def hhg_gather_unique(ctx, level, dt, comps, src, dst):
    _check(ctx, load().hhg_gather_unique(ctx, level, dt, comps, _ptr(src), _ptr(dst)))


def hhg_scatter_unique(ctx, level, dt, comps, src, dst):
    _check(ctx, load().hhg_scatter_unique(ctx, level, dt, comps, _ptr(src), _ptr(dst)))


def hhg_set_coefficient(ctx, k, dt):
    _check(ctx, load().hhg_set_coefficient(ctx, _ptr(k), dt))


def hhg_apply(ctx, level, dt, x, y):
    _check(ctx, load().hhg_apply(ctx, level, dt, _ptr(x), _ptr(y)))


def hhg_residual(ctx, level, dt, f, x, r, want_norm=False):
    nrm = C.c_double()
    _check(ctx, load().hhg_residual(ctx, level, dt, _ptr(f), _ptr(x), _ptr(r), C.byref(nrm) if want_norm else None))
    return nrm.value if want_norm else None


def hhg_apply_host(ctx, level, dt, x_host, y_host):
    _check(ctx, load().hhg_apply_host(ctx, level, dt, _ptr(x_host), _ptr(y_host)))


def hhg_profile(ctx, enable, read=False):
    """Start/stop kernel timing; with read=True returns ([interior_ms, skeleton_ms], [launches])."""
    if read:
        ms = np.zeros(2)
        nl = np.zeros(2, dtype=np.int64)
        _check(ctx, load().hhg_profile(ctx, int(enable), ms.ctypes.data, nl.ctypes.data))
        return ms, nl
    _check(ctx, load().hhg_profile(ctx, int(enable), None, None))
    return None


def hhg_set_interior_kernel(ctx, kernel):
    """0: direct global loads (FP32 on point pairs, packed arithmetic), 1: shared-memory tile."""
    _check(ctx, load().hhg_set_interior_kernel(ctx, int(kernel)))


def hhg_fp32_fma_probe(ctx, packed, iterations, out):
    """Launch the FP32 FMA issue-rate probe on the context's stream; returns (flops, sm_count)."""
    fl = C.c_double()
    sms = C.c_int()
    _check(ctx, load().hhg_fp32_fma_probe(ctx, int(packed), C.c_int64(int(iterations)), _ptr(out), C.byref(fl),
                                          C.byref(sms)))
    return fl.value, sms.value


def hhg_residual_noalloc(ctx, level, dt, f, x, r):
    """Residual and its squared norm with no device allocation (static scratch); returns the norm^2."""
    nrm = C.c_double()
    _check(ctx, load().hhg_residual_noalloc(ctx, level, dt, _ptr(f), _ptr(x), _ptr(r), C.byref(nrm)))
    return nrm.value


def hhg_set_mg_params(ctx, smoother=SMOOTH_CHEBYSHEV, pre=2, post=2, omega=2.0 / 3.0, cheby_lo=1.0 / 8.0,
                      cheby_hi=1.1, power_iters=15, coarse_coeff=0, uzawa_pre=3, uzawa_post=3, uzawa_extra=2,
                      uzawa_vsteps=2, uzawa_omega=0.5):
    p = hhg_mg_params(smoother, pre, post, omega, cheby_lo, cheby_hi, power_iters, coarse_coeff, uzawa_pre,
                      uzawa_post, uzawa_extra, uzawa_vsteps, uzawa_omega)
    _check(ctx, load().hhg_set_mg_params(ctx, C.byref(p)))


def hhg_mg_setup(ctx):
    _check(ctx, load().hhg_mg_setup(ctx))


def hhg_get_lambda_max(ctx, level):
    v = C.c_double()
    _check(ctx, load().hhg_get_lambda_max(ctx, level, C.byref(v)))
    return v.value


def hhg_set_lambda_max(ctx, level, lam):
    _check(ctx, load().hhg_set_lambda_max(ctx, level, float(lam)))


def hhg_diagonal(ctx, level, dt, d):
    _check(ctx, load().hhg_diagonal(ctx, level, dt, _ptr(d)))


def hhg_smooth(ctx, level, dt, steps, f, x):
    _check(ctx, load().hhg_smooth(ctx, level, dt, steps, _ptr(f), _ptr(x)))


def hhg_prolongate_add(ctx, fine_level, dt, xc, xf):
    _check(ctx, load().hhg_prolongate_add(ctx, fine_level, dt, _ptr(xc), _ptr(xf)))


def hhg_restrict(ctx, fine_level, dt, rf, rc):
    _check(ctx, load().hhg_restrict(ctx, fine_level, dt, _ptr(rf), _ptr(rc)))


def hhg_vcycle(ctx, level, dt, f, x):
    _check(ctx, load().hhg_vcycle(ctx, level, dt, _ptr(f), _ptr(x)))


def hhg_solve(ctx, f, x, method=SOLVE_MG_CG, level=None, dt=F64, rtol=1e-8, max_iter=200, inner_rtol=1e-3,
              inner_max_iter=50, allow_not_converged=False):
    """Returns the report as a dict; raises unless converged (or allow_not_converged)."""
    o = hhg_solve_opts(method, level, dt, rtol, max_iter, inner_rtol, inner_max_iter)
    rep = hhg_solve_report()
    st = load().hhg_solve(ctx, C.byref(o), _ptr(f), _ptr(x), C.byref(rep))
    if st == 5 and allow_not_converged:
        return rep.as_dict()
    _check(ctx, st)
    return rep.as_dict()


def hhg_stokes_apply(ctx, level, dt, x, y):
    _check(ctx, load().hhg_stokes_apply(ctx, level, dt, _ptr(x), _ptr(y)))


def hhg_stokes_residual(ctx, level, dt, f, x, r, want_norm=False):
    nrm = C.c_double()
    _check(ctx, load().hhg_stokes_residual(ctx, level, dt, _ptr(f), _ptr(x), _ptr(r),
                                           C.byref(nrm) if want_norm else None))
    return nrm.value if want_norm else None


def hhg_carreau_viscosity(ctx, level, u, mu, eta0=1.0, eta_inf=1e-3, kappa=1.0, r=-0.25):
    p = hhg_carreau(eta0, eta_inf, kappa, r)
    _check(ctx, load().hhg_carreau_viscosity(ctx, level, C.byref(p), _ptr(u), _ptr(mu)))


def hhg_picard(ctx, f, x, level, eta0=1.0, eta_inf=1e-3, kappa=1.0, r=-0.25, picard_tol=1e-3, max_picard=30,
               step_rtol=1e-2, step_max_iter=50, final_rtol=1e-3, allow_not_converged=False):
    o = hhg_picard_opts(hhg_carreau(eta0, eta_inf, kappa, r), level, picard_tol, max_picard, step_rtol,
                        step_max_iter, final_rtol)
    rep = hhg_picard_report()
    st = load().hhg_picard(ctx, C.byref(o), _ptr(f), _ptr(x), C.byref(rep))
    if st == 5 and allow_not_converged:
        return rep.as_dict()
    _check(ctx, st)
    return rep.as_dict()


def hhg_learn_num_params():
    return int(load().hhg_learn_num_params())


def hhg_learn_set_conv_kernel(ctx, kernel):
    """0: warp-level MMA convolution (default), 1: tcgen05 per tile, 2: TMA + tcgen05 pipeline."""
    _check(ctx, load().hhg_learn_set_conv_kernel(ctx, int(kernel)))


def hhg_learn_set_conv_wait(ctx, polls):
    """Bound (polls) of the tensor-core convolution's wait for its MMAs; negative: the default."""
    _check(ctx, load().hhg_learn_set_conv_wait(ctx, C.c_int64(int(polls))))


def hhg_learn_init(ctx, seed=0):
    _check(ctx, load().hhg_learn_init(ctx, int(seed)))


def hhg_learn_get_params(ctx):
    n = hhg_learn_num_params()
    out = np.empty(n, dtype=np.float32)
    _check(ctx, load().hhg_learn_get_params(ctx, out.ctypes.data, n))
    return out


def hhg_learn_set_params(ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, load().hhg_learn_set_params(ctx, p.ctypes.data, p.size))


def hhg_learn_grid(ctx, level):
    """((D, H, W), number of voxels holding a free node) of the level's node grid."""
    dhw = np.zeros(3, dtype=np.int32)
    nf = C.c_int64()
    _check(ctx, load().hhg_learn_grid(ctx, level, dhw.ctypes.data, C.byref(nf)))
    return tuple(int(v) for v in dhw), nf.value


def hhg_learn_set_coarsening(ctx, levels):
    _check(ctx, load().hhg_learn_set_coarsening(ctx, int(levels)))


def hhg_learn_channels(ctx):
    """(input, output) channels of the network for the context's problem kind."""
    ci, co = C.c_int(), C.c_int()
    _check(ctx, load().hhg_learn_channels(ctx, C.byref(ci), C.byref(co)))
    return ci.value, co.value


def hhg_learn_forward(ctx, x, cin, B, D, H, W, out, cout=3):
    _check(ctx, load().hhg_learn_forward(ctx, _ptr(x), cin, cout, B, D, H, W, _ptr(out)))


def hhg_learn_loss_grad(ctx, x, cin, target, B, D, H, W, cout=3):
    """(loss, gradient as FP32 numpy array in the parameter layout)."""
    loss = C.c_double()
    g = np.empty(hhg_learn_num_params(), dtype=np.float32)
    _check(ctx, load().hhg_learn_loss_grad(ctx, _ptr(x), cin, _ptr(target), cout, B, D, H, W, C.byref(loss),
                                           g.ctypes.data))
    return loss.value, g


def hhg_learn_reserve_pairs(ctx, level, capacity):
    _check(ctx, load().hhg_learn_reserve_pairs(ctx, level, int(capacity)))


def hhg_learn_collect(ctx, level, e0_grid, cycles):
    n = C.c_int64()
    _check(ctx, load().hhg_learn_collect(ctx, level, _ptr(e0_grid), cycles, C.byref(n)))
    return n.value


def hhg_learn_collect_cg(ctx, level, f, iters):
    n = C.c_int64()
    _check(ctx, load().hhg_learn_collect_cg(ctx, level, _ptr(f), iters, C.byref(n)))
    return n.value


def hhg_learn_get_pair(ctx, index, dhw, nc=3):
    """(inputs FP32 (D, H, W, 2 nc + 1), targets FP32 (D, H, W, nc)) of stored pair `index`
    (nc = 3 elasticity, 4 Stokes)."""
    D, H, W = dhw
    x = np.empty((D, H, W, 2 * nc + 1), dtype=np.float32)
    y = np.empty((D, H, W, nc), dtype=np.float32)
    _check(ctx, load().hhg_learn_get_pair(ctx, int(index), x.ctypes.data, y.ctypes.data))
    return x, y


def hhg_learn_train(ctx, steps, batch, crop, lr=2e-3, seed=0):
    o = hhg_learn_train_opts(steps, batch, crop, lr, seed)
    rep = hhg_learn_train_report()
    _check(ctx, load().hhg_learn_train(ctx, C.byref(o), C.byref(rep)))
    return rep.as_dict()


def hhg_learn_precondition(ctx, level, use_net, r, z):
    """z = a multigrid step + b correction (FP32 library-layout vectors); returns b / a."""
    a = C.c_double()
    _check(ctx, load().hhg_learn_precondition(ctx, level, int(use_net), _ptr(r), _ptr(z), C.byref(a)))
    return a.value


def hhg_learn_stats(ctx, reset=False):
    rep = hhg_learn_stats_report()
    _check(ctx, load().hhg_learn_stats(ctx, C.byref(rep), int(reset)))
    return rep.as_dict()
