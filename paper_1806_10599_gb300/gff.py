"""Thin ctypes binding of libgff.so (include/gff.h): same names, argument
marshalling only.  Every computation happens in the CUDA library; importing
this module fails loudly when libgff.so has not been built.

Host arrays are numpy arrays (converted to contiguous float64 / int32 /
uint8 as the C signature requires).  Device arguments (`*_dev`) are torch
CUDA tensors (or raw integer addresses).
"""

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgff.so")

GFF_OK = 0
GFF_ERR_ARG = -1
GFF_ERR_OOM = -2
GFF_ERR_CUDA = -3
GFF_ERR_NO_CONVERGENCE = -4
GFF_ERR_CP_FAIL = -5
GFF_ERR_TIMEOUT = -6
GFF_ERR_STATE = -7
GFF_ERR_IO = -8

GFF_PROJ_CONTINUOUS, GFF_PROJ_DISCRETE = 0, 1
GFF_WARM_OFF, GFF_WARM_NET_IF_BETTER, GFF_WARM_NET, GFF_WARM_EXTRAPOLATE = 0, 1, 2, 3
UNET_IN = 32  # input channels of the warm-start network
GFF_PREC_FP64, GFF_PREC_MIXED = 0, 1
GFF_RETURN_MAP_DEFAULT, GFF_RETURN_MAP_EXACT, GFF_RETURN_MAP_F32_FIRST, GFF_RETURN_MAP_FP64 = 0, 1, 2, 3
GFF_STRAIN_FINITE, GFF_STRAIN_SMALL = 0, 1
GFF_MAT_SVK_CUBIC, GFF_MAT_SVK_ISO, GFF_MAT_CP_FCC, GFF_MAT_NEOHOOKE = 0, 1, 2, 3
(GFF_FIELD_F, GFF_FIELD_P, GFF_FIELD_K, GFF_FIELD_FP_INV, GFF_FIELD_CHI,
 GFF_FIELD_GAMMA, GFF_FIELD_PCYC, GFF_FIELD_WCYC) = range(8)
FIELD_COMPONENTS = {0: 9, 1: 9, 2: 81, 3: 9, 4: 12, 5: 12, 6: 1, 7: 12}

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class gff_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("L", c_double * 3)]


class gff_material(ctypes.Structure):
    _fields_ = [("kind", c_int)] + [
        (n, c_double) for n in ("C11", "C12", "C44", "E", "nu", "gdot0", "p_exp", "tau0", "c_af", "d_af")
    ]


class gff_options(ctypes.Structure):
    _fields_ = [
        ("projection", c_int),
        ("precision", c_int),
        ("newton_tol", c_double),
        ("cg_tol", c_double),
        ("newton_max", c_int),
        ("cg_max", c_int),
        ("max_cuts", c_int),
        ("warm_start", c_int),
        ("fs_k", c_double),
        ("fs_sigma_y", c_double),
    ]


class gff_step_report(ctypes.Structure):
    _fields_ = [
        ("newton_iters", c_int),
        ("cg_iters", c_int),
        ("cuts", c_int),
        ("residual", c_double),
        ("Pmacro", c_double * 9),
        ("Fmacro", c_double * 9),
        ("seconds", c_double),
        ("t_constitutive", c_double),
        ("t_residual", c_double),
        ("t_linear", c_double),
        ("warm_start_used", c_int),
        ("residual_first", c_double),
        ("cp_fallbacks", c_int),
        ("cp_local_iters", c_double),
        ("t_tangent", c_double),
    ]


class gff_auto_options(ctypes.Structure):
    _fields_ = [("dt_initial", c_double), ("dt_min", c_double), ("dt_max", c_double), ("grow", c_double),
                ("shrink", c_double), ("easy_newton", c_int), ("hard_newton", c_int)]


class GffError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gff status %d: %s" % (status, msg))
        self.status = status


_P = ctypes.POINTER
_SIGS = {
    "gff_options_default": (None, [_P(gff_options)]),
    "gff_create": (c_int, [_P(gff_grid), _P(gff_options), _P(c_void_p)]),
    "gff_destroy": (None, [c_void_p]),
    "gff_last_error": (ctypes.c_char_p, [c_void_p]),
    "gff_set_stream": (c_int, [c_void_p, c_void_p]),
    "gff_set_options": (c_int, [c_void_p, _P(gff_options)]),
    "gff_set_microstructure": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "gff_set_material": (c_int, [c_void_p, c_int, _P(gff_material)]),
    "gff_set_field": (c_int, [c_void_p, c_int, c_void_p]),
    "gff_get_field": (c_int, [c_void_p, c_int, c_void_p]),
    "gff_constitutive": (c_int, [c_void_p, c_double]),
    "gff_apply_operator": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "gff_project": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "gff_apply_operator_timed": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gff_autotune": (c_int, [c_void_p, c_void_p]),
    "gff_set_tiles": (c_int, [c_void_p, c_void_p]),
    "gff_project_noalloc": (c_int, [_P(gff_grid), c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gff_sync": (c_int, [c_void_p]),
    "gff_apply_operator_host": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "gff_cg_kernels_timed": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "gff_measure_fp64_peak": (c_int, [c_void_p, c_void_p]),
    "gff_set_wait_limit": (c_int, [c_void_p, ctypes.c_longlong]),
    "gff_set_return_map": (c_int, [c_void_p, c_int]),
    "gff_set_strain_measure": (c_int, [c_void_p, c_int]),
    "gff_step": (c_int, [c_void_p, c_double, c_void_p, c_void_p, c_void_p, _P(gff_step_report)]),
    "gff_run_history": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p]),
    "gff_batch_run": (c_int, [c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p]),
    "gff_auto_options_default": (None, [_P(gff_auto_options)]),
    "gff_run_auto": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                             _P(gff_auto_options), c_int, _P(c_int), c_void_p, c_void_p, c_void_p]),
    "gff_unet_create": (c_int, [ctypes.c_uint64, _P(c_void_p)]),
    "gff_unet_destroy": (None, [c_void_p]),
    "gff_unet_last_error": (ctypes.c_char_p, [c_void_p]),
    "gff_unet_num_params": (ctypes.c_size_t, [c_void_p]),
    "gff_unet_get_params": (c_int, [c_void_p, c_void_p]),
    "gff_unet_set_params": (c_int, [c_void_p, c_void_p]),
    "gff_unet_save": (c_int, [c_void_p, ctypes.c_char_p]),
    "gff_unet_load": (c_int, [c_void_p, ctypes.c_char_p]),
    "gff_unet_eval_host": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gff_unet_add_sample": (c_int, [c_void_p, c_void_p]),
    "gff_unet_add_sample_host": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "gff_unet_num_samples": (c_int, [c_void_p]),
    "gff_unet_set_sampling": (c_int, [c_void_p, c_int]),
    "gff_unet_train": (c_int, [c_void_p, c_int, c_double, c_void_p]),
    "gff_set_warm_start": (c_int, [c_void_p, c_void_p, c_int]),
    "gff_reset_fips": (c_int, [c_void_p]),
    "gff_get_fips": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "gff_get_band_fips": (c_int, [c_void_p, c_double, c_void_p, c_void_p]),
    "gff_umat_tangent": (c_int, [ctypes.c_longlong, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gff_save_state": (c_int, [c_void_p, ctypes.c_char_p]),
    "gff_load_state": (c_int, [c_void_p, ctypes.c_char_p]),
}


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libgff.so not built (%s): run `python -m paper_1806_10599_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _check(h, st):
    if st != GFF_OK:
        msg = _lib.gff_last_error(h)
        raise GffError(st, msg.decode() if msg else "")
    return st


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(c_void_p)


def _dev(t):
    if isinstance(t, int):
        return c_void_p(t)
    return c_void_p(t.data_ptr())


# --------------------------------------------------------------------------- same-name wrappers
def gff_options_default():
    o = gff_options()
    _lib.gff_options_default(ctypes.byref(o))
    return o


def gff_create(grid, opt=None):
    h = c_void_p()
    st = _lib.gff_create(ctypes.byref(grid), ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    if st != GFF_OK:
        msg = _lib.gff_last_error(h).decode() if h.value else ""
        if h.value:
            _lib.gff_destroy(h)
        raise GffError(st, msg)
    return h


def gff_destroy(h):
    _lib.gff_destroy(h)


def gff_last_error(h):
    return _lib.gff_last_error(h).decode()


def gff_set_stream(h, stream):
    s = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", 0)
    return _check(h, _lib.gff_set_stream(h, c_void_p(s)))


def gff_set_options(h, opt):
    return _check(h, _lib.gff_set_options(h, ctypes.byref(opt)))


def gff_set_microstructure(h, grain_id, ngrains, quat, grain_phase):
    g, gp = _host(grain_id, np.int32)
    q, qp = _host(quat, np.float64)
    p, pp = _host(grain_phase, np.int32)
    return _check(h, _lib.gff_set_microstructure(h, gp, int(ngrains), qp, pp))


def gff_set_material(h, phase, mat):
    return _check(h, _lib.gff_set_material(h, int(phase), ctypes.byref(mat)))


def gff_set_field(h, which, host):
    a, ap = _host(host, np.float64)
    return _check(h, _lib.gff_set_field(h, int(which), ap))


def gff_get_field(h, which, n_voxels):
    out = np.empty(FIELD_COMPONENTS[which] * n_voxels)
    _check(h, _lib.gff_get_field(h, int(which), out.ctypes.data_as(c_void_p)))
    return out


def gff_constitutive(h, dt):
    return _check(h, _lib.gff_constitutive(h, float(dt)))


def _mask(mask9):
    if mask9 is None:
        return None, None
    return _host(mask9, np.uint8)


def gff_apply_operator(h, precision, mask9, x_dev, y_dev):
    m, mp = _mask(mask9)
    return _check(h, _lib.gff_apply_operator(h, int(precision), mp, _dev(x_dev), _dev(y_dev)))


def gff_apply_operator_timed(h, precision, mask9, x_dev, y_dev):
    """Returns the three kernel durations (ms) of one apply."""
    m, mp = _mask(mask9)
    ms = (ctypes.c_float * 3)()
    _check(h, _lib.gff_apply_operator_timed(h, int(precision), mp, _dev(x_dev), _dev(y_dev),
                                            ctypes.cast(ms, c_void_p)))
    return [ms[0], ms[1], ms[2]]


def gff_autotune(h):
    """Returns {fwd threads, z columns, z threads, inv threads, inv persistent blocks, TMA z blocks}
    for FP64 and FP32."""
    t = (ctypes.c_int * 12)()
    _check(h, _lib.gff_autotune(h, ctypes.cast(t, c_void_p)))
    return {"fp64": list(t[0:5]) + [t[10]], "fp32": list(t[5:10]) + [t[11]]}


def gff_set_tiles(h, fp64, fp32):
    """Launch shapes in the layout gff_autotune returns: 6 ints per precision."""
    t = (ctypes.c_int * 12)(*(list(fp64[:5]) + list(fp32[:5]) + [fp64[5], fp32[5]]))
    return _check(h, _lib.gff_set_tiles(h, ctypes.cast(t, c_void_p)))


def gff_project(h, precision, mask9, x_dev, y_dev):
    m, mp = _mask(mask9)
    return _check(h, _lib.gff_project(h, int(precision), mp, _dev(x_dev), _dev(y_dev)))


def gff_project_noalloc(grid, projection, precision, mask9, x_dev, y_dev, stream=0):
    """y = G_M(x) without any device allocation (scratch inside libgff.so;
    at most 32768 voxels; overlapping calls race -- see gff.h)."""
    m, mp = _mask(mask9)
    s = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", 0)
    st = _lib.gff_project_noalloc(ctypes.byref(grid), int(projection), int(precision), mp, _dev(x_dev),
                                  _dev(y_dev), c_void_p(s))
    if st != GFF_OK:
        raise GffError(st, "gff_project_noalloc failed")
    return st


def gff_apply_operator_host(h, precision, mask9, x_host, y_host):
    """x_host, y_host: host tensors/arrays (pinned torch tensors give asynchronous copies)."""
    m, mp = _mask(mask9)
    return _check(h, _lib.gff_apply_operator_host(h, int(precision), mp, _hostptr(x_host), _hostptr(y_host)))


def _hostptr(a):
    if hasattr(a, "data_ptr"):
        return c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(c_void_p)
    return c_void_p(int(a))


def gff_cg_kernels_timed(h, precision, reps=10):
    ms = (ctypes.c_float * 3)()
    _check(h, _lib.gff_cg_kernels_timed(h, int(precision), int(reps), ctypes.cast(ms, c_void_p)))
    return [ms[0], ms[1], ms[2]]


def gff_measure_fp64_peak():
    """Returns (GFLOP/s, ms of the best launch)."""
    gf, ms = c_double(), c_double()
    st = _lib.gff_measure_fp64_peak(ctypes.byref(gf), ctypes.byref(ms))
    if st != GFF_OK:
        raise GffError(st, "gff_measure_fp64_peak failed")
    return gf.value, ms.value


def gff_sync(h):
    return _check(h, _lib.gff_sync(h))


def gff_set_wait_limit(h, cycles):
    return _check(h, _lib.gff_set_wait_limit(h, int(cycles)))


def gff_set_strain_measure(h, mode):
    return _check(h, _lib.gff_set_strain_measure(h, int(mode)))


def gff_set_return_map(h, mode):
    return _check(h, _lib.gff_set_return_map(h, int(mode)))


def gff_step(h, dt, Fbar, mask, Pbar):
    f, fp = _host(Fbar, np.float64)
    m, mp = _host(mask, np.uint8)
    p, pp = _host(Pbar, np.float64)
    rep = gff_step_report()
    _check(h, _lib.gff_step(h, float(dt), fp, mp, pp, ctypes.byref(rep)))
    return rep


def gff_run_history(h, dt, Fbar, mask, Pbar, cycle_start=None):
    n = int(np.asarray(dt).shape[0])
    d, dp = _host(dt, np.float64)
    f, fp = _host(Fbar, np.float64)
    m, mp = _host(mask, np.uint8)
    p, pp = _host(Pbar, np.float64)
    cs, csp = _host(cycle_start, np.uint8) if cycle_start is not None else (None, None)
    Pm = np.zeros((n, 9))
    reps = (gff_step_report * max(n, 1))()
    _check(h, _lib.gff_run_history(h, n, dp, fp, mp, pp, csp, Pm.ctypes.data_as(c_void_p),
                                   ctypes.cast(reps, c_void_p)))
    return Pm, [reps[k] for k in range(n)]


def gff_auto_options_default(**kw):
    a = gff_auto_options()
    _lib.gff_auto_options_default(ctypes.byref(a))
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def gff_run_auto(h, t_knots, Fbar_knots, mask, Pbar_knots, cycle_start=None, options=None, max_increments=10000):
    """Automatic time incrementation along a piecewise-linear path.  Returns
    (end times [n], Pmacro [n][9], reports [n])."""
    nk = int(np.asarray(t_knots).shape[0])
    t, tp = _host(t_knots, np.float64)
    f, fp = _host(Fbar_knots, np.float64)
    m, mp = _host(mask, np.uint8)
    p, pp = _host(Pbar_knots, np.float64)
    cs, csp = _host(cycle_start, np.uint8) if cycle_start is not None else (None, None)
    ao = options if options is not None else gff_auto_options_default()
    n = c_int(0)
    tout = np.zeros(max_increments)
    Pm = np.zeros((max_increments, 9))
    reps = (gff_step_report * max_increments)()
    _check(h, _lib.gff_run_auto(h, nk, tp, fp, mp, pp, csp, ctypes.byref(ao), int(max_increments), ctypes.byref(n),
                                tout.ctypes.data_as(c_void_p), Pm.ctypes.data_as(c_void_p), ctypes.cast(reps, c_void_p)))
    k = n.value
    return tout[:k].copy(), Pm[:k].copy(), [reps[i] for i in range(k)]


def gff_batch_run(handles, dt, Fbar, mask, Pbar, cycle_start=None, raise_on_error=True):
    """Runs all handles through one history together.  Returns (Pmacro
    [n][nsteps][9], reports [n][nsteps], per-RVE status array)."""
    n = len(handles)
    hs = (c_void_p * n)(*[h.value for h in handles])
    ns = int(np.asarray(dt).shape[0])
    d, dp = _host(dt, np.float64)
    f, fp = _host(Fbar, np.float64)
    m, mp = _host(mask, np.uint8)
    p, pp = _host(Pbar, np.float64)
    cs, csp = _host(cycle_start, np.uint8) if cycle_start is not None else (None, None)
    Pm = np.zeros((n, ns, 9))
    reps = (gff_step_report * max(n * ns, 1))()
    stat = np.zeros(n, dtype=np.int32)
    st = _lib.gff_batch_run(n, ctypes.cast(hs, c_void_p), ns, dp, fp, mp, pp, csp, Pm.ctypes.data_as(c_void_p),
                            ctypes.cast(reps, c_void_p), stat.ctypes.data_as(c_void_p))
    if st != GFF_OK and raise_on_error:
        raise GffError(st, "gff_batch_run: per-RVE status %s; %s" % (stat.tolist(), gff_last_error(handles[0])))
    return Pm, [[reps[r * ns + k] for k in range(ns)] for r in range(n)], stat


def _ucheck(u, st):
    if st != GFF_OK:
        msg = _lib.gff_unet_last_error(u)
        raise GffError(st, msg.decode() if msg else "")
    return st


def gff_unet_create(seed=0):
    u = c_void_p()
    st = _lib.gff_unet_create(ctypes.c_uint64(seed), ctypes.byref(u))
    if st != GFF_OK:
        msg = _lib.gff_unet_last_error(u).decode() if u.value else ""
        if u.value:
            _lib.gff_unet_destroy(u)
        raise GffError(st, msg)
    return u


def gff_unet_destroy(u):
    _lib.gff_unet_destroy(u)


def gff_unet_last_error(u):
    return _lib.gff_unet_last_error(u).decode()


def gff_unet_num_params(u):
    return int(_lib.gff_unet_num_params(u))


def gff_unet_get_params(u):
    w = np.empty(gff_unet_num_params(u), dtype=np.float32)
    _ucheck(u, _lib.gff_unet_get_params(u, w.ctypes.data_as(c_void_p)))
    return w


def gff_unet_set_params(u, w):
    a, ap = _host(w, np.float32)
    return _ucheck(u, _lib.gff_unet_set_params(u, ap))


def gff_unet_save(u, path):
    return _ucheck(u, _lib.gff_unet_save(u, str(path).encode()))


def gff_unet_load(u, path):
    return _ucheck(u, _lib.gff_unet_load(u, str(path).encode()))


def gff_unet_eval_host(u, n, x, target=None):
    """x [V][UNET_IN] -> y [V][9]; with a target also (loss, grads)."""
    V = n ** 3
    xa, xp = _host(np.asarray(x).reshape(V, UNET_IN), np.float32)
    y = np.empty((V, 9), dtype=np.float32)
    if target is None:
        _ucheck(u, _lib.gff_unet_eval_host(u, n, xp, None, y.ctypes.data_as(c_void_p), None, None))
        return y
    ta, tp = _host(np.asarray(target).reshape(V, 9), np.float32)
    loss = c_double()
    grads = np.empty(gff_unet_num_params(u), dtype=np.float32)
    _ucheck(u, _lib.gff_unet_eval_host(u, n, xp, tp, y.ctypes.data_as(c_void_p), ctypes.byref(loss),
                                       grads.ctypes.data_as(c_void_p)))
    return y, loss.value, grads


def gff_unet_add_sample(u, h):
    return _ucheck(u, _lib.gff_unet_add_sample(u, h))


def gff_unet_add_sample_host(u, n, x, target):
    """x [V][UNET_IN], target [V][9] on an n^3 grid."""
    V = n ** 3
    xa, xp = _host(np.asarray(x).reshape(V, UNET_IN), np.float32)
    ta, tp = _host(np.asarray(target).reshape(V, 9), np.float32)
    return _ucheck(u, _lib.gff_unet_add_sample_host(u, int(n), xp, tp))


def gff_unet_set_sampling(u, mode):
    return _ucheck(u, _lib.gff_unet_set_sampling(u, int(mode)))


def gff_unet_num_samples(u):
    return int(_lib.gff_unet_num_samples(u))


def gff_unet_train(u, steps, lr):
    losses = np.zeros(max(steps, 1))
    _ucheck(u, _lib.gff_unet_train(u, int(steps), float(lr), losses.ctypes.data_as(c_void_p)))
    return losses[:steps]


def gff_set_warm_start(h, u, mode):
    return _check(h, _lib.gff_set_warm_start(h, u, int(mode)))


def gff_reset_fips(h):
    return _check(h, _lib.gff_reset_fips(h))


def gff_get_fips(h, ngrains):
    pc = np.zeros(ngrains)
    w = np.zeros((ngrains, 12))
    fs = np.zeros(ngrains)
    _check(h, _lib.gff_get_fips(h, pc.ctypes.data_as(c_void_p), w.ctypes.data_as(c_void_p),
                                fs.ctypes.data_as(c_void_p)))
    return pc, w, fs


def gff_umat_tangent(n, F_dev, sigma_dev, Cab_dev, P_dev, K_dev, stream=0):
    s = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", 0)
    st = _lib.gff_umat_tangent(int(n), _dev(F_dev), _dev(sigma_dev), _dev(Cab_dev), _dev(P_dev), _dev(K_dev),
                               c_void_p(s))
    if st != GFF_OK:
        raise GffError(st, "gff_umat_tangent failed")
    return st


def gff_get_band_fips(h, width, ngrains):
    """Band-averaged W_cyc per grain and its maximum over the RVE."""
    wb = np.zeros(ngrains)
    mx = c_double()
    _check(h, _lib.gff_get_band_fips(h, float(width), wb.ctypes.data_as(c_void_p), ctypes.byref(mx)))
    return wb, mx.value


def gff_save_state(h, path):
    return _check(h, _lib.gff_save_state(h, str(path).encode()))


def gff_load_state(h, path):
    return _check(h, _lib.gff_load_state(h, str(path).encode()))


# --------------------------------------------------------------------------- convenience
def make_grid(nx, ny, nz, L=(1.0, 1.0, 1.0)):
    g = gff_grid()
    g.nx, g.ny, g.nz = nx, ny, nz
    g.L[0], g.L[1], g.L[2] = L
    return g


def make_options(**kw):
    o = gff_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_material(kind, C11=168.4e9, C12=121.4e9, C44=75.4e9, E=400e9, nu=0.2, gdot0=1e-3, p_exp=20.0,
                  tau0=50e6, c_af=20e9, d_af=200.0):
    m = gff_material()
    m.kind = kind
    m.C11, m.C12, m.C44, m.E, m.nu = C11, C12, C44, E, nu
    m.gdot0, m.p_exp, m.tau0, m.c_af, m.d_af = gdot0, p_exp, tau0, c_af, d_af
    return m


def create_rve(ms, materials, options=None, small_strain=False):
    """Handle for a rve_inputs.Microstructure with {phase: gff_material}."""
    h = gff_create(make_grid(ms.nx, ms.ny, ms.nz, ms.L), options)
    try:
        if small_strain:
            gff_set_strain_measure(h, GFF_STRAIN_SMALL)
        for ph, m in materials.items():
            gff_set_material(h, ph, m)
        gff_set_microstructure(h, ms.grain_id.reshape(-1), ms.ngrains, ms.quat, ms.phase)
    except Exception:
        gff_destroy(h)
        raise
    return h
