"""Thin ctypes binding of libcolapm.so (argument marshalling only).

The functions carry the C names of ``include/colapm.h``. Array arguments may be numpy
arrays (host) or torch tensors (host or CUDA); they must be C-contiguous with the dtype
the C call expects. Every call raises ``ColapmError`` on a non-zero return code.
There is no CPU fallback: importing this module fails when the library is missing.
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libcolapm.so")

PHASES = ["deposit", "fft_fwd", "poisson", "fft_inv", "gather", "ics", "power", "fft_inv_x", "sort"]


class ColapmError(RuntimeError):
    def __init__(self, code, call):
        super().__init__(f"{call} failed: {code} ({strerror(code)})")
        self.code = code


class Cosmo(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("omega_b", ctypes.c_double), ("h", ctypes.c_double),
                ("n_s", ctypes.c_double), ("sigma8", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("cosmo", Cosmo), ("box", ctypes.c_double), ("np", ctypes.c_int), ("nm", ctypes.c_int),
                ("z_init", ctypes.c_double), ("z_final", ctypes.c_double), ("n_steps", ctypes.c_int),
                ("spacing", ctypes.c_int), ("stepping", ctypes.c_int), ("nlpt", ctypes.c_double),
                ("cola", ctypes.c_int), ("deconv", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


class NNConfig(ctypes.Structure):
    _fields_ = [("s_in", ctypes.c_float), ("s_out", ctypes.c_float), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("engine", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


class Lightcone(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("z_max", ctypes.c_double), ("rep_lo", ctypes.c_int * 3),
                ("rep_hi", ctypes.c_int * 3)]


# rows of colapm_get_lightcone (colapm_lc_particle)
LC_DTYPE = np.dtype([("x", np.float32), ("y", np.float32), ("z", np.float32), ("a", np.float32),
                     ("px", np.float32), ("py", np.float32), ("pz", np.float32), ("id", np.int32)])

NN_PARAMS = 16467


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libcolapm.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "colapm_default_params": (None, [ctypes.POINTER(Params)]),
        "colapm_create": (I, [ctypes.POINTER(Params), P, ctypes.POINTER(P)]),
        "colapm_destroy": (None, [P]),
        "colapm_make_ics": (I, [P]),
        "colapm_set_displacements": (I, [P, P, P]),
        "colapm_step": (I, [P, I]),
        "colapm_finalize": (I, [P]),
        "colapm_power": (I, [P, I, D, D, P, P, P]),
        "colapm_cross_correlation": (I, [P, P, I, D, D, P, P, P]),
        "colapm_power_rsd": (I, [P, I, I, D, D, P, P, P]),
        "colapm_set_fnl": (I, [P, D]),
        "colapm_set_lightcone": (I, [P, P, ctypes.c_longlong]),
        "colapm_get_lightcone": (I, [P, P, P, ctypes.c_longlong, P]),
        "colapm_get_particles": (I, [P, P, P]),
        "colapm_get_particles_async": (I, [P, P, P]),
        "colapm_wait_particles": (I, [P]),
        "colapm_get_state": (I, [P, P, P, P]),
        "colapm_set_state": (I, [P, P, P, P]),
        "colapm_get_density": (I, [P, P]),
        "colapm_get_force": (I, [P, P]),
        "colapm_get_lpt": (I, [P, P, P]),
        "colapm_get_gaussian_field": (I, [P, P]),
        "colapm_sync": (I, [P]),
        "colapm_reseed": (I, [P, ctypes.c_ulonglong]),
        "colapm_kernel_launches": (ctypes.c_longlong, [P]),
        "colapm_steps_done": (I, [P]),
        "colapm_save_state": (I, [P, P, ctypes.POINTER(Z)]),
        "colapm_load_state": (I, [P, P, Z]),
        "colapm_set_timing": (I, [P, I]),
        "colapm_get_timing": (I, [P, P, P]),
        "colapm_strerror": (ctypes.c_char_p, [I]),
        "colapm_power_noalloc": (I, [P, P, ctypes.c_longlong, I, D, I, D, D, P, P, P, P]),
        "colapm_autotune": (I, [P, P]),
        "colapm_set_engine": (I, [P, I, I, I]),
        "colapm_set_plan": (I, [P, I]),
        "colapm_get_config": (I, [P, P]),
        "colapm_set_sort": (I, [P, I]),
        "colapm_set_deposit_tiles": (I, [P, I]),
        "colapm_set_sort_tiles": (I, [P, I]),
        "colapm_batch_create": (I, [I, P, I, P, ctypes.POINTER(P)]),
        "colapm_batch_run": (I, [P, P, I, D, D, P, P, P]),
        "colapm_batch_streams": (I, [P]),
        "colapm_batch_set_lockstep": (I, [P, I]),
        "colapm_batch_destroy": (None, [P]),
        "colapm_get_displacement": (I, [P, P]),
        "colapm_set_displacement": (I, [P, P]),
        "colapm_nn_default_config": (None, [ctypes.POINTER(NNConfig)]),
        "colapm_nn_create": (I, [I, ctypes.POINTER(NNConfig), P, ctypes.POINTER(P)]),
        "colapm_nn_destroy": (I, [P]),
        "colapm_nn_set_params": (I, [P, P]),
        "colapm_nn_get_params": (I, [P, P]),
        "colapm_nn_forward": (I, [P, P, P, I]),
        "colapm_nn_grads": (I, [P, P, P, P, ctypes.POINTER(D)]),
        "colapm_nn_train_step": (I, [P, P, P, ctypes.POINTER(D)]),
        "colapm_nn_steps": (I, [P]),
        "colapm_nn_launches": (ctypes.c_longlong, [P]),
        "colapm_nn_sync": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()
EXPORTED = [n for n in dir(LIB) if n.startswith("colapm_")]


def strerror(code):
    return LIB.colapm_strerror(code).decode()


def _check(code, call):
    if code != 0:
        raise ColapmError(code, call)


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def default_params(**kw):
    p = Params()
    LIB.colapm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("omega_m", "omega_b", "h", "n_s", "sigma8"):
            setattr(p.cosmo, k, v)
        else:
            setattr(p, k, v)
    return p


def colapm_create(params, stream=0):
    ctx = ctypes.c_void_p()
    _check(LIB.colapm_create(ctypes.byref(params), ctypes.c_void_p(stream or None), ctypes.byref(ctx)),
           "colapm_create")
    return ctx


def colapm_destroy(ctx):
    LIB.colapm_destroy(ctx)


def colapm_make_ics(ctx):
    _check(LIB.colapm_make_ics(ctx), "colapm_make_ics")


def colapm_set_displacements(ctx, psi1, psi2):
    _check(LIB.colapm_set_displacements(ctx, _ptr(psi1), _ptr(psi2)), "colapm_set_displacements")


def colapm_step(ctx, k=-1):
    _check(LIB.colapm_step(ctx, k), "colapm_step")


def colapm_finalize(ctx):
    _check(LIB.colapm_finalize(ctx), "colapm_finalize")


def colapm_power(ctx, nbins, kmin=0.0, kmax=0.0, k_out=None, p_out=None, n_out=None):
    k_out = np.empty(nbins) if k_out is None else k_out
    p_out = np.empty(nbins) if p_out is None else p_out
    n_out = np.empty(nbins, dtype=np.int64) if n_out is None else n_out
    _check(LIB.colapm_power(ctx, nbins, kmin, kmax, _ptr(k_out), _ptr(p_out), _ptr(n_out)), "colapm_power")
    return k_out, p_out, n_out


def colapm_set_lightcone(ctx, origin=None, z_max=1.0, rep_lo=(0, 0, 0), rep_hi=(0, 0, 0), capacity=0):
    """origin None turns the lightcone off."""
    if origin is None:
        _check(LIB.colapm_set_lightcone(ctx, None, 0), "colapm_set_lightcone")
        return
    lc = Lightcone()
    for j in range(3):
        lc.origin[j] = float(origin[j])
        lc.rep_lo[j] = int(rep_lo[j])
        lc.rep_hi[j] = int(rep_hi[j])
    lc.z_max = float(z_max)
    _check(LIB.colapm_set_lightcone(ctx, ctypes.byref(lc), int(capacity)), "colapm_set_lightcone")


def colapm_get_lightcone(ctx, max_rows=None):
    """(count, rows): rows is a numpy structured array (LC_DTYPE) of the stored rows; raises
    ColapmError (code -4) when rows were lost to the capacity."""
    count, copied = ctypes.c_longlong(0), ctypes.c_longlong(0)
    code = LIB.colapm_get_lightcone(ctx, ctypes.byref(count), None, 0, None)
    if code not in (0, -4):
        _check(code, "colapm_get_lightcone")
    n = count.value if max_rows is None else min(count.value, max_rows)
    rows = np.empty(n, dtype=LC_DTYPE)
    _check(LIB.colapm_get_lightcone(ctx, ctypes.byref(count), rows.ctypes.data_as(ctypes.c_void_p), n,
                                    ctypes.byref(copied)), "colapm_get_lightcone")
    return count.value, rows[:copied.value]


def colapm_set_fnl(ctx, fnl):
    _check(LIB.colapm_set_fnl(ctx, float(fnl)), "colapm_set_fnl")


def colapm_power_rsd(ctx, los, nbins, kmin=0.0, kmax=0.0, k_out=None, p_out=None, n_out=None):
    k_out = np.empty(nbins) if k_out is None else k_out
    p_out = np.empty(nbins) if p_out is None else p_out
    n_out = np.empty(nbins, dtype=np.int64) if n_out is None else n_out
    _check(LIB.colapm_power_rsd(ctx, los, nbins, kmin, kmax, _ptr(k_out), _ptr(p_out), _ptr(n_out)), "colapm_power_rsd")
    return k_out, p_out, n_out


def colapm_cross_correlation(a, b, nbins, kmin=0.0, kmax=0.0, k_out=None, r_out=None, n_out=None):
    k_out = np.empty(nbins) if k_out is None else k_out
    r_out = np.empty(nbins) if r_out is None else r_out
    n_out = np.empty(nbins, dtype=np.int64) if n_out is None else n_out
    _check(LIB.colapm_cross_correlation(a, b, nbins, kmin, kmax, _ptr(k_out), _ptr(r_out), _ptr(n_out)),
           "colapm_cross_correlation")
    return k_out, r_out, n_out


def colapm_get_particles(ctx, pos=None, mom=None):
    _check(LIB.colapm_get_particles(ctx, _ptr(pos), _ptr(mom)), "colapm_get_particles")
    return pos, mom


def colapm_get_particles_async(ctx, pos=None, mom=None):
    _check(LIB.colapm_get_particles_async(ctx, _ptr(pos), _ptr(mom)), "colapm_get_particles_async")
    return pos, mom


def colapm_wait_particles(ctx):
    _check(LIB.colapm_wait_particles(ctx), "colapm_wait_particles")


def colapm_get_state(ctx, cell=None, offset=None, mom=None):
    _check(LIB.colapm_get_state(ctx, _ptr(cell), _ptr(offset), _ptr(mom)), "colapm_get_state")
    return cell, offset, mom


def colapm_set_state(ctx, cell=None, offset=None, mom=None):
    _check(LIB.colapm_set_state(ctx, _ptr(cell), _ptr(offset), _ptr(mom)), "colapm_set_state")


def colapm_get_density(ctx, mesh):
    _check(LIB.colapm_get_density(ctx, _ptr(mesh)), "colapm_get_density")
    return mesh


def colapm_get_force(ctx, force):
    _check(LIB.colapm_get_force(ctx, _ptr(force)), "colapm_get_force")
    return force


def colapm_get_lpt(ctx, psi1=None, psi2=None):
    _check(LIB.colapm_get_lpt(ctx, _ptr(psi1), _ptr(psi2)), "colapm_get_lpt")
    return psi1, psi2


def colapm_get_gaussian_field(ctx, dk):
    _check(LIB.colapm_get_gaussian_field(ctx, _ptr(dk)), "colapm_get_gaussian_field")
    return dk


def colapm_reseed(ctx, seed):
    _check(LIB.colapm_reseed(ctx, seed), "colapm_reseed")


def colapm_kernel_launches(ctx):
    return LIB.colapm_kernel_launches(ctx)


def colapm_sync(ctx):
    _check(LIB.colapm_sync(ctx), "colapm_sync")


def colapm_steps_done(ctx):
    return LIB.colapm_steps_done(ctx)


def colapm_save_state(ctx):
    n = ctypes.c_size_t(0)
    _check(LIB.colapm_save_state(ctx, None, ctypes.byref(n)), "colapm_save_state")
    buf = np.empty(n.value, dtype=np.uint8)
    _check(LIB.colapm_save_state(ctx, _ptr(buf), ctypes.byref(n)), "colapm_save_state")
    return buf


def colapm_load_state(ctx, buf):
    _check(LIB.colapm_load_state(ctx, _ptr(buf), buf.nbytes), "colapm_load_state")


def colapm_power_noalloc(cell, offset, n_particles, nm, box, nbins, kmin=0.0, kmax=0.0, k_out=None, p_out=None,
                         n_out=None, stream=0):
    k_out = np.empty(nbins) if k_out is None else k_out
    p_out = np.empty(nbins) if p_out is None else p_out
    n_out = np.empty(nbins, dtype=np.int64) if n_out is None else n_out
    _check(LIB.colapm_power_noalloc(_ptr(cell), _ptr(offset), n_particles, nm, box, nbins, kmin, kmax, _ptr(k_out),
                                    _ptr(p_out), _ptr(n_out), ctypes.c_void_p(stream or None)),
           "colapm_power_noalloc")
    return k_out, p_out, n_out


def colapm_autotune(ctx):
    choice = np.zeros(3, dtype=np.int32)
    _check(LIB.colapm_autotune(ctx, _ptr(choice)), "colapm_autotune")
    return {"two_stage": bool(choice[0]), "block": int(choice[1]), "fused": int(choice[2])}


def colapm_set_engine(ctx, fused=3, two_stage=True, block=256):
    _check(LIB.colapm_set_engine(ctx, int(fused), int(two_stage), int(block)), "colapm_set_engine")


PLAN_XF, PLAN_Y, PLAN_Z, PLAN_XI, PLAN_ALL = 1, 2, 4, 8, 15


def colapm_set_plan(ctx, plan):
    _check(LIB.colapm_set_plan(ctx, int(plan)), "colapm_set_plan")


def colapm_get_config(ctx):
    cfg = np.zeros(7, dtype=np.int32)
    _check(LIB.colapm_get_config(ctx, _ptr(cfg)), "colapm_get_config")
    return {"plan": int(cfg[0]), "block": int(cfg[1]), "fused": int(cfg[2]), "sort_every": int(cfg[3]),
            "sort_tiles": int(cfg[4]), "deposit_tiled": bool(cfg[5]), "sort_first": int(cfg[6])}


def colapm_set_sort_tiles(ctx, t):
    _check(LIB.colapm_set_sort_tiles(ctx, int(t)), "colapm_set_sort_tiles")


def colapm_set_deposit_tiles(ctx, t):
    _check(LIB.colapm_set_deposit_tiles(ctx, int(t)), "colapm_set_deposit_tiles")


def colapm_batch_create(params_list, nstreams=0, stream=0):
    arr = (Params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _check(LIB.colapm_batch_create(len(params_list), ctypes.cast(arr, ctypes.c_void_p), nstreams,
                                   ctypes.c_void_p(stream or None), ctypes.byref(b)), "colapm_batch_create")
    return b


def colapm_batch_run(b, n, nbins, seeds=None, kmin=0.0, kmax=0.0):
    k = np.empty((n, nbins))
    p = np.empty((n, nbins))
    cnt = np.empty((n, nbins), dtype=np.int64)
    sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
    _check(LIB.colapm_batch_run(b, _ptr(sd), nbins, kmin, kmax, _ptr(k), _ptr(p), _ptr(cnt)), "colapm_batch_run")
    return k, p, cnt


def colapm_batch_streams(b):
    return LIB.colapm_batch_streams(b)


def colapm_batch_set_lockstep(b, on=True):
    _check(LIB.colapm_batch_set_lockstep(b, int(bool(on))), "colapm_batch_set_lockstep")


def colapm_batch_destroy(b):
    LIB.colapm_batch_destroy(b)


def colapm_set_sort(ctx, every):
    _check(LIB.colapm_set_sort(ctx, every), "colapm_set_sort")


def colapm_set_timing(ctx, on=True):
    _check(LIB.colapm_set_timing(ctx, 1 if on else 0), "colapm_set_timing")


def colapm_get_timing(ctx):
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    _check(LIB.colapm_get_timing(ctx, _ptr(ms), _ptr(cnt)), "colapm_get_timing")
    return dict(zip(PHASES, ms)), dict(zip(PHASES, cnt))


def colapm_get_displacement(ctx, psi):
    _check(LIB.colapm_get_displacement(ctx, _ptr(psi)), "colapm_get_displacement")
    return psi


def colapm_set_displacement(ctx, psi):
    _check(LIB.colapm_set_displacement(ctx, _ptr(psi)), "colapm_set_displacement")


def nn_default_config(**kw):
    c = NNConfig()
    LIB.colapm_nn_default_config(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def colapm_nn_create(n, cfg=None, stream=0):
    cfg = nn_default_config() if cfg is None else cfg
    h = ctypes.c_void_p()
    _check(LIB.colapm_nn_create(n, ctypes.byref(cfg), stream, ctypes.byref(h)), "colapm_nn_create")
    return h


def colapm_nn_destroy(nn):
    _check(LIB.colapm_nn_destroy(nn), "colapm_nn_destroy")


def colapm_nn_set_params(nn, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != NN_PARAMS:
        raise ValueError(f"expected {NN_PARAMS} parameters")
    _check(LIB.colapm_nn_set_params(nn, _ptr(a)), "colapm_nn_set_params")


def colapm_nn_get_params(nn):
    out = np.empty(NN_PARAMS, np.float32)
    _check(LIB.colapm_nn_get_params(nn, _ptr(out)), "colapm_nn_get_params")
    return out


def colapm_nn_forward(nn, psi, out, add=False):
    _check(LIB.colapm_nn_forward(nn, _ptr(psi), _ptr(out), int(add)), "colapm_nn_forward")
    return out


def colapm_nn_grads(nn, psi, target):
    g = np.empty(NN_PARAMS, np.float32)
    loss = ctypes.c_double()
    _check(LIB.colapm_nn_grads(nn, _ptr(psi), _ptr(target), _ptr(g), ctypes.byref(loss)), "colapm_nn_grads")
    return g, loss.value


def colapm_nn_train_step(nn, psi, target, want_loss=True):
    loss = ctypes.c_double()
    _check(LIB.colapm_nn_train_step(nn, _ptr(psi), _ptr(target), ctypes.byref(loss) if want_loss else None),
           "colapm_nn_train_step")
    return loss.value if want_loss else None


def colapm_nn_steps(nn):
    return LIB.colapm_nn_steps(nn)


def colapm_nn_launches(nn):
    return LIB.colapm_nn_launches(nn)


def colapm_nn_sync(nn):
    _check(LIB.colapm_nn_sync(nn), "colapm_nn_sync")
