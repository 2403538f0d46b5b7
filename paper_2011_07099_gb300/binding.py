"""Thin ctypes binding of libfmm (include/fmm.h).  Argument marshalling only.

The functions carry the C names.  Tensors are torch CUDA tensors (torch is
used for device memory and streams only); the stream defaults to torch's
current stream on the tensors' device.  The library must have been built
(``paper_2011_07099_gb300.build.build()``); there is no fallback path: if the
shared library is missing, loading raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfmm.so")

FMM_OK = 0
FMM_ERR_ARG = 1
FMM_ERR_CUDA = 2
FMM_ERR_TIMEOUT = 3
FMM_ERR_INTERNAL = 4
FMM_ERR_ALLOC = 5
FMM_ERR_UNSUPPORTED = 6

FMM_PREC_FP32 = 0
FMM_PREC_BF16 = 1
FMM_PREC_BF16X3 = 2

FMM_MLP_PARAMS = 8769
FMM_INFER_BF16 = 0
FMM_INFER_FP32 = 1

FMM_FAULT_NONE = 0
FMM_FAULT_TC_STALL = 1

FMM_BOUNDARY_PERIODIC = 0
FMM_BOUNDARY_ISOLATED = 1

FMM_GREEN_S1 = 0
FMM_GREEN_S = 1
FMM_GREEN_X = 2

FMM_M2L_DENSE = 0
FMM_M2L_FFT = 1
FMM_NEAR_DIRECT = 0
FMM_NEAR_FFT = 1

FMM_STAGE_MULTIPOLE = 0
FMM_STAGE_LOCAL = 1
FMM_STAGE_MEAN = 2

# every symbol include/fmm.h declares, with (restype, argtypes)
_VP, _FP, _I, _SZ = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "fmm_plan_create": (_VP, [_I, _I, _I]),
    "fmm_plan_destroy": (None, [_VP]),
    "fmm_solve": (_I, [_VP, _FP, _FP, _FP, _VP]),
    "fmm_solve_host": (_I, [_VP, _FP, _FP, _FP, _VP]),
    "fmm_plan_set_precision": (_I, [_VP, _I]),
    "fmm_plan_get_shape": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                ctypes.POINTER(_I)]),
    "fmm_last_error": (_I, []),
    "fmm_error_string": (ctypes.c_char_p, [_I]),
    "fmm_plan_copy_stage": (_I, [_VP, _I, _I, _FP, _SZ, _VP]),
    "fmm_plan_set_timing": (_I, [_VP, _I]),
    "fmm_plan_check": (_I, [_VP]),
    "fmm_plan_set_m2l_group": (_I, [_VP, _I]),
    "fmm_plan_set_tc_min_level": (_I, [_VP, _I]),
    "fmm_plan_set_timeout_ms": (_I, [_VP, _I]),
    "fmm_plan_inject_fault": (_I, [_VP, _I]),
    "fmm_mean_density_noalloc": (_I, [_FP, _SZ, _FP, _VP]),
    "fmm_probe_fma": (_I, [_FP, _I, _I, _VP]),
    "fmm_plan_table_grid_size": (_I, [_VP, ctypes.POINTER(_SZ)]),
    "fmm_plan_set_boundary": (_I, [_VP, _I]),
    "fmm_plan_set_green": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_double), _I]),
    "fmm_plan_mesh_green": (_I, [_VP, _FP, _VP]),
    "fmm_plan_set_green_mesh": (_I, [_VP, _FP, _SZ]),
    "fmm_plan_set_m2l_algorithm": (_I, [_VP, _I]),
    "fmm_plan_set_near_algorithm": (_I, [_VP, _I]),
    "fmm_plan_set_tc_tile": (_I, [_VP, _I, _I]),
    "fmm_plan_autotune_tiles": (_I, [_VP, _VP, ctypes.POINTER(ctypes.c_int), _I, _VP]),
    "fmm_batch_set_near_algorithm": (_I, [_VP, _I]),
    "fmm_plan_set_table_grid": (_I, [_VP, _FP, _SZ]),
    "fmm_table_grid_grad": (_I, [_VP, _FP, _FP, _FP, ctypes.c_float, ctypes.c_float, _FP, _FP, _VP]),
    "fmm_probe_fma_flops": (ctypes.c_double, [_I, _I]),
    "fmm_plan_set_correction": (_I, [_VP, _FP, _SZ]),
    "fmm_plan_set_correction_inference": (_I, [_VP, _I]),
    "fmm_correction_grad": (_I, [_VP, _FP, _FP, _FP, ctypes.c_float, ctypes.c_float, _FP, _FP, _VP]),
    "fmm_adam_step": (_I, [_FP, _FP, _FP, _FP, _SZ, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, _VP]),
    "fmm_mesh_green": (_I, [_I, _FP, _VP]),
    "fmm_batch_create": (_VP, [_I, _VP, _VP, _VP]),
    "fmm_batch_set_precision": (_I, [_VP, _I]),
    "fmm_batch_get_levels": (_I, [_VP, _VP]),
    "fmm_batch_solve": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "fmm_batch_check": (_I, [_VP]),
    "fmm_batch_destroy": (None, [_VP]),
    "fmm_autotune_levels": (_I, [_I, _I, _I, ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "fmm_plan_stage_times": (_I, [_VP, ctypes.POINTER(ctypes.c_float), _I]),
    "fmm_plan_error_stats": (_I, [_VP, _FP, _FP, _FP, _I, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double),
                                  _VP]),
}

FMM_TIME_MEAN, FMM_TIME_P2M, FMM_TIME_M2M, FMM_TIME_M2L, FMM_TIME_L2L, FMM_TIME_P2P = range(6)
FMM_TIME_M2L_LEVEL0 = 6
FMM_TIME_SLOTS = 16

_lib = None


class FMMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {lib().fmm_error_string(code).decode()} (code {code})")


def lib():
    """Load libfmm once.  Raises OSError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libfmm is not built ({LIB_PATH} missing); run paper_2011_07099_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, where):
    if rc != FMM_OK:
        raise FMMError(rc, where)


def _stream_of(t, stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    import torch
    return torch.cuda.current_stream(t.device).cuda_stream


def fmm_plan_create(N, L, order):
    h = lib().fmm_plan_create(int(N), int(L), int(order))
    if not h:
        raise FMMError(lib().fmm_last_error(), "fmm_plan_create")
    return h


def fmm_plan_destroy(plan):
    lib().fmm_plan_destroy(plan)


def fmm_solve(plan, density, potential, accel, stream=None):
    _check(lib().fmm_solve(plan, density.data_ptr(), potential.data_ptr(), accel.data_ptr(),
                           _stream_of(density, stream)), "fmm_solve")


def fmm_plan_error_stats(plan, density, potential, accel, samples=256, seed=0, stream=None):
    """(relative L2 of the potential, of the acceleration) against the PM
    solution with G_S1, over `samples` sampled cells.  Synchronous."""
    out = (ctypes.c_double * 2)()
    _check(lib().fmm_plan_error_stats(plan, density.data_ptr(), potential.data_ptr(), accel.data_ptr(), int(samples),
                                      int(seed), out, _stream_of(density, stream)), "fmm_plan_error_stats")
    return out[0], out[1]


def fmm_solve_host(plan, density, potential, accel, stream=None):
    """Host tensors (ideally pinned).  Synchronises ``stream`` before returning."""
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().fmm_solve_host(plan, density.data_ptr(), potential.data_ptr(), accel.data_ptr(), s),
           "fmm_solve_host")


def fmm_plan_set_precision(plan, mode):
    _check(lib().fmm_plan_set_precision(plan, int(mode)), "fmm_plan_set_precision")


def fmm_plan_get_shape(plan):
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().fmm_plan_get_shape(plan, *[ctypes.byref(x) for x in v]), "fmm_plan_get_shape")
    return tuple(x.value for x in v)


def fmm_plan_copy_stage(plan, stage, level, dst, stream=None):
    _check(lib().fmm_plan_copy_stage(plan, int(stage), int(level), dst.data_ptr(), dst.numel(),
                                     _stream_of(dst, stream)), "fmm_plan_copy_stage")


def fmm_plan_set_m2l_group(plan, offsets_per_partial):
    _check(lib().fmm_plan_set_m2l_group(plan, int(offsets_per_partial)), "fmm_plan_set_m2l_group")


def fmm_plan_set_tc_min_level(plan, level):
    _check(lib().fmm_plan_set_tc_min_level(plan, int(level)), "fmm_plan_set_tc_min_level")


def fmm_plan_set_timeout_ms(plan, ms):
    _check(lib().fmm_plan_set_timeout_ms(plan, int(ms)), "fmm_plan_set_timeout_ms")


def fmm_plan_inject_fault(plan, kind):
    _check(lib().fmm_plan_inject_fault(plan, int(kind)), "fmm_plan_inject_fault")


def fmm_plan_set_correction(plan, weights):
    """weights: torch tensor (device or host) of FMM_MLP_PARAMS floats, or None."""
    if weights is None:
        _check(lib().fmm_plan_set_correction(plan, None, 0), "fmm_plan_set_correction")
    else:
        _check(lib().fmm_plan_set_correction(plan, weights.data_ptr(), weights.numel()), "fmm_plan_set_correction")


def fmm_plan_set_correction_inference(plan, mode):
    _check(lib().fmm_plan_set_correction_inference(plan, int(mode)), "fmm_plan_set_correction_inference")


def fmm_correction_grad(plan, density, target_phi, target_acc, w_phi, w_g, grad, loss, stream=None):
    _check(lib().fmm_correction_grad(plan, density.data_ptr(), target_phi.data_ptr(), target_acc.data_ptr(),
                                     float(w_phi), float(w_g), grad.data_ptr(), loss.data_ptr(),
                                     _stream_of(density, stream)), "fmm_correction_grad")


def fmm_adam_step(weights, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().fmm_adam_step(weights.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), weights.numel(),
                               int(step), float(lr), float(beta1), float(beta2), float(eps),
                               _stream_of(weights, stream)), "fmm_adam_step")


def fmm_mesh_green(N, out, stream=None):
    _check(lib().fmm_mesh_green(int(N), out.data_ptr(), _stream_of(out, stream)), "fmm_mesh_green")


def fmm_plan_set_boundary(plan, boundary):
    _check(lib().fmm_plan_set_boundary(plan, int(boundary)), "fmm_plan_set_boundary")


def fmm_plan_set_green(plan, kind, a=()):
    arr = (ctypes.c_double * max(1, len(a)))(*[float(x) for x in a])
    _check(lib().fmm_plan_set_green(plan, int(kind), arr if len(a) else None, len(a)), "fmm_plan_set_green")


def fmm_plan_set_m2l_algorithm(plan, algorithm):
    _check(lib().fmm_plan_set_m2l_algorithm(plan, int(algorithm)), "fmm_plan_set_m2l_algorithm")


def fmm_plan_set_near_algorithm(plan, algorithm):
    _check(lib().fmm_plan_set_near_algorithm(plan, int(algorithm)), "fmm_plan_set_near_algorithm")


def fmm_plan_set_tc_tile(plan, level, targets):
    _check(lib().fmm_plan_set_tc_tile(plan, int(level), int(targets)), "fmm_plan_set_tc_tile")


def fmm_plan_autotune_tiles(plan, density, stream=None):
    """Tuned tensor-core tiles: a list, targets per CTA per level (0 where a
    level is not on the tensor cores)."""
    n = 9                                   # levels 0..8, the deepest tree the library builds
    out = (ctypes.c_int * n)()
    _check(lib().fmm_plan_autotune_tiles(plan, density.data_ptr(), out, n, _stream_of(density, stream)),
           "fmm_plan_autotune_tiles")
    return list(out)


def fmm_batch_set_near_algorithm(batch, algorithm):
    _check(lib().fmm_batch_set_near_algorithm(batch, int(algorithm)), "fmm_batch_set_near_algorithm")


def fmm_plan_set_green_mesh(plan, mesh):
    _check(lib().fmm_plan_set_green_mesh(plan, mesh.data_ptr(), mesh.numel()), "fmm_plan_set_green_mesh")


def fmm_plan_mesh_green(plan, out, stream=None):
    _check(lib().fmm_plan_mesh_green(plan, out.data_ptr(), _stream_of(out, stream)), "fmm_plan_mesh_green")


def fmm_plan_table_grid_size(plan):
    n = _SZ(0)
    _check(lib().fmm_plan_table_grid_size(plan, ctypes.byref(n)), "fmm_plan_table_grid_size")
    return int(n.value)


def fmm_plan_set_table_grid(plan, theta):
    if theta is None:
        _check(lib().fmm_plan_set_table_grid(plan, None, 0), "fmm_plan_set_table_grid")
    else:
        _check(lib().fmm_plan_set_table_grid(plan, theta.data_ptr(), theta.numel()), "fmm_plan_set_table_grid")


def fmm_table_grid_grad(plan, density, target_phi, target_acc, w_phi, w_g, grad, loss, stream=None):
    _check(lib().fmm_table_grid_grad(plan, density.data_ptr(), target_phi.data_ptr(), target_acc.data_ptr(),
                                     float(w_phi), float(w_g), grad.data_ptr(), loss.data_ptr(),
                                     _stream_of(density, stream)), "fmm_table_grid_grad")


def fmm_probe_fma(out, blocks, iters, stream=None):
    _check(lib().fmm_probe_fma(out.data_ptr(), int(blocks), int(iters), _stream_of(out, stream)), "fmm_probe_fma")
    return float(lib().fmm_probe_fma_flops(int(blocks), int(iters)))


def fmm_plan_check(plan):
    _check(lib().fmm_plan_check(plan), "fmm_plan_check")


def fmm_plan_set_timing(plan, enable):
    _check(lib().fmm_plan_set_timing(plan, int(bool(enable))), "fmm_plan_set_timing")


def fmm_plan_stage_times(plan):
    buf = (ctypes.c_float * FMM_TIME_SLOTS)()
    _check(lib().fmm_plan_stage_times(plan, buf, FMM_TIME_SLOTS), "fmm_plan_stage_times")
    return list(buf)


def fmm_autotune_levels(N, order, precision, cache_path=None):
    L = ctypes.c_int()
    ms = ctypes.c_float()
    path = cache_path.encode() if cache_path else None
    _check(lib().fmm_autotune_levels(int(N), int(order), int(precision), path, ctypes.byref(L), ctypes.byref(ms)),
           "fmm_autotune_levels")
    return L.value, ms.value


class Batch:
    """Owning wrapper of fmm_batch: fields of uneven size, one graph launch."""

    def __init__(self, N, L, order, precision=FMM_PREC_FP32):
        n = len(N)
        arr = lambda v: (ctypes.c_int * n)(*[int(x) for x in v])
        self.n = n
        self.handle = lib().fmm_batch_create(n, arr(N), arr(L), arr(order))
        if not self.handle:
            raise FMMError(lib().fmm_last_error(), "fmm_batch_create")
        if precision != FMM_PREC_FP32:
            _check(lib().fmm_batch_set_precision(self.handle, int(precision)), "fmm_batch_set_precision")
        lv = (ctypes.c_int * n)()
        _check(lib().fmm_batch_get_levels(self.handle, lv), "fmm_batch_get_levels")
        self.levels = list(lv)

    def solve(self, densities, potentials, accels, stream=None):
        n = self.n
        ptrs = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        s = _stream_of(densities[0], stream)
        _check(lib().fmm_batch_solve(self.handle, ptrs(densities), ptrs(potentials), ptrs(accels), s),
               "fmm_batch_solve")

    def check(self):
        _check(lib().fmm_batch_check(self.handle), "fmm_batch_check")

    def close(self):
        if self.handle:
            lib().fmm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper: ``Plan(N, L, order).solve(rho) -> (phi, accel)``."""

    def __init__(self, N, L, order, precision=FMM_PREC_FP32):
        self.handle = fmm_plan_create(N, L, order)
        self.N, self.L, self.order, self.S = fmm_plan_get_shape(self.handle)
        if precision != FMM_PREC_FP32:
            fmm_plan_set_precision(self.handle, precision)

    def set_precision(self, mode):
        fmm_plan_set_precision(self.handle, mode)

    def solve(self, density, potential=None, accel=None, stream=None):
        import torch
        n = self.N
        if potential is None:
            potential = torch.empty((n, n, n), dtype=torch.float32, device=density.device)
        if accel is None:
            accel = torch.empty((3, n, n, n), dtype=torch.float32, device=density.device)
        fmm_solve(self.handle, density, potential, accel, stream)
        return potential, accel

    def error_stats(self, density, potential, accel, samples=256, seed=0, stream=None):
        return fmm_plan_error_stats(self.handle, density, potential, accel, samples, seed, stream)

    def stage(self, stage, level):
        import torch
        p3 = self.order ** 3
        if stage == FMM_STAGE_MEAN:
            out = torch.empty(1, dtype=torch.float32, device="cuda")
        else:
            k = p3 if stage == FMM_STAGE_MULTIPOLE else 4 * p3
            out = torch.empty((8 ** level) * k, dtype=torch.float32, device="cuda")
        fmm_plan_copy_stage(self.handle, stage, level, out)
        return out

    def close(self):
        if self.handle:
            fmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
