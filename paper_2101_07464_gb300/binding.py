"""Thin ctypes binding of libhd.so (include/hd.h), with the same names as the C ABI.

Argument marshalling only: torch CUDA tensors are checked (device, dtype, length,
contiguity) and passed as raw device pointers; every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing or cannot be
loaded, every call raises.
"""
import ctypes
import os

from . import build as _build

HD_GINIBRE, HD_HAAR = 0, 1
HD_F64, HD_F32 = 0, 1
HD_OK, HD_ERR_ARG, HD_ERR_DIM, HD_ERR_TMAX = 0, 1, 2, 3
HD_ERR_OOM, HD_ERR_CUDA, HD_ERR_TIMEOUT, HD_ERR_STATE = 4, 5, 6, 7

ENSEMBLES = {"ginibre": HD_GINIBRE, "haar": HD_HAAR}
DTYPES = {"f64": HD_F64, "f32": HD_F32}

_LIB = None

HD_DYN_TANH, HD_DYN_SIGN_MEM, HD_DYN_NORM_TANH, HD_DYN_AMP, HD_DYN_ISTA = 1, 2, 3, 4, 5
DYNAMICS = {"tanh": HD_DYN_TANH, "sign_mem": HD_DYN_SIGN_MEM, "norm_tanh": HD_DYN_NORM_TANH, "amp": HD_DYN_AMP,
            "ista": HD_DYN_ISTA}


class hd_run_spec(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("transpose", ctypes.POINTER(ctypes.c_uint8)),
                ("dynamics", ctypes.c_int32), ("a", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("aux", ctypes.c_void_p), ("y_record", ctypes.c_void_p), ("x_record", ctypes.c_void_p),
                ("x_given", ctypes.c_void_p), ("ld_rows", ctypes.c_int64), ("b", ctypes.c_double)]

HD_ENGINE_NO_FUSE, HD_ENGINE_NO_PDL, HD_ENGINE_STEP_KERNEL = 1, 2, 4

_c = ctypes
_P = _c.c_void_p
_PROTOS = {
    "hd_create": (_c.c_int, [_c.c_int, _c.c_int64, _c.c_int64, _c.c_int32, _c.c_uint64, _c.c_int,
                             _c.POINTER(_P)]),
    "hd_set_options": (_c.c_int, [_P, _c.c_double, _c.c_uint32, _P]),
    "hd_create_batched": (_c.c_int, [_c.c_int, _c.c_int32, _P, _P, _c.c_int32, _c.c_uint64, _c.c_int,
                                     _c.POINTER(_P)]),
    "hd_get_batch_layout": (_c.c_int, [_P, _c.POINTER(_c.c_int32), _P, _P]),
    "hd_set_trial_sigmas": (_c.c_int, [_P, _P]),
    "hd_set_engine": (_c.c_int, [_P, _c.c_int]),
    "hd_fp64_fma_rate": (_c.c_int, [_c.c_int32, _c.c_int32, _c.POINTER(_c.c_double), _P]),
    "hd_complex_create": (_c.c_int, [_c.c_int, _c.c_int64, _c.c_int64, _c.c_int32, _c.c_uint64, _c.c_int,
                                     _c.POINTER(_P)]),
    "hd_complex_set_options": (_c.c_int, [_P, _c.c_double, _c.c_uint32, _P]),
    "hd_complex_apply": (_c.c_int, [_P, _P, _c.c_int, _P]),
    "hd_complex_gue_apply": (_c.c_int, [_P, _P, _P]),
    "hd_complex_reset": (_c.c_int, [_P, _c.c_uint64]),
    "hd_complex_get_counts": (_c.c_int, [_P, _c.POINTER(_c.c_int32)]),
    "hd_complex_destroy": (None, [_P]),
    "hd_adjoint_enable": (_c.c_int, [_P, _c.c_int]),
    "hd_adjoint_step": (_c.c_int, [_P, _P, _P, _P]),
    "hd_adjoint_restart": (_c.c_int, [_P]),
    "hd_adjoint_position": (_c.c_int, [_P, _c.POINTER(_c.c_int32)]),
    "hd_first_product_noalloc": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int64, _c.c_int64, _c.c_int,
                                            _c.c_uint64, _c.c_uint32, _c.c_double, _P, _P, _P]),
    "hd_apply": (_c.c_int, [_P, _P, _c.c_int, _P]),
    "hd_probe": (_c.c_int, [_P, _P, _c.c_int, _P, _c.POINTER(_c.c_double)]),
    "hd_probe_at": (_c.c_int, [_P, _c.c_int32, _P, _c.c_int, _P, _c.POINTER(_c.c_double)]),
    "hd_reset": (_c.c_int, [_P, _c.c_uint64]),
    "hd_sync": (_c.c_int, [_P]),
    "hd_check_bounded_wait": (_c.c_int, [_P, _c.c_uint32]),
    "hd_run": (_c.c_int, [_P, _P, _P, _P]),
    "hd_goe_apply": (_c.c_int, [_P, _P, _P]),
    "hd_usv_apply": (_c.c_int, [_P, _P, _P, _P, _c.c_int, _P]),
    "hd_autotune": (_c.c_int, [_P, _P, _P, _P, _c.c_int32]),
    "hd_get_tuning": (_c.c_int, [_P, _P, _c.c_int32]),
    "hd_set_tuning": (_c.c_int, [_P, _P, _c.c_int32]),
    "hd_get_map_options": (_c.c_int, [_P, _c.POINTER(_c.c_int32), _P]),
    "hd_profile_enable": (_c.c_int, [_P, _c.c_int]),
    "hd_profile_read": (_c.c_int, [_P, _c.POINTER(_c.c_double), _c.POINTER(_c.c_int64),
                                   _c.POINTER(_c.c_double), _c.c_int]),
    "hd_get_launches": (_c.c_int, [_P, _c.POINTER(_c.c_int64)]),
    "hd_destroy": (None, [_P]),
    "hd_get_counts": (_c.c_int, [_P, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32),
                                 _c.POINTER(_c.c_int32)]),
    "hd_get_device_bytes": (_c.c_int, [_P, _c.POINTER(_c.c_int64)]),
    "hd_status_string": (_c.c_char_p, [_c.c_int]),
    "hd_last_error": (_c.c_char_p, []),
    "hd_philox_normals": (_c.c_int, [_c.c_uint64, _c.c_uint32, _c.c_uint32, _c.c_uint32, _c.c_int64,
                                     _c.c_int64, _c.c_int, _P, _P]),
    "hd_philox_words": (_c.c_int, [_c.c_uint64, _P, _c.c_int64, _P, _P]),
}


class HDError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().hd_status_string(code).decode() if _LIB is not None else str(code)
        if code in (HD_ERR_CUDA, HD_ERR_TIMEOUT) and _LIB is not None:
            msg += " (%s)" % lib().hd_last_error().decode()
        super().__init__("%s%s" % (where + ": " if where else "", msg))


def library_path():
    return _build.LIB


def lib():
    """Load libhd.so (built in-tree by paper_2101_07464_gb300.build); raises if absent."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libhd.so is not built (%s); run paper_2101_07464_gb300.build.build() "
                               "or __graft_entry__.build() first" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc, where):
    if rc != HD_OK:
        raise HDError(rc, where)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None  # torch.cuda.Stream


def _ptr(t, dtype_code=None, numel=None, what="tensor"):
    """Raw device pointer of a contiguous CUDA tensor (or an int address)."""
    if isinstance(t, int):
        return t
    import torch
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype_code is not None:
        want = torch.float64 if dtype_code == HD_F64 else torch.float32
        if t.dtype != want:
            raise ValueError("%s must be %s" % (what, want))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (what, numel, t.numel()))
    return t.data_ptr()


def hd_create(ensemble, m, n, T_max, seed, dtype):
    ens = ENSEMBLES.get(ensemble, ensemble)
    dt = DTYPES.get(dtype, dtype)
    h = _P()
    _check(lib().hd_create(ens, m, n, T_max, seed & 0xFFFFFFFFFFFFFFFF, dt, ctypes.byref(h)),
           "hd_create")
    return h


def hd_create_batched(ensemble, ms, ns, T_max, seed, dtype):
    import numpy as np
    ens = ENSEMBLES.get(ensemble, ensemble)
    dt = DTYPES.get(dtype, dtype)
    m = np.ascontiguousarray(ms, dtype=np.int64)
    n = np.ascontiguousarray(ns, dtype=np.int64)
    if m.shape != n.shape:
        raise ValueError("m and n must have the same length")
    h = _P()
    _check(lib().hd_create_batched(ens, len(m), m.ctypes.data, n.ctypes.data, T_max,
                                   seed & 0xFFFFFFFFFFFFFFFF, dt, ctypes.byref(h)), "hd_create_batched")
    return h


def hd_get_batch_layout(state):
    """Returns (off_n, off_m) as numpy int64 arrays of count + 1 packed offsets."""
    import numpy as np
    c = ctypes.c_int32()
    _check(lib().hd_get_batch_layout(state, ctypes.byref(c), None, None), "hd_get_batch_layout")
    on = np.zeros(c.value + 1, dtype=np.int64)
    om = np.zeros(c.value + 1, dtype=np.int64)
    _check(lib().hd_get_batch_layout(state, ctypes.byref(c), on.ctypes.data, om.ctypes.data),
           "hd_get_batch_layout")
    return on, om


def hd_first_product_noalloc(ensemble, dtype, m, n, transpose, seed, trial, sigma, x, y,
                             stream=None):
    """y = Q x (or Q^T x) for a fresh matrix, as a new state's step 1; allocates nothing.
    x and y are preallocated CUDA tensors (or raw device addresses) of the dtype."""
    dt = DTYPES.get(dtype, dtype)
    nx, ny = (m, n) if transpose else (n, m)
    _check(lib().hd_first_product_noalloc(ENSEMBLES.get(ensemble, ensemble), dt, m, n,
                                          1 if transpose else 0, seed & 0xFFFFFFFFFFFFFFFF, trial,
                                          float(sigma), _ptr(x, dt, nx, "x"), _ptr(y, dt, ny, "y"),
                                          _stream_ptr(stream)), "hd_first_product_noalloc")


HD_ADJ_RECORD_X = 1


def hd_adjoint_enable(state, record_x=True):
    _check(lib().hd_adjoint_enable(state, HD_ADJ_RECORD_X if record_x else 0), "hd_adjoint_enable")


def hd_adjoint_step(state, ybar, x_t, xbar):
    """ybar, xbar: CUDA tensors (or addresses); x_t: CUDA tensor, address or None (recorded)."""
    _check(lib().hd_adjoint_step(state, _ptr(ybar, what="ybar"), None if x_t is None else _ptr(x_t, what="x_t"),
                                 _ptr(xbar, what="xbar")), "hd_adjoint_step")


def hd_adjoint_restart(state):
    _check(lib().hd_adjoint_restart(state), "hd_adjoint_restart")


def hd_adjoint_position(state):
    v = ctypes.c_int32()
    _check(lib().hd_adjoint_position(state, ctypes.byref(v)), "hd_adjoint_position")
    return v.value


def hd_set_options(state, sigma=1.0, trial=0, stream=None):
    _check(lib().hd_set_options(state, sigma, trial, _stream_ptr(stream)), "hd_set_options")


def hd_apply(state, x, transpose, y):
    _check(lib().hd_apply(state, _ptr(x, what="x"), int(bool(transpose)), _ptr(y, what="y")), "hd_apply")


def hd_probe(state, x, transpose, y):
    u = ctypes.c_double()
    _check(lib().hd_probe(state, _ptr(x, what="x"), int(bool(transpose)), _ptr(y, what="y"),
                          ctypes.byref(u)), "hd_probe")
    return u.value


def _rows_addr(t, what):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous() or t.dim() != 2:
        raise ValueError("%s must be a contiguous 2-D CUDA tensor (T rows)" % what)
    return t.data_ptr()


def hd_probe_at(state, step, x, transpose, y):
    u = ctypes.c_double()
    _check(lib().hd_probe_at(state, int(step), _ptr(x, what="x"), int(bool(transpose)), _ptr(y, what="y"),
                             ctypes.byref(u)), "hd_probe_at")
    return u.value


def make_run_spec(transpose_flags, dynamics, a=0.0, use_graph=True, aux=None, y_record=None,
                  x_record=None, x_given=None, b=0.0):
    """hd_run_spec for a schedule (sequence of 0/1 flags) and a built-in dynamics name/code.
    aux: the noise vector w of HD_DYN_AMP / HD_DYN_ISTA (CUDA or page-locked tensor, or an address);
    b: HD_DYN_ISTA's step size.
    y_record / x_record / x_given: optional T x L CUDA tensors of the state's dtype (row t-1
    for step t; L >= the longest packed vector): records of y_t and of f_t's result, and
    teacher-forced replacements of f_t's result (hd_run_spec)."""
    flags = (ctypes.c_uint8 * len(transpose_flags))(*[1 if f else 0 for f in transpose_flags])
    aux_addr = None
    if aux is not None:
        aux_addr = aux if isinstance(aux, int) else aux.data_ptr()
    rows = [r for r in (y_record, x_record, x_given) if r is not None]
    ld = 0
    for r in rows:
        if isinstance(r, int):
            raise ValueError("record buffers must be tensors")
        if r.shape[0] < len(transpose_flags):
            raise ValueError("record buffers need one row per step")
        if ld and r.stride(0) != ld:
            raise ValueError("record buffers must share one row length")
        ld = r.stride(0)
    spec = hd_run_spec(len(transpose_flags), ctypes.cast(flags, ctypes.POINTER(ctypes.c_uint8)),
                       DYNAMICS.get(dynamics, dynamics), float(a), 1 if use_graph else 0, aux_addr,
                       _rows_addr(y_record, "y_record"), _rows_addr(x_record, "x_record"),
                       _rows_addr(x_given, "x_given"), int(ld), float(b))
    spec._flags = flags  # keep the array alive with the struct
    spec._aux = aux
    spec._rows = rows
    return spec


def hd_fp64_fma_rate(iters=1 << 16, reps=5, stream=None):
    """Measured FP64 FMA pipe rate of the current device in TFLOP/s (hd_fp64_fma_rate)."""
    out = ctypes.c_double()
    _check(lib().hd_fp64_fma_rate(int(iters), int(reps), ctypes.byref(out), _stream_ptr(stream)),
           "hd_fp64_fma_rate")
    return out.value


def hd_set_engine(state, no_fuse=False, no_pdl=False, step_kernel=False):
    """Engine switches (hd_set_engine): keep hd_run's separate sweeps, launch without
    programmatic dependent launch, or run each fused step as one launch (the step kernel)."""
    flags = ((HD_ENGINE_NO_FUSE if no_fuse else 0) | (HD_ENGINE_NO_PDL if no_pdl else 0)
             | (HD_ENGINE_STEP_KERNEL if step_kernel else 0))
    _check(lib().hd_set_engine(state, flags), "hd_set_engine")


def hd_run(state, spec, x1, x_out):
    """x1 / x_out: CUDA tensors, page-locked CPU tensors, or raw addresses."""
    _check(lib().hd_run(state, ctypes.byref(spec), _run_addr(x1, "x1"), _run_addr(x_out, "x_out")),
           "hd_run")


HD_TUNE_WORDS = 134


def hd_goe_apply(state, x, y):
    """y = (Q + Q^T) x / sqrt(2) on a square Ginibre state (two of its products)."""
    _check(lib().hd_goe_apply(state, _ptr(x, what="x"), _ptr(y, what="y")), "hd_goe_apply")


def hd_usv_apply(U, V, s, x, transpose, y):
    """y = U Sigma V x (transpose False) or V^T Sigma^T U^T x (True); s: CUDA float64 tensor."""
    _check(lib().hd_usv_apply(U, V, _ptr(s, HD_F64, what="s"), _ptr(x, what="x"), int(bool(transpose)),
                              _ptr(y, what="y")), "hd_usv_apply")


def _run_addr(t, what):
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if not t.is_cuda and not t.is_pinned():
        raise ValueError("%s must be a CUDA tensor or page-locked host memory" % what)
    return t.data_ptr()


def hd_autotune(state, spec, x1, x_out, reps=2):
    """Measure and keep the fastest launch shapes and CTA split for trajectory `spec`."""
    _check(lib().hd_autotune(state, ctypes.byref(spec), _run_addr(x1, "x1"), _run_addr(x_out, "x_out"),
                             int(reps)), "hd_autotune")


def hd_get_tuning(state):
    w = (ctypes.c_int32 * HD_TUNE_WORDS)()
    _check(lib().hd_get_tuning(state, w, HD_TUNE_WORDS), "hd_get_tuning")
    return list(w)


def hd_set_tuning(state, words):
    """words: a list from hd_get_tuning (same shape of state), or [] for the built-in rules."""
    w = (ctypes.c_int32 * max(1, len(words)))(*[int(v) for v in words])
    _check(lib().hd_set_tuning(state, w, len(words)), "hd_set_tuning")


def hd_get_map_options(state):
    """[(sub-tiles per CTA in the n-space, in the m-space)] of the candidate CTA splits."""
    cnt = ctypes.c_int32()
    _check(lib().hd_get_map_options(state, ctypes.byref(cnt), None), "hd_get_map_options")
    spc = (ctypes.c_int32 * (2 * cnt.value))()
    _check(lib().hd_get_map_options(state, ctypes.byref(cnt), spc), "hd_get_map_options")
    return [(spc[2 * o], spc[2 * o + 1]) for o in range(cnt.value)]


def hd_profile_enable(state, on=True):
    _check(lib().hd_profile_enable(state, 1 if on else 0), "hd_profile_enable")


def hd_profile_read(state, clear=False):
    """Returns {kind: (ms, launches, bytes)} for kinds 'dots', 'update', 'output' and 'step'
    (the step kernel: update and fused output sweep in one launch)."""
    ms = (ctypes.c_double * 4)()
    nl = (ctypes.c_int64 * 4)()
    by = (ctypes.c_double * 4)()
    _check(lib().hd_profile_read(state, ms, nl, by, 1 if clear else 0), "hd_profile_read")
    return {k: (ms[i], nl[i], by[i]) for i, k in enumerate(("dots", "update", "output", "step"))}


def hd_get_launches(state):
    v = ctypes.c_int64()
    _check(lib().hd_get_launches(state, ctypes.byref(v)), "hd_get_launches")
    return v.value


def hd_sync(state):
    _check(lib().hd_sync(state), "hd_sync")


def hd_check_bounded_wait(state, polls=4096):
    """Launch the bounded-wait check (see include/hd.h); hd_sync afterwards reports the expiry."""
    _check(lib().hd_check_bounded_wait(state, int(polls)), "hd_check_bounded_wait")


def hd_reset(state, seed):
    _check(lib().hd_reset(state, seed & 0xFFFFFFFFFFFFFFFF), "hd_reset")


def hd_destroy(state):
    if state:
        lib().hd_destroy(state)


def hd_get_counts(state):
    t, r, l = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().hd_get_counts(state, ctypes.byref(t), ctypes.byref(r), ctypes.byref(l)),
           "hd_get_counts")
    return t.value, r.value, l.value


def hd_get_device_bytes(state):
    b = ctypes.c_int64()
    _check(lib().hd_get_device_bytes(state, ctypes.byref(b)), "hd_get_device_bytes")
    return b.value


def hd_philox_normals(seed, trial, step, stream_id, start, count, dtype, out, stream=None):
    dt = DTYPES.get(dtype, dtype)
    _check(lib().hd_philox_normals(seed & 0xFFFFFFFFFFFFFFFF, trial, step, stream_id, start, count,
                                   dt, _ptr(out, dt, count, "out"), _stream_ptr(stream)),
           "hd_philox_normals")


def hd_philox_words(seed, counters, nblocks, out, stream=None):
    _check(lib().hd_philox_words(seed & 0xFFFFFFFFFFFFFFFF, _ptr(counters, what="counters"), nblocks,
                                 _ptr(out, what="out"), _stream_ptr(stream)), "hd_philox_words")


def hd_set_trial_sigmas(state, sigmas):
    import numpy as np
    a = np.ascontiguousarray(sigmas, dtype=np.float64)
    _check(lib().hd_set_trial_sigmas(state, a.ctypes.data), "hd_set_trial_sigmas")


class HDBatch:
    """Owner of a batched hd_state: `count` independent trials, packed vectors."""

    def __init__(self, ensemble, ms, ns, T_max, seed, dtype="f32", sigma=1.0, trial=0, stream=None):
        import torch
        self.dtype_code = DTYPES.get(dtype, dtype)
        self.torch_dtype = torch.float64 if self.dtype_code == HD_F64 else torch.float32
        self.seed = seed
        self.h = hd_create_batched(ensemble, ms, ns, T_max, seed, self.dtype_code)
        self.off_n, self.off_m = hd_get_batch_layout(self.h)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        hd_set_options(self.h, sigma, trial, stream)

    def apply(self, x, transpose=False, out=None):
        import torch
        dim_in = int(self.off_m[-1] if transpose else self.off_n[-1])
        dim_out = int(self.off_n[-1] if transpose else self.off_m[-1])
        _ptr(x, self.dtype_code, dim_in, "x")
        if out is None:
            out = torch.empty(dim_out, dtype=self.torch_dtype, device=x.device)
        hd_apply(self.h, x, transpose, out)
        return out

    def adjoint_enable(self, record_x=True):
        """Record the following forward steps for hd_adjoint_step (every trial of the batch must
        have the same dimensions; call on a fresh or reset state)."""
        hd_adjoint_enable(self.h, record_x)

    def adjoint_step(self, ybar, transpose, x_t=None):
        """Reverse the latest unreversed step for every trial at once (packed vectors): returns
        dLoss/dx_t through y_t and every later product; x_t=None uses the recorded input."""
        import torch
        n_in, n_out = (int(self.off_m[-1]), int(self.off_n[-1])) if transpose else \
            (int(self.off_n[-1]), int(self.off_m[-1]))
        _ptr(ybar, self.dtype_code, n_out, "ybar")
        if x_t is not None:
            _ptr(x_t, self.dtype_code, n_in, "x_t")
        xbar = torch.empty(n_in, dtype=self.torch_dtype, device=ybar.device)
        hd_adjoint_step(self.h, ybar, x_t, xbar)
        return xbar

    def reset(self, seed=None):
        if seed is not None:
            self.seed = seed
        hd_reset(self.h, self.seed)

    def set_trial_sigmas(self, sigmas):
        hd_set_trial_sigmas(self.h, sigmas)

    def _dims(self):
        return (int(self.off_n[-1]), int(self.off_m[-1]))

    def autotune(self, schedule, dynamics, x1, a=0.0, reps=2, aux=None, b=0.0):
        """hd_autotune on the trajectory (schedule, dynamics, a, b) from x1; leaves the state reset."""
        import torch
        spec = make_run_spec(schedule, dynamics, a, use_graph=False, aux=aux, b=b)
        dmax = int(max(self._dims()))
        out = torch.empty(dmax, dtype=self.torch_dtype, device=x1.device)
        hd_autotune(self.h, spec, x1, out, reps)

    def tuning(self):
        return hd_get_tuning(self.h)

    def set_tuning(self, words):
        hd_set_tuning(self.h, words)

    def map_options(self):
        return hd_get_map_options(self.h)

    def close(self):
        if self.h:
            hd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HD:
    """Convenience owner of one hd_state: y = M_t x through hd_apply.

    HD("haar", n, n, T_max, seed, "f32").apply(x, transpose) returns a new CUDA tensor.
    Work goes on torch's current CUDA stream at construction (or `stream`).
    """

    def __init__(self, ensemble, m, n, T_max, seed, dtype="f64", sigma=1.0, trial=0, stream=None):
        import torch
        self.ensemble, self.m, self.n, self.T_max = ensemble, m, n, T_max
        self.seed = seed
        self.dtype_code = DTYPES.get(dtype, dtype)
        self.torch_dtype = torch.float64 if self.dtype_code == HD_F64 else torch.float32
        self.h = hd_create(ensemble, m, n, T_max, seed, self.dtype_code)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        hd_set_options(self.h, sigma, trial, stream)

    def apply(self, x, transpose=False, out=None):
        import torch
        dim_in, dim_out = (self.m, self.n) if transpose else (self.n, self.m)
        _ptr(x, self.dtype_code, dim_in, "x")
        if out is None:
            out = torch.empty(dim_out, dtype=self.torch_dtype, device=x.device)
        else:
            _ptr(out, self.dtype_code, dim_out, "out")
        hd_apply(self.h, x, transpose, out)
        return out

    def probe(self, x, transpose=False, step=None):
        """Q x (or Q^T x) on the revealed part; with `step`, as the representation stood after
        that product (hd_probe_at)."""
        import torch
        dim_out = self.n if transpose else self.m
        out = torch.empty(dim_out, dtype=self.torch_dtype, device=x.device)
        u = hd_probe(self.h, x, transpose, out) if step is None else hd_probe_at(self.h, step, x, transpose, out)
        return out, u

    def reset(self, seed=None):
        if seed is not None:
            self.seed = seed
        hd_reset(self.h, self.seed)

    def counts(self):
        return hd_get_counts(self.h)

    def adjoint_enable(self, record_x=True):
        """Record the following forward steps for hd_adjoint_step (call on a fresh or reset state)."""
        hd_adjoint_enable(self.h, record_x)

    def adjoint_step(self, ybar, transpose, x_t=None):
        """Reverse the latest unreversed step (a Q^T step when `transpose`): returns dLoss/dx_t
        through y_t and every later product; x_t=None uses the recorded input."""
        import torch
        n_in, n_out = (self.m, self.n) if transpose else (self.n, self.m)
        _ptr(ybar, self.dtype_code, n_out, "ybar")
        if x_t is not None:
            _ptr(x_t, self.dtype_code, n_in, "x_t")
        xbar = torch.empty(n_in, dtype=self.torch_dtype, device=ybar.device)
        hd_adjoint_step(self.h, ybar, x_t, xbar)
        return xbar

    def adjoint_restart(self):
        hd_adjoint_restart(self.h)

    def goe(self, x, out=None):
        """W x for W = (Q + Q^T)/sqrt(2) (square Ginibre state; two products)."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=self.torch_dtype, device=x.device)
        _ptr(x, self.dtype_code, self.n, "x")
        _ptr(out, self.dtype_code, self.n, "out")
        hd_goe_apply(self.h, x, out)
        return out

    def _dims(self):
        return (self.n, self.m)

    def autotune(self, schedule, dynamics, x1, a=0.0, reps=2, aux=None, b=0.0):
        """hd_autotune on the trajectory (schedule, dynamics, a, b) from x1; leaves the state reset."""
        import torch
        spec = make_run_spec(schedule, dynamics, a, use_graph=False, aux=aux, b=b)
        dmax = int(max(self._dims()))
        out = torch.empty(dmax, dtype=self.torch_dtype, device=x1.device)
        hd_autotune(self.h, spec, x1, out, reps)

    def tuning(self):
        return hd_get_tuning(self.h)

    def set_tuning(self, words):
        hd_set_tuning(self.h, words)

    def map_options(self):
        return hd_get_map_options(self.h)

    def close(self):
        if self.h:
            hd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class USV:
    """Q = U Sigma V (eq. inv) from two independent Haar states and singular values s."""

    def __init__(self, m, n, T_max, seed_u, seed_v, s, dtype="f64", stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.m, self.n = m, n
        self.U = HD("haar", m, m, T_max, seed_u, dtype, stream=stream)
        self.V = HD("haar", n, n, T_max, seed_v, dtype, stream=stream)
        self.s = torch.as_tensor(s, dtype=torch.float64).to("cuda").contiguous()
        if self.s.numel() < min(m, n):
            raise ValueError("s needs min(m, n) = %d values" % min(m, n))
        self.torch_dtype = self.U.torch_dtype

    def apply(self, x, transpose=False):
        import torch
        out = torch.empty(self.n if transpose else self.m, dtype=self.torch_dtype, device=x.device)
        hd_usv_apply(self.U.h, self.V.h, self.s, x, transpose, out)
        return out

    def close(self):
        self.U.close()
        self.V.close()


class HDComplex:
    """Owner of a complex Householder Dice state (hd_complex_* of include/hd.h): Q ~ Haar on
    the unitary group U(n) (ensemble "haar", m == n) or Q ~ CGin(m, n) with entries sigma
    CN(0, 1) ("ginibre").  apply(x, adjoint) returns Q x or Q^H x as a new CUDA tensor
    (complex128 for "f64", complex64 for "f32"), on torch's current stream; gue(x) returns
    (Q + Q^H) x / sqrt(2) for a square Ginibre state.
    """

    def __init__(self, ensemble, m, n, T_max, seed, dtype="f64", sigma=1.0, trial=0, stream=None):
        import torch
        self.ensemble, self.m, self.n, self.T_max, self.seed = ensemble, m, n, T_max, seed
        self.dtype_code = DTYPES.get(dtype, dtype)
        self.torch_dtype = torch.complex128 if self.dtype_code == HD_F64 else torch.complex64
        h = ctypes.c_void_p()
        _check(lib().hd_complex_create(ENSEMBLES.get(ensemble, ensemble), int(m), int(n), int(T_max), int(seed),
                                       self.dtype_code, ctypes.byref(h)), "hd_complex_create")
        self.h = h
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        _check(lib().hd_complex_set_options(self.h, float(sigma), int(trial), _stream_ptr(stream)),
               "hd_complex_set_options")

    def _vec(self, t, dim, what):
        if t.dtype != self.torch_dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != dim:
            raise ValueError("%s must be a contiguous CUDA %s tensor of %d elements" % (what, self.torch_dtype, dim))
        return t.data_ptr()

    def apply(self, x, adjoint=False, out=None):
        import torch
        din, dout = (self.m, self.n) if adjoint else (self.n, self.m)
        if out is None:
            out = torch.empty(dout, dtype=self.torch_dtype, device=x.device)
        _check(lib().hd_complex_apply(self.h, self._vec(x, din, "x"), 1 if adjoint else 0,
                                      self._vec(out, dout, "y")), "hd_complex_apply")
        return out

    def gue(self, x, out=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=self.torch_dtype, device=x.device)
        _check(lib().hd_complex_gue_apply(self.h, self._vec(x, self.n, "x"), self._vec(out, self.n, "y")),
               "hd_complex_gue_apply")
        return out

    def reset(self, seed=None):
        if seed is not None:
            self.seed = seed
        _check(lib().hd_complex_reset(self.h, int(self.seed)), "hd_complex_reset")

    def counts(self):
        t = ctypes.c_int32()
        _check(lib().hd_complex_get_counts(self.h, ctypes.byref(t)), "hd_complex_get_counts")
        return t.value

    def close(self):
        if getattr(self, "h", None):
            lib().hd_complex_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
