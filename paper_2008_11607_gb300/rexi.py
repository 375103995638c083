"""Thin ctypes binding of librexi (include/rexi.h), same entry-point names.

Only argument marshalling happens here: every step of the computation runs in
the CUDA library.  PyTorch supplies device memory (the state, the output and
the workspace) and the CUDA stream.  If the library is missing, ``load()``
raises; there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librexi.so")

REXI_OK = 0
REXI_EINVAL = -1
REXI_ENOMEM = -2
REXI_ECUDA = -3
REXI_ENOCONV = -4
REXI_ETIMEOUT = -5
REXI_EUNSUPPORTED = -6

REXI_BATCH_PERSISTENT = 0
REXI_BATCH_PER_INSTANCE = 1

REXI_SYMBOL_CGRID = 0
REXI_SYMBOL_SPECTRAL = 1
REXI_SYMBOL_SCHRODINGER = 2
SYMBOLS = {"cgrid": REXI_SYMBOL_CGRID, "spectral": REXI_SYMBOL_SPECTRAL, "schrodinger": REXI_SYMBOL_SCHRODINGER}

REXI_COEF_REXII = 0
REXI_COEF_REXI = 1
REXI_COEF_REXIE = 2
COEFFICIENT_SETS = {"rexii": REXI_COEF_REXII, "rexi": REXI_COEF_REXI, "rexie": REXI_COEF_REXIE}

REXI_SHIFT_NONE = 0
REXI_SHIFT_MIDPOINT = 1
REXI_SHIFT_VALUE = 2

REXI_FORM_FP64 = 0
REXI_FORM_MIXED = 1
REXI_FORM_PLAIN = 2
FORMS = {"fp64": REXI_FORM_FP64, "mixed": REXI_FORM_MIXED, "plain": REXI_FORM_PLAIN}

REXI_KRYLOV_CG = 0
REXI_KRYLOV_SHARED = 1
KRYLOV_METHODS = {"cg": REXI_KRYLOV_CG, "shared": REXI_KRYLOV_SHARED}


class rexi_step_info(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("n_terms", ctypes.c_int32),
        ("n_poles", ctypes.c_int32),
        ("tau_rho", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("krylov_iters", ctypes.c_int32),
        ("krylov_unconverged", ctypes.c_int32),
        ("krylov_max_rel_res", ctypes.c_double),
        ("krylov_term_iters", ctypes.c_int64),
    ]


_c_int = ctypes.c_int32
_c_dbl = ctypes.c_double
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)

SIGNATURES = {
    "rexi_pole_count": (_c_int, [_c_dbl, _c_dbl, _c_dbl, _ip]),
    "rexi_rexii_terms": (_c_int, [_c_int, _c_dbl, _dp, _ip, _dp, _dp, _c_int]),
    "rexi_coeffs": (_c_int, [_c_dbl, _c_dbl, _c_dbl, _c_int, _ip, _ip, _dp, _dp, _c_int]),
    "rexi_plan_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl,
                                  _c_dbl, _vp, _c_int, _c_dbl]),
    "rexi_plan_destroy": (None, [_vp]),
    "rexi_spectral_radius": (_c_int, [_vp, _dp]),
    "rexi_plan_set_krylov": (_c_int, [_vp, _c_dbl, _c_int, _c_int]),
    "rexi_plan_set_krylov_method": (_c_int, [_vp, _c_int]),
    "rexi_plan_set_symbol": (_c_int, [_vp, _c_int]),
    "rexi_plan_set_rho": (_c_int, [_vp, _c_dbl]),
    "rexi_plan_set_coefficients": (_c_int, [_vp, _c_int]),
    "rexi_gaussian_fit_table": (_c_int, [_dp, _dp]),
    "rexi_gaussian_refit": (_c_int, [_c_dbl, _c_int, _c_dbl, _c_int, _dp, _dp]),
    "rexi_plan_set_gaussian_fit": (_c_int, [_vp, _c_dbl, _dp]),
    "rexi_plan_set_shift": (_c_int, [_vp, _c_int, _c_dbl]),
    "rexi_plan_get_shift": (_c_int, [_vp, _dp]),
    "rexi_workspace_size": (_c_int, [_vp, _c_dbl, _c_dbl, _c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "rexi_workspace_size_grad_depth": (_c_int, [_vp, _c_dbl, _c_dbl, _c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "rexi_step": (_c_int, [_vp, _vp, _vp, _c_dbl, _c_dbl, _c_int, _c_int, _c_int, _vp, ctypes.c_size_t, _vp,
                           ctypes.POINTER(rexi_step_info)]),
    "rexi_step_adjoint": (_c_int, [_vp, _vp, _vp, _c_dbl, _c_dbl, _c_int, _vp, ctypes.c_size_t, _vp]),
    "rexi_step_grad_depth": (_c_int, [_vp, _vp, _vp, _vp, _c_dbl, _c_dbl, _c_int, _vp, ctypes.c_size_t, _vp,
                                      ctypes.POINTER(rexi_step_info)]),
    "rexi_step_host_async": (_c_int, [_vp, _vp, _vp, _c_dbl, _c_dbl, _c_int, _vp, ctypes.c_size_t, _vp]),
    "rexi_step_host": (_c_int, [_vp, _vp, _vp, _c_dbl, _c_dbl, _c_int, _vp, ctypes.c_size_t, _vp,
                                ctypes.POINTER(rexi_step_info)]),
    "rexi_workspace_size_host": (_c_int, [_vp, _c_dbl, _c_dbl, _c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "rexi_plan_set_profiling": (_c_int, [_vp, _c_int]),
    "rexi_plan_read_profile": (_c_int, [_vp, _dp, _ip, ctypes.POINTER(ctypes.c_int64)]),
    "rexi_step_noalloc": (_c_int, [_c_int, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _vp, _vp,
                                   _c_dbl, _c_dbl, _c_int, _vp]),
    "rexi_batch_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _ip, _ip, _dp, _c_dbl, _c_dbl, _c_dbl, _c_dbl,
                                   _c_dbl, _c_dbl, _c_int, _c_dbl]),
    "rexi_batch_destroy": (None, [_vp]),
    "rexi_batch_layout": (_c_int, [_vp, ctypes.POINTER(ctypes.c_int64), _ip, ctypes.POINTER(ctypes.c_size_t)]),
    "rexi_batch_step": (_c_int, [_vp, _vp, _vp, _c_int, _vp, ctypes.c_size_t, _c_int, _vp]),
    "rexi_batch_autotune": (_c_int, [_vp, _vp, _vp, _c_int, _vp, ctypes.c_size_t, _vp, _ip, _ip, _dp]),
    "rexi_batch_info": (_c_int, [_vp, _ip, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64)]),
    "rexi_alu_probe": (_c_int, [_c_int, _c_int, _c_int, _vp, _vp]),
    "rexi_status_string": (ctypes.c_char_p, [_c_int]),
    "rexi_version": (ctypes.c_char_p, []),
    "rexi_last_error_message": (ctypes.c_char_p, []),
}

_LIB = None


def load(path=LIB_PATH):
    """Load librexi.so and declare the C signatures.  Raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("librexi.so not found at %s: build it with __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class RexiError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.rexi_last_error_message().decode()
        super().__init__("%s: %s (%s)" % (where, lib.rexi_status_string(status).decode(), msg))
        self.status = status


def _check(status, where):
    if status != REXI_OK:
        raise RexiError(status, where)


# ---- host coefficient entry points -----------------------------------------

def rexi_pole_count(tau_rho, h=0.5, tol=1e-10):
    M = ctypes.c_int32()
    _check(load().rexi_pole_count(tau_rho, h, tol, ctypes.byref(M)), "rexi_pole_count")
    return M.value


def rexi_rexii_terms(M, h=0.5):
    """Returns (mu, c1, c2) with c1, c2 complex lists for n = -N..N."""
    import numpy as np

    lib = load()
    mu = ctypes.c_double()
    nt = ctypes.c_int32()
    _check(lib.rexi_rexii_terms(M, h, ctypes.byref(mu), ctypes.byref(nt), None, None, 0), "rexi_rexii_terms")
    c1 = np.zeros(2 * nt.value)
    c2 = np.zeros(2 * nt.value)
    _check(lib.rexi_rexii_terms(M, h, ctypes.byref(mu), ctypes.byref(nt),
                                c1.ctypes.data_as(_dp), c2.ctypes.data_as(_dp), nt.value), "rexi_rexii_terms")
    return mu.value, c1[0::2] + 1j * c1[1::2], c2[0::2] + 1j * c2[1::2]


def rexi_coeffs(tau_rho, tol=1e-10, h=0.5, real_input=True):
    """Returns (M, poles, weights) of the single-shift partial-fraction form."""
    import numpy as np

    lib = load()
    M = ctypes.c_int32()
    J = ctypes.c_int32()
    _check(lib.rexi_coeffs(tau_rho, tol, h, int(real_input), ctypes.byref(M), ctypes.byref(J), None, None, 0),
           "rexi_coeffs")
    p = np.zeros(2 * J.value)
    w = np.zeros(2 * J.value)
    _check(lib.rexi_coeffs(tau_rho, tol, h, int(real_input), ctypes.byref(M), ctypes.byref(J),
                           p.ctypes.data_as(_dp), w.ctypes.data_as(_dp), J.value), "rexi_coeffs")
    return M.value, p[0::2] + 1j * p[1::2], w[0::2] + 1j * w[1::2]


def gaussian_fit_table():
    """(mu, a) of Table tab:coef_al, a[l + 24] = a_l for l = -24..24 (complex)."""
    import numpy as np

    mu = ctypes.c_double()
    arr = (ctypes.c_double * 98)()
    _check(load().rexi_gaussian_fit_table(ctypes.byref(mu), arr), "rexi_gaussian_fit_table")
    v = np.frombuffer(arr, dtype=np.float64).copy()
    return mu.value, v[0::2] + 1j * v[1::2]


def gaussian_refit(mu=None, K=200, xmax=40.0, n_candidates=20001):
    """Least-squares refit on Leja points (host FP64, in the library): returns (mu, a, max_err)."""
    import numpy as np

    if mu is None:
        mu = gaussian_fit_table()[0]
    arr = (ctypes.c_double * 98)()
    err = ctypes.c_double()
    _check(load().rexi_gaussian_refit(float(mu), int(K), float(xmax), int(n_candidates), arr, ctypes.byref(err)),
           "rexi_gaussian_refit")
    v = np.frombuffer(arr, dtype=np.float64).copy()
    return mu, v[0::2] + 1j * v[1::2], err.value


def term_partition(n_terms, world, rank):
    """Contiguous slice [begin, end) of the REXII term indices |n| = 0..n_terms-1
    for `rank` of `world` devices, balanced by count.  Each device passes it to
    rexi_step as term_begin/term_end; the step is linear in the terms, so the
    outputs sum (one all-reduce) to the full step."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(int(n_terms), int(world))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


# ---- plans and the step -----------------------------------------------------

def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def alu_probe(kind, blocks, iters, out, stream=None):
    """Enqueue the multiply-add throughput probe (kind "fp32", "fp64" or
    "fp32x2"); returns the flops it performs (blocks * 256 threads * 256 * iters
    * 2, twice that for the packed kind)."""
    k = {"fp32": 0, "fp64": 1, "fp32x2": 2}[kind]
    _check(load().rexi_alu_probe(k, int(blocks), int(iters), _ptr(out), _stream_handle(stream)), "rexi_alu_probe")
    return blocks * 256 * 256 * iters * 2 * (2 if k == 2 else 1)


class Plan:
    """Owns one rexi_plan_t.  ``depth`` (torch float64 CUDA tensor, (ny, nx))
    selects the variable-depth path; it must stay alive as long as the plan."""

    def __init__(self, nx, ny, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, depth=None, form="fp64", h=0.5):
        lib = load()
        self._lib = lib
        self.nx, self.ny, self.h = int(nx), int(ny), float(h)
        self.form = form
        self._depth = depth
        handle = ctypes.c_void_p()
        dptr = _ptr(depth) if depth is not None else None
        _check(lib.rexi_plan_create(ctypes.byref(handle), self.nx, self.ny, Lx, Ly, g, f, H, dptr,
                                    FORMS[form] if isinstance(form, str) else int(form), self.h),
               "rexi_plan_create")
        self._h = handle

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rexi_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def rho(self):
        r = ctypes.c_double()
        _check(self._lib.rexi_spectral_radius(self._h, ctypes.byref(r)), "rexi_spectral_radius")
        return r.value

    def set_symbol(self, symbol):
        """"cgrid", "spectral" or "schrodinger" (constant-depth plans)."""
        code = SYMBOLS.get(symbol, symbol)
        _check(self._lib.rexi_plan_set_symbol(self._h, int(code)), "rexi_plan_set_symbol")

    def set_coefficients(self, name):
        """"rexii" (default), "rexi" (original, eq. originalREXImatrix) or "rexie" (eq. REXIE)."""
        _check(self._lib.rexi_plan_set_coefficients(self._h, int(COEFFICIENT_SETS.get(name, name))),
               "rexi_plan_set_coefficients")

    def set_gaussian_fit(self, mu=None, a=None):
        """Use (mu, a) (a: 49 complex values a_-24..a_24) instead of the table; no arguments restore it."""
        if a is None:
            _check(self._lib.rexi_plan_set_gaussian_fit(self._h, 0.0, None), "rexi_plan_set_gaussian_fit")
            return
        import numpy as np

        a = np.asarray(a, dtype=np.complex128)
        arr = (ctypes.c_double * 98)(*np.column_stack([a.real, a.imag]).ravel().tolist())
        _check(self._lib.rexi_plan_set_gaussian_fit(self._h, float(mu), arr), "rexi_plan_set_gaussian_fit")

    def set_shift(self, mode="none", sigma=0.0):
        """Spectral shift nu = i sigma: mode "none", "midpoint" or "value" (with sigma)."""
        code = {"none": REXI_SHIFT_NONE, "midpoint": REXI_SHIFT_MIDPOINT, "value": REXI_SHIFT_VALUE}.get(mode, mode)
        _check(self._lib.rexi_plan_set_shift(self._h, int(code), float(sigma)), "rexi_plan_set_shift")

    @property
    def shift(self):
        v = ctypes.c_double()
        _check(self._lib.rexi_plan_get_shift(self._h, ctypes.byref(v)), "rexi_plan_get_shift")
        return v.value

    def set_rho(self, rho):
        """Override rho for the pole count (0 restores the plan's own value)."""
        _check(self._lib.rexi_plan_set_rho(self._h, float(rho)), "rexi_plan_set_rho")

    def set_krylov(self, rtol=1e-10, max_iters=20000, term_batch=64):
        _check(self._lib.rexi_plan_set_krylov(self._h, rtol, max_iters, term_batch), "rexi_plan_set_krylov")

    def set_krylov_method(self, method):
        """Variable-depth solver: "cg" (one CG per REXII term) or "shared" (one Lanczos basis for all poles)."""
        code = KRYLOV_METHODS[method] if isinstance(method, str) else int(method)
        _check(self._lib.rexi_plan_set_krylov_method(self._h, code), "rexi_plan_set_krylov_method")

    def krylov_vector_bytes(self, real_input=True):
        """Bytes of one kept Lanczos vector of the shared-Krylov method (extra workspace beyond
        workspace_size() holds as many as fit)."""
        return (3 * self.nx * self.ny * (8 if real_input else 16) + 255) // 256 * 256

    def workspace_size(self, dt, tol=1e-10, real_input=True, grad_depth=False):
        b = ctypes.c_size_t()
        fn = "rexi_workspace_size_grad_depth" if grad_depth else "rexi_workspace_size"
        _check(getattr(self._lib, fn)(self._h, dt, tol, int(real_input), ctypes.byref(b)), fn)
        return b.value

    def workspace(self, dt, tol=1e-10, real_input=True, device=None, grad_depth=False):
        import torch

        n = self.workspace_size(dt, tol, real_input, grad_depth=grad_depth)
        return torch.empty(max(n, 256), dtype=torch.uint8, device=device or "cuda")

    def step(self, state, dt, tol=1e-10, real_input=True, out=None, workspace=None, stream=None,
             terms=(0, -1), want_info=False):
        """out = r(dt A) state; ``state`` complex128 CUDA tensor (3, ny, nx)."""
        import torch

        if out is None:
            out = torch.empty_like(state)
        if workspace is None:
            workspace = self.workspace(dt, tol, real_input, device=state.device)
        info = rexi_step_info() if want_info else None
        st = self._lib.rexi_step(self._h, _ptr(state), _ptr(out), dt, tol, int(real_input), int(terms[0]),
                                 int(terms[1]), _ptr(workspace), workspace.numel(), _stream_handle(stream),
                                 ctypes.byref(info) if info is not None else None)
        _check(st, "rexi_step")
        return (out, info) if want_info else out

    def workspace_host(self, dt, tol=1e-10, real_input=True, device=None):
        import torch

        b = ctypes.c_size_t()
        _check(self._lib.rexi_workspace_size_host(self._h, dt, tol, int(real_input), ctypes.byref(b)),
               "rexi_workspace_size_host")
        return torch.empty(max(b.value, 256), dtype=torch.uint8, device=device or "cuda")

    def step_host(self, state_host, out_host, dt, tol=1e-10, real_input=True, workspace=None, stream=None,
                  blocking=True):
        """Host-buffer step: ``state_host``/``out_host`` are CPU tensors (pinned for full speed).
        With blocking=False the copies and the step are only enqueued on ``stream``
        (rexi_step_host_async): ``out_host`` is ready once the stream gets there."""
        if workspace is None:
            workspace = self.workspace_host(dt, tol, real_input)
        if blocking:
            st = self._lib.rexi_step_host(self._h, ctypes.c_void_p(state_host.data_ptr()),
                                          ctypes.c_void_p(out_host.data_ptr()), dt, tol, int(real_input),
                                          _ptr(workspace), workspace.numel(), _stream_handle(stream), None)
            _check(st, "rexi_step_host")
        else:
            st = self._lib.rexi_step_host_async(self._h, ctypes.c_void_p(state_host.data_ptr()),
                                                ctypes.c_void_p(out_host.data_ptr()), dt, tol, int(real_input),
                                                _ptr(workspace), workspace.numel(), _stream_handle(stream))
            _check(st, "rexi_step_host_async")
        return out_host

    def set_profiling(self, enable=True):
        _check(self._lib.rexi_plan_set_profiling(self._h, int(enable)), "rexi_plan_set_profiling")

    def read_profile(self):
        """Returns (ms per phase [fwd, poles, inv, upload, combine part of poles], calls, kernel
        launches) since the last read."""
        ms = (ctypes.c_double * 5)()
        n = ctypes.c_int32()
        L = ctypes.c_int64()
        _check(self._lib.rexi_plan_read_profile(self._h, ms, ctypes.byref(n), ctypes.byref(L)),
               "rexi_plan_read_profile")
        return list(ms), n.value, L.value

    def grad_depth(self, state, grad_out, dt, tol=1e-10, real_input=True, grad=None, workspace=None, stream=None,
                   want_info=False):
        """grad += dL/dH for out = r(dt A(H)) state and grad_out = dL/d out (variable depth)."""
        import torch

        if grad is None:
            grad = torch.zeros((self.ny, self.nx), dtype=torch.float64, device=state.device)
        if workspace is None:
            workspace = self.workspace(dt, tol, real_input, device=state.device, grad_depth=True)
        info = rexi_step_info() if want_info else None
        st = self._lib.rexi_step_grad_depth(self._h, _ptr(state), _ptr(grad_out), _ptr(grad), dt, tol,
                                            int(real_input), _ptr(workspace), workspace.numel(),
                                            _stream_handle(stream), ctypes.byref(info) if info is not None else None)
        _check(st, "rexi_step_grad_depth")
        return (grad, info) if want_info else grad

    def step_adjoint(self, grad_out, dt, tol=1e-10, real_input=True, out=None, workspace=None, stream=None):
        import torch

        if out is None:
            out = torch.empty_like(grad_out)
        if workspace is None:
            workspace = self.workspace(dt, tol, real_input, device=grad_out.device)
        st = self._lib.rexi_step_adjoint(self._h, _ptr(grad_out), _ptr(out), dt, tol, int(real_input),
                                         _ptr(workspace), workspace.numel(), _stream_handle(stream))
        _check(st, "rexi_step_adjoint")
        return out


class Batch:
    """Owns one rexi_batch_t: many constant-depth instances stepped together.

    ``sizes`` is a list of (nx, ny), ``dts`` the per-instance time steps.
    ``pack``/``unpack`` move per-instance (3, ny, nx) tensors in and out of the
    packed device buffer (plain tensor copies; the step itself is one call)."""

    def __init__(self, sizes, dts, Lx=1.0, Ly=1.0, g=1.0, f=1.0, H=1.0, tol=1e-10, form="fp64", h=0.5):
        import numpy as np

        lib = load()
        self._lib = lib
        self.n = len(sizes)
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        nx = (ctypes.c_int32 * self.n)(*[s[0] for s in self.sizes])
        ny = (ctypes.c_int32 * self.n)(*[s[1] for s in self.sizes])
        dt = (ctypes.c_double * self.n)(*[float(d) for d in dts])
        handle = ctypes.c_void_p()
        _check(lib.rexi_batch_create(ctypes.byref(handle), self.n, nx, ny, dt, Lx, Ly, g, f, H, tol,
                                     FORMS[form] if isinstance(form, str) else int(form), h), "rexi_batch_create")
        self._h = handle
        offs = (ctypes.c_int64 * (self.n + 1))()
        Ms = (ctypes.c_int32 * self.n)()
        ws = ctypes.c_size_t()
        _check(lib.rexi_batch_layout(handle, offs, Ms, ctypes.byref(ws)), "rexi_batch_layout")
        self.offsets = np.array(offs[:], dtype=np.int64)
        self.M = list(Ms[:])
        self.workspace_bytes = ws.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rexi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, device="cuda"):
        import torch

        return torch.empty(int(self.offsets[-1]), dtype=torch.complex128, device=device)

    def workspace(self, device="cuda"):
        import torch

        return torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)

    def pack(self, states, out=None):
        buf = self.empty(states[0].device) if out is None else out
        for i, (nx, ny) in enumerate(self.sizes):
            buf[int(self.offsets[i]):int(self.offsets[i]) + 3 * nx * ny].copy_(states[i].reshape(-1))
        return buf

    def unpack(self, buf):
        return [buf[int(self.offsets[i]):int(self.offsets[i]) + 3 * nx * ny].view(3, ny, nx)
                for i, (nx, ny) in enumerate(self.sizes)]

    def step(self, packed_in, packed_out=None, workspace=None, real_input=True, mode=REXI_BATCH_PERSISTENT,
             stream=None):
        if packed_out is None:
            packed_out = packed_in.new_empty(packed_in.shape)
        if workspace is None:
            workspace = self.workspace(packed_in.device)
        _check(self._lib.rexi_batch_step(self._h, _ptr(packed_in), _ptr(packed_out), int(real_input),
                                         _ptr(workspace), workspace.numel(), int(mode), _stream_handle(stream)),
               "rexi_batch_step")
        return packed_out

    def autotune(self, packed_in, packed_out, workspace, real_input=True, stream=None):
        t = ctypes.c_int32()
        p = ctypes.c_int32()
        ms = ctypes.c_double()
        _check(self._lib.rexi_batch_autotune(self._h, _ptr(packed_in), _ptr(packed_out), int(real_input),
                                             _ptr(workspace), workspace.numel(), _stream_handle(stream),
                                             ctypes.byref(t), ctypes.byref(p), ctypes.byref(ms)),
               "rexi_batch_autotune")
        return t.value, p.value, ms.value

    def info(self):
        vals = [ctypes.c_int32() for _ in range(4)] + [ctypes.c_int64(), ctypes.c_int64()]
        _check(self._lib.rexi_batch_info(self._h, *[ctypes.byref(v) for v in vals]), "rexi_batch_info")
        keys = ["threads", "orbits_per_thread", "ctas", "n_items", "terms_orbits", "launches"]
        return {k: v.value for k, v in zip(keys, vals)}
