"""Python binding of libsfista (ctypes; argument marshalling only).

Every function here forwards to the C entry point of the same name declared
in ``include/sfista.h``; all arithmetic runs in the library's CUDA kernels and
host setup.  PyTorch provides device memory and streams.  If the shared
library is missing or fails to load, ``load()`` raises: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfista.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTSUP, ENUMERIC, ETIMEOUT = range(7)
BC = {"zero": 0, "reflexive": 1, "reflective": 1, "periodic": 2}
PREC = {"fp32": 0, "tf32": 1, "tf32x3": 2, "bf16": 3, "bf16x3": 4}
OP = {"auto": 0, "banded": 1, "gemm_band": 2, "gemm_dense": 3, "banded_persistent": 4, "banded_fused": 5,
      "fft": 6, "exact_fft": 7}
PREC_NAME = {v: k for k, v in PREC.items()}
OP_NAME = {v: k for k, v in OP.items()}

_lib = None


class SfistaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("sfista status %d (%s): %s" % (status, _strerror(status), msg))
        self.status = status


class TuneEntry(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("stage", ctypes.c_int), ("chunk", ctypes.c_int), ("ms", ctypes.c_float)]


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("op", ctypes.c_int), ("project_nonneg", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("lipschitz", ctypes.c_double),
                ("lipschitz_tol", ctypes.c_double), ("lipschitz_maxit", ctypes.c_int),
                ("device", ctypes.c_int), ("l1", ctypes.c_double), ("refine_every", ctypes.c_int),
                ("tile_override", ctypes.c_int), ("gemm_bn", ctypes.c_int),
                ("gemm_resident_panels", ctypes.c_int)]


def load(path=None):
    """Load libsfista.so (raises OSError if it is missing: no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError("libsfista.so not built (%s); run paper_1901_00913_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    vp, i, d, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    L.sfista_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.sfista_default_opts.restype = None
    L.sfista_setup.argtypes = [vp, i, i, i, i, i, i, i, i, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    L.sfista_setup_exact.argtypes = [vp, i, i, i, i, i, i, i, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    L.sfista_factorize.argtypes = [vp, i, i, i, i, i, i, i, i, vp, vp, vp, D]
    L.sfista_factor_bands.argtypes = [vp, i, i, i, i, i, i, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), vp, vp]
    L.sfista_destroy.argtypes = [vp]
    L.sfista_destroy.restype = None
    L.sfista_solve.argtypes = [vp, vp, d, i, vp]
    L.sfista_solve_device.argtypes = [vp, vp, d, i, vp, vp]
    L.sfista_solve_state.argtypes = [vp, vp, d, i, i, vp, vp, vp]
    L.sfista_sync.argtypes = [vp, vp]
    L.sfista_apply.argtypes = [vp, vp, vp, i, vp]
    L.sfista_info.argtypes = [vp, D, vp, D, vp]
    L.sfista_get_profiles.argtypes = [vp, vp, vp]
    L.sfista_get_factors.argtypes = [vp, vp, vp]
    L.sfista_set_factors.argtypes = [vp, vp, vp]
    L.sfista_blur.argtypes = [vp, i, i, i, i, i, vp, i, i, vp, vp]
    L.sfista_time_stages.argtypes = [vp, vp, d, i, vp]
    L.sfista_objective.argtypes = [vp, vp, vp, d, ctypes.POINTER(ctypes.c_double), vp]
    L.sfista_tune.argtypes = [vp, i, ctypes.POINTER(TuneEntry), i, ctypes.POINTER(ctypes.c_int)]
    L.sfista_batch_tune.argtypes = [vp, i, ctypes.POINTER(TuneEntry), i, ctypes.POINTER(ctypes.c_int)]
    L.sfista_apply_static.argtypes = [vp, vp, i, i, i, vp, i, i, vp, i, i, vp]
    L.sfista_batch_create.argtypes = [vp, i, ctypes.POINTER(vp)]
    L.sfista_batch_solve.argtypes = [vp, vp, vp, i, vp, vp]
    L.sfista_batch_sync.argtypes = [vp, vp]
    L.sfista_batch_destroy.argtypes = [vp]
    L.sfista_batch_destroy.restype = None
    L.sfista_solve_batched.argtypes = [vp, vp, vp, i, i, vp, vp]
    L.sfista_selftest_wait_timeout.argtypes = [vp]
    L.sfista_unrolled_fwd.argtypes = [vp, vp, d, i, i, vp, vp, vp]
    L.sfista_unrolled_bwd.argtypes = [vp, vp, d, i, i, vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp]
    L.sfista_strerror.argtypes = [i]
    L.sfista_strerror.restype = ctypes.c_char_p
    L.sfista_last_error.argtypes = []
    L.sfista_last_error.restype = ctypes.c_char_p
    for name in ("sfista_setup", "sfista_setup_exact", "sfista_factorize", "sfista_solve", "sfista_solve_device", "sfista_solve_state",
                 "sfista_sync", "sfista_apply", "sfista_info", "sfista_get_profiles",
                 "sfista_get_factors", "sfista_set_factors", "sfista_blur", "sfista_time_stages",
                 "sfista_apply_static", "sfista_batch_create", "sfista_batch_solve", "sfista_batch_sync",
                 "sfista_solve_batched", "sfista_unrolled_fwd", "sfista_unrolled_bwd", "sfista_selftest_wait_timeout"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _strerror(s):
    try:
        return load().sfista_strerror(s).decode()
    except OSError:
        return "?"


def _check(status):
    if status != OK:
        raise SfistaError(status, load().sfista_last_error().decode())


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def default_opts():
    o = Opts()
    load().sfista_default_opts(ctypes.byref(o))
    return o


# ------------------------------------------------------------------ C-named calls
def sfista_setup(psf, img_rows, img_cols, bc, r, center=(-1, -1), opts=None):
    """Returns an opaque context handle (int).  See include/sfista.h."""
    P = np.ascontiguousarray(psf, dtype=np.float64)
    h = ctypes.c_void_p()
    o = opts if opts is not None else default_opts()
    _check(load().sfista_setup(P.ctypes.data, P.shape[0], P.shape[1], int(center[0]), int(center[1]),
                               int(img_rows), int(img_cols), int(bc), int(r), ctypes.byref(o),
                               ctypes.byref(h)))
    return h.value


def sfista_setup_exact(psf, img_rows, img_cols, bc, center=(-1, -1), opts=None):
    """Context whose operator is the exact blur A (Alg. 1 on the unapproximated problem); see include/sfista.h."""
    P = np.ascontiguousarray(psf, dtype=np.float64)
    h = ctypes.c_void_p()
    o = opts if opts is not None else default_opts()
    _check(load().sfista_setup_exact(P.ctypes.data, P.shape[0], P.shape[1], int(center[0]), int(center[1]),
                                     int(img_rows), int(img_cols), int(bc), ctypes.byref(o), ctypes.byref(h)))
    return h.value


def sfista_factorize(psf, img_rows, img_cols, bc, r, center=(-1, -1)):
    """Host-only FP64 factorisation; returns (sigma, C, D, approx_err)."""
    P = np.ascontiguousarray(psf, dtype=np.float64)
    p, q = P.shape
    sig = np.zeros(min(p, q))
    C = np.zeros((r, p))
    D = np.zeros((r, q))
    err = ctypes.c_double()
    _check(load().sfista_factorize(P.ctypes.data, p, q, int(center[0]), int(center[1]), int(img_rows),
                                   int(img_cols), int(bc), int(r), sig.ctypes.data, C.ctypes.data,
                                   D.ctypes.data, ctypes.byref(err)))
    return sig, C, D, err.value


def sfista_factor_bands(psf, img_rows, img_cols, bc, r, which, center=(-1, -1)):
    """Host-only band storage of one factor family (which: 0 A, 1 A^T, 2 B,
    3 B^T); returns (band r x w x len, lo, (i0, i1) interior rows)."""
    P = np.ascontiguousarray(psf, dtype=np.float64)
    p, q = P.shape
    lo, w = ctypes.c_int(), ctypes.c_int()
    args = (P.ctypes.data, p, q, int(center[0]), int(center[1]), int(img_rows), int(img_cols), int(bc), int(r),
            int(which))
    _check(load().sfista_factor_bands(*args, ctypes.byref(lo), ctypes.byref(w), None, None))
    length = int(img_cols) if which in (0, 1) else int(img_rows)
    band = np.zeros((int(r), w.value, length))
    inter = (ctypes.c_int * 2)()
    _check(load().sfista_factor_bands(*args, ctypes.byref(lo), ctypes.byref(w), band.ctypes.data, inter))
    return band, lo.value, (inter[0], inter[1])


def sfista_destroy(ctx):
    load().sfista_destroy(ctypes.c_void_p(ctx))


def sfista_solve(ctx, b, lam, iters, x):
    """Host buffers: b, x float32 contiguous numpy arrays of the image shape."""
    assert b.dtype == np.float32 and x.dtype == np.float32 and b.flags.c_contiguous and x.flags.c_contiguous
    _check(load().sfista_solve(ctypes.c_void_p(ctx), b.ctypes.data, float(lam), int(iters), x.ctypes.data))


def sfista_solve_device(ctx, d_b, lam, iters, d_x, stream=None):
    _check(load().sfista_solve_device(ctypes.c_void_p(ctx), _ptr(d_b), float(lam), int(iters), _ptr(d_x),
                                      _stream_ptr(stream)))


def sfista_solve_state(ctx, d_b, lam, k0, iters, d_X, d_Xprev, stream=None):
    _check(load().sfista_solve_state(ctypes.c_void_p(ctx), _ptr(d_b), float(lam), int(k0), int(iters),
                                     _ptr(d_X), _ptr(d_Xprev), _stream_ptr(stream)))


def sfista_sync(ctx, stream=None):
    _check(load().sfista_sync(ctypes.c_void_p(ctx), _stream_ptr(stream)))


def sfista_apply(ctx, d_x, d_y, transpose=False, stream=None):
    _check(load().sfista_apply(ctypes.c_void_p(ctx), _ptr(d_x), _ptr(d_y), int(bool(transpose)),
                               _stream_ptr(stream)))


def sfista_info(ctx, kmax):
    L = ctypes.c_double()
    err = ctypes.c_double()
    sig = np.zeros(kmax)
    cfg = np.zeros(8, dtype=np.int32)
    _check(load().sfista_info(ctypes.c_void_p(ctx), ctypes.byref(L), sig.ctypes.data, ctypes.byref(err),
                              cfg.ctypes.data))
    return {"lipschitz": L.value, "sigma": sig, "approx_err": err.value,
            "prec": PREC_NAME[int(cfg[0])], "op": OP_NAME[int(cfg[1])],
            "band_right": int(cfg[2]), "band_left": int(cfg[3]),
            "lo": {"A": int(cfg[4]), "B": int(cfg[5]), "AT": int(cfg[6]), "BT": int(cfg[7])}}


def sfista_get_profiles(ctx, r, p, q):
    C = np.zeros((r, p))
    D = np.zeros((r, q))
    _check(load().sfista_get_profiles(ctypes.c_void_p(ctx), C.ctypes.data, D.ctypes.data))
    return C, D


def sfista_get_factors(ctx, r, m, n):
    A = np.zeros((r, n, n))
    B = np.zeros((r, m, m))
    _check(load().sfista_get_factors(ctypes.c_void_p(ctx), A.ctypes.data, B.ctypes.data))
    return A, B


def _host_f64(t):
    """Host FP64 contiguous copy of a numpy array or torch tensor (marshalling)."""
    if hasattr(t, "detach"):
        t = t.detach().double().cpu().numpy()
    return np.ascontiguousarray(t, dtype=np.float64)


def sfista_set_factors(ctx, A=None, B=None):
    """Replace the dense factors (A: r x n x n, B: r x m x m; None keeps them); see include/sfista.h."""
    Ah = _host_f64(A) if A is not None else None
    Bh = _host_f64(B) if B is not None else None
    _check(load().sfista_set_factors(ctypes.c_void_p(ctx), Ah.ctypes.data if Ah is not None else None,
                                     Bh.ctypes.data if Bh is not None else None))


def sfista_blur(psf, d_x, bc, center=(-1, -1), d_y=None, stream=None):
    """Exact blur of Eq. (1.1) of a CUDA float32 image; returns d_y."""
    import torch
    P = np.ascontiguousarray(psf, dtype=np.float64)
    if d_y is None:
        d_y = torch.empty_like(d_x)
    m, n = d_x.shape
    _check(load().sfista_blur(P.ctypes.data, P.shape[0], P.shape[1], int(center[0]), int(center[1]), int(bc),
                              _ptr(d_x), m, n, _ptr(d_y), _stream_ptr(stream)))
    return d_y


def sfista_time_stages(ctx, d_b, lam, reps):
    """Mean ms of the four per-iteration stages (see include/sfista.h)."""
    ms = np.zeros(4, dtype=np.float32)
    _check(load().sfista_time_stages(ctypes.c_void_p(ctx), _ptr(d_b), float(lam), int(reps), ms.ctypes.data))
    return ms


def sfista_objective(ctx, d_b, d_x, lam, stream=None):
    """Phi_s(X) = 1/2 ||A_s X - B||^2 + 1/2 lam^2 ||X||^2 on the device (see include/sfista.h)."""
    phi = ctypes.c_double()
    _check(load().sfista_objective(ctypes.c_void_p(ctx), _ptr(d_b), _ptr(d_x), float(lam), ctypes.byref(phi),
                                   _stream_ptr(stream)))
    return phi.value


def sfista_tune(ctx, iters=10, max_entries=64):
    """Autotuner (see include/sfista.h): returns every measurement as dicts."""
    buf = (TuneEntry * max_entries)()
    cnt = ctypes.c_int(0)
    _check(load().sfista_tune(ctypes.c_void_p(ctx), int(iters), buf, int(max_entries), ctypes.byref(cnt)))
    return [{"op": OP_NAME.get(e.op, e.op), "stage": e.stage, "chunk": e.chunk, "ms": e.ms}
            for e in buf[:min(cnt.value, max_entries)]]


def sfista_batch_tune(handle, iters=5, max_entries=64):
    """Batch autotuner (see include/sfista.h): one dict per plan; "op" names the
    plan's form (banded: grouped launches with a shared-memory budget of
    budget_kb KB; banded_persistent: the whole batch in one launch; tensor-core
    forms: "chunk" 1 / 0 for resident / streamed factor panels)."""
    buf = (TuneEntry * max_entries)()
    cnt = ctypes.c_int(0)
    _check(load().sfista_batch_tune(ctypes.c_void_p(handle), int(iters), buf, int(max_entries), ctypes.byref(cnt)))
    return [{"op": OP_NAME.get(e.op, e.op), "budget_kb": e.chunk, "chunk": e.chunk, "ms": e.ms}
            for e in buf[:min(cnt.value, max_entries)]]


def sfista_apply_static(d_x, d_y, r, band_right, lo_right, band_left, lo_left, stream=None):
    """Operator without allocation; band tables are CUDA float32 tensors (r, w, len)."""
    m, n = d_x.shape
    _check(load().sfista_apply_static(_ptr(d_x), _ptr(d_y), m, n, int(r), _ptr(band_right), int(lo_right),
                                      int(band_right.shape[1]), _ptr(band_left), int(lo_left),
                                      int(band_left.shape[1]), _stream_ptr(stream)))


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t).value
    return arr


def sfista_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    h = ctypes.c_void_p()
    _check(load().sfista_batch_create(arr, len(ctxs), ctypes.byref(h)))
    return h.value


def sfista_batch_solve(batch, d_bs, lambdas, iters, d_xs, stream=None):
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    _check(load().sfista_batch_solve(ctypes.c_void_p(batch), _ptr_array(d_bs), lam.ctypes.data, int(iters),
                                     _ptr_array(d_xs), _stream_ptr(stream)))


def sfista_batch_sync(batch, stream=None):
    _check(load().sfista_batch_sync(ctypes.c_void_p(batch), _stream_ptr(stream)))


def sfista_batch_destroy(batch):
    load().sfista_batch_destroy(ctypes.c_void_p(batch))


def sfista_solve_batched(ctxs, d_bs, lambdas, iters, d_xs, stream=None):
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    _check(load().sfista_solve_batched(arr, _ptr_array(d_bs), lam.ctypes.data, len(ctxs), int(iters),
                                       _ptr_array(d_xs), _stream_ptr(stream)))


class Batch:
    """Groups Sfista objects: ``Batch([s1, s2, ...]).solve([b1, b2, ...], [lam1, ...], iters)``."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.handle = sfista_batch_create([s.ctx for s in self.solvers])

    def solve(self, d_bs, lambdas, iters, outs=None, stream=None, sync=True):
        import torch
        outs = [torch.empty_like(b) for b in d_bs] if outs is None else outs
        sfista_batch_solve(self.handle, d_bs, lambdas, iters, outs, stream)
        if sync:
            sfista_batch_sync(self.handle, stream)
        return outs

    def tune(self, iters=5):
        """Chooses the batch plan by measurement (grouped launches and their shared-memory budget, or one
        launch for the whole batch); returns the measurements."""
        return sfista_batch_tune(self.handle, iters)

    def close(self):
        if self.handle:
            sfista_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfista_selftest_wait_timeout(ctx):
    """Returns the status of the bounded-wait self-test (SFISTA_ETIMEOUT when the guard works)."""
    return load().sfista_selftest_wait_timeout(ctypes.c_void_p(ctx))


def sfista_unrolled_fwd(ctx, d_b, lam, iters, ckpt_every, d_ckpt, d_x, stream=None):
    _check(load().sfista_unrolled_fwd(ctypes.c_void_p(ctx), _ptr(d_b), float(lam), int(iters), int(ckpt_every),
                                      _ptr(d_ckpt), _ptr(d_x), _stream_ptr(stream)))


def sfista_unrolled_bwd(ctx, d_b, lam, iters, ckpt_every, d_ckpt, d_gX, d_gb, d_gA=None, d_gB=None, stream=None):
    gl = ctypes.c_double()
    _check(load().sfista_unrolled_bwd(ctypes.c_void_p(ctx), _ptr(d_b), float(lam), int(iters), int(ckpt_every),
                                      _ptr(d_ckpt), _ptr(d_gX), _ptr(d_gb), ctypes.byref(gl),
                                      _ptr(d_gA) if d_gA is not None else None,
                                      _ptr(d_gB) if d_gB is not None else None, _stream_ptr(stream)))
    return gl.value


def _unrolled_function():
    import torch

    class SfistaUnrolled(torch.autograd.Function):
        """X_iters of Alg. 2 as a differentiable function of (b, lambda, A, B).

        A (r x n x n) and B (r x m x m) are the dense factors the solve uses:
        when given, they are loaded into the context first (sfista_set_factors;
        they must be zero outside the band of the context's factors), so the
        forward and the gradients dl/dA_i, dl/dB_i follow the tensors passed.
        None keeps the context's current factors.  L is held fixed.
        """

        @staticmethod
        def forward(fctx, solver, b, lam, A, B, iters, ckpt_every):
            if A is not None or B is not None:
                sfista_set_factors(solver.ctx, A, B)
            m, n = b.shape
            nseg = (iters + ckpt_every - 1) // ckpt_every
            ck = torch.empty(2 * nseg, m, n, dtype=torch.float64, device=b.device)
            x = torch.empty_like(b)
            lam_v = float(lam)
            sfista_unrolled_fwd(solver.ctx, b.contiguous(), lam_v, iters, ckpt_every, ck, x)
            sfista_sync(solver.ctx)
            fctx.solver, fctx.iters, fctx.ckpt, fctx.lam = solver, iters, ckpt_every, lam_v
            fctx.save_for_backward(b.contiguous(), ck, lam)
            fctx.want = (A.requires_grad if A is not None else False, B.requires_grad if B is not None else False)
            fctx.shapes = (None if A is None else A.shape, None if B is None else B.shape)
            fctx.dtypes = (None if A is None else A.dtype, None if B is None else B.dtype)
            return x

        @staticmethod
        def backward(fctx, gX):
            b, ck, lam = fctx.saved_tensors
            gb = torch.empty_like(b)
            gA = torch.empty(fctx.shapes[0], dtype=torch.float32, device=b.device) if fctx.want[0] else None
            gB = torch.empty(fctx.shapes[1], dtype=torch.float32, device=b.device) if fctx.want[1] else None
            gl = sfista_unrolled_bwd(fctx.solver.ctx, b, fctx.lam, fctx.iters, fctx.ckpt, ck,
                                     gX.contiguous().float(), gb, gA, gB)
            glam = torch.tensor(gl, dtype=lam.dtype, device=lam.device).reshape(lam.shape)
            gA = gA.to(fctx.dtypes[0]) if gA is not None else None
            gB = gB.to(fctx.dtypes[1]) if gB is not None else None
            return None, gb, glam, gA, gB, None, None

    return SfistaUnrolled


_UNROLLED = None


def unrolled_solve(solver, b, lam, iters, ckpt_every=10, A=None, B=None):
    """Differentiable X_iters = sFISTA(b, lambda; A, B) for ``solver`` (banded FP32 form)."""
    global _UNROLLED
    import torch
    if _UNROLLED is None:
        _UNROLLED = _unrolled_function()
    if not torch.is_tensor(lam):
        lam = torch.tensor(float(lam), dtype=torch.float64, device=b.device)
    return _UNROLLED.apply(solver, b, lam, A, B, iters, ckpt_every)


# ------------------------------------------------------------------ convenience wrapper
class Sfista:
    """Owns one context: ``Sfista(psf, (m, n), 'reflexive', r=3, prec='bf16x3')``."""

    def __init__(self, psf, shape, bc, r, center=(-1, -1), prec="fp32", op="auto", project=False,
                 use_graph=True, lipschitz=None, lipschitz_tol=1e-10, lipschitz_maxit=1000, device=-1, l1=0.0,
                 refine_every=0, tile_override=0, exact=False, gemm_bn=0, gemm_resident_panels=False):
        """exact=True: the exact blur A instead of the rank-r approximation (sfista_setup_exact; r unused)."""
        o = default_opts()
        o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        o.op = OP[op] if isinstance(op, str) else int(op)
        o.project_nonneg = int(bool(project))
        o.use_graph = int(bool(use_graph))
        o.lipschitz = float(lipschitz) if lipschitz else 0.0
        o.lipschitz_tol = float(lipschitz_tol)
        o.lipschitz_maxit = int(lipschitz_maxit)
        o.device = int(device)
        o.l1 = float(l1)
        o.refine_every = int(refine_every)
        o.tile_override = int(tile_override)
        o.gemm_bn = int(gemm_bn)
        o.gemm_resident_panels = int(bool(gemm_resident_panels))
        bcv = BC[bc] if isinstance(bc, str) else int(bc)
        self.shape = (int(shape[0]), int(shape[1]))
        self.psf_shape = np.asarray(psf).shape
        self.r = int(r)
        self.exact = bool(exact)
        if self.exact:
            self.ctx = sfista_setup_exact(psf, self.shape[0], self.shape[1], bcv, center, o)
        else:
            self.ctx = sfista_setup(psf, self.shape[0], self.shape[1], bcv, r, center, o)

    def close(self):
        if self.ctx:
            sfista_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return sfista_info(self.ctx, 0 if self.exact else min(self.psf_shape))

    def objective(self, d_b, d_x, lam):
        """Phi_s(X) for device tensors B and X."""
        return sfista_objective(self.ctx, d_b, d_x, lam)

    def tune(self, iters=10):
        """Times the candidate configurations and keeps the fastest; returns the measurements
        (for one-launch solver entries, ``chunk`` is the tile height)."""
        return sfista_tune(self.ctx, iters)

    def profiles(self):
        return sfista_get_profiles(self.ctx, self.r, *self.psf_shape)

    def factors(self):
        return sfista_get_factors(self.ctx, self.r, *self.shape)

    def set_factors(self, A=None, B=None):
        """Use the given dense factors (zero outside the band) from now on; see include/sfista.h."""
        sfista_set_factors(self.ctx, A, B)

    def solve(self, b, lam, iters):
        b = np.ascontiguousarray(b, dtype=np.float32)
        x = np.empty_like(b)
        sfista_solve(self.ctx, b, lam, iters, x)
        return x

    def solve_device(self, d_b, lam, iters, out=None, stream=None, sync=True):
        import torch
        out = torch.empty_like(d_b) if out is None else out
        sfista_solve_device(self.ctx, d_b, lam, iters, out, stream)
        if sync:
            sfista_sync(self.ctx, stream)
        return out

    def solve_state(self, d_b, lam, k0, iters, X, Xprev, stream=None, sync=True):
        sfista_solve_state(self.ctx, d_b, lam, k0, iters, X, Xprev, stream)
        if sync:
            sfista_sync(self.ctx, stream)
        return X, Xprev

    def apply(self, d_x, transpose=False, out=None, stream=None, sync=True):
        import torch
        out = torch.empty_like(d_x) if out is None else out
        sfista_apply(self.ctx, d_x, out, transpose, stream)
        if sync:
            sfista_sync(self.ctx, stream)
        return out
