"""ctypes binding of libdgfs.so: argument marshalling only.

The functions mirror the C ABI of ``include/dgfs.h`` one to one (same names, same
arguments, pointers passed as integers).  ``Plan`` is a convenience holder that builds the
descriptor, owns the handle and accepts torch tensors (their ``data_ptr()``) for device
memory and ``torch.cuda.Stream`` objects for streams.  Every evaluation runs in the CUDA
library; there is no other implementation behind this module, and a missing library is an
error.
"""

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdgfs.so")

DGFS_OK = 0
DGFS_ERR_INVALID_ARG = -1
DGFS_ERR_UNSUPPORTED_N = -2
DGFS_ERR_OOM = -3
DGFS_ERR_BUDGET = -4
DGFS_ERR_CUDA = -5
DGFS_ERR_DEVICE_TIMEOUT = -6
DGFS_ERR_UNSUPPORTED = -7
DGFS_FP64 = 0
DGFS_FP32 = 1
DGFS_BF16X3 = 2
DGFS_CONSERVE = 1
DGFS_SUM_SPECIES = 2
DGFS_LOSS_ACCURATE = 4
DGFS_PER_PAIR_R = 8
DGFS_BC_PERIODIC = 0
DGFS_BC_WALLS = 1
DGFS_SIDE_WALL = 0
DGFS_SIDE_INFLOW = 1

EXPORTS = ("dgfs_create_plan", "dgfs_destroy_plan", "dgfs_eval_collision",
           "dgfs_eval_collision_host", "dgfs_plan_bytes", "dgfs_plan_radius",
           "dgfs_plan_launches", "dgfs_plan_check", "dgfs_strerror", "dgfs_eval_collision_noalloc",
           "dgfs_plan_set_sm_share", "dgfs_ssp_rk2_step", "dgfs_dg_create", "dgfs_dg_destroy",
           "dgfs_dg_nodes", "dgfs_dg_transport", "dgfs_dg_step", "dgfs_measure_fma_rate",
           "dgfs_dft3_bf16x3", "dgfs_check_bounded_wait")

_dptr = ctypes.POINTER(ctypes.c_double)


class dgfs_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("s", ctypes.c_int),
                ("mass", _dptr), ("omega", _dptr), ("alpha", _dptr), ("b_override", _dptr),
                ("M", ctypes.c_int), ("sigma", _dptr), ("w_sigma", _dptr),
                ("N_rho", ctypes.c_int), ("R", ctypes.c_double), ("precision", ctypes.c_int),
                ("flags", ctypes.c_uint), ("max_batch", ctypes.c_int), ("kappa", _dptr)]


class DgfsError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, dgfs_strerror(code), code))
        self.code = code


class dgfs_dg_desc(ctypes.Structure):
    _fields_ = [("Ne", ctypes.c_int), ("K", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("bc", ctypes.c_int), ("Tw", ctypes.c_double * 2),
                ("uw", ctypes.c_double * 6), ("acc", ctypes.c_double * 2),
                ("side", ctypes.c_int * 2), ("n_in", _dptr)]


_lib = None


def load():
    """Load libdgfs.so (built by ``paper_1903_03056_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdgfs.so has not been built (python -m paper_1903_03056_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cs = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.dgfs_create_plan.argtypes = [ctypes.POINTER(dgfs_plan_desc), ctypes.POINTER(vp)]
    lib.dgfs_destroy_plan.argtypes = [vp]
    lib.dgfs_eval_collision.argtypes = [vp, vp, vp, ci, vp]
    lib.dgfs_eval_collision_host.argtypes = [vp, vp, vp, ci, vp]
    lib.dgfs_plan_bytes.argtypes = [vp, ci, ctypes.POINTER(cs), ctypes.POINTER(cs)]
    lib.dgfs_plan_radius.argtypes = [vp, _dptr]
    lib.dgfs_plan_launches.argtypes = [vp, ctypes.POINTER(ci)]
    lib.dgfs_plan_check.argtypes = [vp, ctypes.POINTER(ci)]
    lib.dgfs_eval_collision_noalloc.argtypes = [ctypes.POINTER(dgfs_plan_desc), vp, vp, ci, vp]
    lib.dgfs_plan_set_sm_share.argtypes = [vp, ctypes.c_double]
    lib.dgfs_ssp_rk2_step.argtypes = [vp, vp, ctypes.c_double, ci, vp]
    lib.dgfs_dg_create.argtypes = [ctypes.POINTER(dgfs_dg_desc), vp, ctypes.POINTER(vp)]
    lib.dgfs_dg_destroy.argtypes = [vp]
    lib.dgfs_dg_nodes.argtypes = [vp, _dptr]
    lib.dgfs_dg_transport.argtypes = [vp, vp, vp, vp]
    lib.dgfs_dg_step.argtypes = [vp, vp, ctypes.c_double, vp]
    lib.dgfs_measure_fma_rate.argtypes = [ci, _dptr]
    lib.dgfs_dft3_bf16x3.argtypes = [ci, ci, vp, vp, ci, vp]
    lib.dgfs_check_bounded_wait.argtypes = [ctypes.c_double]
    lib.dgfs_strerror.argtypes = [ci]
    lib.dgfs_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "dgfs_strerror":
            getattr(lib, name).restype = ci
    _lib = lib
    return lib


def _check(code, where):
    if code != DGFS_OK:
        raise DgfsError(code, where)


# ---- one-to-one wrappers of the C ABI -------------------------------------------------------

def dgfs_create_plan(desc):
    h = ctypes.c_void_p()
    code = load().dgfs_create_plan(ctypes.byref(desc), ctypes.byref(h))
    return code, h.value


def dgfs_destroy_plan(plan):
    return load().dgfs_destroy_plan(plan)


def dgfs_eval_collision(plan, f_dev, Q_dev, batch, stream):
    return load().dgfs_eval_collision(plan, f_dev, Q_dev, batch, stream)


def dgfs_eval_collision_host(plan, f_host, Q_host, batch, stream):
    return load().dgfs_eval_collision_host(plan, f_host, Q_host, batch, stream)


def dgfs_plan_bytes(plan, batch):
    t, w = ctypes.c_size_t(), ctypes.c_size_t()
    code = load().dgfs_plan_bytes(plan, batch, ctypes.byref(t), ctypes.byref(w))
    return code, t.value, w.value


def dgfs_plan_radius(plan):
    r = ctypes.c_double()
    code = load().dgfs_plan_radius(plan, ctypes.byref(r))
    return code, r.value


def dgfs_plan_launches(plan):
    n = ctypes.c_int()
    code = load().dgfs_plan_launches(plan, ctypes.byref(n))
    return code, n.value


def dgfs_plan_check(plan):
    ok = ctypes.c_int()
    code = load().dgfs_plan_check(plan, ctypes.byref(ok))
    return code, bool(ok.value)


def dgfs_strerror(code):
    return load().dgfs_strerror(code).decode()


def dgfs_ssp_rk2_step(plan, f_dev, dt, batch, stream):
    return load().dgfs_ssp_rk2_step(plan, f_dev, dt, batch, stream)


def dgfs_plan_set_sm_share(plan, share):
    return load().dgfs_plan_set_sm_share(plan, share)


def dgfs_dg_create(desc, collision_plan):
    h = ctypes.c_void_p()
    code = load().dgfs_dg_create(ctypes.byref(desc), collision_plan, ctypes.byref(h))
    return code, h.value


def dgfs_dg_destroy(plan):
    return load().dgfs_dg_destroy(plan)


def dgfs_dg_nodes(plan, n):
    x = np.zeros(n)
    code = load().dgfs_dg_nodes(plan, x.ctypes.data_as(_dptr))
    return code, x


def dgfs_dg_transport(plan, f_dev, rhs_dev, stream):
    return load().dgfs_dg_transport(plan, f_dev, rhs_dev, stream)


def dgfs_dg_step(plan, f_dev, dt, stream):
    return load().dgfs_dg_step(plan, f_dev, dt, stream)


def dgfs_eval_collision_noalloc(desc, f_dev, Q_dev, batch, stream):
    return load().dgfs_eval_collision_noalloc(ctypes.byref(desc), f_dev, Q_dev, batch, stream)


# ---- convenience holder -----------------------------------------------------------------------

def _arr(x, n):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), (n,)).copy())
    return a, a.ctypes.data_as(_dptr)


def dgfs_measure_fma_rate(precision):
    """(code, flop/s) of the current device's FP32 or FP64 multiply-add pipe."""
    out = ctypes.c_double(0.0)
    code = load().dgfs_measure_fma_rate(DGFS_FP32 if precision in ("fp32", DGFS_FP32) else DGFS_FP64,
                                        ctypes.byref(out))
    return code, out.value


def precision_code(precision):
    """"fp64" / "fp32" / "bf16x3" (or the DGFS_* code itself) -> the DGFS_* code."""
    names = {"fp64": DGFS_FP64, "fp32": DGFS_FP32, "bf16x3": DGFS_BF16X3}
    if precision in names:
        return names[precision]
    if precision in (DGFS_FP64, DGFS_FP32, DGFS_BF16X3):
        return int(precision)
    raise ValueError("unknown precision %r" % (precision,))


def dgfs_check_bounded_wait(seconds):
    return load().dgfs_check_bounded_wait(float(seconds))


def dgfs_dft3_bf16x3(N, direction, x_dev, y_dev, count, stream):
    return load().dgfs_dft3_bf16x3(N, direction, x_dev, y_dev, count, _stream_handle(stream))


def make_desc(N, L, masses, omega, alpha=1.0, M=12, N_rho=None, R=0.0, precision="fp32",
              b_override=None, sigma=None, w_sigma=None, max_batch=0, flags=0, kappa=None):
    """Build a dgfs_plan_desc; returns (desc, keepalive) -- keep the second alive until the
    plan is created."""
    s = len(masses)
    keep = []
    mass, pm = _arr(masses, s)
    om, po = _arr(np.asarray(omega, dtype=np.float64).reshape(-1) if np.ndim(omega) else omega, s * s)
    al, pa = _arr(np.asarray(alpha, dtype=np.float64).reshape(-1) if np.ndim(alpha) else alpha, s * s)
    keep += [mass, om, al]
    d = dgfs_plan_desc()
    d.N, d.L, d.s = int(N), float(L), s
    d.mass, d.omega, d.alpha = pm, po, pa
    if b_override is not None:
        bo, pb = _arr(np.asarray(b_override, dtype=np.float64).reshape(-1), s * s)
        keep.append(bo)
        d.b_override = pb
    if sigma is not None:
        sg = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        keep.append(sg)
        d.sigma = sg.ctypes.data_as(_dptr)
        M = sg.size // 3
        if w_sigma is not None:
            ws, pw = _arr(w_sigma, M)
            keep.append(ws)
            d.w_sigma = pw
    d.M = int(M)
    d.N_rho = int(N if N_rho is None else N_rho)
    d.R = float(R)
    d.precision = precision_code(precision)
    d.flags = int(flags)
    d.max_batch = int(max_batch)
    if kappa is not None:
        ka, pk = _arr(np.asarray(kappa, dtype=np.float64).reshape(-1), s * s)
        keep.append(ka)
        d.kappa = pk
    return d, keep


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Plan:
    """Owns one dgfs plan.  ``precision`` is "fp32", "fp64" or "bf16x3"."""

    def __init__(self, N, L, masses, omega, **kw):
        desc, keep = make_desc(N, L, masses, omega, **kw)
        code, h = dgfs_create_plan(desc)
        del keep
        _check(code, "dgfs_create_plan")
        self.handle = h
        self.N, self.L, self.s = int(N), float(L), len(masses)
        self.precision = kw.get("precision", "fp32")
        self.max_batch = int(kw.get("max_batch", 0))
        self.flags = int(kw.get("flags", 0))

    @property
    def dtype_name(self):
        return "float64" if precision_code(self.precision) == DGFS_FP64 else "float32"

    def radius(self):
        code, r = dgfs_plan_radius(self.handle)
        _check(code, "dgfs_plan_radius")
        return r

    def launches(self):
        code, n = dgfs_plan_launches(self.handle)
        _check(code, "dgfs_plan_launches")
        return n

    def ssp_rk2_step(self, f, dt, stream=None):
        """One SSP-RK2 step of d_t f_i = sum_j kappa_ij Q_ij, in place on the CUDA tensor f."""
        _check(dgfs_ssp_rk2_step(self.handle, f.data_ptr(), float(dt), int(f.shape[0]),
                                 _stream_handle(stream)), "dgfs_ssp_rk2_step")

    def check(self):
        """True when the guard blocks around the plan's workspace are intact after its most
        recent evaluation (no kernel wrote outside the workspace)."""
        code, ok = dgfs_plan_check(self.handle)
        _check(code, "dgfs_plan_check")
        return ok

    def set_sm_share(self, share):
        _check(dgfs_plan_set_sm_share(self.handle, float(share)), "dgfs_plan_set_sm_share")

    def bytes(self, batch=0):
        code, t, w = dgfs_plan_bytes(self.handle, batch)
        _check(code, "dgfs_plan_bytes")
        return t, w

    def eval_ptr(self, f_dev, Q_dev, batch, stream=None):
        _check(dgfs_eval_collision(self.handle, f_dev, Q_dev, int(batch), _stream_handle(stream)),
               "dgfs_eval_collision")

    def eval(self, f, Q=None, stream=None):
        """f: CUDA tensor [B, s, N, N, N] of the plan's dtype; returns Q [B, s, s, N, N, N]."""
        import torch
        assert f.is_cuda and f.is_contiguous() and str(f.dtype).endswith(self.dtype_name)
        B = f.shape[0]
        if Q is None:
            pairs = (self.s,) if self.flags & DGFS_SUM_SPECIES else (self.s, self.s)
            Q = torch.empty((B,) + pairs + tuple(f.shape[2:]), dtype=f.dtype, device=f.device)
        self.eval_ptr(f.data_ptr(), Q.data_ptr(), B, stream)
        return Q

    def capture(self, f, Q, stream=None):
        """Capture one evaluation of device tensors f -> Q into a CUDA graph (torch.cuda.CUDAGraph)
        that replays the same launches; f and Q must stay allocated while the graph is used."""
        import torch
        st = stream if stream is not None else torch.cuda.Stream()
        B = f.shape[0]
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):  # warm the launch path outside the capture
            self.eval_ptr(f.data_ptr(), Q.data_ptr(), B, st)
        torch.cuda.current_stream().wait_stream(st)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            self.eval_ptr(f.data_ptr(), Q.data_ptr(), B, torch.cuda.current_stream())
        return g

    def eval_host(self, f_host, Q_host, stream=None):
        """Host arrays or tensors (contiguous, plan dtype); copies in, evaluates, copies out."""
        fp = f_host.data_ptr() if hasattr(f_host, "data_ptr") else f_host.ctypes.data
        qp = Q_host.data_ptr() if hasattr(Q_host, "data_ptr") else Q_host.ctypes.data
        _check(dgfs_eval_collision_host(self.handle, fp, qp, int(f_host.shape[0]),
                                        _stream_handle(stream)), "dgfs_eval_collision_host")
        return Q_host

    def close(self):
        if getattr(self, "handle", None):
            dgfs_destroy_plan(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DGPlan:
    """Owns one 1D DG plan built on a collision ``Plan`` (which must outlive it)."""

    def __init__(self, collision, Ne, K, x0=0.0, x1=1.0, bc="periodic", Tw=(1.0, 1.0),
                 uw=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)), acc=(1.0, 1.0), side_kind=("wall", "wall"),
                 n_in=None):
        d = dgfs_dg_desc()
        for k, kind in enumerate(side_kind):
            d.side[k] = DGFS_SIDE_INFLOW if kind == "inflow" else DGFS_SIDE_WALL
        keep = None
        if n_in is not None:
            keep = np.ascontiguousarray(np.asarray(n_in, dtype=np.float64).reshape(-1))
            d.n_in = keep.ctypes.data_as(_dptr)
        d.Ne, d.K, d.x0, d.x1 = int(Ne), int(K), float(x0), float(x1)
        d.bc = DGFS_BC_WALLS if bc == "walls" else DGFS_BC_PERIODIC
        d.Tw[0], d.Tw[1] = float(Tw[0]), float(Tw[1])
        for k, u in enumerate(np.asarray(uw, dtype=np.float64).reshape(-1)):
            d.uw[k] = float(u)
        d.acc[0], d.acc[1] = float(acc[0]), float(acc[1])
        code, h = dgfs_dg_create(d, collision.handle)
        del keep
        _check(code, "dgfs_dg_create")
        self.handle, self.collision = h, collision
        self.Ne, self.K = int(Ne), int(K)

    def nodes(self):
        code, x = dgfs_dg_nodes(self.handle, self.Ne * self.K)
        _check(code, "dgfs_dg_nodes")
        return x.reshape(self.Ne, self.K)

    def transport(self, f, rhs=None, stream=None):
        """f: CUDA tensor [Ne*K, s, N, N, N]; returns the transport part of d_t f."""
        import torch
        if rhs is None:
            rhs = torch.empty_like(f)
        _check(dgfs_dg_transport(self.handle, f.data_ptr(), rhs.data_ptr(), _stream_handle(stream)),
               "dgfs_dg_transport")
        return rhs

    def step(self, f, dt, stream=None):
        """One SSP-RK2 step of the full equation, in place on f."""
        _check(dgfs_dg_step(self.handle, f.data_ptr(), float(dt), _stream_handle(stream)),
               "dgfs_dg_step")

    def close(self):
        if getattr(self, "handle", None):
            dgfs_dg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
