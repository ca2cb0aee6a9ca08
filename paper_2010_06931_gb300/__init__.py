"""GB300-native orthogonal-raster OCT/OCTA motion correction (Ploner et al.,
arXiv 2010.06931): the joint registration objective, its per-A-scan
displacement gradient and the multi-resolution L-BFGS solve.

Thin Python binding of the C ABI in ``include/octmc.h``: every method below
marshals arguments and calls the function of the same name (``octmc_`` +
name); all arithmetic runs in the CUDA kernels of ``liboctmc.so``.  PyTorch
provides device memory and the stream only.  There is no CPU fallback: the
calls raise if the library is not built or no sm_103a GPU is present.

Layouts (see the header): volumes float32 ``[h][w][d]``, en-face images
``[h][w]``, validity ``vx[h]``, ``vy[w]``, time maps float64 ``[h][w]``,
displacements and gradients float64 ``[2][3][h][w]`` on the GPU.
"""
import ctypes as C

import numpy as np
import torch

from . import _native as N
from ._native import BF16, F16, F32, LOSS_PSEUDO_HUBER, LOSS_SSD, OctmcError  # noqa: F401

__all__ = ["Problem", "Lbfgs", "Server", "create_problem", "estimate_bytes", "OctmcError", "F32", "BF16",
           "F16", "LOSS_PSEUDO_HUBER", "LOSS_SSD", "library_path"]


def library_path():
    return N.LIB_PATH


def _stream_ptr():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _as_tensor(a, dtype, device):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    return a.to(device=device, dtype=dtype).contiguous()


def _check_disp(t, shape):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("displacement buffers must be contiguous float64 CUDA tensors")
    if tuple(t.shape) != shape and t.numel() < int(np.prod(shape)):
        raise ValueError("displacement buffer of shape %s, need %s" % (tuple(t.shape), shape))


class Problem:
    """One orthogonal scan pair on the GPU (``octmc_problem``).

    Inputs may be numpy arrays or torch tensors (host or CUDA); if all the
    given inputs are CUDA tensors they are read on the device, otherwise from
    host memory.  Keyword arguments are the fields of ``octmc_desc``.
    """

    def __init__(self, sx, sy, tx, ty, ax=None, ay=None, vx=None, vy=None, *, storage=F32,
                 alpha=0.1, delta0=0.5, eps_h=1e-3, eps_r=1e-2, mu=0.0, loss=LOSS_PSEUDO_HUBER,
                 levels=1, lbfgs_m=8, max_iter=5000, max_ls=20, gtol=1e-6, ftol=1e-7,
                 persistent_ascans=0):
        L = N.lib()
        arrays = [sx, sy, tx, ty, ax, ay, vx, vy]
        on_dev = all(isinstance(a, torch.Tensor) and a.is_cuda for a in arrays if a is not None)
        dev = torch.device("cuda") if on_dev else torch.device("cpu")
        f32 = lambda a: _as_tensor(a, torch.float32, dev)
        f64 = lambda a: _as_tensor(a, torch.float64, dev)
        self._keep = dict(sx=f32(sx), sy=f32(sy), tx=f64(tx), ty=f64(ty), ax=f32(ax), ay=f32(ay),
                          vx=f32(vx), vy=f32(vy))
        k = self._keep
        h, w, d = k["sx"].shape
        desc = N.Desc()
        L.octmc_desc_defaults(C.byref(desc))
        desc.w, desc.h, desc.d, desc.storage = w, h, d, storage
        for name in ("sx", "sy", "ax", "ay", "vx", "vy", "tx", "ty"):
            setattr(desc, name, None if k[name] is None else k[name].data_ptr())
        desc.inputs_on_device = 1 if on_dev else 0
        desc.alpha, desc.delta0, desc.eps_h, desc.eps_r, desc.mu = alpha, delta0, eps_h, eps_r, mu
        desc.loss, desc.levels, desc.lbfgs_m = loss, levels, lbfgs_m
        desc.max_iter, desc.max_ls, desc.gtol, desc.ftol = max_iter, max_ls, gtol, ftol
        desc.persistent_ascans = persistent_ascans
        desc.stream = _stream_ptr().value
        self.levels = levels
        self._h = C.c_void_p()
        N.check(L.octmc_create_problem(C.byref(desc), C.byref(self._h)), "octmc_create_problem")
        self._keep = None  # the library copied the inputs

    # -- lifetime
    def destroy_problem(self):
        if self._h:
            N.lib().octmc_destroy_problem(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy_problem()
        except Exception:
            pass

    # -- queries
    def level_shape(self, level=0):
        w, h, d = C.c_int(), C.c_int(), C.c_int()
        N.check(N.lib().octmc_level_shape(self._h, level, C.byref(w), C.byref(h), C.byref(d)),
                "octmc_level_shape")
        return w.value, h.value, d.value

    def disp_shape(self, level=0):
        w, h, _ = self.level_shape(level)
        return (2, 3, h, w)

    def zeros(self, level=0):
        return torch.zeros(self.disp_shape(level), dtype=torch.float64, device="cuda")

    # -- eta (Eq. 9-10)
    def set_eta(self, level, eta):
        N.check(N.lib().octmc_set_eta(self._h, level, float(eta)), "octmc_set_eta")

    def compute_eta(self, level, disp0):
        _check_disp(disp0, self.disp_shape(level))
        e = C.c_double()
        N.check(N.lib().octmc_compute_eta(self._h, level, _ptr(disp0), C.byref(e)), "octmc_compute_eta")
        return e.value

    # -- objective (Eq. 1-10)
    def eval_objective_grad(self, level, disp, grad=None):
        """f (float) and, if ``grad`` is a tensor, the gradient written into it."""
        _check_disp(disp, self.disp_shape(level))
        if grad is not None:
            _check_disp(grad, self.disp_shape(level))
        f = C.c_double()
        N.check(N.lib().octmc_eval_objective_grad(self._h, level, _ptr(disp), C.byref(f), _ptr(grad)),
                "octmc_eval_objective_grad")
        return f.value

    def eval_objective_grad_async(self, level, disp, grad=None, terms=None, stream=None):
        """Enqueues the evaluation on ``stream`` (a torch.cuda.Stream; default:
        the current stream) and returns at once.  ``terms`` (float64 CUDA
        tensor of 6, optional) receives [S^str, S^ang, R, M, f, eta] in stream
        order; ``grad`` as for eval_objective_grad."""
        _check_disp(disp, self.disp_shape(level))
        if grad is not None:
            _check_disp(grad, self.disp_shape(level))
        if terms is not None and (terms.dtype != torch.float64 or not terms.is_cuda or terms.numel() < 6
                                  or not terms.is_contiguous()):
            raise ValueError("terms must be a contiguous float64 CUDA tensor of at least 6 values")
        st = stream if stream is not None else torch.cuda.current_stream()
        N.check(N.lib().octmc_eval_objective_grad_async(self._h, level, _ptr(disp), _ptr(grad), _ptr(terms),
                                                        C.c_void_p(st.cuda_stream)),
                "octmc_eval_objective_grad_async")

    def eval_terms(self, level, disp, grad=None):
        """[S^str, S^ang, R, M, f, eta] as a numpy array; optional gradient as above."""
        _check_disp(disp, self.disp_shape(level))
        if grad is not None:
            _check_disp(grad, self.disp_shape(level))
        t = (C.c_double * 6)()
        N.check(N.lib().octmc_eval_terms(self._h, level, _ptr(disp), t, _ptr(grad)), "octmc_eval_terms")
        return np.array(t[:])

    # -- solves (Sec. 2.1)
    def solve_level(self, level, disp):
        """In-place L-BFGS solve of ``disp``; returns the statistics dict."""
        _check_disp(disp, self.disp_shape(level))
        st = N.Stats()
        rc = N.check(N.lib().octmc_solve_level(self._h, level, _ptr(disp), C.byref(st)), "octmc_solve_level")
        out = st.as_dict()
        out["rc"] = rc
        return out

    def solve_full(self, out=None):
        """Coarse-to-fine solve from zero; returns (level-0 field, per-level stats)."""
        if out is None:
            out = self.zeros(0)
        _check_disp(out, self.disp_shape(0))
        st = (N.Stats * self.levels)()
        rc = N.check(N.lib().octmc_solve_full(self._h, _ptr(out), st), "octmc_solve_full")
        stats = [s.as_dict() for s in st]
        for s in stats:
            s["rc"] = rc
        return out, stats

    def prolong(self, level, coarse):
        _check_disp(coarse, self.disp_shape(level))
        fine = self.zeros(level - 1)
        N.check(N.lib().octmc_prolong(self._h, level, _ptr(coarse), _ptr(fine)), "octmc_prolong")
        return fine

    def level_data(self, level=0):
        w, h, d = self.level_shape(level)
        out = {k: torch.empty(s, dtype=torch.float32, device="cuda") for k, s in
               (("sx", (h, w, d)), ("sy", (h, w, d)), ("ax", (h, w)), ("ay", (h, w)), ("vx", (h,)), ("vy", (w,)))}
        N.check(N.lib().octmc_level_data(self._h, level, *[_ptr(out[k]) for k in ("sx", "sy", "ax", "ay", "vx", "vy")]),
                "octmc_level_data")
        return out

    # -- rough axial prealignment (stage 1): parameters [aX(h), tX(h), aY(w), tY(w)] float64
    def prealign_size(self, level=0):
        w, h, _ = self.level_shape(level)
        return 2 * (w + h)

    def _check_prm(self, t, level):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() >= self.prealign_size(level)):
            raise ValueError("prealignment parameters must be a contiguous float64 CUDA tensor of %d values"
                             % self.prealign_size(level))

    def prealign_disp(self, level, prm):
        """``octmc_prealign_disp``: the induced field [2][3][h][w]."""
        self._check_prm(prm, level)
        out = self.zeros(level)
        N.check(N.lib().octmc_prealign_disp(self._h, level, _ptr(prm), _ptr(out)), "octmc_prealign_disp")
        return out

    def prealign_eval(self, level, prm, grad=None):
        """``octmc_prealign_eval``: f of the stage-1 objective (gradient into ``grad``)."""
        self._check_prm(prm, level)
        if grad is not None:
            self._check_prm(grad, level)
        f = C.c_double()
        N.check(N.lib().octmc_prealign_eval(self._h, level, _ptr(prm), C.byref(f), _ptr(grad)),
                "octmc_prealign_eval")
        return f.value

    def prealign_level(self, level, prm):
        """``octmc_prealign_level``: solve one level in place; returns the stats dict."""
        self._check_prm(prm, level)
        st = N.Stats()
        rc = N.check(N.lib().octmc_prealign_level(self._h, level, _ptr(prm), C.byref(st)), "octmc_prealign_level")
        out = st.as_dict()
        out["rc"] = rc
        return out

    def prealign_full(self, want_disp=True):
        """``octmc_prealign_full``: (level-0 parameters, induced level-0 field or None, per-level stats)."""
        prm = torch.zeros(self.prealign_size(0), dtype=torch.float64, device="cuda")
        disp = self.zeros(0) if want_disp else None
        st = (N.Stats * self.levels)()
        rc = N.check(N.lib().octmc_prealign_full(self._h, _ptr(prm), _ptr(disp), st), "octmc_prealign_full")
        stats = [s.as_dict() for s in st]
        for s in stats:
            s["rc"] = rc
        return prm, disp, stats

    def merge(self, disp0, beta=2.0, tau=0.05, outputs=("merged", "weights", "angio"), out=None):
        """``octmc_merge``: final resampling and merging at level 0 (Sec. 2.1, 2.5).

        ``outputs`` picks any of "merged", "corrected_x", "corrected_y",
        "weights", "angio"; returns a dict of float32 device tensors (those of
        ``out`` when given, a dict returned by an earlier call)."""
        _check_disp(disp0, self.disp_shape(0))
        w, h, d = self.level_shape(0)
        shapes = {"merged": (h, w, d), "corrected_x": (h, w, d), "corrected_y": (h, w, d), "weights": (2, h, w),
                  "angio": (h, w)}
        unknown = set(outputs) - set(shapes)
        if unknown:
            raise ValueError("unknown merge outputs %s" % sorted(unknown))
        if out is None:
            out = {k: torch.empty(shapes[k], dtype=torch.float32, device="cuda") for k in outputs}
        else:
            out = {k: out[k] for k in outputs}
            for k, t in out.items():
                if tuple(t.shape) != shapes[k] or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                    raise ValueError("merge output %s must be a contiguous float32 CUDA tensor of shape %s"
                                     % (k, shapes[k]))
        N.check(N.lib().octmc_merge(self._h, _ptr(disp0), float(beta), float(tau),
                                    *[_ptr(out.get(k)) for k in ("merged", "corrected_x", "corrected_y", "weights",
                                                                 "angio")]), "octmc_merge")
        return out

    # -- kernel timing
    def profile_enable(self, enable=True):
        N.check(N.lib().octmc_profile_enable(self._h, 1 if enable else 0), "octmc_profile_enable")

    def profile_read(self):
        """(total ms, launches) of the data-term kernel since profiling was enabled."""
        ms, n = C.c_double(), C.c_longlong()
        N.check(N.lib().octmc_profile_read(self._h, C.byref(ms), C.byref(n)), "octmc_profile_read")
        return ms.value, n.value


def _fvol(a, ndim):
    t = _as_tensor(a, torch.float32, "cuda")
    if t.dim() != ndim or not t.is_contiguous():
        raise ValueError("expected a contiguous %d-d float32 array" % ndim)
    return t


def saccade_validity(octa, fast_axis):
    """``octmc_saccade_validity`` (Sec. 2.2): (validity per B-scan float32,
    mean decorrelation per B-scan float64) of an OCTA volume [h][w][d];
    fast_axis 0 for an X-fast scan (B-scans are rows), 1 for Y-fast."""
    A = _fvol(octa, 3)
    h, w, d = A.shape
    nb = h if fast_axis == 0 else w
    v = torch.empty(nb, dtype=torch.float32, device="cuda")
    m = torch.empty(nb, dtype=torch.float64, device="cuda")
    N.check(N.lib().octmc_saccade_validity(_ptr(A), w, h, d, int(fast_axis), _ptr(v), _ptr(m), _stream_ptr()),
            "octmc_saccade_validity")
    return v, m


def enface(octa, oct, fast_axis, v, q_lo=0.05, q_hi=0.95, thresh=0.1, t_oct=None, out=None, filtered=None):
    """``octmc_enface`` (Sec. 2.3): the en-face OCTA image [h][w] of one scan.
    Returns (image, info dict with the two quantiles, the OCT threshold and
    the voxels kept).  ``filtered`` (optional [h][w][d] float32 CUDA tensor)
    receives the rank-filtered volume."""
    A, S = _fvol(octa, 3), _fvol(oct, 3)
    if A.shape != S.shape:
        raise ValueError("OCTA and OCT volumes differ in shape")
    h, w, d = A.shape
    vv = _fvol(v, 1)
    if vv.numel() != (h if fast_axis == 0 else w):
        raise ValueError("validity needs one value per B-scan")
    E = out if out is not None else torch.empty((h, w), dtype=torch.float32, device="cuda")
    if filtered is not None and (tuple(filtered.shape) != (h, w, d) or filtered.dtype != torch.float32
                                 or not filtered.is_cuda or not filtered.is_contiguous()):
        raise ValueError("filtered must be a contiguous float32 CUDA tensor of the volume's shape")
    info = (C.c_double * 4)()
    N.check(N.lib().octmc_enface(_ptr(A), _ptr(S), w, h, d, int(fast_axis), _ptr(vv), float(q_lo), float(q_hi),
                                 float(thresh), float("nan") if t_oct is None else float(t_oct), _ptr(E),
                                 _ptr(filtered), info, _stream_ptr()), "octmc_enface")
    return E, dict(p_lo=info[0], p_hi=info[1], t_oct=info[2], kept=int(info[3]))


def eval_batch(problems, levels, disps, grads=None):
    """Objectives of several problems in one batched evaluation
    (``octmc_eval_batch``): ``problems``, ``levels``, ``disps`` (and
    optionally ``grads``, tensors receiving the gradients, or None entries)
    are sequences of equal length; returns the list of f values."""
    k = len(problems)
    if not (len(levels) == len(disps) == k) or (grads is not None and len(grads) != k):
        raise ValueError("problems, levels, disps and grads must have the same length")
    for P, l, D in zip(problems, levels, disps):
        _check_disp(D, P.disp_shape(l))
    if grads is not None:
        for P, l, g in zip(problems, levels, grads):
            if g is not None:
                _check_disp(g, P.disp_shape(l))
    hs = (C.c_void_p * k)(*[P._h.value for P in problems])
    lv = (C.c_int * k)(*[int(l) for l in levels])
    dp = (C.c_void_p * k)(*[D.data_ptr() for D in disps])
    gp = None if grads is None else (C.c_void_p * k)(*[None if g is None else g.data_ptr() for g in grads])
    f = (C.c_double * k)()
    N.check(N.lib().octmc_eval_batch(hs, k, lv, dp, gp, f), "octmc_eval_batch")
    return list(f)


def create_problem(*args, **kw):
    """``octmc_create_problem``: see :class:`Problem`."""
    return Problem(*args, **kw)


class Lbfgs:
    """Stand-alone on-device L-BFGS direction (``octmc_lbfgs_*``) over n float64 values."""

    def __init__(self, n, m=8):
        self.n = int(n)
        self._h = C.c_void_p()
        N.check(N.lib().octmc_lbfgs_create(self.n, int(m), _stream_ptr(), C.byref(self._h)), "octmc_lbfgs_create")

    def push(self, s, y):
        return N.check(N.lib().octmc_lbfgs_push(self._h, _ptr(s), _ptr(y)), "octmc_lbfgs_push")

    def direction(self, g):
        out = torch.empty_like(g)
        gtd = C.c_double()
        N.check(N.lib().octmc_lbfgs_direction(self._h, _ptr(g), _ptr(out), C.byref(gtd)), "octmc_lbfgs_direction")
        return out, gtd.value

    def reset(self):
        N.check(N.lib().octmc_lbfgs_reset(self._h), "octmc_lbfgs_reset")

    def destroy(self):
        if self._h:
            N.lib().octmc_lbfgs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Server:
    """Continuous-batching solver (``octmc_server_*``).

    ``submit`` queues a full coarse-to-fine solve of one scan pair and returns
    a ticket; ``step`` retires finished requests and admits what fits the
    device-memory budget (each admitted request's whole solve runs on the
    device, concurrently with the others; the call does not wait for it);
    ``poll`` returns the result of a finished request (and releases it).
    """

    QUEUED, RUNNING, DONE, UNKNOWN = 0, 1, 2, -1

    def __init__(self, budget_bytes, max_slots=32):
        self._h = C.c_void_p()
        N.check(N.lib().octmc_server_create(int(budget_bytes), int(max_slots), _stream_ptr(), C.byref(self._h)),
                "octmc_server_create")
        self._inputs = {}  # ticket -> (tensors kept alive until admission, levels, shape)

    def submit(self, sx, sy, tx, ty, ax=None, ay=None, vx=None, vy=None, *, storage=F32, alpha=0.1,
               delta0=0.5, eps_h=1e-3, eps_r=1e-2, mu=0.0, loss=LOSS_PSEUDO_HUBER, levels=1, lbfgs_m=8,
               max_iter=5000, max_ls=20, gtol=1e-6, ftol=1e-7):
        arrays = [sx, sy, tx, ty, ax, ay, vx, vy]
        on_dev = all(isinstance(a, torch.Tensor) and a.is_cuda for a in arrays if a is not None)
        dev = torch.device("cuda") if on_dev else torch.device("cpu")
        f32 = lambda a: _as_tensor(a, torch.float32, dev)
        f64 = lambda a: _as_tensor(a, torch.float64, dev)
        keep = dict(sx=f32(sx), sy=f32(sy), tx=f64(tx), ty=f64(ty), ax=f32(ax), ay=f32(ay), vx=f32(vx), vy=f32(vy))
        h, w, d = keep["sx"].shape
        desc = N.Desc()
        N.lib().octmc_desc_defaults(C.byref(desc))
        desc.w, desc.h, desc.d, desc.storage = w, h, d, storage
        for name in ("sx", "sy", "ax", "ay", "vx", "vy", "tx", "ty"):
            setattr(desc, name, None if keep[name] is None else keep[name].data_ptr())
        desc.inputs_on_device = 1 if on_dev else 0
        desc.alpha, desc.delta0, desc.eps_h, desc.eps_r, desc.mu = alpha, delta0, eps_h, eps_r, mu
        desc.loss, desc.levels, desc.lbfgs_m = loss, levels, lbfgs_m
        desc.max_iter, desc.max_ls, desc.gtol, desc.ftol = max_iter, max_ls, gtol, ftol
        t = C.c_int64()
        N.check(N.lib().octmc_server_submit(self._h, C.byref(desc), C.byref(t)), "octmc_server_submit")
        self._inputs[t.value] = (keep, levels, (h, w))
        return t.value

    def step(self):
        a, q = C.c_int(), C.c_int()
        N.check(N.lib().octmc_server_step(self._h, C.byref(a), C.byref(q)), "octmc_server_step")
        # inputs of admitted requests are no longer needed
        return a.value, q.value

    def state(self, ticket):
        st = C.c_int()
        N.check(N.lib().octmc_server_state(self._h, int(ticket), C.byref(st)), "octmc_server_state")
        return st.value

    def poll(self, ticket):
        """(state, field or None, stats or None, return code or None).  A finished
        request is released by this call."""
        if self.state(ticket) != self.DONE:
            return self.state(ticket), None, None, None
        keep, levels, (h, w) = self._inputs.get(ticket, (None, 1, (0, 0)))
        state = C.c_int()
        if keep is None:
            N.check(N.lib().octmc_server_poll(self._h, int(ticket), C.byref(state), None, None, 0, None),
                    "octmc_server_poll")
            return state.value, None, None, None
        # poll releases a finished request, so the result buffer goes with it
        out = torch.empty((2, 3, h, w), dtype=torch.float64, device="cuda")
        st = (N.Stats * levels)()
        rc = C.c_int()
        N.check(N.lib().octmc_server_poll(self._h, int(ticket), C.byref(state), _ptr(out), st, levels, C.byref(rc)),
                "octmc_server_poll")
        if state.value != self.DONE:
            return state.value, None, None, None
        del self._inputs[ticket]
        return state.value, out, [s.as_dict() for s in st], rc.value

    def destroy(self):
        if self._h:
            N.lib().octmc_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def estimate_bytes(w, h, d, levels=1, storage=F32, lbfgs_m=8):
    """``octmc_estimate_bytes`` for a problem of this size."""
    desc = N.Desc()
    N.lib().octmc_desc_defaults(C.byref(desc))
    desc.w, desc.h, desc.d, desc.levels, desc.storage, desc.lbfgs_m = w, h, d, levels, storage, lbfgs_m
    return int(N.lib().octmc_estimate_bytes(C.byref(desc)))
