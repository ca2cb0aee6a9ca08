"""ctypes wrapper and multi-resolution driver for the C oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy;
volumes are float32 ``[h][w][d]``, en-face images float32 ``[h][w]``,
validity float32 ``vx[h]``, ``vy[w]``, time maps float64 ``[h][w]``,
displacements float64 ``[2][3][h][w]`` (volume X/Y, component x/y/z).
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "octmc_oracle.c"), os.path.join(_HERE, "octa_oracle.c")]
_LIB = os.path.join(_HERE, "liboctmc_oracle.so")
_lock = threading.Lock()
_lib = None

LOSS_PSEUDO_HUBER = 0
LOSS_SSD = 1

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


class _Level(C.Structure):
    _fields_ = [
        ("w", C.c_int), ("h", C.c_int), ("d", C.c_int),
        ("sx", C.c_void_p), ("sy", C.c_void_p),
        ("ax", C.c_void_p), ("ay", C.c_void_p),
        ("vx", C.c_void_p), ("vy", C.c_void_p),
        ("tx", C.c_void_p), ("ty", C.c_void_p),
        ("alpha", C.c_double), ("delta0", C.c_double), ("eps_h", C.c_double),
        ("eps_r", C.c_double), ("mu", C.c_double), ("eta", C.c_double),
        ("loss", C.c_int),
    ]


class _Solver(C.Structure):
    _fields_ = [("m", C.c_int), ("max_iter", C.c_int), ("max_ls", C.c_int),
                ("gtol", C.c_double), ("ftol", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("evals", C.c_int), ("status", C.c_int), ("f", C.c_double)]


# objective callback of the stand-alone minimiser: fn(n, x, f, g)
_FG = C.CFUNCTYPE(None, C.c_long, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double))


def build(force=False):
    """Compile the oracle shared library (gcc, OpenMP) if it is missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS)
        if force or stale:
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                                   "-o", tmp] + _SRCS + ["-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.oracle_cr_weights.argtypes = [C.c_double, _dp, _dp]
        lib.oracle_interp1.argtypes = [_fp, C.c_int, C.c_double, C.POINTER(C.c_double)]
        lib.oracle_interp1.restype = C.c_double
        lib.oracle_validity_interp.argtypes = [_fp, C.c_int, C.c_double, C.POINTER(C.c_double)]
        lib.oracle_validity_interp.restype = C.c_double
        lib.oracle_interp2.argtypes = [_fp, C.c_int, C.c_int, C.c_double, C.c_double, _dp]
        lib.oracle_interp2.restype = C.c_double
        lib.oracle_interp3.argtypes = [_fp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                       C.c_double, _dp]
        lib.oracle_interp3.restype = C.c_double
        lib.oracle_loss.argtypes = [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double)]
        lib.oracle_loss.restype = C.c_double
        lib.oracle_chain.argtypes = [_dp, C.c_long, np.ctypeslib.ndpointer(dtype=np.int64), _dp]
        lib.oracle_eval.argtypes = [C.POINTER(_Level), _dp, C.POINTER(C.c_double), C.c_void_p,
                                    C.c_void_p]
        lib.oracle_eval.restype = C.c_int
        lib.oracle_data_rows.argtypes = [C.POINTER(_Level), _dp, C.c_int, C.c_int, _dp]
        lib.oracle_eta.argtypes = [C.POINTER(_Level), _dp]
        lib.oracle_eta.restype = C.c_double
        lib.oracle_pyramid_volume.argtypes = [_fp, C.c_int, C.c_int, C.c_int, _fp]
        lib.oracle_pyramid_image.argtypes = [_fp, C.c_int, C.c_int, _fp]
        lib.oracle_pyramid_line.argtypes = [_fp, C.c_int, _fp]
        lib.oracle_pyramid_time.argtypes = [_dp, C.c_int, C.c_int, _dp]
        lib.oracle_prolong.argtypes = [_dp, C.c_int, C.c_int, _dp, C.c_int, C.c_int]
        lib.oracle_lbfgs_direction.argtypes = [C.c_long, C.c_int, C.POINTER(C.c_void_p),
                                               C.POINTER(C.c_void_p), _dp, _dp]
        lib.oracle_solve_level.argtypes = [C.POINTER(_Level), _dp, C.POINTER(_Solver),
                                           C.POINTER(_Stats)]
        lib.oracle_solve_level.restype = C.c_int
        lib.oracle_num_threads.restype = C.c_int
        lib.oracle_lbfgs_minimize_fn.argtypes = [C.c_long, _dp, _FG, C.POINTER(_Solver), C.POINTER(_Stats)]
        lib.oracle_lbfgs_minimize_fn.restype = C.c_int
        lib.oracle_merge.argtypes = [C.POINTER(_Level), _dp, C.c_double, C.c_double] + [C.c_void_p] * 5 + [C.c_void_p]
        lib.oracle_prealign_disp.argtypes = [C.POINTER(_Level), _dp, _dp]
        lib.oracle_prealign_eval.argtypes = [C.POINTER(_Level), _dp, C.POINTER(C.c_double), C.c_void_p, C.c_void_p]
        lib.oracle_prealign_level.argtypes = [C.POINTER(_Level), _dp, C.POINTER(_Solver), C.POINTER(_Stats)]
        lib.oracle_prealign_level.restype = C.c_int
        lib.oracle_prealign_prolong.argtypes = [_dp, C.c_int, C.c_int, _dp, C.c_int, C.c_int]
        lib.oracle_saccade_validity.argtypes = [_fp, C.c_int, C.c_int, C.c_int, C.c_int, _fp, _dp]
        lib.oracle_median3.argtypes = [_fp, C.c_int, C.c_int, C.c_int, _fp]
        lib.oracle_rank_filter.argtypes = [_fp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _fp]
        lib.oracle_percentile.argtypes = [_fp, C.c_long, C.c_double]
        lib.oracle_percentile.restype = C.c_double
        lib.oracle_bscan_median_subtract.argtypes = [_fp, C.c_int, C.c_int, C.c_int]
        lib.oracle_replace_invalid.argtypes = [_fp, C.c_int, C.c_int, C.c_int, _fp]
        lib.oracle_enface.argtypes = [_fp, _fp, C.c_int, C.c_int, C.c_int, C.c_int, _fp, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_void_p, _fp, _dp]
        _lib = lib
    return _lib


def num_threads():
    return _load().oracle_num_threads()


# ---------------------------------------------------------------- primitives
def cr_weights(t):
    w = np.zeros(4)
    dw = np.zeros(4)
    _load().oracle_cr_weights(float(t), w, dw)
    return w, dw


def interp1(v, u):
    v = np.ascontiguousarray(v, dtype=np.float32)
    du = C.c_double()
    val = _load().oracle_interp1(v, v.shape[0], float(u), C.byref(du))
    return val, du.value


def validity_interp(v, u):
    """Validity line resampled at u (Eq. 7): (value, d value / du)."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    du = C.c_double()
    val = _load().oracle_validity_interp(v, v.shape[0], float(u), C.byref(du))
    return val, du.value


def interp2(img, x, y):
    img = np.ascontiguousarray(img, dtype=np.float32)
    g = np.zeros(2)
    val = _load().oracle_interp2(img, img.shape[1], img.shape[0], float(x), float(y), g)
    return val, g


def interp3(vol, x, y, z):
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    g = np.zeros(3)
    h, w, d = vol.shape
    val = _load().oracle_interp3(vol, w, h, d, float(x), float(y), float(z), g)
    return val, g


def loss(x, eps, kind=LOSS_PSEUDO_HUBER):
    dl = C.c_double()
    val = _load().oracle_loss(float(x), float(eps), int(kind), C.byref(dl))
    return val, dl.value


def chain(t):
    """Time-ordered chain of a [h][w] time map: (order[n], omega[n-1])."""
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    order = np.zeros(t.size, dtype=np.int64)
    omega = np.zeros(max(t.size - 1, 1))
    _load().oracle_chain(t, t.size, order, omega)
    return order, omega[: t.size - 1]


def _half(n):
    return (n + 1) // 2


def pyramid_volume(vol):
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    h, w, d = vol.shape
    out = np.zeros((_half(h), _half(w), _half(d)), dtype=np.float32)
    _load().oracle_pyramid_volume(vol, w, h, d, out)
    return out


def pyramid_image(img):
    img = np.ascontiguousarray(img, dtype=np.float32)
    h, w = img.shape
    out = np.zeros((_half(h), _half(w)), dtype=np.float32)
    _load().oracle_pyramid_image(img, w, h, out)
    return out


def pyramid_line(v):
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.zeros(_half(v.shape[0]), dtype=np.float32)
    _load().oracle_pyramid_line(v, v.shape[0], out)
    return out


def pyramid_time(t):
    t = np.ascontiguousarray(t, dtype=np.float64)
    h, w = t.shape
    out = np.zeros((_half(h), _half(w)))
    _load().oracle_pyramid_time(t, w, h, out)
    return out


def prealign_prolong(prm, wc, hc, wf, hf):
    out = np.zeros(2 * (wf + hf))
    _load().oracle_prealign_prolong(np.ascontiguousarray(prm, dtype=np.float64), wc, hc, out, wf, hf)
    return out


def prolong(coarse, hf, wf):
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    hc, wc = coarse.shape[-2:]
    fine = np.zeros((2, 3, hf, wf))
    _load().oracle_prolong(coarse, wc, hc, fine, wf, hf)
    return fine


def lbfgs_direction(S, Y, g):
    """-H g by the two-loop recursion; S, Y lists of pairs, oldest first."""
    g = np.ascontiguousarray(g, dtype=np.float64).ravel()
    S = [np.ascontiguousarray(s, dtype=np.float64).ravel() for s in S]
    Y = [np.ascontiguousarray(y, dtype=np.float64).ravel() for y in Y]
    k = len(S)
    sp = (C.c_void_p * max(k, 1))(*[s.ctypes.data for s in S])
    yp = (C.c_void_p * max(k, 1))(*[y.ctypes.data for y in Y])
    out = np.zeros_like(g)
    _load().oracle_lbfgs_direction(g.size, k, sp, yp, g, out)
    return out


def lbfgs_minimize(fg, x0, m=8, max_iter=200, max_ls=20, gtol=1e-6, ftol=1e-9):
    """The oracle's L-BFGS (the level solver's minimiser) on fg(x) -> (f, g)
    from x0; returns (x, stats dict)."""
    x = np.array(x0, dtype=np.float64).ravel()
    n = x.size

    def cb(n_, xp, fp, gp):
        xv = np.ctypeslib.as_array(xp, shape=(n_,)).copy()
        f, g = fg(xv)
        fp[0] = float(f)
        np.ctypeslib.as_array(gp, shape=(n_,))[:] = np.asarray(g, dtype=np.float64).ravel()

    cfn = _FG(cb)
    opt = _Solver(m, max_iter, max_ls, gtol, ftol)
    st = _Stats()
    _load().oracle_lbfgs_minimize_fn(n, x, cfn, C.byref(opt), C.byref(st))
    return x, {"iters": st.iters, "evals": st.evals, "status": st.status, "f": st.f}


# ---------------------------------------------------------------- problem
class OracleProblem:
    """One registration problem (two orthogonal scans) on the CPU, FP64.

    Parameters follow the objective f = eta S^str + S^ang/eta + alpha R + M
    (Eq. 1, 9).  ``mu=None`` selects mu = 1/(2 w h) of each level.
    """

    def __init__(self, sx, sy, tx, ty, ax=None, ay=None, vx=None, vy=None, alpha=0.1,
                 delta0=0.5, eps_h=1e-3, eps_r=1e-2, mu=None, loss=LOSS_PSEUDO_HUBER):
        self.sx = np.ascontiguousarray(sx, dtype=np.float32)
        self.sy = np.ascontiguousarray(sy, dtype=np.float32)
        self.h, self.w, self.d = self.sx.shape
        assert self.sy.shape == self.sx.shape
        self.tx = np.ascontiguousarray(tx, dtype=np.float64)
        self.ty = np.ascontiguousarray(ty, dtype=np.float64)
        f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
        self.ax, self.ay, self.vx, self.vy = f32(ax), f32(ay), f32(vx), f32(vy)
        self.alpha, self.delta0, self.eps_h, self.eps_r = alpha, delta0, eps_h, eps_r
        self.mu = mu
        self.loss = loss
        self.eta = 1.0

    # -- level plumbing
    def _level(self):
        L = _Level()
        L.w, L.h, L.d = self.w, self.h, self.d
        ptr = lambda a: None if a is None else a.ctypes.data
        L.sx, L.sy = ptr(self.sx), ptr(self.sy)
        L.ax, L.ay = ptr(self.ax), ptr(self.ay)
        L.vx, L.vy = ptr(self.vx), ptr(self.vy)
        L.tx, L.ty = ptr(self.tx), ptr(self.ty)
        L.alpha, L.delta0, L.eps_h, L.eps_r = self.alpha, self.delta0, self.eps_h, self.eps_r
        L.mu = self.mu if self.mu is not None else 1.0 / (2.0 * self.w * self.h)
        L.eta = self.eta
        L.loss = self.loss
        return L

    def shape_disp(self):
        return (2, 3, self.h, self.w)

    def eval(self, disp, grad=True):
        """Returns (f, grad or None, terms) with terms = [S^str, S^ang, R, M, f, eta]."""
        disp = np.ascontiguousarray(disp, dtype=np.float64)
        assert disp.shape == self.shape_disp()
        L = self._level()
        f = C.c_double()
        g = np.zeros(self.shape_disp()) if grad else None
        terms = np.zeros(6)
        _load().oracle_eval(C.byref(L), disp, C.byref(f), None if g is None else g.ctypes.data,
                            terms.ctypes.data)
        return f.value, g, terms

    def data_rows(self, disp, j0, j1):
        """[S^str, S^ang] over rows j0..j1-1 only (bounded timing sample)."""
        disp = np.ascontiguousarray(disp, dtype=np.float64)
        out = np.zeros(2)
        L = self._level()
        _load().oracle_data_rows(C.byref(L), disp, int(j0), int(j1), out)
        return out

    def compute_eta(self, disp0):
        disp0 = np.ascontiguousarray(disp0, dtype=np.float64)
        L = self._level()
        return _load().oracle_eta(C.byref(L), disp0)

    def solve_level(self, disp, m=8, max_iter=5000, max_ls=20, gtol=1e-6, ftol=1e-7, set_eta=True):
        """L-BFGS solve of this level from disp; returns (disp, stats dict)."""
        x = np.array(disp, dtype=np.float64, order="C", copy=True)
        if set_eta:
            self.eta = self.compute_eta(x)
        L = self._level()
        opt = _Solver(m, max_iter, max_ls, gtol, ftol)
        st = _Stats()
        _load().oracle_solve_level(C.byref(L), x, C.byref(opt), C.byref(st))
        return x, dict(iters=st.iters, evals=st.evals, status=st.status, f=st.f, eta=self.eta)

    def merge(self, disp, beta=2.0, tau=0.05):
        """Final resampling and merging (Sec. 2.1, 2.5): dict with merged, cx, cy
        [h][w][d], weights [2][h][w], angio [h][w] (if angiography), density [2][h][w]."""
        disp = np.ascontiguousarray(disp, dtype=np.float64)
        h, w, d = self.h, self.w, self.d
        out = dict(merged=np.zeros((h, w, d), np.float32), cx=np.zeros((h, w, d), np.float32),
                   cy=np.zeros((h, w, d), np.float32), weights=np.zeros((2, h, w), np.float32),
                   angio=np.zeros((h, w), np.float32), density=np.zeros((2, h, w)))
        L = self._level()
        _load().oracle_merge(C.byref(L), disp, float(beta), float(tau), out["merged"].ctypes.data,
                             out["cx"].ctypes.data, out["cy"].ctypes.data, out["weights"].ctypes.data,
                             out["angio"].ctypes.data if self.ax is not None else None,
                             out["density"].ctypes.data)
        if self.ax is None:
            out["angio"] = None
        return out

    def downsample(self):
        """The next coarser pyramid level (Sec. 2.1, factor 2)."""
        p = OracleProblem.__new__(OracleProblem)
        p.__dict__.update(self.__dict__)
        p.sx, p.sy = pyramid_volume(self.sx), pyramid_volume(self.sy)
        p.h, p.w, p.d = p.sx.shape
        p.tx, p.ty = pyramid_time(self.tx), pyramid_time(self.ty)
        p.ax = None if self.ax is None else pyramid_image(self.ax)
        p.ay = None if self.ay is None else pyramid_image(self.ay)
        p.vx = None if self.vx is None else pyramid_line(self.vx)
        p.vy = None if self.vy is None else pyramid_line(self.vy)
        p.eta = 1.0
        return p

    # -- rough axial prealignment (stage 1): parameters [aX(h), tX(h), aY(w), tY(w)]
    def n_prealign(self):
        return 2 * (self.h + self.w)

    def prealign_disp(self, prm):
        """The displacement field [2][3][h][w] the B-scan offsets and tilts induce."""
        prm = np.ascontiguousarray(prm, dtype=np.float64)
        assert prm.shape == (self.n_prealign(),)
        out = np.zeros(self.shape_disp())
        L = self._level()
        _load().oracle_prealign_disp(C.byref(L), prm, out)
        return out

    def prealign_eval(self, prm, grad=True):
        """(f, gradient or None, terms [S^str, R, M, T, f]) of the stage-1 objective."""
        prm = np.ascontiguousarray(prm, dtype=np.float64)
        assert prm.shape == (self.n_prealign(),)
        L = self._level()
        f = C.c_double()
        g = np.zeros(self.n_prealign()) if grad else None
        terms = np.zeros(5)
        _load().oracle_prealign_eval(C.byref(L), prm, C.byref(f), None if g is None else g.ctypes.data,
                                     terms.ctypes.data)
        return f.value, g, terms

    def prealign_level(self, prm, m=8, max_iter=200, max_ls=20, gtol=1e-6, ftol=1e-9):
        x = np.array(prm, dtype=np.float64, order="C", copy=True)
        L = self._level()
        opt = _Solver(m, max_iter, max_ls, gtol, ftol)
        st = _Stats()
        _load().oracle_prealign_level(C.byref(L), x, C.byref(opt), C.byref(st))
        return x, dict(iters=st.iters, evals=st.evals, status=st.status, f=st.f)

    def prealign_full(self, levels, **kw):
        """Coarse-to-fine stage-1 solve from zero parameters."""
        pyr = self.pyramid(levels)
        prm = np.zeros(pyr[-1].n_prealign())
        stats = []
        for lv in range(levels - 1, -1, -1):
            P = pyr[lv]
            if lv != levels - 1:
                C_ = pyr[lv + 1]
                fine = np.zeros(P.n_prealign())
                _load().oracle_prealign_prolong(np.ascontiguousarray(prm), C_.w, C_.h, fine, P.w, P.h)
                prm = fine
            prm, st = P.prealign_level(prm, **kw)
            st["level"] = lv
            stats.append(st)
        return prm, stats

    def pyramid(self, levels):
        out = [self]
        for _ in range(levels - 1):
            out.append(out[-1].downsample())
        return out

    def solve_full(self, levels, **kw):
        """Coarse-to-fine solve from zero displacement (Sec. 2.1)."""
        pyr = self.pyramid(levels)
        disp = np.zeros(pyr[-1].shape_disp())
        stats = []
        for lv in range(levels - 1, -1, -1):
            P = pyr[lv]
            if lv != levels - 1:
                disp = prolong(disp, P.h, P.w)
            disp, st = P.solve_level(disp, **kw)
            st["level"] = lv
            stats.append(st)
        return disp, stats


# ---------------------------------------------------------------- angiography preprocessing (Sec. 2.2, 2.3)
def _vol(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def saccade_validity(A, fast_axis):
    """(validity per B-scan float32, mean decorrelation per B-scan float64) of an
    OCTA volume [h][w][d]; fast_axis 0 (X-fast, B-scans are rows) or 1."""
    A = _vol(A)
    h, w, d = A.shape
    nb = h if fast_axis == 0 else w
    v = np.zeros(nb, np.float32)
    m = np.zeros(nb)
    _load().oracle_saccade_validity(A, w, h, d, int(fast_axis), v, m)
    return v, m


def median3(A):
    A = _vol(A)
    out = np.empty_like(A)
    h, w, d = A.shape
    _load().oracle_median3(A, w, h, d, out)
    return out


def rank_filter(A, axis, width=15, rank=3):
    """rank-th smallest (1-based) of `width` samples along axis 0 (x) or 1 (y)."""
    A = _vol(A)
    out = np.empty_like(A)
    h, w, d = A.shape
    _load().oracle_rank_filter(A, w, h, d, int(axis), int(width), int(rank), out)
    return out


def percentile(x, q):
    x = _vol(np.ravel(x))
    return _load().oracle_percentile(x, x.size, float(q))


def bscan_median_subtract(E, fast_axis):
    E = _vol(E).copy()
    h, w = E.shape
    _load().oracle_bscan_median_subtract(E, w, h, int(fast_axis))
    return E


def replace_invalid(E, fast_axis, v):
    E = _vol(E).copy()
    h, w = E.shape
    _load().oracle_replace_invalid(E, w, h, int(fast_axis), _vol(v))
    return E


def enface(A, S, fast_axis, v, q_lo=0.05, q_hi=0.95, thresh=0.1, t_oct=None, want_filtered=False):
    """En-face OCTA image of one scan (Sec. 2.3).  Returns (E [h][w], info dict,
    rank-filtered volume or None)."""
    A, S = _vol(A), _vol(S)
    h, w, d = A.shape
    E = np.zeros((h, w), np.float32)
    info = np.zeros(4)
    filt = np.empty_like(A) if want_filtered else None
    _load().oracle_enface(A, S, w, h, d, int(fast_axis), _vol(v), float(q_lo), float(q_hi), float(thresh),
                          float("nan") if t_oct is None else float(t_oct),
                          None if filt is None else filt.ctypes.data, E, info)
    return E, dict(p_lo=info[0], p_hi=info[1], t_oct=info[2], kept=int(info[3])), filt
