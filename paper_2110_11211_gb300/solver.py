"""Python handle around the C-ABI: torch tensors provide device memory and the
stream; every step of the solver runs in the CUDA library."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import Info, Options, Stats, Tuning, check


def _dev_ptr(t: torch.Tensor, dtype=torch.float64) -> int:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return t.data_ptr()


class Solver:
    """Two-level SFC Schwarz-preconditioned CG for the anisotropic FD Poisson
    operator on levels `levels` with P subdomains and overlap gamma."""

    def __init__(self, levels, P, overlap, *, precision="fp64", variant="additive",
                 weighting="omega", q=0, coeffs=None, flexible=-1, stream=None,
                 profile=False, local_order="lex", slabs_local=0, slabs_coarse=0,
                 tensor_cores=-1, coarse_block=0):
        L = _lib.lib()
        self.levels = tuple(int(l) for l in levels)
        self.d = len(self.levels)
        self.P = int(P)
        self.overlap = float(overlap)
        self.shape = tuple((1 << l) - 1 for l in self.levels)
        opt = Options()
        L.sfcdd_default_options(C.byref(opt))
        self._coeffs = None
        if coeffs is not None:
            vals = [float(c) for c in coeffs]
            self._coeffs = (C.c_double * self.d)(*vals)
            opt.coeffs = C.cast(self._coeffs, C.POINTER(C.c_double))
        opt.q = int(q)
        opt.variant = _lib.VARIANT[variant]
        opt.weighting = _lib.WEIGHTING[weighting]
        opt.precision = _lib.PRECISION[precision]
        opt.flexible = int(flexible)
        opt.profile = int(bool(profile))
        opt.local_order = {"lex": 0, "curve": 1}[local_order]
        opt.slabs_local = int(slabs_local)
        opt.slabs_coarse = int(slabs_coarse)
        opt.tensor_cores = int(tensor_cores)
        opt.coarse_block = int(coarse_block)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = C.c_void_p(stream.cuda_stream)
        lv = (C.c_int * self.d)(*self.levels)
        h = C.c_void_p()
        check("sfcdd_setup_ex", L.sfcdd_setup_ex(lv, self.d, self.P, self.overlap, C.byref(opt),
                                                  C.byref(h)))
        self._h = h
        self._L = L
        self.info = self.get_info()
        self.N = int(self.info.N)

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None):
            self._L.sfcdd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- solves ----
    def solve(self, f: torch.Tensor, rtol=1e-10, maxit=1000, out=None, check_status=True):
        f = f.reshape(-1)
        u = torch.empty_like(f) if out is None else out
        st = Stats()
        rc = self._L.sfcdd_solve(self._h, _dev_ptr(f), _dev_ptr(u), float(rtol), int(maxit),
                                 C.byref(st))
        self.last_stats = st
        if check_status:
            check("sfcdd_solve", rc)
        return u, st

    def solve_host(self, f, rtol=1e-10, maxit=1000):
        import numpy as np
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        u = np.empty_like(f)
        st = Stats()
        rc = self._L.sfcdd_solve_host(self._h, f.ctypes.data, u.ctypes.data, float(rtol),
                                      int(maxit), C.byref(st))
        check("sfcdd_solve_host", rc)
        return u, st

    def solve_backward(self, u: torch.Tensor, gu: torch.Tensor, rtol=1e-10, maxit=1000):
        u = u.reshape(-1).contiguous()
        gu = gu.reshape(-1).contiguous()
        gf = torch.empty_like(gu)
        gc = (C.c_double * self.d)()
        st = Stats()
        rc = self._L.sfcdd_solve_backward(self._h, _dev_ptr(u), _dev_ptr(gu), _dev_ptr(gf), gc,
                                          float(rtol), int(maxit), C.byref(st))
        check("sfcdd_solve_backward", rc)
        return gf, [gc[j] for j in range(self.d)], st

    def estimate_spectrum(self, f: torch.Tensor, steps=200):
        """(lambda_min, lambda_max) estimates of C^{-1} A from a PCG run on f."""
        lo, hi = C.c_double(), C.c_double()
        check("sfcdd_estimate_spectrum",
              self._L.sfcdd_estimate_spectrum(self._h, _dev_ptr(f.reshape(-1).contiguous()),
                                              int(steps), C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def richardson(self, f: torch.Tensor, xi, rtol=1e-8, maxit=100000, check_status=True):
        """Algorithm 3: damped preconditioned Richardson iteration from x = 0."""
        f = f.reshape(-1).contiguous()
        u = torch.empty_like(f)
        st = Stats()
        rc = self._L.sfcdd_richardson(self._h, _dev_ptr(f), _dev_ptr(u), float(xi), float(rtol),
                                      int(maxit), C.byref(st))
        if check_status:
            check("sfcdd_richardson", rc)
        return u, st

    def solve_homogeneous(self, x0: torch.Tensor, method="pcg", xi=0.0, tol=1e-8, maxit=100000,
                          check_status=True):
        """Sec. 4 protocol: A x = 0 from x0, until ||x_K||_A <= tol ||x0||_A.
        method 'pcg' or 'richardson' (damping xi).  Returns (x_K, stats)."""
        m = {"pcg": 0, "richardson": 1}[method]
        x0 = x0.reshape(-1).contiguous()
        u = torch.empty_like(x0)
        st = Stats()
        rc = self._L.sfcdd_solve_homogeneous(self._h, _dev_ptr(x0), _dev_ptr(u), m, float(xi),
                                             float(tol), int(maxit), C.byref(st))
        if check_status:
            check("sfcdd_solve_homogeneous", rc)
        return u, st

    def autotune(self, reps=5):
        """Pick the substitution shapes (whole-matrix local items, slabs_local = -1,
        or row slabs) by timing preconditioner applies."""
        t = Tuning()
        check("sfcdd_autotune", self._L.sfcdd_autotune(self._h, int(reps), C.byref(t)))
        return {"slabs_local": t.slabs_local, "slabs_coarse": t.slabs_coarse,
                "apply_ms": t.apply_ms, "candidates": t.candidates}

    def selftest(self, kind):
        """Failure-detection self-test ('wait_timeout' or 'breakdown'): returns
        (status the device recorded, index or site)."""
        k = {"wait_timeout": 1, "breakdown": 2}[kind]
        d = C.c_int(-1)
        rc = self._L.sfcdd_selftest(self._h, k, C.byref(d))
        return rc, d.value

    def apply_operator(self, x: torch.Tensor, curve_order=False):
        y = torch.empty_like(x)
        check("sfcdd_apply_operator",
              self._L.sfcdd_apply_operator(self._h, _dev_ptr(x), _dev_ptr(y), int(curve_order)))
        return y

    def apply_precond(self, g: torch.Tensor, curve_order=False):
        z = torch.empty_like(g)
        check("sfcdd_apply_precond",
              self._L.sfcdd_apply_precond(self._h, _dev_ptr(g), _dev_ptr(z), int(curve_order)))
        return z

    # ---- introspection ----
    def get_info(self) -> Info:
        info = Info()
        check("sfcdd_get_info", self._L.sfcdd_get_info(self._h, C.byref(info)))
        return info

    def curve(self):
        keys = torch.empty(self.N, dtype=torch.int64, device="cuda")
        perm = torch.empty(self.N, dtype=torch.int32, device="cuda")
        check("sfcdd_get_curve", self._L.sfcdd_get_curve(self._h, keys.data_ptr(), perm.data_ptr()))
        return keys, perm

    def partition(self):
        import numpy as np
        start = np.zeros(self.P, dtype=np.int64)
        length = np.zeros(self.P, dtype=np.int64)
        omega = np.zeros(self.P, dtype=np.float64)
        check("sfcdd_get_partition", self._L.sfcdd_get_partition(
            self._h, start.ctypes.data_as(C.POINTER(C.c_longlong)),
            length.ctypes.data_as(C.POINTER(C.c_longlong)),
            omega.ctypes.data_as(C.POINTER(C.c_double))))
        return start, length, omega

    def coarse_matrix(self):
        n0 = int(self.info.N0)
        A0 = torch.empty(n0 * n0, dtype=torch.float64, device="cuda")
        check("sfcdd_get_coarse_matrix", self._L.sfcdd_get_coarse_matrix(self._h, A0.data_ptr()))
        return A0.reshape(n0, n0)

    def local_matrix(self, i: int):
        _, length, _ = self.partition()
        n = int(length[i])
        Ai = torch.empty(n * n, dtype=torch.float64, device="cuda")
        check("sfcdd_get_local_matrix", self._L.sfcdd_get_local_matrix(self._h, int(i), Ai.data_ptr()))
        return Ai.reshape(n, n)

    def set_profiling(self, on: bool):
        check("sfcdd_set_profiling", self._L.sfcdd_set_profiling(self._h, int(bool(on))))

    def kernel_stats(self, reset=False):
        n = len(_lib.KERNEL_CLASSES)
        ms = (C.c_double * n)()
        la = (C.c_longlong * n)()
        check("sfcdd_get_kernel_stats", self._L.sfcdd_get_kernel_stats(self._h, ms, la, int(reset)))
        return {k: (ms[i], la[i]) for i, k in enumerate(_lib.KERNEL_CLASSES)}

    def kernel_work(self, cls: str) -> float:
        return float(self._L.sfcdd_kernel_work(self._h, _lib.KERNEL_CLASSES.index(cls)))


class BatchSolver:
    """Many independent subgrid problems (same d, overlap, options; P shared or
    one per subgrid), set up together and solved in one CUDA-graph launch
    (sfcdd_batch_*).  Vectors are the concatenation of the subgrids'
    lexicographic vectors at `offsets`."""

    def __init__(self, levels_list, P, overlap, *, precision="fp64", weighting="omega", q=0,
                 coeffs=None, flexible=-1, stream=None, local_order="lex", slabs_local=0,
                 slabs_coarse=0, tensor_cores=-1, variant="additive"):
        L = _lib.lib()
        self.levels = [tuple(int(l) for l in lv) for lv in levels_list]
        self.nsub = len(self.levels)
        self.d = len(self.levels[0])
        if any(len(lv) != self.d for lv in self.levels):
            raise ValueError("all subgrids must have the same dimension")
        opt = Options()
        L.sfcdd_default_options(C.byref(opt))
        self._coeffs = None
        if coeffs is not None:
            self._coeffs = (C.c_double * self.d)(*[float(c) for c in coeffs])
            opt.coeffs = C.cast(self._coeffs, C.POINTER(C.c_double))
        opt.q = int(q)
        opt.variant = _lib.VARIANT[variant]
        opt.weighting = _lib.WEIGHTING[weighting]
        opt.precision = _lib.PRECISION[precision]
        opt.flexible = int(flexible)
        opt.local_order = {"lex": 0, "curve": 1}[local_order]
        opt.slabs_local = int(slabs_local)
        opt.slabs_coarse = int(slabs_coarse)
        opt.tensor_cores = int(tensor_cores)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = C.c_void_p(stream.cuda_stream)
        flat = (C.c_int * (self.nsub * self.d))(*[l for lv in self.levels for l in lv])
        h = C.c_void_p()
        if isinstance(P, (int, np.integer)):
            check("sfcdd_batch_setup", L.sfcdd_batch_setup(flat, self.nsub, self.d, int(P),
                                                           float(overlap), C.byref(opt),
                                                           C.byref(h)))
        else:
            if len(P) != self.nsub:
                raise ValueError("one subdomain count per subgrid")
            Ps = (C.c_int * self.nsub)(*[int(p) for p in P])
            check("sfcdd_batch_setup_each",
                  L.sfcdd_batch_setup_each(flat, Ps, self.nsub, self.d, float(overlap),
                                           C.byref(opt), C.byref(h)))
        self._h = h
        self._L = L
        offs = (C.c_longlong * (self.nsub + 1))()
        check("sfcdd_batch_offsets", L.sfcdd_batch_offsets(h, offs))
        self.offsets = [int(offs[i]) for i in range(self.nsub + 1)]
        self.N = self.offsets[-1]

    def info(self):
        n = C.c_longlong()
        fb = C.c_longlong()
        ms = C.c_double()
        check("sfcdd_batch_info", self._L.sfcdd_batch_info(self._h, C.byref(n), C.byref(fb),
                                                           C.byref(ms)))
        return {"N": n.value, "factor_bytes": fb.value, "setup_ms": ms.value}

    def solve(self, f: torch.Tensor, rtol=1e-10, maxit=1000, check_status=True):
        f = f.reshape(-1)
        u = torch.empty_like(f)
        per = (Stats * self.nsub)()
        tot = Stats()
        rc = self._L.sfcdd_batch_solve(self._h, _dev_ptr(f), _dev_ptr(u), float(rtol), int(maxit),
                                       per, C.byref(tot))
        if check_status:
            check("sfcdd_batch_solve", rc)
        return u, tot, [per[i] for i in range(self.nsub)]

    def autotune(self, reps=3):
        """Pick the substitution slab shapes by timing batched substitution pairs."""
        t = Tuning()
        check("sfcdd_batch_autotune", self._L.sfcdd_batch_autotune(self._h, int(reps), C.byref(t)))
        return {"slabs_local": t.slabs_local, "slabs_coarse": t.slabs_coarse,
                "apply_ms": t.apply_ms, "candidates": t.candidates}

    def combine(self, coef, u: torch.Tensor, points: torch.Tensor):
        """eq. combi at points (npts x d, device): sum_s coef[s] I_s u_s."""
        cf = (C.c_double * self.nsub)(*[float(c) for c in coef])
        pts = points.reshape(-1, self.d).contiguous()
        out = torch.empty(pts.shape[0], dtype=torch.float64, device=pts.device)
        check("sfcdd_batch_combine",
              self._L.sfcdd_batch_combine(self._h, cf, _dev_ptr(u.contiguous()), _dev_ptr(pts),
                                          int(pts.shape[0]), _dev_ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._L.sfcdd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
