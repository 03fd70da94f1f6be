"""Thin ctypes binding of libbmg (include/bmg.h): argument marshalling only.

Every computation runs inside libbmg's CUDA kernels.  Device buffers are torch CUDA
tensors (float64, contiguous) passed by pointer together with the current torch
stream; host outputs are numpy arrays.  Importing this module loads libbmg.so and
raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbmg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bmg.h")

SMOOTHERS = {"jacobi": 0, "mcgs": 1, "mcsgs": 2, "kaczmarz": 3}
FORMS = {"shifted": 0, "homogeneous": 1}
PRECISIONS = {"fp64": 0, "fp32": 1}
STATUS = {0: "BMG_OK", 1: "BMG_ERR_INVALID_ARG", 2: "BMG_ERR_CUDA", 3: "BMG_ERR_OOM",
          4: "BMG_ERR_SINGULAR", 5: "BMG_ERR_NOT_CONVERGED", 6: "BMG_ERR_NONFINITE",
          7: "BMG_ERR_MESH", 8: "BMG_ERR_STATE", 9: "BMG_ERR_TIMEOUT"}


class BmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Options(C.Structure):
    _fields_ = [("smoother", C.c_int), ("nu", C.c_int), ("omega", C.c_double), ("form", C.c_int),
                ("vcycle_depth", C.c_int), ("cycles_intermediate", C.c_int),
                ("tol_intermediate", C.c_double), ("max_cycles", C.c_int), ("precision", C.c_int),
                ("switch_tol", C.c_double), ("stop_after_cycles", C.c_int), ("resume", C.c_int),
                ("tensor_cores", C.c_int), ("autotune", C.c_int), ("graphs", C.c_int),
                ("adaptive_shift", C.c_int), ("selection", C.c_int), ("index_first", C.c_int),
                ("coarse_start", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("levels", C.c_int), ("cycles", C.c_int * 32), ("total_cycles", C.c_int),
                ("converged", C.c_int), ("max_resid", C.c_double), ("max_dense_err", C.c_double),
                ("fp32_cycles", C.c_int), ("n_history", C.c_int), ("history_level", C.c_int * 256),
                ("history_fp32", C.c_int * 256), ("history_resid", C.c_double * 256),
                ("final_shift", C.c_double)]

    def history(self):
        """[(level, fp32, max wanted residual)] per cycle (first 256 cycles)."""
        return [(self.history_level[q], self.history_fp32[q], self.history_resid[q])
                for q in range(self.n_history)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libbmg.so not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
                          "(expected at %s)" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, ip, dp, i, d = C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double
    P = C.POINTER
    sig = {
        "bmg_default_options": (None, [P(Options)]),
        "bmg_last_error": (C.c_char_p, []),
        "bmg_destroy": (None, [vp]),
        "bmg_assemble": (i, [vp, i, vp, i, i, d, vp, vp, P(vp)]),
        "bmg_hierarchy": (i, [vp, i]),
        "bmg_solve": (i, [vp, i, i, d, d, P(Options), vp, i, vp, vp, i, vp, P(SolveInfo)]),
        "bmg_solve_batched": (i, [i, P(vp), P(C.c_double), i, i, d, P(Options), P(vp), P(vp), P(vp), P(vp),
                                  P(SolveInfo), i]),
        "bmg_get_sizes": (i, [vp, i, P(C.c_int), P(C.c_int), P(C.c_int)]),
        "bmg_get_mesh": (i, [vp, i, vp, vp, vp]),
        "bmg_get_csr": (i, [vp, i, vp, vp, vp, vp]),
        "bmg_get_galerkin": (i, [vp, i, i, vp, vp]),
        "bmg_get_colouring": (i, [vp, i, vp, P(C.c_int)]),
        "bmg_get_colouring2": (i, [vp, i, vp, P(C.c_int)]),
        "bmg_spmm": (i, [vp, i, i, vp, i, i, vp, vp, vp]),
        "bmg_smooth": (i, [vp, i, i, vp, vp, vp, i, i, i, i, d, vp, vp]),
        "bmg_spmm_f32": (i, [vp, i, i, vp, i, i, vp, vp, vp]),
        "bmg_smooth_f32": (i, [vp, i, i, vp, vp, vp, i, i, i, i, d, vp, vp]),
        "bmg_gram_f32": (i, [vp, vp, i, i, i, vp, vp]),
        "bmg_prolong": (i, [vp, i, vp, vp, i, i, i, vp]),
        "bmg_restrict": (i, [vp, i, vp, vp, i, i, vp]),
        "bmg_gram": (i, [vp, vp, i, i, i, vp, vp]),
        "bmg_gram_noalloc": (i, [vp, vp, i, i, i, vp, vp]),
        "bmg_gram_tc": (i, [vp, vp, i, i, i, vp, vp]),
        "bmg_gram_tc_f32": (i, [vp, vp, i, i, i, vp, vp]),
        "bmg_tc_timeout_selftest": (i, [vp]),
        "bmg_expand": (i, [vp, vp, vp, i, i, i, i, vp, i, vp]),
        "bmg_expand_f32": (i, [vp, vp, vp, i, i, i, i, vp, i, vp]),
        "bmg_dense_eig": (i, [vp, vp, i, d, i, vp, vp, vp, vp]),
        "bmg_profile_enable": (i, [i]),
        "bmg_profile_reset": (i, []),
        "bmg_profile_read": (i, [i, P(C.c_double), P(C.c_longlong), P(C.c_double), P(C.c_double)]),
        "bmg_kernel_class_name": (C.c_char_p, [i]),
        "bmg_launch_count": (C.c_longlong, []),
        "bmg_autotune_report": (i, [C.c_char_p, i]),
        "bmg_get_state": (i, [vp, i, vp, C.c_size_t, P(C.c_size_t)]),
        "bmg_set_state": (i, [vp, i, vp, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def header_symbols():
    """Function names declared in include/bmg.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bmg_[a-z_0-9]+)\s*\(", text)))


def _check(code):
    if code != 0:
        raise BmgError(code, LIB.bmg_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def options(smoother="jacobi", nu=2, omega=2.0 / 3.0, form="shifted", vcycle_depth=99,
            cycles_intermediate=6, tol_intermediate=-1.0, max_cycles=200, precision="fp64",
            switch_tol=1e-7, stop_after_cycles=0, resume=False, tensor_cores=True, autotune=True,
            graphs=True, adaptive_shift=False, selection="nearest", index_first=0, init="given") -> Options:
    o = Options()
    LIB.bmg_default_options(C.byref(o))
    o.smoother = SMOOTHERS[smoother]
    o.nu = nu
    o.omega = omega
    o.form = FORMS[form]
    o.vcycle_depth = vcycle_depth
    o.cycles_intermediate = cycles_intermediate
    o.tol_intermediate = tol_intermediate
    o.max_cycles = max_cycles
    o.precision = PRECISIONS[precision]
    o.switch_tol = switch_tol
    o.stop_after_cycles = stop_after_cycles
    o.resume = int(bool(resume))
    o.tensor_cores = int(bool(tensor_cores))
    o.autotune = int(bool(autotune))
    o.graphs = int(bool(graphs))
    o.adaptive_shift = int(bool(adaptive_shift))
    o.selection = {"nearest": 0, "index": 1}[selection]
    o.index_first = int(index_first)
    o.coarse_start = {"given": 0, "coarse": 1}[init]
    return o


class Problem:
    """A surface hierarchy and its operators, owned by libbmg on the GPU."""

    def __init__(self, verts, tris, refinements, amplitude=0.0, coefs=None, stream=None):
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        cf = None if coefs is None else np.ascontiguousarray(coefs, dtype=np.float64)
        h = C.c_void_p()
        s = _stream() if stream is None else stream
        _check(LIB.bmg_assemble(_ptr(v), v.shape[0], _ptr(t), t.shape[0], refinements, float(amplitude),
                                _ptr(cf), s, C.byref(h)))
        self.h = h
        self.refinements = refinements
        self.levels = 0

    def close(self):
        if getattr(self, "h", None):
            LIB.bmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hierarchy(self, levels):
        _check(LIB.bmg_hierarchy(self.h, levels))
        self.levels = levels

    def level_refinement(self, level):
        return self.refinements - self.levels + level

    def sizes(self, refinement):
        n, nt, nnz = C.c_int(), C.c_int(), C.c_int()
        _check(LIB.bmg_get_sizes(self.h, refinement, C.byref(n), C.byref(nt), C.byref(nnz)))
        return n.value, nt.value, nnz.value

    def mesh(self, refinement):
        n, nt, _ = self.sizes(refinement)
        v = np.empty((n, 3)); t = np.empty((nt, 3), np.int32); p = np.empty((n, 2), np.int32)
        _check(LIB.bmg_get_mesh(self.h, refinement, _ptr(v), _ptr(t), _ptr(p)))
        return v, t, p

    def csr(self, refinement, values=True):
        n, _, nnz = self.sizes(refinement)
        rp = np.empty(n + 1, np.int32); col = np.empty(nnz, np.int32)
        a = np.empty(nnz) if values else None
        m = np.empty(nnz) if values else None
        _check(LIB.bmg_get_csr(self.h, refinement, _ptr(rp), _ptr(col), _ptr(a), _ptr(m)))
        return rp, col, a, m

    def galerkin(self, f, j):
        _, _, nnz = self.sizes(self.level_refinement(j))
        a = np.empty(nnz); m = np.empty(nnz)
        _check(LIB.bmg_get_galerkin(self.h, f, j, _ptr(a), _ptr(m)))
        return a, m

    def colouring(self, level):
        n, _, _ = self.sizes(self.level_refinement(level))
        c = np.empty(n, np.int32)
        nc = C.c_int()
        _check(LIB.bmg_get_colouring(self.h, level, _ptr(c), C.byref(nc)))
        return c, nc.value

    def colouring2(self, level):
        """Distance-2 colouring of a level (the Kaczmarz smoother's)."""
        n, _, _ = self.sizes(self.level_refinement(level))
        c = np.empty(n, np.int32)
        nc = C.c_int()
        _check(LIB.bmg_get_colouring2(self.h, level, _ptr(c), C.byref(nc)))
        return c, nc.value

    # ---- individual cycle steps on torch CUDA tensors ([N][ld] float64) -------
    def spmm(self, f, level, X, k, AX, MX):
        _check(LIB.bmg_spmm(self.h, f, level, _ptr(X), k, X.shape[1], _ptr(AX), _ptr(MX), _stream()))

    def smooth(self, f, level, X, B, shift, k, smoother, nu, omega, work):
        _check(LIB.bmg_smooth(self.h, f, level, _ptr(X), _ptr(B), _ptr(shift), k, X.shape[1],
                              SMOOTHERS[smoother], nu, omega, _ptr(work), _stream()))

    def spmm_f32(self, f, level, X, k, AX, MX):
        """float32 blocks ([N][ld] with ld % 4 == 0), float32 operators."""
        _check(LIB.bmg_spmm_f32(self.h, f, level, _ptr(X), k, X.shape[1], _ptr(AX), _ptr(MX), _stream()))

    def smooth_f32(self, f, level, X, B, shift, k, smoother, nu, omega, work):
        _check(LIB.bmg_smooth_f32(self.h, f, level, _ptr(X), _ptr(B), _ptr(shift), k, X.shape[1],
                                  SMOOTHERS[smoother], nu, omega, _ptr(work), _stream()))

    def prolong(self, level, Xc, Y, k, add=False):
        _check(LIB.bmg_prolong(self.h, level, _ptr(Xc), _ptr(Y), k, Y.shape[1], int(add), _stream()))

    def restrict(self, level, R, Zc, k):
        _check(LIB.bmg_restrict(self.h, level, _ptr(R), _ptr(Zc), k, R.shape[1], _stream()))

    def solve_host(self, X0_host, U_host, k, n_wanted, sigma, tol, opt=None):
        """BFMG solve with host buffers (e.g. pinned torch CPU tensors): X0 [N_2, k] in,
        eigenvectors [N_L, n_wanted] out; copies happen inside the call."""
        ev, rs, info = _solve_raw(self.h, _ptr(X0_host), 0, _ptr(U_host), 0, k, n_wanted, sigma, tol, opt)
        return ev, U_host, rs, info

    def solve(self, X0, k, n_wanted, sigma, tol, opt=None, evecs=True, evecs_device=None):
        """BFMG solve.  X0: numpy [N_2, k] (host) or torch CUDA tensor (device); None
        with options(resume=True), which continues from the state given to set_state,
        or with options(init="coarse"), which starts from the coarse eigenvectors.

        Returns (evals, evecs, resid, info) with evecs a numpy array, or the
        caller's torch tensor `evecs_device` when given.
        """
        on_dev = X0 is not None and not isinstance(X0, np.ndarray)
        X0c = X0 if (on_dev or X0 is None) else np.ascontiguousarray(X0, dtype=np.float64)
        nL = self.sizes(self.refinements)[0]
        ev = np.empty(n_wanted)
        rs = np.empty(n_wanted)
        if evecs_device is not None:
            U, udev = evecs_device, 1
        elif evecs:
            U, udev = np.empty((nL, n_wanted)), 0
        else:
            U, udev = None, 0
        info = SolveInfo()
        o = opt if opt is not None else options()
        code = LIB.bmg_solve(self.h, k, n_wanted, float(sigma), float(tol), C.byref(o), _ptr(X0c),
                             int(on_dev), _ptr(ev), _ptr(U), udev, _ptr(rs), C.byref(info))
        if code not in (0, 5):
            _check(code)
        return ev, U, rs, info

    def get_state(self, k):
        """State of the last solve of block size k stopped by stop_after_cycles (bytes)."""
        n = C.c_size_t(0)
        _check(LIB.bmg_get_state(self.h, k, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(LIB.bmg_get_state(self.h, k, buf, n.value, C.byref(n)))
        return buf.raw[:n.value]

    def set_state(self, k, state):
        """Loads a state; the next solve with options(resume=True) continues from it."""
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(LIB.bmg_set_state(self.h, k, buf, len(state)))


def solve_batched(problems, sigmas, X0s, k, n_wanted, tol, opt=None, evecs=False, concurrency=0):
    """Batched form: job j solves problems[j] near sigmas[j] from X0s[j] (numpy
    [N_2, k]).  Returns (evals list, evecs list or None, resid list, infos, status)
    where status is 0 or 5 (some job hit its cycle cap)."""
    n = len(problems)
    x0 = [np.ascontiguousarray(x, dtype=np.float64) for x in X0s]
    ev = [np.empty(n_wanted) for _ in range(n)]
    rs = [np.empty(n_wanted) for _ in range(n)]
    U = [np.empty((p.sizes(p.refinements)[0], n_wanted)) for p in problems] if evecs else None
    infos = (SolveInfo * n)()
    arr = lambda xs: (C.c_void_p * n)(*[_ptr(x) for x in xs])
    o = opt if opt is not None else options()
    code = LIB.bmg_solve_batched(n, (C.c_void_p * n)(*[p.h for p in problems]),
                                 (C.c_double * n)(*[float(x) for x in sigmas]), k, n_wanted, float(tol),
                                 C.byref(o), arr(x0), arr(ev), arr(U) if evecs else None, arr(rs), infos,
                                 int(concurrency))
    if code not in (0, 5):
        _check(code)
    return ev, U, rs, list(infos), code


KERNEL_CLASSES = 8


def profile_enable(on=True):
    _check(LIB.bmg_profile_enable(int(bool(on))))


def profile_reset():
    _check(LIB.bmg_profile_reset())


def profile_read():
    """{class name: dict(ms, launches, bytes, flops)} summed since the last reset."""
    out = {}
    for c in range(KERNEL_CLASSES):
        ms, n, b, f = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        _check(LIB.bmg_profile_read(c, C.byref(ms), C.byref(n), C.byref(b), C.byref(f)))
        out[LIB.bmg_kernel_class_name(c).decode()] = dict(ms=ms.value, launches=n.value,
                                                          bytes=b.value, flops=f.value)
    return out


def autotune_report():
    """Row-kernel shapes chosen so far: [(kind, bytes, nch, rows, lanes, chunks, warps)]."""
    n = LIB.bmg_autotune_report(None, 0)
    buf = C.create_string_buffer(n + 1)
    LIB.bmg_autotune_report(buf, n + 1)
    out = []
    for line in buf.value.decode().splitlines():
        a, b = line.split(" -> ")
        k = a.split()
        v = b.split()
        out.append((k[0], int(k[1]), int(k[2]), int(k[3]), int(v[0]), int(v[1]), int(v[2])))
    return out


def launch_count():
    return int(LIB.bmg_launch_count())


def _solve_raw(h, X0_ptr, x0_dev, U_ptr, u_dev, k, n_wanted, sigma, tol, opt):
    ev = np.empty(n_wanted)
    rs = np.empty(n_wanted)
    info = SolveInfo()
    o = opt if opt is not None else options()
    code = LIB.bmg_solve(h, k, n_wanted, float(sigma), float(tol), C.byref(o), X0_ptr, x0_dev,
                         _ptr(ev), U_ptr, u_dev, _ptr(rs), C.byref(info))
    if code not in (0, 5):
        _check(code)
    return ev, rs, info


def gram(X, Y, k, G):
    _check(LIB.bmg_gram(_ptr(X), _ptr(Y), X.shape[0], k, X.shape[1], _ptr(G), _stream()))


def gram_f32(X, Y, k, G):
    """G (float64) = X^T Y for float32 blocks, compensated accumulation."""
    _check(LIB.bmg_gram_f32(_ptr(X), _ptr(Y), X.shape[0], k, X.shape[1], _ptr(G), _stream()))


def gram_tc(X, Y, k, G):
    """G = X^T Y on the tensor cores (exact BF16 digit products; k <= 128)."""
    _check(LIB.bmg_gram_tc(_ptr(X), _ptr(Y), X.shape[0], k, X.shape[1], _ptr(G), _stream()))


def gram_tc_f32(X, Y, k, G):
    """G (float64) = X^T Y for float32 blocks on the tensor cores (k <= 128)."""
    _check(LIB.bmg_gram_tc_f32(_ptr(X), _ptr(Y), X.shape[0], k, X.shape[1], _ptr(G), _stream()))


def tc_timeout_selftest():
    """Status code of bmg_tc_timeout_selftest (BMG_ERR_TIMEOUT when the waits expired)."""
    return int(LIB.bmg_tc_timeout_selftest(_stream()))


def expand(Z, X, Yx, k, U, tensor_cores=True):
    """U = Z + X Yx (Z may be None) for [n][ld] blocks; Yx float64 [k][ldy]."""
    fn = LIB.bmg_expand if X.dtype.itemsize == 8 else LIB.bmg_expand_f32
    _check(fn(_ptr(Z), _ptr(X), _ptr(Yx), X.shape[0], k, X.shape[1], Yx.shape[1], _ptr(U),
              int(bool(tensor_cores)), _stream()))


def gram_noalloc(X, Y, k, G):
    """G = X^T Y through bmg_gram_noalloc (no device allocation; see include/bmg.h)."""
    _check(LIB.bmg_gram_noalloc(_ptr(X), _ptr(Y), X.shape[0], k, X.shape[1], _ptr(G), _stream()))


def dense_eig(Ahat, Mhat, sigma, k, theta, Y, rank=None):
    _check(LIB.bmg_dense_eig(_ptr(Ahat), _ptr(Mhat), Ahat.shape[0], float(sigma), k, _ptr(theta),
                             _ptr(Y), _ptr(rank), _stream()))
