"""Python binding of the GB300 FETI library (``libfeti_gb300.so``).

Argument marshalling only: every function forwards to the C entry point of
the same name declared in ``include/feti.h``; all arithmetic runs in the
library's CUDA kernels.  There is no fallback: if the library is missing,
``lib()`` raises.

Device buffers are passed as torch CUDA tensors (their ``data_ptr()``),
host buffers as numpy arrays.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfeti_gb300.so")

(FETI_OK, FETI_EINVAL, FETI_ENOMEM, FETI_ESTATE, FETI_ENOTCONV, FETI_EBREAKDOWN, FETI_ECUDA, FETI_ENOTSUP,
 FETI_ETIMEOUT) = range(9)
FETI_TFETI, FETI_FETIDP = 0, 1
FETI_SCALING_K, FETI_SCALING_MULT = 0, 1
FETI_PCG, FETI_FO, FETI_RRS = 0, 1, 2
FETI_FP64, FETI_TF32, FETI_TF32X3, FETI_BF16, FETI_BF16X3 = 0, 1, 2, 3, 4
FETI_PRECOND_DIRICHLET, FETI_PRECOND_LUMPED, FETI_PRECOND_SUPERLUMPED = 0, 1, 2
FETI_PRIMAL_CORNERS, FETI_PRIMAL_EDGES, FETI_PRIMAL_ADAPTIVE = 0, 1, 2
FETI_REFINE_DUAL, FETI_REFINE_PRIMAL = 0, 1
(FETI_Q_N_LAMBDA, FETI_Q_N_SUBDOMAINS, FETI_Q_N_PRIMAL, FETI_Q_N_MODULES, FETI_Q_N_B_TOTAL, FETI_Q_N_DOFS,
 FETI_Q_N_ELEMENTS, FETI_Q_MAX_NB, FETI_Q_DEVICE_BYTES, FETI_Q_N_RBM, FETI_Q_LAUNCHES, FETI_Q_N_PROBLEMS,
 FETI_Q_GEMV_CONFIG, FETI_Q_TC_BYTES_F, FETI_Q_TC_BYTES_PER_COL, FETI_Q_APPLY1_BYTES,
 FETI_Q_BATCH_ROW_TILE) = range(17)

STATUS_NAMES = {0: "FETI_OK", 1: "FETI_EINVAL", 2: "FETI_ENOMEM", 3: "FETI_ESTATE", 4: "FETI_ENOTCONV",
                5: "FETI_EBREAKDOWN", 6: "FETI_ECUDA", 7: "FETI_ENOTSUP",
                8: "FETI_ETIMEOUT"}

EXPORTS = [
    "feti_options_default", "feti_create", "feti_set_allocator", "feti_setup_subdomains", "feti_setup_batch", "feti_problem_result",
    "feti_set_density", "feti_factorize",
    "feti_solve_dual", "feti_recover_displacements", "feti_compliance_grad", "feti_primal_residual", "feti_apply_dual",
    "feti_apply_precond", "feti_apply_precond_noalloc", "feti_test_skip_copy", "feti_query", "feti_profile_begin", "feti_profile_end", "feti_profile_tensor", "feti_profile_phases", "feti_lambda_layout", "feti_local_blocks", "feti_last_error",
    "feti_destroy",
]


class feti_options(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("scaling", ctypes.c_int), ("krylov", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("dedup_modules", ctypes.c_int),
                ("tol", ctypes.c_double), ("rr_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("precond", ctypes.c_int),
                ("primal", ctypes.c_int), ("primal_jump", ctypes.c_double), ("refine", ctypes.c_int)]


class feti_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("tiles", ctypes.c_int * 3), ("elems", ctypes.c_int * 3),
                ("E0", ctypes.c_double), ("Emin", ctypes.c_double), ("nu", ctypes.c_double),
                ("p", ctypes.c_double), ("rho", ctypes.c_void_p), ("dirichlet", ctypes.c_void_p),
                ("f", ctypes.c_void_p), ("on_device", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class feti_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class feti_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("f_applies", ctypes.c_int),
                ("last_rank", ctypes.c_int), ("eps0", ctypes.c_double), ("eps", ctypes.c_double),
                ("refinements", ctypes.c_int)]


_LIB = None


def lib():
    """Load the library (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2111_11728_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "feti_options_default": ([ctypes.POINTER(feti_options)], i),
            "feti_create": ([ctypes.POINTER(vp), ctypes.POINTER(feti_options), vp], i),
            "feti_set_allocator": ([vp, ctypes.POINTER(feti_allocator)], i),
            "feti_setup_subdomains": ([vp, ctypes.POINTER(feti_problem)], i),
            "feti_setup_batch": ([vp, ctypes.POINTER(feti_problem), i], i),
            "feti_problem_result": ([vp, i, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                     ctypes.POINTER(feti_stats), ctypes.POINTER(d)], i),
            "feti_set_density": ([vp, vp, i], i),
            "feti_factorize": ([vp], i),
            "feti_solve_dual": ([vp, vp, ctypes.POINTER(feti_stats)], i),
            "feti_recover_displacements": ([vp, vp, i, ctypes.POINTER(d)], i),
            "feti_compliance_grad": ([vp, vp, i], i),
            "feti_primal_residual": ([vp, vp, vp, ctypes.POINTER(d)], i),
            "feti_apply_dual": ([vp, vp, i, i, vp, i], i),
            "feti_apply_precond": ([vp, vp, vp, i, vp], i),
            "feti_apply_precond_noalloc": ([vp, vp, vp, i, vp], i),
            "feti_test_skip_copy": ([vp, i], i),
            "feti_query": ([vp, i, ctypes.POINTER(i64)], i),
            "feti_profile_begin": ([vp], i),
            "feti_profile_end": ([vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(i64)], i),
            "feti_profile_tensor": ([vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(i64)], i),
            "feti_profile_phases": ([vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(i64)], i),
            "feti_lambda_layout": ([vp, vp], i),
            "feti_local_blocks": ([vp, i, ctypes.POINTER(i), ctypes.POINTER(i), vp, vp, vp, vp, vp], i),
            "feti_last_error": ([vp], ctypes.c_char_p),
            "feti_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


class FetiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(type(x))


def _check(ctx, status, ok=(FETI_OK,)):
    if status not in ok:
        msg = lib().feti_last_error(ctx)
        raise FetiError(status, msg.decode() if msg else "")
    return status


def feti_options_default():
    o = feti_options()
    lib().feti_options_default(ctypes.byref(o))
    return o


def feti_create(opt=None, stream=None):
    ctx = ctypes.c_void_p()
    st = lib().feti_create(ctypes.byref(ctx), ctypes.byref(opt) if opt is not None else None,
                           ctypes.c_void_p(stream) if stream else None)
    if st != FETI_OK:
        raise FetiError(st, "feti_create failed")
    return ctx


def feti_destroy(ctx):
    lib().feti_destroy(ctx)


def feti_last_error(ctx):
    return lib().feti_last_error(ctx).decode()


def make_problem(dim, tiles, elems, E0, Emin, nu, p, rho, dirichlet, f, on_device):
    """feti_problem from arrays; the caller keeps rho/dirichlet/f alive during the call."""
    pr = feti_problem()
    pr.dim = dim
    for a in range(3):
        pr.tiles[a] = int(tiles[a]) if a < len(tiles) else 1
        pr.elems[a] = int(elems[a]) if a < len(elems) else 1
    pr.E0, pr.Emin, pr.nu, pr.p = float(E0), float(Emin), float(nu), float(p)
    pr.rho = _ptr(rho).value
    pr.dirichlet = _ptr(dirichlet).value
    pr.f = _ptr(f).value
    pr.on_device = int(on_device)
    return pr


class TorchAllocator:
    """A feti_allocator backed by PyTorch's caching allocator (device memory of
    the current CUDA device, on the stream the library passes).  Counts the
    allocations and the bytes still held, for tests.  Keep the object alive as
    long as any context that uses it."""

    def __init__(self):
        import torch
        self._torch = torch
        self.live = {}
        self.n_alloc = 0
        self.n_free = 0

        def _alloc(user, nbytes, stream):
            try:
                ptr = self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:            # out of memory: the library reports FETI_ENOMEM
                return None
            self.live[ptr] = int(nbytes)
            self.n_alloc += 1
            return ptr

        def _free(user, ptr, nbytes, stream):
            self._torch.cuda.caching_allocator_delete(ptr)
            self.live.pop(ptr, None)
            self.n_free += 1

        self._cb_alloc = ALLOC_FN(_alloc)
        self._cb_free = FREE_FN(_free)
        self.struct = feti_allocator(self._cb_alloc, self._cb_free, None)

    @property
    def bytes_held(self):
        return sum(self.live.values())


def feti_set_allocator(ctx, allocator):
    """allocator: a TorchAllocator (or any object with a feti_allocator ``struct``), or None."""
    ptr = ctypes.byref(allocator.struct) if allocator is not None else None
    _check(ctx, lib().feti_set_allocator(ctx, ptr))


def feti_setup_subdomains(ctx, problem):
    return _check(ctx, lib().feti_setup_subdomains(ctx, ctypes.byref(problem)))


def feti_setup_batch(ctx, problems):
    """problems: a list of feti_problem structures (see make_problem)."""
    arr = (feti_problem * len(problems))(*problems)
    return _check(ctx, lib().feti_setup_batch(ctx, arr, len(problems)))


def feti_problem_result(ctx, p):
    """Returns (dof_offset, elem_offset, lambda_offset, stats, compliance) of problem p."""
    a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    st = feti_stats()
    comp = ctypes.c_double(0.0)
    _check(ctx, lib().feti_problem_result(ctx, int(p), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(st), ctypes.byref(comp)))
    return a.value, b.value, c.value, st, comp.value


def feti_set_density(ctx, rho, on_device):
    return _check(ctx, lib().feti_set_density(ctx, _ptr(rho), int(on_device)))


def feti_factorize(ctx):
    return _check(ctx, lib().feti_factorize(ctx))


def feti_solve_dual(ctx, lambda_inout=None, allow_notconv=False):
    s = feti_stats()
    ok = (FETI_OK, FETI_ENOTCONV) if allow_notconv else (FETI_OK,)
    status = _check(ctx, lib().feti_solve_dual(ctx, _ptr(lambda_inout), ctypes.byref(s)), ok)
    return status, s


def feti_recover_displacements(ctx, u_out, on_device):
    c = ctypes.c_double(0.0)
    _check(ctx, lib().feti_recover_displacements(ctx, _ptr(u_out), int(on_device), ctypes.byref(c)))
    return c.value


def feti_primal_residual(ctx, u=None, r=None):
    """r = f - K u over the free DOFs (device tensors; u None: u = 0); returns
    ||r|| / ||f|| over the free DOFs."""
    rel = ctypes.c_double(0.0)
    _check(ctx, lib().feti_primal_residual(ctx, _ptr(u), _ptr(r), ctypes.byref(rel)))
    return rel.value


def feti_compliance_grad(ctx, out, on_device):
    return _check(ctx, lib().feti_compliance_grad(ctx, _ptr(out), int(on_device)))


def feti_apply_dual(ctx, X, ldx, m, Y, ldy):
    return _check(ctx, lib().feti_apply_dual(ctx, _ptr(X), int(ldx), int(m), _ptr(Y), int(ldy)))


def feti_apply_precond(ctx, r, Z, ldz, z):
    return _check(ctx, lib().feti_apply_precond(ctx, _ptr(r), _ptr(Z), int(ldz), _ptr(z)))


def feti_apply_precond_noalloc(ctx, r, Z, ldz, z):
    return _check(ctx, lib().feti_apply_precond_noalloc(ctx, _ptr(r), _ptr(Z), int(ldz), _ptr(z)))


def feti_test_skip_copy(ctx, chunk):
    _check(ctx, lib().feti_test_skip_copy(ctx, int(chunk)))


def feti_query(ctx, key):
    v = ctypes.c_int64(0)
    _check(ctx, lib().feti_query(ctx, int(key), ctypes.byref(v)))
    return v.value


def feti_profile_begin(ctx):
    return _check(ctx, lib().feti_profile_begin(ctx))


def feti_profile_end(ctx):
    """Returns (algorithmic flops, device ms, launches) of the profiled FP64 GEMMs."""
    f, t, n = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int64(0)
    _check(ctx, lib().feti_profile_end(ctx, ctypes.byref(f), ctypes.byref(t), ctypes.byref(n)))
    return f.value, t.value, n.value


PHASES = ("apply", "precond", "project", "gram", "step", "ortho", "factor", "recover")
(FETI_PHASE_APPLY, FETI_PHASE_PRECOND, FETI_PHASE_PROJECT, FETI_PHASE_GRAM, FETI_PHASE_STEP, FETI_PHASE_ORTHO,
 FETI_PHASE_FACTOR, FETI_PHASE_RECOVER) = range(8)
FETI_N_PHASES = len(PHASES)


def feti_profile_phases(ctx):
    """Per phase of the last profile: {name: (work, ms, regions)}; work is flops or bytes."""
    w = (ctypes.c_double * 8)()
    t = (ctypes.c_double * 8)()
    n = (ctypes.c_int64 * 8)()
    _check(ctx, lib().feti_profile_phases(ctx, w, t, n))
    return {PHASES[q]: (w[q], t[q], n[q]) for q in range(8)}


def feti_profile_tensor(ctx):
    """(flops, ms, launches) of the tensor-core products in the last completed profile."""
    f, t, n = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int64(0)
    _check(ctx, lib().feti_profile_tensor(ctx, ctypes.byref(f), ctypes.byref(t), ctypes.byref(n)))
    return f.value, t.value, n.value


def feti_lambda_layout(ctx):
    n = feti_query(ctx, FETI_Q_N_LAMBDA)
    out = np.zeros(6 * n, np.int32)
    _check(ctx, lib().feti_lambda_layout(ctx, _ptr(out)))
    return out.reshape(n, 6)


def feti_local_blocks(ctx, s):
    nb, nc = ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, lib().feti_local_blocks(ctx, int(s), ctypes.byref(nb), ctypes.byref(nc), None, None, None, None,
                                        None))
    b = np.zeros(nb.value, np.int32)
    c = np.zeros(max(nc.value, 1), np.int32)
    F = np.zeros((nb.value, nb.value))
    S = np.zeros((nb.value, nb.value))
    Frc = np.zeros((nb.value, max(nc.value, 1)))
    _check(ctx, lib().feti_local_blocks(ctx, int(s), ctypes.byref(nb), ctypes.byref(nc), _ptr(b), _ptr(c), _ptr(F),
                                        _ptr(S), _ptr(Frc)))
    return dict(bdofs=b, cdofs=c[:nc.value], F=F, S=S, Frc=Frc[:, :nc.value])


class Solver:
    """Convenience owner of one context: setup -> factorize -> solve -> recover.

    ``problem`` follows the ``workloads.Problem`` fields (dim, tiles, elems,
    E0, Emin, nu, p, rho, dirichlet, f).  ``device`` arrays are torch CUDA
    tensors; pass host numpy arrays with ``on_device=False``.
    """

    def __init__(self, method=FETI_FETIDP, scaling=FETI_SCALING_K, krylov=FETI_RRS, tol=1e-6, max_iter=500,
                 rr_tol=1e-10, dedup=True, stream=None, precision=FETI_FP64, inner_tol=None,
                 precond=FETI_PRECOND_DIRICHLET, primal=FETI_PRIMAL_CORNERS, allocator=None, primal_jump=None,
                 refine=FETI_REFINE_DUAL, max_refine=None):
        o = feti_options_default()
        o.method, o.scaling, o.krylov, o.precision = method, scaling, krylov, precision
        o.precond = precond
        o.primal = primal
        o.refine = refine
        if max_refine is not None:
            o.max_refine = max_refine
        if primal_jump is not None:
            o.primal_jump = primal_jump
        if inner_tol is not None:
            o.inner_tol = inner_tol
        o.tol, o.max_iter, o.rr_tol, o.dedup_modules = tol, max_iter, rr_tol, int(dedup)
        self.ctx = feti_create(o, stream)
        self.allocator = allocator
        if allocator is not None:
            feti_set_allocator(self.ctx, allocator)

    def setup(self, problem, rho=None, dirichlet=None, f=None, on_device=False):
        rho = problem.rho if rho is None else rho
        dirichlet = np.ascontiguousarray(problem.dirichlet, np.uint8) if dirichlet is None else dirichlet
        f = problem.f if f is None else f
        if not on_device:
            rho = np.ascontiguousarray(rho, np.float64)
            f = np.ascontiguousarray(f, np.float64)
        self._keep = (rho, dirichlet, f)
        pr = make_problem(problem.dim, problem.tiles, problem.elems, problem.E0, problem.Emin, problem.nu,
                          problem.p, rho, dirichlet, f, on_device)
        feti_setup_subdomains(self.ctx, pr)
        return self

    def query(self, key):
        return feti_query(self.ctx, key)

    def close(self):
        if self.ctx:
            feti_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
