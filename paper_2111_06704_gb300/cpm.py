"""Thin ctypes binding of libcpm.so (include/cpm.h): argument marshalling only.

Arrays may be numpy arrays (host) or CUDA torch tensors (device, float64, contiguous);
the library stages host arrays itself.  Every compute step runs in the CUDA library;
there is no Python or CPU fallback, and loading fails loudly when the library is absent.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CPM_OK = 0
CPM_EINVAL = -1
CPM_ENOMEM = -2
CPM_ECUDA = -3
CPM_ENOCONV = -4
CPM_EBREAKDOWN = -5
CPM_ENOTBUILT = -7
CPM_EIO = -8
CPM_MLP_FEATURES = 32
CPM_MLP_PARAMS = 10497

CPM_PREC_FP64 = 0
CPM_PREC_FP32 = 1
CPM_PREC_BF16X6 = 2

CPM_PRECOND_NONE = 0
CPM_PRECOND_JACOBI = 1
CPM_PRECOND_DC = 2
CPM_PRECOND_NORMAL = 3
CPM_PRECOND_FULL = 4

CPM_E_STORED = 0
CPM_E_PAPER = 1

CPM_GCD_MAX_ELECTRODES = 16
CPM_SMATRIX_MAX_ATOMS = 8192

KE = 14.399645478  # V A / e

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class cpm_params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("g_ewald", ctypes.c_double),
        ("rcut_real", ctypes.c_double),
        ("kspace_eps", ctypes.c_double),
        ("slab", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("precond", ctypes.c_int),
        ("g_dc", ctypes.c_double),
        ("rcut_dc", ctypes.c_double),
        ("p_gap", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("stream_operand", ctypes.c_int),
        ("k_window", ctypes.c_int),
        ("matvec_mode", ctypes.c_int),
        ("solver_path", ctypes.c_int),
    ]


class cpm_info_t(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("m", ctypes.c_int),
        ("nnz_p", ctypes.c_int64),
        ("p_gap", ctypes.c_double),
        ("c_ele", ctypes.c_double),
        ("t_kspace_ms", ctypes.c_double),
        ("t_phase_ms", ctypes.c_double),
        ("t_precond_ms", ctypes.c_double),
        ("t_dsolve_ms", ctypes.c_double),
        ("d_iters", ctypes.c_int),
        ("launches", ctypes.c_int64),
        ("t_tc_ms", ctypes.c_double),
        ("head_cols", ctypes.c_int),
        ("t_matvec_ms", ctypes.c_double),
        ("tc_blocks", ctypes.c_int * 3),
        ("t_head_ms", ctypes.c_double),
        ("t_tc_light_ms", ctypes.c_double),
        ("tc_blocks_fp8", ctypes.c_int),
        ("t_tc_loop_ms", ctypes.c_double),
        ("t_solve_ms", ctypes.c_double),
        ("t_solve_matvec_ms", ctypes.c_double),
        ("t_solve_replace_ms", ctypes.c_double),
        ("solve_replacements", ctypes.c_int),
        ("t_pot_sf_ms", ctypes.c_double),
        ("t_pot_kspace_ms", ctypes.c_double),
        ("t_pot_real_ms", ctypes.c_double),
        ("solve_path", ctypes.c_int),
        ("t_solve_dc_ms", ctypes.c_double),
    ]


class cpm_kspace_plan(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int),
        ("m_pad", ctypes.c_int),
        ("head_cols", ctypes.c_int),
        ("kb_begin", ctypes.c_int),
        ("kb6_end", ctypes.c_int),
        ("kb3_end", ctypes.c_int),
        ("kb8_begin", ctypes.c_int),
        ("kb_end", ctypes.c_int),
        ("chunks", ctypes.c_int),
    ]


EXPORTS = ["cpm_default_params", "cpm_create", "cpm_destroy", "cpm_build_E", "cpm_potential",
           "cpm_solve", "cpm_solve_static", "cpm_neutralize", "cpm_get_E", "cpm_get_info",
           "cpm_get_d", "cpm_guess_features", "cpm_mlp_forward", "cpm_mlp_grad",
           "cpm_mlp_adam", "cpm_guess_apply", "cpm_apply_E", "cpm_get_precond",
           "cpm_last_error", "cpm_batch_create", "cpm_batch_destroy", "cpm_batch_solve",
           "cpm_batch_neutralize", "cpm_batch_last_error", "cpm_get_E_rows",
           "cpm_guess", "cpm_release_workspace", "cpm_plan_kspace", "cpm_gcd_setup",
           "cpm_gcd_charges", "cpm_smatrix_build", "cpm_smatrix_charges",
           "cpm_build_E_copy", "cpm_guess_init", "cpm_guess_norm", "cpm_guess_save",
           "cpm_guess_load", "cpm_ion_forces", "cpm_guess_train_step"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libcpm.so (building it first when asked and it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libcpm.so is not built ({path})")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, d, i, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    lib.cpm_default_params.argtypes = [P(cpm_params)]
    lib.cpm_default_params.restype = None
    lib.cpm_create.argtypes = [P(vp), P(cpm_params)]
    lib.cpm_destroy.argtypes = [vp]
    lib.cpm_release_workspace.argtypes = [vp]
    lib.cpm_build_E.argtypes = [vp, i, vp, vp]
    lib.cpm_build_E_copy.argtypes = [vp, vp]
    lib.cpm_ion_forces.argtypes = [vp, i, i, vp, vp, vp, vp]
    lib.cpm_guess_init.argtypes = [vp, ctypes.c_uint64, vp]
    lib.cpm_guess_norm.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.cpm_guess_save.argtypes = [ctypes.c_char_p, vp, vp, ctypes.c_float]
    lib.cpm_guess_load.argtypes = [ctypes.c_char_p, vp, vp, vp]
    lib.cpm_potential.argtypes = [vp, i, i, vp, vp, vp, vp, vp]
    lib.cpm_solve.argtypes = [vp, i, vp, vp, i, d, i, vp, vp]
    lib.cpm_solve_static.argtypes = [vp, i, vp, vp, i, d, i, vp, vp]
    lib.cpm_neutralize.argtypes = [vp, i, vp, vp]
    lib.cpm_get_E.argtypes = [vp, i, vp, i64]
    lib.cpm_get_E_rows.argtypes = [vp, i, i, vp, vp, i64]
    lib.cpm_get_info.argtypes = [vp, P(cpm_info_t)]
    lib.cpm_get_d.argtypes = [vp, vp]
    lib.cpm_get_precond.argtypes = [vp, vp, vp, vp]
    lib.cpm_batch_create.argtypes = [P(vp), i, P(vp)]
    lib.cpm_batch_destroy.argtypes = [vp]
    lib.cpm_batch_solve.argtypes = [vp, vp, vp, i, d, i, vp, vp]
    lib.cpm_batch_neutralize.argtypes = [vp, vp, vp]
    lib.cpm_batch_last_error.argtypes = [vp]
    lib.cpm_batch_last_error.restype = ctypes.c_char_p
    lib.cpm_guess_features.argtypes = [vp, i, vp, vp, vp, vp]
    lib.cpm_mlp_forward.argtypes = [vp, vp, vp, i, i64, vp, vp]
    lib.cpm_mlp_grad.argtypes = [vp, vp, vp, i, i64, vp, vp, vp, vp]
    lib.cpm_mlp_adam.argtypes = [vp, vp, vp, vp, vp, i, ctypes.c_float]
    lib.cpm_guess_train_step.argtypes = [vp, vp, vp, i, i64, vp, vp, vp, vp, vp, vp, i,
                                         ctypes.c_float, vp]
    lib.cpm_guess_apply.argtypes = [vp, i64, vp, ctypes.c_float, vp, vp]
    lib.cpm_guess.argtypes = [vp, vp, vp, i, i, vp, vp, vp, ctypes.c_float, vp, vp]
    lib.cpm_apply_E.argtypes = [vp, i, vp, vp]
    lib.cpm_plan_kspace.argtypes = [P(cpm_params), P(cpm_kspace_plan), vp, vp, vp, vp]
    lib.cpm_gcd_setup.argtypes = [vp, i, vp, d, i, vp, vp, vp]
    lib.cpm_gcd_charges.argtypes = [vp, i, vp, vp, vp, vp]
    lib.cpm_smatrix_build.argtypes = [vp, d, i, vp]
    lib.cpm_smatrix_charges.argtypes = [vp, i, vp, vp, vp]
    lib.cpm_last_error.argtypes = [vp]
    lib.cpm_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("cpm_default_params", "cpm_last_error", "cpm_batch_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class CpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cpm status {status}: {msg}")
        self.status = status


def _ptr(a):
    """(pointer, keep-alive) for a numpy array or a CUDA torch tensor (float64/int)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a.ctypes.data_as(ctypes.c_void_p), a
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensors passed to libcpm must be contiguous")
    return ctypes.c_void_p(a.data_ptr()), a


def default_params(box, **kw) -> cpm_params:
    lib = load()
    p = cpm_params()
    lib.cpm_default_params(ctypes.byref(p))
    p.box[0], p.box[1], p.box[2] = (float(x) for x in box)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def cpm_plan_kspace(box, **params) -> dict:
    """The host plan of the k-space sum for these parameters (no GPU needed): the plan's
    sizes and region bounds, and the arrays hkl [m, 3], w [m], kexp [kb_end] and
    chunk_end [kb_end] (bool)."""
    lib = load()
    p = default_params(box, **params)
    plan = cpm_kspace_plan()
    st = lib.cpm_plan_kspace(ctypes.byref(p), ctypes.byref(plan), None, None, None, None)
    if st != CPM_OK:
        raise CpmError(st, "cpm_plan_kspace: invalid parameters")
    hkl = np.zeros((plan.m, 3), dtype=np.int32)
    w = np.zeros(plan.m, dtype=np.float64)
    kexp = np.zeros(plan.kb_end, dtype=np.int32)
    chunk_end = np.zeros(plan.kb_end, dtype=np.uint8)
    vp = ctypes.c_void_p
    st = lib.cpm_plan_kspace(ctypes.byref(p), ctypes.byref(plan), hkl.ctypes.data_as(vp),
                             w.ctypes.data_as(vp), kexp.ctypes.data_as(vp),
                             chunk_end.ctypes.data_as(vp))
    if st != CPM_OK:
        raise CpmError(st, "cpm_plan_kspace failed")
    out = {name: getattr(plan, name) for name, _ in cpm_kspace_plan._fields_}
    out.update(hkl=hkl, w=w, kexp=kexp, chunk_end=chunk_end.astype(bool))
    return out


class Context:
    """One libcpm context (one electrode geometry, one CUDA device and stream)."""

    def __init__(self, box, stream=None, torch_allocator: bool = False, allocator=None,
                 **params):
        """allocator: optional (alloc(nbytes) -> device address or None, free(address))
        pair of Python callables behind the library's allocator callback."""
        self.lib = load()
        self.params = default_params(box, **params)
        if stream is not None:
            self.params.stream = ctypes.c_void_p(int(stream))
        self._cb = None
        if allocator is not None:
            alloc_py, free_py = allocator
            self._cb = (ALLOC_FN(lambda nbytes, _user: alloc_py(int(nbytes))),
                        FREE_FN(lambda ptr, _user: free_py(ptr)))
            self.params.alloc, self.params.free = self._cb
        elif torch_allocator:
            import torch
            dev = torch.cuda.current_device()

            def _alloc(nbytes, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:  # noqa: BLE001 - reported to C as NULL
                    return None

            def _free(ptr, _user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            self.params.alloc, self.params.free = self._cb
        h = ctypes.c_void_p()
        self._check(self.lib.cpm_create(ctypes.byref(h), ctypes.byref(self.params)), None)
        self.h = h
        self.n = 0
        self.gcd_m = 0

    def _check(self, st, h=-1):
        if st != CPM_OK:
            hh = self.h if h == -1 else h
            msg = self.lib.cpm_last_error(hh).decode() if hh else "create failed"
            raise CpmError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.cpm_destroy(self.h)
            self.h = None

    def cpm_release_workspace(self):
        """Frees the kept build, solve and potential workspaces (E, P, d and A stay)."""
        self._check(self.lib.cpm_release_workspace(self.h))

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # -- the four calls of the boundary ---------------------------------------------
    def cpm_build_E(self, xyz, alpha):
        n = int(xyz.shape[0])
        px, kx = _ptr(xyz)
        pa, ka = _ptr(alpha)
        self._check(self.lib.cpm_build_E(self.h, n, px, pa))
        self.n = n
        self.gcd_m = 0  # a rebuild drops the electrodes' solves

    def cpm_build_E_copy(self, src: "Context"):
        """This context takes src's built E (in this context's storage precision), d and
        diagonal, and its PCG-DC preconditioner when this context selects PCG-DC: the
        solve-side build, with no k-space tables (no cpm_potential here)."""
        self._check(self.lib.cpm_build_E_copy(self.h, src.h))
        self.n = src.n
        self.gcd_m = 0

    def cpm_potential(self, ion_xyz, ion_q, chi, b_out=None, qsol_out=None):
        frames, n_ion = int(ion_q.shape[0]), int(ion_q.shape[1])
        if b_out is None:
            b_out = np.empty((frames, self.n))
        if qsol_out is None and isinstance(b_out, np.ndarray):
            qsol_out = np.empty(frames)
        p1, k1 = _ptr(ion_xyz)
        p2, k2 = _ptr(ion_q)
        p3, k3 = _ptr(chi)
        p4, k4 = _ptr(b_out)
        p5, k5 = _ptr(qsol_out)
        self._check(self.lib.cpm_potential(self.h, frames, n_ion, p1, p2, p3, p4, p5))
        if isinstance(b_out, np.ndarray) and k4 is not b_out:
            b_out[...] = k4
        if isinstance(qsol_out, np.ndarray) and k5 is not qsol_out:
            qsol_out[...] = k5
        return b_out, qsol_out

    def cpm_ion_forces(self, ion_xyz, ion_q, q, f_out=None):
        """Forces on the ions from the electrode charges q [frames, n] (e^2/A^2)."""
        frames, n_ion = int(ion_q.shape[0]), int(ion_q.shape[1])
        if f_out is None:
            f_out = np.empty((frames, n_ion, 3))
        p1, k1 = _ptr(ion_xyz)
        p2, k2 = _ptr(ion_q)
        p3, k3 = _ptr(q)
        p4, k4 = _ptr(f_out)
        self._check(self.lib.cpm_ion_forces(self.h, frames, n_ion, p1, p2, p3, p4))
        if isinstance(f_out, np.ndarray) and k4 is not f_out:
            f_out[...] = k4
        return f_out

    def cpm_solve(self, b, q=None, use_guess=False, tol=1e-6, maxit=1000, allow_noconv=False):
        nrhs = int(b.shape[0]) if b.ndim == 2 else 1
        if q is None:
            q = np.zeros((nrhs, self.n))
        pb, kb = _ptr(b)
        pq, kq = _ptr(q)
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs)
        st = self.lib.cpm_solve(self.h, nrhs, pb, pq, 1 if use_guess else 0, float(tol),
                                int(maxit), iters.ctypes.data_as(ctypes.c_void_p),
                                rel.ctypes.data_as(ctypes.c_void_p))
        if not (st == CPM_ENOCONV and allow_noconv):
            self._check(st)
        if isinstance(q, np.ndarray) and kq is not q:
            q[...] = kq
        return q, iters, rel

    def cpm_solve_static(self, b, q, use_guess=False, tol=1e-6, maxit=1000):
        """cpm_solve on the library's fixed device workspace: no allocation.  b and q
        must be CUDA tensors (device pointers); returns (iterations, relative residual)."""
        nrhs = int(b.shape[0]) if b.ndim == 2 else 1
        pb, kb = _ptr(b)
        pq, kq = _ptr(q)
        iters = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs)
        self._check(self.lib.cpm_solve_static(self.h, nrhs, pb, pq, 1 if use_guess else 0,
                                              float(tol), int(maxit),
                                              iters.ctypes.data_as(ctypes.c_void_p),
                                              rel.ctypes.data_as(ctypes.c_void_p)))
        return iters, rel

    def cpm_neutralize(self, q, qsol=None):
        nrhs = int(q.shape[0]) if q.ndim == 2 else 1
        pq, kq = _ptr(q)
        ps, ks = _ptr(qsol)
        self._check(self.lib.cpm_neutralize(self.h, nrhs, pq, ps))
        if isinstance(q, np.ndarray) and kq is not q:
            q[...] = kq
        return q

    # -- fixed charge per electrode (GCD, Eq. S14-S24) ------------------------------
    def cpm_gcd_setup(self, labels, m=None, tol=1e-10, maxit=2000):
        """Splits the electrode into electrodes by labels [n] (0 .. m-1) and prepares
        their capacitance coefficients.  Returns (C [m, m] in e/V of the stored form,
        iterations [m], relative residuals [m])."""
        if hasattr(labels, "is_cuda") and labels.is_cuda:
            lab, plab = labels, ctypes.c_void_p(labels.data_ptr())
            if m is None:
                m = int(labels.max().item()) + 1
        else:
            lab = np.ascontiguousarray(labels, dtype=np.int32)
            plab = lab.ctypes.data_as(ctypes.c_void_p)
            if m is None:
                m = int(lab.max()) + 1
        c = np.zeros((m, m))
        iters = np.zeros(m, dtype=np.int32)
        rel = np.zeros(m)
        self._check(self.lib.cpm_gcd_setup(self.h, int(m), plab, float(tol), int(maxit),
                                           c.ctypes.data_as(ctypes.c_void_p),
                                           iters.ctypes.data_as(ctypes.c_void_p),
                                           rel.ctypes.data_as(ctypes.c_void_p)))
        self.gcd_m = m
        return c, iters, rel

    def cpm_gcd_charges(self, q, q0, qsol=None):
        """q holds q^b [nrhs, n] (cpm_solve); on return the charges with the totals
        q0 [nrhs, m] on the electrodes.  Returns (q, Delta mu [nrhs, m] in V)."""
        nrhs = int(q.shape[0]) if q.ndim == 2 else 1
        pq, kq = _ptr(q)
        p0, k0 = _ptr(q0)
        ps, ks = _ptr(qsol)
        dmu = np.zeros((nrhs, self.gcd_m))
        self._check(self.lib.cpm_gcd_charges(self.h, nrhs, pq, p0, ps,
                                             dmu.ctypes.data_as(ctypes.c_void_p)))
        if isinstance(q, np.ndarray) and kq is not q:
            q[...] = kq
        return q, dmu

    # -- the matrix path (Eq. 33 with Eq. 35) ----------------------------------------
    def cpm_smatrix_build(self, tol=1e-12, maxit=2000):
        """Forms S = E^-1 (I - 1 d^T) once; returns the most PCG iterations a column took."""
        it = ctypes.c_int(0)
        self._check(self.lib.cpm_smatrix_build(self.h, float(tol), int(maxit), ctypes.byref(it)))
        return it.value

    def cpm_smatrix_charges(self, b, qsol=None, q_out=None):
        """Neutral charges q = S b - Q^sol d for b [frames, n] in volts."""
        frames = int(b.shape[0]) if b.ndim == 2 else 1
        if q_out is None:
            q_out = np.empty((frames, self.n))
        pb, kb = _ptr(b)
        ps, ks = _ptr(qsol)
        pq, kq = _ptr(q_out)
        self._check(self.lib.cpm_smatrix_charges(self.h, frames, pb, ps, pq))
        if isinstance(q_out, np.ndarray) and kq is not q_out:
            q_out[...] = kq
        return q_out

    # -- inspection -----------------------------------------------------------------
    def cpm_get_E(self, form=CPM_E_STORED):
        out = np.empty((self.n, self.n))
        self._check(self.lib.cpm_get_E(self.h, int(form), out.ctypes.data_as(ctypes.c_void_p),
                                       self.n))
        return out

    def cpm_get_E_rows(self, rows, form=CPM_E_STORED):
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((len(rows), self.n))
        self._check(self.lib.cpm_get_E_rows(self.h, int(form), len(rows),
                                            rows.ctypes.data_as(ctypes.c_void_p),
                                            out.ctypes.data_as(ctypes.c_void_p), self.n))
        return out

    def cpm_apply_E(self, p, q=None):
        """q = E_n p (stored neutral-equivalent form) through the solver's matvec."""
        nrhs = int(p.shape[0]) if p.ndim == 2 else 1
        if q is None:
            q = np.empty((nrhs, self.n))
        pp, kp = _ptr(p)
        pq, kq = _ptr(q)
        self._check(self.lib.cpm_apply_E(self.h, nrhs, pp, pq))
        if isinstance(q, np.ndarray) and kq is not q:
            q[...] = kq
        return q

    def cpm_get_d(self):
        out = np.empty(self.n)
        self._check(self.lib.cpm_get_d(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def cpm_get_precond(self):
        """PCG-DC P in row form (Eq. 36): (off int64[n+1], idx int32[nnz], val f64[nnz])."""
        nnz = int(self.cpm_get_info()["nnz_p"])
        off = np.empty(self.n + 1, dtype=np.int64)
        idx = np.empty(max(nnz, 1), dtype=np.int32)
        val = np.empty(max(nnz, 1))
        vp = ctypes.c_void_p
        self._check(self.lib.cpm_get_precond(self.h, off.ctypes.data_as(vp),
                                             idx.ctypes.data_as(vp), val.ctypes.data_as(vp)))
        return off, idx[:nnz], val[:nnz]

    def cpm_get_info(self) -> dict:
        info = cpm_info_t()
        self._check(self.lib.cpm_get_info(self.h, ctypes.byref(info)))
        return {k: getattr(info, k) for k, _ in cpm_info_t._fields_}


class Batch:
    """A ragged batch over built contexts (cpm_batch_*): one PCG over all systems.
    Vectors are the systems' vectors concatenated in batch order."""

    def __init__(self, contexts):
        self.lib = load()
        self.contexts = list(contexts)  # kept alive: the batch refers to their builds
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = ctypes.c_void_p()
        st = self.lib.cpm_batch_create(ctypes.byref(h), len(self.contexts), arr)
        if st != CPM_OK:
            raise CpmError(st, "cpm_batch_create failed")
        self.h = h
        self.sizes = [c.n for c in self.contexts]

    def _check(self, st):
        if st != CPM_OK:
            raise CpmError(st, self.lib.cpm_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.cpm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def solve(self, b, q=None, use_guess=False, tol=1e-6, maxit=1000):
        count = len(self.contexts)
        if q is None:
            q = np.zeros(sum(self.sizes))
        pb, kb = _ptr(b)
        pq, kq = _ptr(q)
        iters = np.zeros(count, dtype=np.int32)
        rel = np.zeros(count)
        self._check(self.lib.cpm_batch_solve(self.h, pb, pq, 1 if use_guess else 0, float(tol),
                                             int(maxit), iters.ctypes.data_as(ctypes.c_void_p),
                                             rel.ctypes.data_as(ctypes.c_void_p)))
        if isinstance(q, np.ndarray) and kq is not q:
            q[...] = kq
        return q, iters, rel

    def neutralize(self, q, qsol=None):
        pq, kq = _ptr(q)
        ps, ks = _ptr(qsol)
        self._check(self.lib.cpm_batch_neutralize(self.h, pq, ps))
        if isinstance(q, np.ndarray) and kq is not q:
            q[...] = kq
        return q


def charges(ctx: Context, ion_xyz, ion_q, chi, tol=1e-6, maxit=1000, q0=None):
    """One charge solve per frame through the boundary: b, q^b, neutral q (Eq. 25, 35)."""
    b, qsol = ctx.cpm_potential(ion_xyz, ion_q, chi)
    q, iters, rel = ctx.cpm_solve(b, q0, use_guess=q0 is not None, tol=tol, maxit=maxit)
    ctx.cpm_neutralize(q, qsol)
    return q, iters, rel, b, qsol


__all__ = ["Context", "CpmError", "load", "charges", "EXPORTS", "KE"] + [
    n for n in dir() if n.startswith("CPM_")]
