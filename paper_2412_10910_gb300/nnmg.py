"""Thin Python binding of libnnmg (include/nnmg.h).

Functions carry the C names and only marshal arguments: device vectors are
torch CUDA tensors passed by data pointer together with torch's current CUDA
stream; host arrays are numpy arrays.  Every computation runs in the CUDA
library; if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi

_lib = _abi.load()

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "BAD_MESH", 3: "POINT_NOT_FOUND", 4: "CHOLESKY_FAIL",
          5: "OUT_OF_MEMORY", 6: "CUDA_ERROR", 7: "NOT_CONVERGED", 8: "BREAKDOWN"}


class NNMGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.nnmg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


def _check(status, where, allow=()):
    if status != 0 and status not in allow:
        raise NNMGError(status, where)
    return status


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype=None, numel=None, name="vector"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return C.c_void_p(t.data_ptr())


def _prec(t):
    import torch
    if t.dtype == torch.float64:
        return _abi.F64
    if t.dtype == torch.float32:
        return _abi.F32
    raise ValueError("vectors must be float32 or float64")


def nnmg_default_options():
    o = _abi.Options()
    _lib.nnmg_default_options(C.byref(o))
    return o


def _descs_and_options(levels, degree, n_components, lame, cheb_degree, smoothing_range,
                       lanczos_steps, eig_safety, max_nrhs, level_degrees, deterministic=False):
    keep = []
    descs = (_abi.LevelDesc * len(levels))()
    for i, lv in enumerate(levels):
        v = np.ascontiguousarray(lv.vertices, dtype=np.float64)
        c = np.ascontiguousarray(lv.cells, dtype=np.int32)
        dm = None if lv.dirichlet is None else np.ascontiguousarray(lv.dirichlet, dtype=np.uint8)
        keep += [v, c, dm]
        descs[i] = _abi.LevelDesc(int(lv.dim), v.shape[0], v.ctypes.data, c.shape[0], c.ctypes.data,
                                  None if dm is None else dm.ctypes.data,
                                  int(level_degrees[i]) if level_degrees else 0)
    o = nnmg_default_options()
    o.degree, o.n_components = int(degree), int(n_components)
    o.lam, o.mu = float(lame[0]), float(lame[1])
    o.cheb_degree, o.smoothing_range = int(cheb_degree), float(smoothing_range)
    o.lanczos_steps, o.eig_safety, o.max_nrhs = int(lanczos_steps), float(eig_safety), int(max_nrhs)
    o.deterministic = 1 if deterministic else 0
    return descs, o, keep


def nnmg_setup_hierarchy(levels, degree, n_components=1, lame=(1.0, 1.0), cheb_degree=3,
                         smoothing_range=20.0, lanczos_steps=12, eig_safety=1.2, max_nrhs=16,
                         stream=None, level_degrees=None, deterministic=False):
    """levels: sequence with .dim, .vertices [nv,dim] f64, .cells [nc,2^dim] i32, .dirichlet [nv] u8.

    level_degrees: optional per-level degrees (0 = `degree`), coarse -> fine.
    deterministic: bitwise reproducible results (cells stored grouped by color)."""
    descs, o, keep = _descs_and_options(levels, degree, n_components, lame, cheb_degree,
                                        smoothing_range, lanczos_steps, eig_safety, max_nrhs,
                                        level_degrees, deterministic)
    h = C.c_void_p()
    _check(_lib.nnmg_setup_hierarchy(descs, len(levels), C.byref(o), _stream(stream), C.byref(h)),
           "nnmg_setup_hierarchy")
    del keep
    return h


def nnmg_estimate_bytes(levels, degree, n_components=1, nrhs=16, level_degrees=None, **kw):
    """(hierarchy bytes, solve bytes for nrhs columns) before anything is built
    (host only: no CUDA call)."""
    opts = dict(lame=(1.0, 1.0), cheb_degree=3, smoothing_range=20.0, lanczos_steps=12,
                eig_safety=1.2, max_nrhs=16, deterministic=False)
    opts.update(kw)
    descs, o, keep = _descs_and_options(levels, degree, n_components, opts["lame"],
                                        opts["cheb_degree"], opts["smoothing_range"],
                                        opts["lanczos_steps"], opts["eig_safety"],
                                        opts["max_nrhs"], level_degrees, opts["deterministic"])
    hb, sb = C.c_size_t(), C.c_size_t()
    _check(_lib.nnmg_estimate_bytes(descs, len(levels), C.byref(o), int(nrhs), C.byref(hb),
                                    C.byref(sb)), "nnmg_estimate_bytes")
    del keep
    return hb.value, sb.value


def nnmg_color_cells(cells, n_vertices):
    """Greedy vertex-disjoint cell colors (host only): (color [n_cells] u8, n_colors)."""
    c = np.ascontiguousarray(cells, dtype=np.int32)
    dim = {4: 2, 8: 3}[c.shape[1]]
    color = np.zeros(c.shape[0], dtype=np.uint8)
    n = C.c_int()
    _check(_lib.nnmg_color_cells(c.ctypes.data, c.shape[0], int(n_vertices), dim, color.ctypes.data,
                                 C.byref(n)), "nnmg_color_cells")
    return color, n.value


def nnmg_level_colors(h, level):
    """First stored cell of every color and the cell count [n_colors + 1]
    (empty if the hierarchy was not built deterministic)."""
    n = C.c_int()
    _check(_lib.nnmg_level_colors(h, level, None, C.byref(n)), "nnmg_level_colors")
    if n.value == 0:
        return np.zeros(0, dtype=np.int64)
    out = np.zeros(n.value + 1, dtype=np.int64)
    _check(_lib.nnmg_level_colors(h, level, out.ctypes.data, C.byref(n)), "nnmg_level_colors")
    return out


def nnmg_destroy(h):
    _lib.nnmg_destroy(h)


def nnmg_n_levels(h):
    return _lib.nnmg_n_levels(h)


def nnmg_level_info(h, level):
    n, f, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.nnmg_level_info(h, level, C.byref(n), C.byref(f), C.byref(c)), "nnmg_level_info")
    return n.value, f.value, c.value


def nnmg_hierarchy_bytes(h):
    return _lib.nnmg_hierarchy_bytes(h)


def nnmg_solve_bytes(h, nrhs):
    return _lib.nnmg_solve_bytes(h, nrhs)


def nnmg_support_points(h, level, dim):
    n, _, _ = nnmg_level_info(h, level)
    out = np.empty((n, dim))
    _check(_lib.nnmg_support_points(h, level, out.ctypes.data), "nnmg_support_points")
    return out


def nnmg_constrained_nodes(h, level):
    n, _, _ = nnmg_level_info(h, level)
    out = np.empty(n, dtype=np.uint8)
    _check(_lib.nnmg_constrained_nodes(h, level, out.ctypes.data), "nnmg_constrained_nodes")
    return out


def nnmg_cell_nodes(h, level, nloc):
    _, _, nc = nnmg_level_info(h, level)
    out = np.empty((nc, nloc), dtype=np.int32)
    _check(_lib.nnmg_cell_nodes(h, level, out.ctypes.data), "nnmg_cell_nodes")
    return out


def nnmg_quadrature_points(h, level, nq, dim):
    _, _, nc = nnmg_level_info(h, level)
    out = np.empty((nc, nq, dim))
    _check(_lib.nnmg_quadrature_points(h, level, out.ctypes.data), "nnmg_quadrature_points")
    return out


def nnmg_transfer_points(h, fine_level, dim):
    _, nfree, _ = nnmg_level_info(h, fine_level)
    cell = np.empty(nfree, dtype=np.int32)
    xi = np.empty((nfree, dim))
    _check(_lib.nnmg_transfer_points(h, fine_level, cell.ctypes.data, xi.ctypes.data),
           "nnmg_transfer_points")
    return cell, xi


def nnmg_pcg_device_loop(h, mode, nrhs):
    out = C.c_int(0)
    _check(_lib.nnmg_pcg_device_loop(h, mode, nrhs, C.byref(out)), "nnmg_pcg_device_loop")
    return out.value


SETUP_PHASES = ("numbering", "level_geometry", "point_location", "gather_lists", "lanczos",
                "coarse_inverse")


def nnmg_setup_seconds(h):
    out = np.zeros(len(SETUP_PHASES))
    _check(_lib.nnmg_setup_seconds(h, out.ctypes.data), "nnmg_setup_seconds")
    return dict(zip(SETUP_PHASES, out.tolist()))


def nnmg_operator_choice(h, level, precision, nrhs):
    out = C.c_int(0)
    _check(_lib.nnmg_operator_choice(h, level, precision, nrhs, C.byref(out)), "nnmg_operator_choice")
    return out.value


def nnmg_eigen_estimates(h):
    out = np.empty(nnmg_n_levels(h))
    _check(_lib.nnmg_eigen_estimates(h, out.ctypes.data), "nnmg_eigen_estimates")
    return out


def nnmg_load_vector(h, level, f, f_per_qp, b, nrhs, col, stream=None, ncomp=1):
    import torch
    _need(h, level, b, nrhs, ncomp, "b")
    n, _, nc = nnmg_level_info(h, level)
    fa = np.ascontiguousarray(f, dtype=np.float64)
    if fa.size < ncomp or (f_per_qp and fa.size != nc * (fa.size // max(nc, 1))):
        raise ValueError("f has the wrong size")
    _check(_lib.nnmg_load_vector(h, level, fa.ctypes.data, int(f_per_qp),
                                 _dev(b, torch.float64, name="b"), nrhs, col, _stream(stream)),
           "nnmg_load_vector")


def _need(h, level, t, nrhs, ncomp, name):
    n = C.c_int64()
    _check(_lib.nnmg_level_info(h, level, C.byref(n), None, None), "nnmg_level_info")
    if t.numel() != n.value * ncomp * nrhs:
        raise ValueError(f"{name} must hold rows*nrhs = {n.value * ncomp * nrhs} values")


def nnmg_apply_operator(h, level, x, y, nrhs, stream=None, ncomp=1, double_word=False):
    """y = A_l x; double_word=True (FP64 vectors) computes in double-word arithmetic."""
    _need(h, level, x, nrhs, ncomp, "x")
    prec = _prec(x)
    if double_word:
        if prec != _abi.F64:
            raise ValueError("double-word operator takes float64 vectors")
        prec = _abi.F64_DW
    _check(_lib.nnmg_apply_operator(h, level, prec, _dev(x, name="x"),
                                    _dev(y, x.dtype, x.numel(), name="y"), nrhs, _stream(stream)),
           "nnmg_apply_operator")


def nnmg_prolongate(h, fine_level, coarse, fine, nrhs, stream=None, ncomp=1):
    _need(h, fine_level - 1, coarse, nrhs, ncomp, "coarse")
    _need(h, fine_level, fine, nrhs, ncomp, "fine")
    _check(_lib.nnmg_prolongate(h, fine_level, _prec(coarse), _dev(coarse, name="coarse"),
                                _dev(fine, coarse.dtype, name="fine"), nrhs, _stream(stream)),
           "nnmg_prolongate")


def nnmg_restrict(h, fine_level, fine, coarse, nrhs, stream=None, ncomp=1):
    _need(h, fine_level - 1, coarse, nrhs, ncomp, "coarse")
    _need(h, fine_level, fine, nrhs, ncomp, "fine")
    _check(_lib.nnmg_restrict(h, fine_level, _prec(fine), _dev(fine, name="fine"),
                              _dev(coarse, fine.dtype, name="coarse"), nrhs, _stream(stream)),
           "nnmg_restrict")


def nnmg_restrict_noalloc(h, fine_level, fine, coarse, nrhs, stream=None, ncomp=1):
    """coarse = P^T fine without any device allocation (scratch is a fixed
    array inside the library; see include/nnmg.h for its limit)."""
    _need(h, fine_level - 1, coarse, nrhs, ncomp, "coarse")
    _need(h, fine_level, fine, nrhs, ncomp, "fine")
    _check(_lib.nnmg_restrict_noalloc(h, fine_level, _prec(fine), _dev(fine, name="fine"),
                                      _dev(coarse, fine.dtype, name="coarse"), nrhs,
                                      _stream(stream)), "nnmg_restrict_noalloc")


def nnmg_set_nested(h, fine_level, parent_cell=None, child_index=None):
    """Use the nested (sum-factorized) transfer for this level pair; None to undo."""
    if parent_cell is None:
        _check(_lib.nnmg_set_nested(h, fine_level, None, None), "nnmg_set_nested")
        return
    p = np.ascontiguousarray(parent_cell, dtype=np.int32)
    c = np.ascontiguousarray(child_index, dtype=np.uint8)
    _check(_lib.nnmg_set_nested(h, fine_level, p.ctypes.data, c.ctypes.data), "nnmg_set_nested")


def nnmg_vcycle(h, r, z, nrhs, stream=None, ncomp=1):
    _need(h, nnmg_n_levels(h) - 1, r, nrhs, ncomp, "r")
    _check(_lib.nnmg_vcycle(h, _prec(r), _dev(r, name="r"), _dev(z, r.dtype, r.numel(), name="z"),
                            nrhs, _stream(stream)), "nnmg_vcycle")


def nnmg_vcycle_profile(h, r, z, nrhs, stream=None, ncomp=1):
    """One V-cycle as nnmg_vcycle, timed per level and component; returns
    (ms, launches), numpy arrays [n_levels][len(_abi.PROF_COLUMNS)]."""
    _need(h, nnmg_n_levels(h) - 1, r, nrhs, ncomp, "r")
    nl = nnmg_n_levels(h)
    ms = np.zeros((nl, len(_abi.PROF_COLUMNS)), dtype=np.float64)
    cnt = np.zeros((nl, len(_abi.PROF_COLUMNS)), dtype=np.int32)
    _check(_lib.nnmg_vcycle_profile(h, _prec(r), _dev(r, name="r"),
                                    _dev(z, r.dtype, r.numel(), name="z"), nrhs, _stream(stream),
                                    ms.ctypes.data, cnt.ctypes.data), "nnmg_vcycle_profile")
    return ms, cnt


def nnmg_pcg_solve(h, mode, b, x, nrhs, rtol=1e-8, maxit=200, stream=None, allow_fail=False,
                   ncomp=1):
    """Returns (status, iters[nrhs], relres[nrhs])."""
    import torch
    _need(h, nnmg_n_levels(h) - 1, b, nrhs, ncomp, "b")
    its = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs)
    st = _lib.nnmg_pcg_solve(h, mode, _dev(b, torch.float64, name="b"),
                             _dev(x, torch.float64, b.numel(), name="x"), nrhs, rtol, maxit,
                             its.ctypes.data, rel.ctypes.data, _stream(stream))
    _check(st, "nnmg_pcg_solve", allow=(7, 8) if allow_fail else ())
    return st, its, rel


def nnmg_pcg_solve_host(h, mode, b, x, nrhs, rtol=1e-8, maxit=200, stream=None, allow_fail=False,
                        ncomp=1):
    """b, x: host float64 arrays (numpy, or pinned torch CPU tensors) of rows*nrhs values."""
    def ptr(a):
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("host vectors must be C-contiguous float64")
            return a.ctypes.data
        if a.dtype.is_floating_point and a.element_size() == 8 and not a.is_cuda and a.is_contiguous():
            return a.data_ptr()
        raise ValueError("host vectors must be float64 numpy arrays or CPU tensors")
    n = C.c_int64()
    _check(_lib.nnmg_level_info(h, nnmg_n_levels(h) - 1, C.byref(n), None, None), "nnmg_level_info")
    size = b.size if isinstance(b, np.ndarray) else b.numel()
    xsize = x.size if isinstance(x, np.ndarray) else x.numel()
    if size != n.value * ncomp * nrhs or xsize != size:
        raise ValueError("b and x must hold rows*nrhs values")
    its = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs)
    st = _lib.nnmg_pcg_solve_host(h, mode, ptr(b), ptr(x), nrhs, rtol, maxit, its.ctypes.data,
                                  rel.ctypes.data, _stream(stream))
    _check(st, "nnmg_pcg_solve_host", allow=(7, 8) if allow_fail else ())
    return st, its, rel


def nnmg_pipe_rate(kind, iters=20000, stream=None):
    """Fused multiply-adds per second of the FP64 (kind 0), FP32 (1) or packed
    FP32 (2) pipe, from an FMA-chain kernel timed with CUDA events."""
    r = C.c_double()
    _check(_lib.nnmg_pipe_rate(int(kind), int(iters), _stream(stream), C.byref(r)), "nnmg_pipe_rate")
    return r.value


def nnmg_last_error():
    return _lib.nnmg_last_error().decode(errors="replace")


class Hierarchy:
    """Owner of one device hierarchy; methods forward to the functions above."""

    def __init__(self, levels, degree, n_components=1, lame=(1.0, 1.0), cheb_degree=3,
                 max_nrhs=16, level_degrees=None, **kw):
        self.dim = int(levels[0].dim)
        self.degree = int(degree)
        self.ncomp = int(n_components)
        self.degrees = [int(d) if d else int(degree) for d in (level_degrees or [0] * len(levels))]
        self.nloc = (degree + 1) ** self.dim
        self.h = nnmg_setup_hierarchy(levels, degree, n_components, lame, cheb_degree,
                                      max_nrhs=max_nrhs, level_degrees=level_degrees, **kw)
        self.n_levels = nnmg_n_levels(self.h)

    def close(self):
        if self.h:
            nnmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _nrhs(t):
        return t.shape[1] if t.dim() > 1 else 1

    def rows(self, level):
        return nnmg_level_info(self.h, level)[0] * self.ncomp

    def info(self, level):
        return nnmg_level_info(self.h, level)

    def vector(self, level, nrhs=1, dtype=None):
        import torch
        return torch.zeros(self.rows(level), nrhs, dtype=dtype or torch.float64, device="cuda")

    def support_points(self, level):
        return nnmg_support_points(self.h, level, self.dim)

    def constrained(self, level):
        return nnmg_constrained_nodes(self.h, level).astype(bool)

    def cell_nodes(self, level):
        return nnmg_cell_nodes(self.h, level, (self.degrees[level] + 1) ** self.dim)

    def quadrature_points(self, level):
        return nnmg_quadrature_points(self.h, level, (self.degrees[level] + 1) ** self.dim, self.dim)

    def transfer_points(self, fine_level):
        return nnmg_transfer_points(self.h, fine_level, self.dim)

    def eigen_estimates(self):
        return nnmg_eigen_estimates(self.h)

    def pcg_device_loop(self, mode, nrhs):
        """1: solves for (mode, nrhs) run as one device-side graph loop; 0: not
        built yet; -1: could not be built (host-driven loop)."""
        return nnmg_pcg_device_loop(self.h, mode, nrhs)

    def setup_seconds(self):
        """Wall seconds of the setup phases, by name."""
        return nnmg_setup_seconds(self.h)

    def operator_choice(self, level, precision, nrhs):
        """-1 register kernel, -2 paired FP32 register kernel, U > 0 shared-memory
        kernel with U units per block, -100 - U its paired FP32 form, 0 default
        rule / not chosen yet."""
        return nnmg_operator_choice(self.h, level, precision, nrhs)

    def load_vector(self, level, f, b, col=0, per_qp=False):
        nnmg_load_vector(self.h, level, f, per_qp, b, self._nrhs(b), col, ncomp=self.ncomp)

    def apply(self, level, x, y, double_word=False):
        nnmg_apply_operator(self.h, level, x, y, self._nrhs(x), ncomp=self.ncomp,
                            double_word=double_word)

    def prolongate(self, fine_level, xc, xf):
        nnmg_prolongate(self.h, fine_level, xc, xf, self._nrhs(xc), ncomp=self.ncomp)

    def restrict(self, fine_level, rf, rc):
        nnmg_restrict(self.h, fine_level, rf, rc, self._nrhs(rf), ncomp=self.ncomp)

    def set_nested(self, fine_level, parent_cell=None, child_index=None):
        nnmg_set_nested(self.h, fine_level, parent_cell, child_index)

    def vcycle(self, r, z):
        nnmg_vcycle(self.h, r, z, self._nrhs(r), ncomp=self.ncomp)

    def vcycle_profile(self, r, z):
        """(ms, launches) per level and component of one V-cycle (see
        _abi.PROF_COLUMNS)."""
        return nnmg_vcycle_profile(self.h, r, z, self._nrhs(r), ncomp=self.ncomp)

    def pcg(self, b, x, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=200, allow_fail=False):
        return nnmg_pcg_solve(self.h, mode, b, x, self._nrhs(b), rtol, maxit,
                              allow_fail=allow_fail, ncomp=self.ncomp)

    def pcg_host(self, b, x, nrhs, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=200,
                 allow_fail=False):
        return nnmg_pcg_solve_host(self.h, mode, b, x, nrhs, rtol, maxit, allow_fail=allow_fail,
                                   ncomp=self.ncomp)

    def hierarchy_bytes(self):
        return nnmg_hierarchy_bytes(self.h)

    def solve_bytes(self, nrhs):
        return nnmg_solve_bytes(self.h, nrhs)
