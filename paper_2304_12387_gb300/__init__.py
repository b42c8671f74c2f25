"""Python binding of libhdivsp (matrix-free H(div) saddle-point operators on GB300).

A thin ctypes layer over the C ABI declared in include/hdivsp.h: every hd_*
function of the header is exported here under the same name and only marshals
arguments (device vectors are torch CUDA tensors passed by data pointer; the
handle runs on torch's current stream). All arithmetic happens in the CUDA
library; there is no fallback path. Building: ``python -m
paper_2304_12387_gb300.build`` (or ``__graft_entry__.build()``).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhdivsp.so")

HD_OK, HD_ERR_INVALID_ARG, HD_ERR_CUDA, HD_ERR_OOM, HD_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
HD_ERR_PREC_INDEFINITE, HD_ERR_NAN, HD_ERR_STAGNATION, HD_ERR_BOUNDS, HD_ERR_NOT_IMPLEMENTED = 5, 6, 7, 8, 9
HD_GRAD_DIV, HD_DARCY = 0, 1
HD_WINV_DENSE, HD_WINV_CG, HD_WINV_CG_HIST, HD_WINV_CHOL = 0, 1, 2, 3
HD_GMRES_BLOCK_DIAG, HD_GMRES_BLOCK_TRI = 0, 1
STATUS_NAMES = {0: "HD_OK", 1: "HD_ERR_INVALID_ARG", 2: "HD_ERR_CUDA", 3: "HD_ERR_OOM",
                4: "HD_ERR_NOT_CONVERGED", 5: "HD_ERR_PREC_INDEFINITE", 6: "HD_ERR_NAN",
                7: "HD_ERR_STAGNATION", 8: "HD_ERR_BOUNDS", 9: "HD_ERR_NOT_IMPLEMENTED"}


class HdError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__("%s%s" % (STATUS_NAMES.get(status, status), (": " + msg) if msg else ""))
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("k", ctypes.c_int32), ("q", ctypes.c_int32),
                ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
                ("vz", ctypes.POINTER(ctypes.c_double)), ("coef0", ctypes.POINTER(ctypes.c_double)),
                ("coef1", ctypes.POINTER(ctypes.c_double)), ("ess_mask", ctypes.c_uint32),
                ("affine", ctypes.c_int32), ("tau", ctypes.c_double), ("winv_mode", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("coarse_max", ctypes.c_int32), ("cycle", ctypes.c_int32),
                ("fp64_emulation", ctypes.c_int32), ("smooth_levels", ctypes.c_int32),
                ("w_levels", ctypes.c_int32), ("elem_rotation", ctypes.POINTER(ctypes.c_int8)),
                ("aggregation", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int32), ("use_x0", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("outer_rtol", ctypes.c_double), ("max_outer", ctypes.c_int32), ("resume", ctypes.c_int32)]


class GmresOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("use_x0", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("inner_rtol", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("eta_ratio", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("ms_total", ctypes.c_double), ("status", ctypes.c_int32),
                ("fallback", ctypes.c_int32)]


class MassInvDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("k", ctypes.c_int32),
                ("q", ctypes.c_int32), ("vx", ctypes.POINTER(ctypes.c_double)),
                ("vy", ctypes.POINTER(ctypes.c_double)), ("vz", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("method", ctypes.c_int32),
                ("fp64_emulation", ctypes.c_int32)]


class RadDesc(ctypes.Structure):
    _fields_ = [("mesh", ProblemDesc), ("sigma", ctypes.POINTER(ctypes.c_double)), ("rho", ctypes.c_double),
                ("cv", ctypes.c_double), ("a", ctypes.c_double), ("c", ctypes.c_double), ("dt", ctypes.c_double),
                ("outer_rtol", ctypes.c_double), ("outer_maxit", ctypes.c_int32), ("newton_rtol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int32), ("linear_rtol", ctypes.c_double),
                ("linear_maxit", ctypes.c_int32), ("linear_precision", ctypes.c_int32)]


class RadInfo(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int32), ("outer", ctypes.c_int32), ("outer_max", ctypes.c_int32),
                ("newton_max", ctypes.c_int32), ("linear_solves", ctypes.c_int32),
                ("linear_iterations", ctypes.c_int32), ("relres", ctypes.c_double), ("ms_newton", ctypes.c_double),
                ("ms_linear", ctypes.c_double), ("ms_residual", ctypes.c_double), ("status", ctypes.c_int32)]


class Slab(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("P", ctypes.c_int32), ("ez0", ctypes.c_int32), ("ez1", ctypes.c_int32),
                ("xf", ctypes.c_int64 * 2), ("yf", ctypes.c_int64 * 2), ("zf", ctypes.c_int64 * 2),
                ("cell", ctypes.c_int64 * 2), ("halo", ctypes.c_int64 * 2)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("npairs", ctypes.c_int32), ("capture_every", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("lr", ctypes.c_double), ("seed", ctypes.c_uint64)]


class TrainInfo(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int32), ("loss_initial", ctypes.c_double), ("loss_final", ctypes.c_double),
                ("pcg_max_iterations", ctypes.c_int32), ("ms_total", ctypes.c_double)]


_lib = None

_VP, _H = ctypes.c_void_p, ctypes.c_void_p
_SIGS = {
    "hd_create": [ctypes.POINTER(ProblemDesc), ctypes.POINTER(ctypes.c_void_p)],
    "hd_destroy": [_H],
    "hd_set_stream": [_H, _VP],
    "hd_get_sizes": [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                     ctypes.POINTER(ctypes.c_int64)],
    "hd_get_setup_times": [_H, ctypes.POINTER(ctypes.c_double), ctypes.c_int32],
    "hd_get_e2d_map": [_H, _VP],
    "hd_get_ess_dofs": [_H, _VP, ctypes.POINTER(ctypes.c_int64)],
    "hd_lattice_e2d_map": [ctypes.c_int32] * 4 + [_VP],
    "hd_lattice_e2d_map_rot": [ctypes.c_int32] * 4 + [_VP, _VP],
    "hd_lattice_e2l_map": [ctypes.c_int32] * 4 + [_VP, _VP],
    "hd_get_e2l_map": [_H, _VP],
    "hd_lattice_is_affine": [ctypes.c_int32] * 3 + [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_int32)],
    "hd_lattice_ess_dofs": [ctypes.c_int32] * 4 + [ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_int64)],
    "hd_apply_A": [_H, _VP, _VP],
    "hd_apply_B": [_H, _VP, _VP],
    "hd_apply_Bt": [_H, _VP, _VP],
    "hd_apply_C": [_H, _VP, _VP],
    "hd_apply_op": [_H, _VP, _VP],
    "hd_apply_op_host": [_H, _VP, _VP],
    "hd_apply_prec": [_H, _VP, _VP],
    "hd_apply_schur": [_H, _VP, _VP],
    "hd_vcycle": [_H, _VP, _VP],
    "hd_get_diagonals": [_H, _VP, _VP],
    "hd_get_level": [_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "hd_minres_solve": [_H, _VP, _VP, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)],
    "hd_gmres_solve": [_H, _VP, _VP, ctypes.POINTER(GmresOpts), ctypes.POINTER(SolveInfo)],
    "hd_minres_solve_noalloc": [_H, _VP, _VP, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)],
    "hd_profile": [_H, ctypes.c_int32],
    "hd_profile_read": [_H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)],
    "hd_learned_init": [_H, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double],
    "hd_learned_set_weights": [_H, _VP, _VP],
    "hd_learned_get_weights": [_H, _VP, _VP],
    "hd_learned_apply": [_H, _VP, _VP],
    "hd_coarse_correction": [_H, _VP, _VP],
    "hd_learned_grad": [_H, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double)],
    "hd_learned_train": [_H, ctypes.POINTER(TrainOpts), ctypes.POINTER(TrainInfo)],
    "hd_set_schur_prec": [_H, ctypes.c_int32],
    "hd_enable_learned": [_H, ctypes.c_int32],
    "hd_learned_save": [_H, ctypes.c_char_p],
    "hd_learned_load": [_H, ctypes.c_char_p],
    "hd_checkpoint_minres": [_H, ctypes.c_char_p],
    "hd_resume_minres": [_H, ctypes.c_char_p],
    "hd_apply_op_f32": [_H, _VP, _VP],
    "hd_apply_prec_f32": [_H, _VP, _VP],
    "hd_apply_op_tc": [_H, _VP, _VP],
    "hd_apply_op_tc_f32": [_H, _VP, _VP],
    "hd_set_inner_operator": [_H, ctypes.c_int32],
    "hd_tc_status": [_H],
    "hd_slab_plan": [ctypes.c_int32] * 6 + [ctypes.POINTER(Slab)],
    "hd_apply_op_partitioned": [_H, ctypes.c_int32, _VP, _VP],
    "hd_minres_solve_partitioned": [_H, ctypes.c_int32, _VP, _VP, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)],
    "hd_learned_conv_engine": [_H, ctypes.c_int32],
    "hd_massinv_create": [ctypes.POINTER(MassInvDesc), ctypes.POINTER(ctypes.c_void_p)],
    "hd_massinv_set_stream": [_H, _VP],
    "hd_massinv_apply": [_H, _VP, _VP],
    "hd_massinv_setup_ms": [_H, ctypes.POINTER(ctypes.c_double)],
    "hd_massinv_iterations": [_H, ctypes.POINTER(ctypes.c_int32)],
    "hd_massinv_destroy": [_H],
    "hd_rad_create": [ctypes.POINTER(RadDesc), ctypes.POINTER(ctypes.c_void_p)],
    "hd_rad_destroy": [_H],
    "hd_rad_set_stream": [_H, _VP],
    "hd_rad_get_sizes": [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)],
    "hd_rad_get_op": [_H, ctypes.POINTER(ctypes.c_void_p)],
    "hd_rad_points": [_H, _VP],
    "hd_rad_load": [_H, _VP, _VP],
    "hd_rad_winv": [_H, _VP, _VP],
    "hd_rad_residual": [_H, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double)],
    "hd_rad_stage": [_H, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(RadInfo)],
    "hd_rad_step": [_H, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(RadInfo)],
}


def lib():
    """The loaded libhdivsp (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhdivsp.so is not built: run python -m paper_2304_12387_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int32
        L.hd_last_error.argtypes = [_H]
        L.hd_last_error.restype = ctypes.c_char_p
        L.hd_rad_last_error.argtypes = [_H]
        L.hd_rad_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(st, h=None):
    if st != HD_OK:
        msg = lib().hd_last_error(h).decode() if h else ""
        raise HdError(st, msg)


def _ptr(t):
    """Device (or host numpy) pointer of a contiguous array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# -- same-name wrappers of the C ABI -------------------------------------------

def hd_lattice_e2d_map(nx, ny, nz, k):
    out = np.zeros((nx * ny * nz, 3 * (k + 1) * k * k), dtype=np.int32)
    _check(lib().hd_lattice_e2d_map(nx, ny, nz, k, out.ctypes.data))
    return out


def _rot_codes(rot, E):
    """Rotation codes as a contiguous int8 array of length E (None stays None)."""
    if rot is None:
        return None
    r = np.ascontiguousarray(rot, dtype=np.int64)
    if r.shape != (E,):
        raise ValueError("elem_rotation needs one code per element")
    if (r < -128).any() or (r > 127).any():
        raise ValueError("rotation codes must fit int8 (valid codes: 0..23)")
    return np.ascontiguousarray(r.astype(np.int8))


def hd_lattice_e2d_map_rot(nx, ny, nz, k, rot):
    rot = _rot_codes(rot, nx * ny * nz)
    out = np.zeros((nx * ny * nz, 3 * (k + 1) * k * k), dtype=np.int32)
    _check(lib().hd_lattice_e2d_map_rot(nx, ny, nz, k, _ptr(rot), out.ctypes.data))
    return out


def hd_lattice_e2l_map(nx, ny, nz, k, rot=None):
    rot = _rot_codes(rot, nx * ny * nz)
    out = np.zeros((nx * ny * nz, k ** 3), dtype=np.int32)
    _check(lib().hd_lattice_e2l_map(nx, ny, nz, k, _ptr(rot), out.ctypes.data))
    return out


def hd_lattice_is_affine(nx, ny, nz, vx, vy, vz):
    """True when every element of the lattice mesh is a parallelepiped (the affine fast path's test)."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (vx, vy, vz)]
    nv = (nx + 1) * (ny + 1) * (nz + 1)
    if any(a.shape != (nv,) for a in arrs):
        raise ValueError("vertex arrays need (nx+1)(ny+1)(nz+1) entries")
    out = ctypes.c_int32(0)
    _check(lib().hd_lattice_is_affine(nx, ny, nz, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                                      ctypes.byref(out)))
    return bool(out.value)


def hd_slab_plan(nx, ny, nz, k, P, p):
    """Owned id ranges of z-slab p of P (host only): a dict of half-open (lo, hi) pairs."""
    s = Slab()
    _check(lib().hd_slab_plan(nx, ny, nz, k, P, p, ctypes.byref(s)))
    return {"p": s.p, "P": s.P, "ez": (s.ez0, s.ez1), "xf": tuple(s.xf), "yf": tuple(s.yf), "zf": tuple(s.zf),
            "cell": tuple(s.cell), "halo": tuple(s.halo)}


def hd_lattice_ess_dofs(nx, ny, nz, k, ess_mask):
    n = ctypes.c_int64(0)
    _check(lib().hd_lattice_ess_dofs(nx, ny, nz, k, ess_mask, None, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.int64)
    _check(lib().hd_lattice_ess_dofs(nx, ny, nz, k, ess_mask, out.ctypes.data, ctypes.byref(n)))
    return out


class Operator:
    """Owns an hd_handle. Vectors are torch CUDA tensors (float64, or float32 for *_f32)."""

    def __init__(self, nx, ny, nz, k, vx, vy, vz, coef0, coef1, kind=HD_GRAD_DIV, ess_mask=0, q=0,
                 affine=False, tau=0.0, winv_mode=HD_WINV_DENSE, nu=0, coarse_max=0, cycle=1,
                 fp64_emulation=0, smooth_levels=0, w_levels=0, elem_rotation=None, aggregation=0, stream=None):
        E = nx * ny * nz
        self._keep = []
        rot = _rot_codes(elem_rotation, E)
        self._keep.append(rot)
        arrs = []
        for a, n in ((vx, None), (vy, None), (vz, None), (coef0, E), (coef1, E)):
            a = np.asarray(a, dtype=np.float64)
            if n is not None:
                a = np.broadcast_to(a, (n,))
            a, p = _dptr(a)
            self._keep.append(a)
            arrs.append(p)
        d = ProblemDesc(kind, nx, ny, nz, k, q, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4], ess_mask,
                        int(affine), tau, winv_mode, nu, coarse_max, cycle, int(fp64_emulation),
                        int(smooth_levels), int(w_levels),
                        None if rot is None else rot.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                        int(aggregation))
        h = ctypes.c_void_p()
        st = lib().hd_create(ctypes.byref(d), ctypes.byref(h))
        _check(st)
        self.h = h
        self.k, self.kind = k, kind
        self.dims = (nx, ny, nz)
        nrt, nl2, ne = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().hd_get_sizes(h, ctypes.byref(nrt), ctypes.byref(nl2), ctypes.byref(ne)), h)
        self.n_rt, self.n_l2, self.n_elem = nrt.value, nl2.value, ne.value
        self.n = self.n_rt + self.n_l2
        if stream is not None:
            self.set_stream(stream)

    def hd_get_setup_times(self):
        """Setup phase times of hd_create in ms: geometric factors, W^-1 data, diag(M),
        Schur preconditioner hierarchies, double-float copies, total."""
        ms = (ctypes.c_double * 6)()
        _check(lib().hd_get_setup_times(self.h, ms, 6), self.h)
        return {k: ms[i] for i, k in enumerate(("geometry", "winv", "diag_m", "schur", "double_float", "total"))}

    def close(self):
        if getattr(self, "h", None):
            lib().hd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream or a raw cudaStream_t integer."""
        s = getattr(stream, "cuda_stream", stream)
        _check(lib().hd_set_stream(self.h, ctypes.c_void_p(s)), self.h)

    def _call(self, name, *args):
        _check(getattr(lib(), name)(self.h, *[_ptr(a) for a in args]), self.h)

    def hd_apply_A(self, u, y): self._call("hd_apply_A", u, y)
    def hd_apply_B(self, u, yq): self._call("hd_apply_B", u, yq)
    def hd_apply_Bt(self, q, yu): self._call("hd_apply_Bt", q, yu)
    def hd_apply_C(self, q, yq): self._call("hd_apply_C", q, yq)
    def hd_apply_op(self, x, y): self._call("hd_apply_op", x, y)
    def hd_apply_op_host(self, x, y): self._call("hd_apply_op_host", x, y)
    def hd_apply_prec(self, r, z): self._call("hd_apply_prec", r, z)
    def hd_apply_schur(self, x, y): self._call("hd_apply_schur", x, y)
    def hd_vcycle(self, b, x): self._call("hd_vcycle", b, x)
    def hd_apply_op_f32(self, x, y): self._call("hd_apply_op_f32", x, y)
    def hd_apply_op_tc(self, x, y): self._call("hd_apply_op_tc", x, y)
    def hd_apply_op_tc_f32(self, x, y): self._call("hd_apply_op_tc_f32", x, y)

    def hd_apply_op_partitioned(self, P, x, y):
        _check(lib().hd_apply_op_partitioned(self.h, int(P), _ptr(x), _ptr(y)), self.h)

    def hd_minres_solve_partitioned(self, P, b, x, rtol=1e-8, maxit=1000, use_x0=False, check_every=8,
                                    outer_rtol=0.0, max_outer=1):
        """MINRES through P emulated z-slab partitions (see the header)."""
        o = SolveOpts(rtol, maxit, int(use_x0), check_every, 0, outer_rtol, max_outer)
        info = SolveInfo()
        st = lib().hd_minres_solve_partitioned(self.h, int(P), _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info))
        return st, {"iterations": info.iterations, "outer": info.outer, "true_relres": info.true_relres,
                    "ms_total": info.ms_total, "status": info.status}

    def hd_set_inner_operator(self, mode):
        """0: FP32 element kernel (CUDA cores); 1: tensor-core operator (affine meshes, k = 2..4)."""
        _check(lib().hd_set_inner_operator(self.h, int(mode)), self.h)

    def hd_tc_status(self):
        """Status of the tensor-core kernel's bounded waits since the last call (HD_OK or HD_ERR_CUDA)."""
        return lib().hd_tc_status(self.h)
    def hd_apply_prec_f32(self, r, z): self._call("hd_apply_prec_f32", r, z)
    def hd_get_diagonals(self, mt, ct): self._call("hd_get_diagonals", mt, ct)

    def hd_minres_solve_noalloc(self, b, x, rtol=1e-8, maxit=1000, use_x0=False, check_every=8,
                                outer_rtol=0.0, max_outer=1):
        """Allocation-free FP64 MINRES (work space in a fixed device array; see the header)."""
        o = SolveOpts(rtol, maxit, int(use_x0), check_every, 0, outer_rtol, max_outer)
        info = SolveInfo()
        st = lib().hd_minres_solve_noalloc(self.h, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info))
        return st, {"iterations": info.iterations, "outer": info.outer, "eta_ratio": info.eta_ratio,
                    "true_relres": info.true_relres, "ms_total": info.ms_total, "status": info.status}

    def hd_profile(self, enable):
        _check(lib().hd_profile(self.h, int(enable)), self.h)

    def hd_profile_read(self):
        n, ms = ctypes.c_int32(), ctypes.c_double()
        _check(lib().hd_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms)), self.h)
        return n.value, ms.value

    def hd_get_e2d_map(self):
        out = np.zeros((self.n_elem, 3 * (self.k + 1) * self.k ** 2), dtype=np.int32)
        _check(lib().hd_get_e2d_map(self.h, out.ctypes.data), self.h)
        return out

    def hd_get_e2l_map(self):
        out = np.zeros((self.n_elem, self.k ** 3), dtype=np.int32)
        _check(lib().hd_get_e2l_map(self.h, out.ctypes.data), self.h)
        return out

    def hd_get_ess_dofs(self):
        n = ctypes.c_int64(0)
        _check(lib().hd_get_ess_dofs(self.h, None, ctypes.byref(n)), self.h)
        out = np.zeros(n.value, dtype=np.int64)
        _check(lib().hd_get_ess_dofs(self.h, out.ctypes.data, ctypes.byref(n)), self.h)
        return out

    def hd_get_level(self, l=0):
        nl = ctypes.c_int32()
        dims = (ctypes.c_int32 * 3)()
        _check(lib().hd_get_level(self.h, l, ctypes.byref(nl), dims), self.h)
        return nl.value, tuple(dims)

    def hd_minres_solve(self, b, x, rtol=1e-8, maxit=1000, use_x0=False, check_every=8, precision=0,
                        outer_rtol=0.0, max_outer=1, raise_on_error=False, resume=False):
        """MINRES on AA x = b. max_outer > 1 or precision = 1 wraps it in an FP64
        residual correction that stops at ||b - AA x|| <= outer_rtol ||b||. resume:
        continue the recurrence that the handle keeps (a stopped solve or
        hd_resume_minres) for up to maxit more iterations."""
        o = SolveOpts(rtol, maxit, int(use_x0), check_every, precision, outer_rtol, max_outer, int(resume))
        info = SolveInfo()
        st = lib().hd_minres_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info))
        if raise_on_error:
            _check(st, self.h)
        return st, {"iterations": info.iterations, "outer": info.outer, "eta_ratio": info.eta_ratio,
                    "true_relres": info.true_relres, "ms_total": info.ms_total, "status": info.status,
                    "fallback": info.fallback}

    def hd_gmres_solve(self, b, x, rtol=1e-8, maxit=1000, restart=64, prec=1, use_x0=False, precision=0,
                       inner_rtol=1e-4):
        """Restarted right-preconditioned GMRES on AA x = b; prec = HD_GMRES_BLOCK_TRI (1,
        the block upper-triangular preconditioner) or HD_GMRES_BLOCK_DIAG (0); precision 1:
        FP32 operator and V-cycle inside the cycles, FP64 residual at every restart."""
        o = GmresOpts(rtol, maxit, restart, prec, int(use_x0), precision, inner_rtol)
        info = SolveInfo()
        st = lib().hd_gmres_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info))
        return st, {"iterations": info.iterations, "cycles": info.outer, "estimate_ratio": info.eta_ratio,
                    "true_relres": info.true_relres, "ms_total": info.ms_total, "status": info.status}

    # -- learned Schur preconditioner ----------------------------------------
    def hd_learned_init(self, nc=32, seed=2304, delta=0.0):
        _check(lib().hd_learned_init(self.h, nc, seed, delta), self.h)

    def hd_learned_set_weights(self, W1, W2):
        W1 = np.ascontiguousarray(W1, dtype=np.float32)
        W2 = np.ascontiguousarray(W2, dtype=np.float32)
        _check(lib().hd_learned_set_weights(self.h, W1.ctypes.data, W2.ctypes.data), self.h)

    def hd_learned_get_weights(self, nc=32):
        W1 = np.zeros((nc, 27), dtype=np.float32)
        W2 = np.zeros((nc, nc, 27), dtype=np.float32)
        _check(lib().hd_learned_get_weights(self.h, W1.ctypes.data, W2.ctypes.data), self.h)
        return W1, W2

    def hd_learned_apply(self, r, z): self._call("hd_learned_apply", r, z)
    def hd_coarse_correction(self, r, z): self._call("hd_coarse_correction", r, z)

    def hd_learned_grad(self, r, e, qr, nc=32):
        """r, e, qr: (npairs, n_l2) device tensors (qr may be None). Returns (loss, gW1, gW2)."""
        g1 = np.zeros((nc, 27), dtype=np.float32)
        g2 = np.zeros((nc, nc, 27), dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().hd_learned_grad(self.h, r.shape[0], _ptr(r), _ptr(e), _ptr(qr), g1.ctypes.data,
                                     g2.ctypes.data, ctypes.byref(loss)), self.h)
        return loss.value, g1, g2

    def hd_learned_train(self, npairs=8, capture_every=4, steps=100, lr=1e-3, seed=2304):
        o = TrainOpts(npairs, capture_every, steps, lr, seed)
        info = TrainInfo()
        _check(lib().hd_learned_train(self.h, ctypes.byref(o), ctypes.byref(info)), self.h)
        return {"pairs": info.pairs, "loss_initial": info.loss_initial, "loss_final": info.loss_final,
                "pcg_max_iterations": info.pcg_max_iterations, "ms_total": info.ms_total}

    def hd_set_schur_prec(self, mode):
        _check(lib().hd_set_schur_prec(self.h, int(mode)), self.h)

    def hd_enable_learned(self, on):
        _check(lib().hd_enable_learned(self.h, int(bool(on))), self.h)

    def hd_learned_conv_engine(self, engine):
        """0: tcgen05 tensor cores (default); 1: mma.sync."""
        _check(lib().hd_learned_conv_engine(self.h, int(engine)), self.h)

    def hd_learned_save(self, path):
        """Returns the status (HD_OK or HD_ERR_INVALID_ARG)."""
        return lib().hd_learned_save(self.h, os.fsencode(path))

    def hd_learned_load(self, path):
        return lib().hd_learned_load(self.h, os.fsencode(path))

    # -- MINRES checkpoints ----------------------------------------------------
    def hd_checkpoint_minres(self, path):
        """Writes the recurrence that a stopped plain FP64 solve left on the handle;
        returns the status."""
        return lib().hd_checkpoint_minres(self.h, os.fsencode(path))

    def hd_resume_minres(self, path):
        """Loads a checkpoint; the next hd_minres_solve(..., resume=True) continues it."""
        return lib().hd_resume_minres(self.h, os.fsencode(path))


class MassInverse:
    """The DG mass inverse W^-1 of any degree k = 2..9 (hd_massinv_*): vectors are torch
    CUDA float64 tensors of n_l2 = (nx k)(ny k)(nz k) entries in lattice order."""

    def __init__(self, nx, ny, nz, k, vx, vy, vz, alpha=None, method=HD_WINV_CG, q=0, fp64_emulation=0,
                 stream=None):
        E = nx * ny * nz
        self._keep = []
        ptrs = []
        for a in (vx, vy, vz):
            a, pa = _dptr(a)
            self._keep.append(a)
            ptrs.append(pa)
        pal = None
        if alpha is not None:
            al, pal = _dptr(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (E,)))
            self._keep.append(al)
        d = MassInvDesc(nx, ny, nz, k, q, ptrs[0], ptrs[1], ptrs[2], pal, method, int(fp64_emulation))
        h = ctypes.c_void_p()
        _check(lib().hd_massinv_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.k, self.dims = k, (nx, ny, nz)
        self.n_l2 = E * k ** 3
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        s = getattr(stream, "cuda_stream", stream)
        _check(lib().hd_massinv_set_stream(self.h, ctypes.c_void_p(s)))

    def apply(self, x, y):
        _check(lib().hd_massinv_apply(self.h, _ptr(x), _ptr(y)))

    def setup_ms(self):
        v = ctypes.c_double()
        _check(lib().hd_massinv_setup_ms(self.h, ctypes.byref(v)))
        return v.value

    def iterations(self):
        v = ctypes.c_int32()
        _check(lib().hd_massinv_iterations(self.h, ctypes.byref(v)))
        return v.value

    def close(self):
        if self.h:
            lib().hd_massinv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rad_info(i):
    return {f: getattr(i, f) for f, _ in RadInfo._fields_}


class RadDiff:
    """Grey nonlinear radiation diffusion (hd_rad_*, Sec. 4.3) on a structured hex mesh with
    reflecting walls: the SDIRK3 stages, the outer iteration of element-wise Newton and
    Darcy solves. Vectors are torch CUDA float64 tensors: e, Eh and loads n_l2, F n_rt,
    point values [E][q^3]."""

    def __init__(self, nx, ny, nz, k, vx, vy, vz, sigma, dt, rho=1.0, cv=1.0, a=1.0, c=1.0, q=0, cycle=2,
                 smooth_levels=2, fp64_emulation=1, aggregation=0, outer_rtol=0.0, outer_maxit=0,
                 newton_rtol=0.0, newton_maxit=0, linear_rtol=0.0, linear_maxit=0, linear_precision=0,
                 stream=None):
        E = nx * ny * nz
        self._keep = []
        ptrs = []
        for arr in (vx, vy, vz):
            arr, pa = _dptr(arr)
            self._keep.append(arr)
            ptrs.append(pa)
        sg, psg = _dptr(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (E,)))
        self._keep.append(sg)
        mesh = ProblemDesc(HD_DARCY, nx, ny, nz, k, q, ptrs[0], ptrs[1], ptrs[2], None, None, 0, 0, 0.0,
                           HD_WINV_DENSE, 0, 0, cycle, int(fp64_emulation), int(smooth_levels), 0, None,
                           int(aggregation))
        d = RadDesc(mesh, psg, rho, cv, a, c, dt, outer_rtol, outer_maxit, newton_rtol, newton_maxit, linear_rtol,
                    linear_maxit, int(linear_precision))
        h = ctypes.c_void_p()
        _check(lib().hd_rad_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        nrt, nl2, ne, qq = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        self._call("hd_rad_get_sizes", ctypes.byref(nrt), ctypes.byref(nl2), ctypes.byref(ne), ctypes.byref(qq))
        self.n_rt, self.n_l2, self.n_elem, self.q = nrt.value, nl2.value, ne.value, qq.value
        self.k, self.dims = k, (nx, ny, nz)
        if stream is not None:
            self.set_stream(stream)

    def _call(self, name, *args):
        st = getattr(lib(), name)(self.h, *args)
        if st != HD_OK:
            raise HdError(st, lib().hd_rad_last_error(self.h).decode())

    def set_stream(self, stream):
        s = getattr(stream, "cuda_stream", stream)
        self._call("hd_rad_set_stream", ctypes.c_void_p(s))

    def points(self):
        """Physical coordinates of the Gauss points (E, q^3, 3), host numpy."""
        out = np.zeros((self.n_elem, self.q ** 3, 3))
        self._call("hd_rad_points", out.ctypes.data)
        return out

    def load(self, values, out):
        self._call("hd_rad_load", _ptr(values), _ptr(out))

    def winv(self, x, y):
        self._call("hd_rad_winv", _ptr(x), _ptr(y))

    def residual(self, e_star, Eh_star, q_load, s_load, e, Eh, F, r=None):
        v = ctypes.c_double()
        self._call("hd_rad_residual", *[_ptr(t) for t in (e_star, Eh_star, q_load, s_load, e, Eh, F, r)],
                   ctypes.byref(v))
        return v.value

    def stage(self, e_star, Eh_star, q_load, s_load, e, Eh, F):
        info = RadInfo()
        self._call("hd_rad_stage", *[_ptr(t) for t in (e_star, Eh_star, q_load, s_load, e, Eh, F)],
                   ctypes.byref(info))
        return _rad_info(info)

    def step(self, e, Eh, F, q_loads=None, s_loads=None):
        info = RadInfo()
        self._call("hd_rad_step", *[_ptr(t) for t in (e, Eh, F, q_loads, s_loads)], ctypes.byref(info))
        return _rad_info(info)

    def close(self):
        if getattr(self, "h", None):
            lib().hd_rad_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
