"""ctypes binding of libosm.so (include/osm.h).  Argument marshalling only:
every step of the solve runs in the library's CUDA kernels.  PyTorch is used
for device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libosm.so")

OSM_OK, OSM_E_ARG, OSM_E_CUDA, OSM_E_NOMEM, OSM_E_NOCONV, OSM_E_BREAKDOWN, OSM_E_STATE, OSM_E_TIMEOUT = range(8)
OSM_FP64, OSM_MIXED, OSM_FP64_REFINE = 0, 1, 2

EXPORTED = (
    "osm_default_opts", "osm_setup", "osm_info", "osm_set_density", "osm_set_robin",
    "osm_set_robin_sub", "osm_solve", "osm_sample_p", "osm_log_uniform_p", "osm_apply",
    "osm_apply_noalloc", "osm_reset", "osm_iterate", "osm_get_local", "osm_get_lambda",
    "osm_set_lambda", "osm_inner_iters", "osm_stats", "osm_set_density_dev", "osm_set_stations",
    "osm_gravity", "osm_potential_vjp", "osm_grad", "osm_grad_p", "osm_host_local_system", "osm_host_face_system",
    "osm_profile_spmv", "osm_status_string", "osm_last_error", "osm_destroy", "osm_setup_batch",
    "osm_batch_info", "osm_set_robin_inst", "osm_solve_batch", "osm_set_transmission",
    "osm_host_local_system_tc", "osm_host_face_stiffness", "osm_sample_p_ex",
)


class OsmMesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("xc", C.c_void_p), ("yc", C.c_void_p), ("zc", C.c_void_p)]


class OsmDecomp(C.Structure):
    _fields_ = [("sx", C.c_int32), ("sy", C.c_int32), ("sz", C.c_int32),
                ("cx", C.c_void_p), ("cy", C.c_void_p), ("cz", C.c_void_p)]


class OsmOpts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("inner_rtol", C.c_double), ("mixed_inner_rtol", C.c_double),
                ("max_outer", C.c_int32), ("max_inner", C.c_int32), ("use_graph", C.c_int32),
                ("max_seconds", C.c_int32), ("autotune", C.c_int32), ("index16", C.c_int32),
                ("fp32_operator", C.c_int32), ("fp64_start", C.c_int32), ("tensor_zchunk", C.c_int32)]


class OsmInfo(C.Structure):
    _fields_ = [("n_sub", C.c_int32), ("n_face", C.c_int32), ("n_nodes", C.c_int64),
                ("n_dofs", C.c_int64), ("n_local", C.c_int64), ("n_face_vals", C.c_int64),
                ("nnz", C.c_int64), ("sell_entries", C.c_int64), ("n_slices", C.c_int64),
                ("vec_rows", C.c_int64),
                ("device_bytes", C.c_int64), ("setup_seconds", C.c_double),
                ("spmv_variant_fp64", C.c_int32), ("spmv_variant_fp32", C.c_int32),
                ("spmv_ms_fp64", C.c_double * 2), ("spmv_ms_fp32", C.c_double * 2),
                ("spmv_ms16_fp64", C.c_double * 2), ("spmv_ms16_fp32", C.c_double * 2),
                ("col_bytes_fp64", C.c_int32), ("col_bytes_fp32", C.c_int32),
                ("fp32_operator", C.c_int32), ("fp32_operator_tuned", C.c_int32),
                ("tensor_ms_fp32", C.c_double), ("tensor_zchunk", C.c_int32), ("reserved_i", C.c_int32),
                ("tensor_ms_zchunk", C.c_double * 4), ("fp64_start", C.c_int32), ("reserved_j", C.c_int32),
                ("start_ms", C.c_double * 3), ("box_rows", C.c_int64),
                ("tensor_ms_zchunk_tail", C.c_double * 4)]


def _info_dict(info):
    out = {}
    for k, _ in OsmInfo._fields_:
        v = getattr(info, k)
        out[k] = list(v) if hasattr(v, "__len__") else v
    return out


class OsmStats(C.Structure):
    _fields_ = [("n_outer", C.c_int32), ("n_cg_steps", C.c_int32), ("n_launches", C.c_int64),
                ("relres", C.c_double), ("status", C.c_int32), ("reserved", C.c_int32),
                ("sub_row_steps", C.c_int64), ("op_row_steps", C.c_int64)]


class OsmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libosm.so; fails loudly if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libosm.so is missing ({LIB_PATH}); build it with "
                          "paper_2112_03851_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "osm_default_opts": (None, [vp]),
        "osm_setup": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "osm_info": (C.c_int, [vp, vp]),
        "osm_set_density": (C.c_int, [vp, vp]),
        "osm_set_robin": (C.c_int, [vp, d]),
        "osm_set_robin_sub": (C.c_int, [vp, vp]),
        "osm_set_transmission": (C.c_int, [vp, d, d, d, d]),
        "osm_solve": (C.c_int, [vp, d, vp, vp, vp]),
        "osm_sample_p": (C.c_int, [vp, i32, vp, d, i32, vp, vp, vp]),
        "osm_sample_p_ex": (C.c_int, [vp, i32, vp, d, i32, i32, vp, vp, vp]),
        "osm_log_uniform_p": (C.c_int, [C.c_uint64, i32, d, d, vp]),
        "osm_apply": (C.c_int, [vp, i32, vp, vp]),
        "osm_apply_noalloc": (C.c_int, [vp, i32, vp, vp]),
        "osm_reset": (C.c_int, [vp]),
        "osm_iterate": (C.c_int, [vp, i32, vp]),
        "osm_get_local": (C.c_int, [vp, vp]),
        "osm_get_lambda": (C.c_int, [vp, vp]),
        "osm_set_lambda": (C.c_int, [vp, vp]),
        "osm_inner_iters": (C.c_int, [vp, vp]),
        "osm_stats": (C.c_int, [vp, vp]),
        "osm_set_density_dev": (C.c_int, [vp, vp]),
        "osm_set_stations": (C.c_int, [vp, i32, vp]),
        "osm_gravity": (C.c_int, [vp, vp, vp]),
        "osm_potential_vjp": (C.c_int, [vp, d, vp, vp]),
        "osm_grad": (C.c_int, [vp, d, vp, vp, vp, vp]),
        "osm_grad_p": (C.c_int, [vp, i32, vp, vp, vp]),
        "osm_host_local_system": (C.c_int, [vp, vp, vp, d, i32, vp, vp, vp, vp, vp, vp]),
        "osm_host_face_system": (C.c_int, [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]),
        "osm_host_local_system_tc": (C.c_int, [vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]),
        "osm_host_face_stiffness": (C.c_int, [vp, vp, vp, i32, vp]),
        "osm_profile_spmv": (C.c_int, [vp, i32, i32, vp]),
        "osm_setup_batch": (C.c_int, [i32, vp, vp, vp, vp, vp, vp]),
        "osm_batch_info": (C.c_int, [vp, vp, vp]),
        "osm_set_robin_inst": (C.c_int, [vp, vp]),
        "osm_solve_batch": (C.c_int, [vp, d, vp, vp, vp]),
        "osm_status_string": (C.c_char_p, [C.c_int]),
        "osm_last_error": (C.c_char_p, [vp]),
        "osm_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _status_name(st):
    try:
        return load().osm_status_string(st).decode()
    except Exception:
        return f"status {st}"


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dptr(t):
    return C.c_void_p(t.data_ptr())


def check_local_vector(t, n, device, name):
    """Refuse, before any launch, a tensor the C ABI would read or write out
    of bounds: it must be float64, contiguous, on the handle's device and
    hold exactly n values (the canonical local layout)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if t.device != torch.device(device):
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != n:
        raise ValueError(f"{name} must have {n} values (canonical local layout), got {t.numel()}")


class _Inputs:
    """Host copies of mesh / density / cuts kept alive for a call."""

    def __init__(self, xc, yc, zc, drho, cx, cy, cz):
        self.xc = np.ascontiguousarray(xc, dtype=np.float64)
        self.yc = np.ascontiguousarray(yc, dtype=np.float64)
        self.zc = np.ascontiguousarray(zc, dtype=np.float64)
        self.drho = np.ascontiguousarray(drho, dtype=np.float64).reshape(-1)
        self.cx = np.ascontiguousarray(cx, dtype=np.int32)
        self.cy = np.ascontiguousarray(cy, dtype=np.int32)
        self.cz = np.ascontiguousarray(cz, dtype=np.int32)
        nx, ny, nz = len(self.xc) - 1, len(self.yc) - 1, len(self.zc) - 1
        if self.drho.size != nx * ny * nz:
            raise ValueError("density must have nx*ny*nz entries")
        self.mesh = OsmMesh(nx, ny, nz, _ptr(self.xc).value, _ptr(self.yc).value, _ptr(self.zc).value)
        self.dec = OsmDecomp(len(self.cx) - 1, len(self.cy) - 1, len(self.cz) - 1,
                             _ptr(self.cx).value, _ptr(self.cy).value, _ptr(self.cz).value)


def default_opts(**kw) -> OsmOpts:
    o = OsmOpts()
    load().osm_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = {"fp64": OSM_FP64, "mixed": OSM_MIXED, "fp64_refine": OSM_FP64_REFINE}[v]
        setattr(o, k, v)
    return o


class Solver:
    """One gravimetry problem on the GPU (a libosm handle).

    ``xc, yc, zc``: element vertex coordinates; ``drho``: per-element density
    (x fastest); ``cx, cy, cz``: element-index cuts of the subdomain grid.
    """

    def __init__(self, xc, yc, zc, drho, cx, cy, cz, p=1.0, stream=None, tc=None, **opts):
        import torch
        L = load()
        self._torch = torch
        self._in = _Inputs(xc, yc, zc, drho, cx, cy, cz)
        self.opts = default_opts(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        st = L.osm_setup(C.byref(self._in.mesh), _ptr(self._in.drho), C.byref(self._in.dec),
                         C.byref(self.opts), C.c_void_p(stream.cuda_stream), C.byref(h))
        self._h = h
        if st != OSM_OK:
            msg = L.osm_last_error(h).decode() if h.value else ""
            self.close()
            raise OsmError(st, msg)
        if tc is not None:
            self.set_transmission(*tc)
        elif p is not None:
            if np.ndim(p) == 0:
                self.set_robin(float(p))
            else:
                self.set_robin_sub(p)

    @classmethod
    def from_problem(cls, prob, p=None, tc=None, **opts):
        return cls(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz,
                   p=prob.p if p is None else p, tc=tc, **opts)

    @property
    def info(self):
        """osm_info of the handle as it is now: the FP32 operator and the
        refinement start follow set_transmission / set_robin (a second-order
        condition moves a tensor-form handle back to the SELL matrix)."""
        info = OsmInfo()
        self._check(load().osm_info(self._h, C.byref(info)))
        return _info_dict(info)

    # ------------------------------------------------------------ plumbing
    def _check(self, st, allow=()):
        if st != OSM_OK and st not in allow:
            raise OsmError(st, load().osm_last_error(self._h).decode())
        return st

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().osm_destroy(h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _zeros(self, n, dtype=None):
        t = self._torch
        return t.zeros(int(n), dtype=dtype or t.float64, device=self.device)

    # ----------------------------------------------------------------- API
    def set_robin(self, p: float):
        self._check(load().osm_set_robin(self._h, float(p)))

    def set_robin_sub(self, p_sub):
        p_sub = np.ascontiguousarray(p_sub, dtype=np.float64)
        self._check(load().osm_set_robin_sub(self._h, _ptr(p_sub)))

    def set_transmission(self, p_lo: float, q_lo: float, p_hi: float, q_hi: float):
        """Second-order / unsymmetric condition p + q(-d^2/dtau^2): (p_lo, q_lo)
        on the lower side of every face, (p_hi, q_hi) on the upper side."""
        self._check(load().osm_set_transmission(self._h, float(p_lo), float(q_lo), float(p_hi), float(q_hi)))

    def set_density(self, drho):
        drho = np.ascontiguousarray(drho, dtype=np.float64).reshape(-1)
        self._check(load().osm_set_density(self._h, _ptr(drho)))

    def solve(self, rtol=1e-8, phi=None, allow_noconv=False):
        """Full Schwarz solve; returns (phi on the node grid, iterations, relres)."""
        if phi is None:
            phi = self._zeros(self.info["n_nodes"])
        it = C.c_int32()
        rel = C.c_double()
        allow = (OSM_E_NOCONV,) if allow_noconv else ()
        self._check(load().osm_solve(self._h, float(rtol), _dptr(phi), C.byref(it), C.byref(rel)), allow)
        return phi, it.value, rel.value

    def apply(self, x, op=0):
        """y = A x (op 0: Robin matrix, op 1: Neumann stiffness, op 2: the FP32
        inner operator of a mixed handle), canonical local layout."""
        check_local_vector(x, self.info["n_local"], self.device, "x")
        y = self._zeros(self.info["n_local"])
        self._check(load().osm_apply(self._h, int(op), _dptr(x), _dptr(y)))
        return y

    def apply_noalloc(self, x, y=None, op=0):
        """y = A x like apply(), using only the library's fixed scratch (no
        device allocation by the library).  Pass a preallocated y to avoid
        the one allocation this wrapper would otherwise make for it."""
        check_local_vector(x, self.info["n_local"], self.device, "x")
        if y is None:
            y = self._zeros(self.info["n_local"])
        else:
            check_local_vector(y, self.info["n_local"], self.device, "y")
        self._check(load().osm_apply_noalloc(self._h, int(op), _dptr(x), _dptr(y)))
        return y

    def reset(self):
        self._check(load().osm_reset(self._h))

    def iterate(self, n):
        hist = np.zeros(max(int(n), 1))
        self._check(load().osm_iterate(self._h, int(n), _ptr(hist)))
        return hist[:n]

    def get_local(self):
        u = self._zeros(self.info["n_local"])
        self._check(load().osm_get_local(self._h, _dptr(u)))
        return u

    def get_lambda(self):
        lam = self._zeros(self.info["n_face_vals"])
        self._check(load().osm_get_lambda(self._h, _dptr(lam)))
        return lam

    def set_lambda(self, lam):
        lam = lam.contiguous()
        self._check(load().osm_set_lambda(self._h, _dptr(lam)))

    # ------------------------------------------------------ adjoint gradient
    @property
    def n_elements(self):
        return (len(self._in.xc) - 1) * (len(self._in.yc) - 1) * (len(self._in.zc) - 1)

    def set_density_dev(self, drho):
        """Density from a device tensor (float64, nx*ny*nz); load built on the GPU."""
        drho = drho.detach().to(dtype=self._torch.float64).contiguous()
        assert drho.numel() == self.n_elements and drho.is_cuda
        self._check(load().osm_set_density_dev(self._h, _dptr(drho)))

    def set_stations(self, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self._check(load().osm_set_stations(self._h, len(xyz), _ptr(xyz)))
        self.n_stations = len(xyz)

    def gravity(self, phi):
        g = self._zeros(self.n_stations)
        self._check(load().osm_gravity(self._h, _dptr(phi.contiguous()), _dptr(g)))
        return g

    def potential_vjp(self, v, rtol=1e-8):
        """dL/d drho for v = dL/dphi (device, full node grid), by one adjoint solve."""
        v = v.detach().to(dtype=self._torch.float64).contiguous()
        grad = self._zeros(self.n_elements)
        self._check(load().osm_potential_vjp(self._h, float(rtol), _dptr(v), _dptr(grad)))
        return grad

    def grad(self, g_obs, rtol=1e-8):
        """(J, dJ/d drho, dJ/dp) of J = 1/2 ||B phi - g_obs||^2 at the current density."""
        g_obs = g_obs.detach().to(dtype=self._torch.float64).contiguous()
        J = C.c_double()
        dp = C.c_double()
        grad = self._zeros(self.n_elements)
        self._check(load().osm_grad(self._h, float(rtol), _dptr(g_obs), C.byref(J), _dptr(grad), C.byref(dp)))
        return J.value, grad, dp.value

    def grad_p(self, g_obs, n_iter):
        """(J_N, dJ_N/dp): misfit after exactly n_iter Schwarz iterations from
        zero and its derivative w.r.t. p by reverse-mode Schwarz."""
        g_obs = g_obs.detach().to(dtype=self._torch.float64).contiguous()
        J = C.c_double()
        dp = C.c_double()
        self._check(load().osm_grad_p(self._h, int(n_iter), _dptr(g_obs), C.byref(J), C.byref(dp)))
        return J.value, dp.value

    def stats(self):
        st = OsmStats()
        self._check(load().osm_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in OsmStats._fields_ if k != "reserved"}

    def inner_iters(self):
        it = np.zeros(self.info["n_sub"], dtype=np.int32)
        self._check(load().osm_inner_iters(self._h, _ptr(it)))
        return it

    def profile_spmv(self, reps=20, prec=0):
        """Median time (ms) of one batched SELL SpMV launch (CUDA events).
        prec 0: plain FP64 operator; 1: plain FP32 operator (mixed handles);
        2: the FP32 CG-step kernel k_cg_spmv_dir32 (mixed handles); 3: the FP64
        CG-step kernel k_cg_spmv<double>.  2 and 3 overwrite the CG state."""
        ms = C.c_double()
        self._check(load().osm_profile_spmv(self._h, int(prec), int(reps), C.byref(ms)))
        return ms.value

    def spmv_bytes(self, prec=0):
        """Algorithmic bytes of one launch of profile_spmv's kernel `prec`: per
        nonzero the value (8 B FP64 or 4 B FP32) and its column index (4 B, or
        2 B on a handle with 16-bit indices), 8 B per slice offset, the input
        vector read once and the output written once; the FP32 CG-step kernel
        (2) also reads p and q and writes p (12 B per row).  The tensor-product
        FP32 operator (info fp32_operator == 2) reads no matrix: per box row
        the input read once and the output written once (+ 12 B for the CG
        step's p, q epilogue); its 1-D bands (40 B per node of a box edge)
        are under 0.1% of that and not counted."""
        i = self.info
        if prec in (1, 2) and i.get("fp32_operator") == 2:
            return i["box_rows"] * (8 + (12 if prec == 2 else 0))
        vb = 8 if prec in (0, 3) else 4
        cb = i["col_bytes_fp64"] if prec in (0, 3) else (i["col_bytes_fp32"] or 4)
        extra = 12 * i["n_local"] if prec == 2 else 0
        return i["nnz"] * (vb + cb) + i["n_slices"] * 8 + i["n_local"] * 2 * vb + extra

    def sample_p(self, p_values, rtol=1e-8, max_outer=None, race=False):
        """Batched evaluation of Robin parameters: (iterations, relres, best
        index).  race=True stops each batch when its first candidate converges
        (osm_sample_p_ex with OSM_SAMPLE_RACE)."""
        p = np.ascontiguousarray(p_values, dtype=np.float64)
        n = len(p)
        iters = np.zeros(n, dtype=np.int32)
        rel = np.zeros(n)
        best = C.c_int32(-1)
        mo = self.opts.max_outer if max_outer is None else int(max_outer)
        self._check(load().osm_sample_p_ex(self._h, n, _ptr(p), float(rtol), mo, 1 if race else 0, _ptr(iters),
                                           _ptr(rel), C.byref(best)), (OSM_E_NOCONV,))
        return iters, rel, best.value


class BatchSolver(Solver):
    """Several independent problems in one handle (one CUDA graph per solve).

    ``problems``: objects with xc, yc, zc, drho, cx, cy, cz (and p)."""

    def __init__(self, problems, p=None, stream=None, **opts):
        import torch
        L = load()
        self._torch = torch
        self._ins = [_Inputs(q.xc, q.yc, q.zc, q.drho, q.cx, q.cy, q.cz) for q in problems]
        self._in = self._ins[0]
        n = len(problems)
        meshes = (OsmMesh * n)(*[i.mesh for i in self._ins])
        decs = (OsmDecomp * n)(*[i.dec for i in self._ins])
        dptrs = (C.c_void_p * n)(*[_ptr(i.drho).value for i in self._ins])
        self.opts = default_opts(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        st = L.osm_setup_batch(n, meshes, dptrs, decs, C.byref(self.opts), C.c_void_p(stream.cuda_stream),
                               C.byref(h))
        self._h = h
        if st != OSM_OK:
            msg = L.osm_last_error(h).decode() if h.value else ""
            self.close()
            raise OsmError(st, msg)
        self.n_inst = n
        off = np.zeros(n + 1, dtype=np.int64)
        ni = C.c_int32()
        L.osm_batch_info(h, C.byref(ni), _ptr(off))
        self.node_offsets = off
        ps = [q.p for q in problems] if p is None else (np.broadcast_to(p, (n,)))
        self.set_robin_inst(ps)

    def set_robin_inst(self, p_inst):
        p_inst = np.ascontiguousarray(p_inst, dtype=np.float64)
        self._check(load().osm_set_robin_inst(self._h, _ptr(p_inst)))

    def solve(self, rtol=1e-8, phi=None, allow_noconv=False):
        """Returns (phi of all instances concatenated, iterations[n], relres[n])."""
        if phi is None:
            phi = self._zeros(self.info["n_nodes"])
        it = np.zeros(self.n_inst, dtype=np.int32)
        rel = np.zeros(self.n_inst)
        allow = (OSM_E_NOCONV,) if allow_noconv else ()
        self._check(load().osm_solve_batch(self._h, float(rtol), _dptr(phi), _ptr(it), _ptr(rel)), allow)
        return phi, it, rel

    def instance_phi(self, phi, i):
        return phi[int(self.node_offsets[i]):int(self.node_offsets[i + 1])]


def log_uniform_p(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.zeros(n)
    st = load().osm_log_uniform_p(C.c_uint64(seed), int(n), float(lo), float(hi), _ptr(out))
    if st != OSM_OK:
        raise OsmError(st, "bad arguments")
    return out


def host_local_system(xc, yc, zc, drho, cx, cy, cz, p, sub, tc=None):
    """(A_i as scipy CSR, f_i) unpacked from the GPU packing (host only);
    tc = (p_lo, q_lo, p_hi, q_hi) selects the second-order form."""
    import scipy.sparse as sp
    L = load()
    inp = _Inputs(xc, yc, zc, drho, cx, cy, cz)
    n, nnz = C.c_int64(), C.c_int64()
    if tc is None:
        fn = L.osm_host_local_system
        args = (C.byref(inp.mesh), _ptr(inp.drho), C.byref(inp.dec), float(p), int(sub))
    else:
        tcv = np.ascontiguousarray(tc, dtype=np.float64)
        fn = L.osm_host_local_system_tc
        args = (C.byref(inp.mesh), _ptr(inp.drho), C.byref(inp.dec), _ptr(tcv), int(sub))
    st = fn(*args, C.byref(n), C.byref(nnz), None, None, None, None)
    if st != OSM_OK:
        raise OsmError(st, "host_local_system")
    rp = np.zeros(n.value + 1, dtype=np.int64)
    ci = np.zeros(nnz.value, dtype=np.int32)
    v = np.zeros(nnz.value)
    f = np.zeros(n.value)
    fn(*args, C.byref(n), C.byref(nnz), _ptr(rp), _ptr(ci), _ptr(v), _ptr(f))
    return sp.csr_matrix((v, ci, rp), shape=(n.value, n.value)), f


def host_face_system(xc, yc, zc, drho, cx, cy, cz, face):
    """(node indices, face mass as scipy CSR) of one face (host only)."""
    import scipy.sparse as sp
    L = load()
    inp = _Inputs(xc, yc, zc, drho, cx, cy, cz)
    n, nnz = C.c_int64(), C.c_int64()
    args = (C.byref(inp.mesh), _ptr(inp.drho), C.byref(inp.dec), int(face))
    st = L.osm_host_face_system(*args, C.byref(n), C.byref(nnz), None, None, None, None)
    if st != OSM_OK:
        raise OsmError(st, "host_face_system")
    node = np.zeros(n.value, dtype=np.int32)
    rp = np.zeros(n.value + 1, dtype=np.int64)
    ci = np.zeros(nnz.value, dtype=np.int32)
    v = np.zeros(nnz.value)
    L.osm_host_face_system(*args, C.byref(n), C.byref(nnz), _ptr(node), _ptr(rp), _ptr(ci), _ptr(v))
    return node, sp.csr_matrix((v, ci, rp), shape=(n.value, n.value))


def host_face_stiffness(xc, yc, zc, drho, cx, cy, cz, face):
    """Tangential stiffness of one face, same CSR as host_face_system."""
    import scipy.sparse as sp
    node, Mf = host_face_system(xc, yc, zc, drho, cx, cy, cz, face)
    inp = _Inputs(xc, yc, zc, drho, cx, cy, cz)
    v = np.zeros(Mf.nnz)
    st = load().osm_host_face_stiffness(C.byref(inp.mesh), _ptr(inp.drho), C.byref(inp.dec), int(face), _ptr(v))
    if st != OSM_OK:
        raise OsmError(st, "host_face_stiffness")
    return node, sp.csr_matrix((v, Mf.indices, Mf.indptr), shape=Mf.shape)


def _autograd():
    import torch

    class GravityPotential(torch.autograd.Function):
        """phi(drho) through the Schwarz solve; backward = one adjoint solve."""

        @staticmethod
        def forward(ctx, drho, solver, rtol):
            solver.set_density_dev(drho)
            phi, _, _ = solver.solve(rtol)
            ctx.solver, ctx.rtol = solver, rtol
            return phi

        @staticmethod
        def backward(ctx, gphi):
            return ctx.solver.potential_vjp(gphi, ctx.rtol), None, None

    class GravityMisfit(torch.autograd.Function):
        """J(drho) = 1/2 ||B phi(drho) - g_obs||^2; gradient by the adjoint solve."""

        @staticmethod
        def forward(ctx, drho, g_obs, solver, rtol):
            solver.set_density_dev(drho)
            J, grad, _ = solver.grad(g_obs, rtol)
            ctx.save_for_backward(grad)
            return torch.tensor(J, dtype=torch.float64, device=drho.device)

        @staticmethod
        def backward(ctx, gJ):
            (grad,) = ctx.saved_tensors
            return gJ * grad, None, None, None

    return GravityPotential, GravityMisfit


def gravity_potential(drho, solver, rtol=1e-8):
    """Differentiable phi(drho) (torch.autograd)."""
    return _autograd()[0].apply(drho, solver, rtol)


def gravity_misfit(drho, g_obs, solver, rtol=1e-8):
    """Differentiable misfit J(drho) = 1/2 ||B phi - g_obs||^2 (torch.autograd)."""
    return _autograd()[1].apply(drho, g_obs, solver, rtol)
