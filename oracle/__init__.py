"""Oracle: plain FP64 CPU implementation of the optimized Schwarz gravimetry
solver.  TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_2112_03851_gb300``) never calls it and shares no code with it.

The arithmetic lives in ``orc.c`` (plain loops, FP64).  This module compiles
it with gcc on first use and wraps it with ctypes:

* :func:`element`         Q2 element stiffness / mass / basis integrals by
                          3x3x3 Gauss quadrature (Sec. 6, "high order finite
                          elements" on hexahedra).
* :class:`GlobalSystem`   global assembly of K and of the load 4 pi G drho
                          (Sec. 2), Dirichlet nodes eliminated (Sec. 3).
* :func:`pcg`             diagonal-preconditioned CG, relative 2-norm stop
                          (Sec. 6).
* :class:`Schwarz`        the non-overlapping Robin ("oo0") Schwarz iteration
                          of Sec. 3 on a box grid of subdomains, parallel
                          (Jacobi-type) updates, global residual stop test.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SRC = os.path.join(_HERE, "orc.c")
_lock = threading.Lock()
_lib = None

G_NEWTON = 6.672e-11


def build(force: bool = False) -> str:
    """Compile ``orc.c`` into ``_build/liborc.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _P(t):
    return C.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(build())
        d, i32, i64, vp = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        sig = {
            "orc_basis_1d": (None, [d, vp, vp]),
            "orc_element": (None, [d, d, d, vp, vp, vp]),
            "orc_face_element": (None, [d, d, vp]),
            "orc_face_stiffness": (None, [d, d, vp]),
            "orc_gauss_points": (None, [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]),
            "orc_global_create": (vp, [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, C.c_int]),
            "orc_global_n": (i64, [vp]),
            "orc_global_nnz": (i64, [vp]),
            "orc_global_export": (None, [vp, vp, vp, vp, vp, vp]),
            "orc_global_load_gauss": (None, [vp, vp, vp]),
            "orc_global_destroy": (None, [vp]),
            "orc_spmv": (None, [i64, vp, vp, vp, vp, vp]),
            "orc_pcg": (C.c_int, [i64, vp, vp, vp, vp, vp, d, C.c_int, vp]),
            "orc_sz_create": (vp, [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, C.c_int, C.c_int,
                                   C.c_int, vp, vp, vp, vp]),
            "orc_sz_create_tc": (vp, [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, C.c_int, C.c_int,
                                      C.c_int, vp, vp, vp, vp]),
            "orc_sz_face_stiffness_export": (None, [vp, C.c_int, vp]),
            "orc_sz_nsub": (C.c_int, [vp]),
            "orc_sz_nface": (C.c_int, [vp]),
            "orc_sz_global_n": (i64, [vp]),
            "orc_sz_sub_n": (i64, [vp, C.c_int]),
            "orc_sz_sub_nnz": (i64, [vp, C.c_int]),
            "orc_sz_status": (C.c_int, [vp]),
            "orc_sz_face_info": (None, [vp, C.c_int, vp, vp, vp, vp]),
            "orc_sz_get_lambda": (None, [vp, C.c_int, C.c_int, vp]),
            "orc_sz_set_lambda": (None, [vp, C.c_int, C.c_int, vp]),
            "orc_sz_face_export": (None, [vp, C.c_int, vp, vp, vp, vp]),
            "orc_sz_sub_export": (None, [vp, C.c_int, vp, vp, vp, vp, vp, vp]),
            "orc_sz_set_rhs": (None, [vp, C.c_int, vp]),
            "orc_sz_set_global_rhs": (None, [vp, vp]),
            "orc_sz_iterate": (None, [vp, d, C.c_int, vp]),
            "orc_sz_residual": (d, [vp, vp]),
            "orc_sz_solve": (C.c_int, [vp, d, C.c_int, d, C.c_int, vp, vp, vp]),
            "orc_sz_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------ elements ----

def basis_1d(s: float):
    phi = np.zeros(3)
    dphi = np.zeros(3)
    lib().orc_basis_1d(float(s), _ptr(phi), _ptr(dphi))
    return phi, dphi


def element(hx: float, hy: float, hz: float):
    """(K[27,27], M[27,27], w[27]) of a box element; node a + 3b + 9c."""
    K = np.zeros((27, 27))
    M = np.zeros((27, 27))
    w = np.zeros(27)
    lib().orc_element(hx, hy, hz, _ptr(K), _ptr(M), _ptr(w))
    return K, M, w


def face_element(ha: float, hb: float):
    M = np.zeros((9, 9))
    lib().orc_face_element(ha, hb, _ptr(M))
    return M


def face_stiffness(ha: float, hb: float):
    """Tangential Q2 stiffness S[9,9] of an ha x hb face element."""
    S = np.zeros((9, 9))
    lib().orc_face_stiffness(ha, hb, _ptr(S))
    return S


def gauss_points(xc, yc, zc):
    xc, yc, zc = _f64(xc), _f64(yc), _f64(zc)
    nx, ny, nz = len(xc) - 1, len(yc) - 1, len(zc) - 1
    pts = np.zeros((nx * ny * nz, 27, 3))
    lib().orc_gauss_points(nx, ny, nz, _ptr(xc), _ptr(yc), _ptr(zc), _ptr(pts))
    return pts


# -------------------------------------------------------- global system ----

class GlobalSystem:
    """Assembled Q2 stiffness and constant-density load on the whole mesh.

    ``keep_boundary=False`` eliminates the homogeneous-Dirichlet nodes (the
    problem of Sec. 3); ``True`` keeps every node (used for inhomogeneous
    Dirichlet tests).
    """

    def __init__(self, xc, yc, zc, drho=None, keep_boundary=False):
        self.xc, self.yc, self.zc = _f64(xc), _f64(yc), _f64(zc)
        self.nx, self.ny, self.nz = len(xc) - 1, len(yc) - 1, len(zc) - 1
        drho_a = None if drho is None else _f64(drho)
        L = lib()
        h = L.orc_global_create(self.nx, self.ny, self.nz, _ptr(self.xc), _ptr(self.yc),
                                _ptr(self.zc), _ptr(drho_a), int(keep_boundary))
        if not h:
            raise RuntimeError("oracle assembly failed")
        try:
            n = L.orc_global_n(h)
            nnz = L.orc_global_nnz(h)
            self.rp = np.zeros(n + 1, dtype=np.int64)
            self.ci = np.zeros(nnz, dtype=np.int32)
            self.v = np.zeros(nnz)
            self.f = np.zeros(n)
            self.gnode = np.zeros(n, dtype=np.int32)
            L.orc_global_export(h, _ptr(self.rp), _ptr(self.ci), _ptr(self.v), _ptr(self.f), _ptr(self.gnode))
            self._h = h
        except Exception:
            L.orc_global_destroy(h)
            raise
        self.n = n
        self.nnz = nnz

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_global_destroy(h)
            self._h = None

    @property
    def n_nodes(self):
        return (2 * self.nx + 1) * (2 * self.ny + 1) * (2 * self.nz + 1)

    def load_gauss(self, fq):
        """Load vector of a source sampled at Gauss points, fq[(e, q)]."""
        fq = _f64(fq).reshape(-1)
        out = np.zeros(self.n)
        lib().orc_global_load_gauss(self._h, _ptr(fq), _ptr(out))
        return out

    def matvec(self, x):
        x = _f64(x)
        y = np.zeros(self.n)
        lib().orc_spmv(self.n, _ptr(self.rp), _ptr(self.ci), _ptr(self.v), _ptr(x), _ptr(y))
        return y

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.v, self.ci, self.rp), shape=(self.n, self.n))

    def solve(self, b=None, tol=1e-13, maxit=100000, x0=None):
        b = self.f if b is None else _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        rel = C.c_double(0.0)
        it = lib().orc_pcg(self.n, _ptr(self.rp), _ptr(self.ci), _ptr(self.v), _ptr(b), _ptr(x),
                           tol, maxit, C.byref(rel))
        if it < 0:
            raise RuntimeError(f"oracle PCG failed (status {it}, relres {rel.value})")
        return x, it, rel.value

    def to_grid(self, u):
        """Scatter unknowns onto the full node grid (zeros elsewhere), x fastest."""
        phi = np.zeros(self.n_nodes)
        phi[self.gnode] = u
        return phi

    def residual(self, phi_grid):
        """||f - K u|| / ||f|| for a full-grid field (Dirichlet nodes ignored)."""
        u = _f64(phi_grid)[self.gnode]
        r = self.f - self.matvec(u)
        return float(np.linalg.norm(r) / np.linalg.norm(self.f))


def pcg(rp, ci, v, b, x0=None, tol=1e-10, maxit=100000):
    n = len(rp) - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    rel = C.c_double(0.0)
    it = lib().orc_pcg(n, _ptr(_np64(rp)), _ptr(_i32(ci)), _ptr(_f64(v)), _ptr(_f64(b)), _ptr(x),
                       tol, maxit, C.byref(rel))
    return x, it, rel.value


def _np64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# -------------------------------------------------------------- Schwarz ----

class Schwarz:
    """Sequential optimized Schwarz iteration (Sec. 3).

    ``p`` is a scalar or one value per subdomain (subdomain s = a + sx(b + sy c)):
    the zeroth-order Robin condition.  ``tc = (p_lo, q_lo, p_hi, q_hi)``
    instead selects the second-order / unsymmetric condition on every face:
    operator p + q(-d^2/dtau^2), (p_lo, q_lo) on the lower side of the face,
    (p_hi, q_hi) on the upper side.
    """

    def __init__(self, xc, yc, zc, drho, cx, cy, cz, p=None, tc=None):
        self.xc, self.yc, self.zc = _f64(xc), _f64(yc), _f64(zc)
        self.cx, self.cy, self.cz = _i32(cx), _i32(cy), _i32(cz)
        sx, sy, sz = len(cx) - 1, len(cy) - 1, len(cz) - 1
        self.drho = _f64(drho)
        L = lib()
        args = (len(xc) - 1, len(yc) - 1, len(zc) - 1, _ptr(self.xc), _ptr(self.yc),
                _ptr(self.zc), _ptr(self.drho), sx, sy, sz, _ptr(self.cx), _ptr(self.cy), _ptr(self.cz))
        if tc is not None:
            self.tc = _f64(tc)
            assert self.tc.shape == (4,)
            self.p_sub = None
            h = L.orc_sz_create_tc(*args, _ptr(self.tc))
        else:
            self.tc = None
            self.p_sub = _f64(np.broadcast_to(np.asarray(p, dtype=np.float64), (sx * sy * sz,)))
            h = L.orc_sz_create(*args, _ptr(self.p_sub))
        if not h:
            raise RuntimeError("oracle decomposition failed")
        self._h = h
        self.nsub = L.orc_sz_nsub(h)
        self.nface = L.orc_sz_nface(h)
        self.n_nodes = (2 * len(xc) - 1) * (2 * len(yc) - 1) * (2 * len(zc) - 1)

    @classmethod
    def from_problem(cls, prob, p=None, tc=None):
        if tc is not None:
            return cls(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, tc=tc)
        return cls(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz,
                   prob.p if p is None else p)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_sz_destroy(h)
            self._h = None

    def solve(self, inner_rtol=1e-10, rtol=1e-8, max_outer=1000, max_inner=100000):
        phi = np.zeros(self.n_nodes)
        rel = C.c_double(0.0)
        hist = np.zeros(max_outer)
        n = lib().orc_sz_solve(self._h, inner_rtol, max_inner, rtol, max_outer, _ptr(phi),
                               C.byref(rel), _ptr(hist))
        return phi, n, rel.value, hist[:n].copy()

    def iterate(self, inner_rtol=1e-10, max_inner=100000):
        it = np.zeros(self.nsub, dtype=np.int32)
        lib().orc_sz_iterate(self._h, inner_rtol, max_inner, _ptr(it))
        return it

    def residual(self):
        phi = np.zeros(self.n_nodes)
        rel = lib().orc_sz_residual(self._h, _ptr(phi))
        return phi, rel

    def status(self):
        return lib().orc_sz_status(self._h)

    def face_info(self, f):
        s, t, ax = C.c_int32(), C.c_int32(), C.c_int32()
        n = C.c_int64()
        lib().orc_sz_face_info(self._h, f, C.byref(s), C.byref(t), C.byref(ax), C.byref(n))
        return s.value, t.value, ax.value, n.value

    def face_export(self, f):
        import scipy.sparse as sp
        n = self.face_info(f)[3]
        g = np.zeros(n, dtype=np.int32)
        rp = np.zeros(n + 1, dtype=np.int64)
        lib().orc_sz_face_export(self._h, f, _ptr(g), _ptr(rp), None, None)
        ci = np.zeros(rp[-1], dtype=np.int32)
        m = np.zeros(rp[-1])
        lib().orc_sz_face_export(self._h, f, _ptr(g), _ptr(rp), _ptr(ci), _ptr(m))
        return g, sp.csr_matrix((m, ci, rp), shape=(n, n))

    def face_stiffness_export(self, f):
        """Tangential stiffness of face f, same node order as face_export."""
        import scipy.sparse as sp
        g, Mf = self.face_export(f)
        sv = np.zeros(Mf.nnz)
        lib().orc_sz_face_stiffness_export(self._h, f, _ptr(sv))
        return sp.csr_matrix((sv, Mf.indices, Mf.indptr), shape=Mf.shape)

    def get_lambda(self, f, side):
        out = np.zeros(self.face_info(f)[3])
        lib().orc_sz_get_lambda(self._h, f, side, _ptr(out))
        return out

    def set_lambda(self, f, side, data):
        data = _f64(data)
        assert data.shape == (self.face_info(f)[3],)
        lib().orc_sz_set_lambda(self._h, f, side, _ptr(data))

    def sub_export(self, s):
        import scipy.sparse as sp
        L = lib()
        n = L.orc_sz_sub_n(self._h, s)
        nnz = L.orc_sz_sub_nnz(self._h, s)
        rp = np.zeros(n + 1, dtype=np.int64)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz)
        f = np.zeros(n)
        g = np.zeros(n, dtype=np.int32)
        u = np.zeros(n)
        L.orc_sz_sub_export(self._h, s, _ptr(rp), _ptr(ci), _ptr(v), _ptr(f), _ptr(g), _ptr(u))
        return sp.csr_matrix((v, ci, rp), shape=(n, n)), f, g, u

    def set_rhs(self, s, f):
        f = _f64(f)
        lib().orc_sz_set_rhs(self._h, s, _ptr(f))

    def set_global_rhs(self, fG):
        fG = _f64(fG)
        lib().orc_sz_set_global_rhs(self._h, _ptr(fG))


# ------------------------------------------------------------- gradient ----
# Surface-gravity misfit J = 1/2 ||B phi - g_obs||^2 with K phi = F drho
# (F: 4 pi G times the element integrals of the basis functions) and its
# gradient dJ/d drho = F^T K^-1 B^T (B phi - g_obs), written from these
# definitions with the oracle's own basis, element routine and PCG.

def _locate(c, v):
    """Element holding coordinate v: the upper-side element on an element
    boundary, the last element on the upper mesh boundary."""
    e = int(np.searchsorted(c, v, side="right")) - 1
    return min(max(e, 0), len(c) - 2)


def station_matrix(G, stations):
    """B (n_st x unknowns of G): d/dz of the Q2 interpolant at each station;
    Dirichlet nodes (phi = 0) are dropped."""
    import scipy.sparse as sp
    NX, NY = 2 * G.nx + 1, 2 * G.ny + 1
    unk = np.full(G.n_nodes, -1, dtype=np.int64)
    unk[G.gnode] = np.arange(G.n)
    rows, cols, vals = [], [], []
    for s, (x, y, z) in enumerate(np.asarray(stations, dtype=np.float64)):
        ex, ey, ez = _locate(G.xc, x), _locate(G.yc, y), _locate(G.zc, z)
        hx, hy, hz = G.xc[ex + 1] - G.xc[ex], G.yc[ey + 1] - G.yc[ey], G.zc[ez + 1] - G.zc[ez]
        Lx, _ = basis_1d((x - G.xc[ex]) / hx)
        Ly, _ = basis_1d((y - G.yc[ey]) / hy)
        _, dLz = basis_1d((z - G.zc[ez]) / hz)
        for c in range(3):
            for b in range(3):
                for a in range(3):
                    node = (2 * ex + a) + NX * ((2 * ey + b) + NY * (2 * ez + c))
                    if unk[node] >= 0:
                        rows.append(s)
                        cols.append(unk[node])
                        vals.append(Lx[a] * Ly[b] * dLz[c] / hz)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(stations), G.n))


def load_matrix(G):
    """F (unknowns x elements): F[a, e] = 4 pi G_newton int_e phi_a."""
    import scipy.sparse as sp
    NX, NY = 2 * G.nx + 1, 2 * G.ny + 1
    unk = np.full(G.n_nodes, -1, dtype=np.int64)
    unk[G.gnode] = np.arange(G.n)
    cache = {}
    rows, cols, vals = [], [], []
    e = 0
    for ez in range(G.nz):
        for ey in range(G.ny):
            for ex in range(G.nx):
                h = (G.xc[ex + 1] - G.xc[ex], G.yc[ey + 1] - G.yc[ey], G.zc[ez + 1] - G.zc[ez])
                if h not in cache:
                    cache[h] = element(*h)[2]
                w = cache[h]
                for I in range(27):
                    a, b, c = I % 3, (I // 3) % 3, I // 9
                    node = (2 * ex + a) + NX * ((2 * ey + b) + NY * (2 * ez + c))
                    if unk[node] >= 0:
                        rows.append(unk[node])
                        cols.append(e)
                        vals.append(4.0 * np.pi * G_NEWTON * w[I])
                e += 1
    return sp.csr_matrix((vals, (rows, cols)), shape=(G.n, G.nx * G.ny * G.nz))


class Misfit:
    """J(drho) = 1/2 ||B K^-1 F drho - g_obs||^2 on the monolithic system."""

    def __init__(self, xc, yc, zc, stations, tol=1e-14):
        self.G = GlobalSystem(xc, yc, zc)
        self.B = station_matrix(self.G, stations)
        self.F = load_matrix(self.G)
        self.tol = tol

    def potential(self, drho):
        u, _, _ = self.G.solve(self.F @ np.asarray(drho, dtype=np.float64), tol=self.tol)
        return u

    def gravity(self, drho):
        return self.B @ self.potential(drho)

    def value_and_grad(self, drho, g_obs):
        r = self.gravity(drho) - g_obs
        w, _, _ = self.G.solve(self.B.T @ r, tol=self.tol)
        return 0.5 * float(r @ r), self.F.T @ w
