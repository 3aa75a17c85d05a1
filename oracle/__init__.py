"""FP64 CPU oracle for the grid-hopping polygonizer -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``oracle.c`` (plain C, double precision);
this module only builds it with gcc and marshals numpy arrays through ctypes.

Paper sections followed (see the header of ``oracle.c`` for details):
Sec. 1 (SDB definition), Sec. 2 (enumeration), Sec. 3 (Eq. 1-4 and
Algorithm 1: the grid hopper), Sec. 4 (plane, box and union bounds),
Sec. 5.2 (neural SDB shrunk by lambda).  Marching Cubes uses the oracle's own
table generated from a per-face rule.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# result slots (oracle.c: enum R_*)
R_CELL, R_CASE, R_TKEY, R_TPOS, R_TCELL, R_COLEVAL, R_MARK = range(7)

PRIM_STRIDE = 17
SPHERE, TORUS, BOX = 0, 1, 2
UNION, SUBTRACT, INTERSECT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            L.or_csg_new.restype = P
            L.or_csg_new.argtypes = [I, P]
            L.or_mlp_new.restype = P
            L.or_mlp_new.argtypes = [I, I, P, D, D, D, D, D]
            L.or_lattice_new.restype = P
            L.or_lattice_new.argtypes = [I, P, D, P]
            L.or_sdb_free.argtypes = [P]
            L.or_eval.argtypes = [P, I64, P, P]
            L.or_mc_table.restype = I
            L.or_mc_table.argtypes = [P, P, I]
            L.or_mc.restype = P
            L.or_mc.argtypes = [P, I, P, D, I64, P]
            L.or_enum.restype = P
            L.or_enum.argtypes = [P, I, P, D, I, I]
            L.or_hop.restype = P
            L.or_cont.restype = P
            L.or_cont.argtypes = [P, I, P, D, I64, P]
            L.or_hop.argtypes = [P, I, P, D, D, D, I64, P]
            L.or_res_count.restype = I64
            L.or_res_count.argtypes = [P, I]
            L.or_res_copy.argtypes = [P, I, P]
            L.or_res_minabs.restype = D
            L.or_res_minabs.argtypes = [P]
            L.or_res_free.argtypes = [P]
            L.or_grad_x.restype = I
            L.or_grad_x.argtypes = [P, I64, P, P]
            L.or_grad_theta_point.restype = I
            L.or_grad_theta_point.argtypes = [P, P, P, I64]
            L.or_adjoint.restype = I
            L.or_adjoint.argtypes = [P, I64, P, P, P, I64]
            L.or_csg_adjoint.restype = I
            L.or_csg_adjoint.argtypes = [P, I64, P, P, P]
            L.or_num_threads.restype = I
            L.or_set_threads.argtypes = [I]
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    """Host threads of later oracle calls (n < 1: all cores)."""
    lib().or_set_threads(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class SDB:
    """An SDB held by the oracle (double precision)."""

    def __init__(self, handle, kind, nparam=0, keep=None):
        self.h = handle
        self.kind = kind
        self.nparam = nparam
        self._keep = keep

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_sdb_free(self.h)
            self.h = None

    def eval(self, pts) -> np.ndarray:
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.empty(p.shape[0], np.float64)
        lib().or_eval(self.h, p.shape[0], _ptr(p), _ptr(out))
        return out

    def eval_many(self, pts, chunk: int = 1 << 16) -> np.ndarray:
        """f at many points: the C evaluator, except for a neural SDB, whose
        layers then run as numpy matrix products (np_eval: the same
        definition, a matrix product per layer as the only library step;
        about 3x faster than the C loops for 10^6 points)."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        args = getattr(self, "np_args", None)
        if args is None or p.shape[0] < 4096:
            return self.eval(p)
        params, width, nmid, kw = args
        out = np.empty(p.shape[0], np.float64)
        for s in range(0, p.shape[0], chunk):
            out[s:s + chunk] = np_eval(params, width, nmid, p[s:s + chunk], **kw)
        return out

    def grad_x(self, pts) -> np.ndarray:
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.empty_like(p)
        if lib().or_grad_x(self.h, p.shape[0], _ptr(p), _ptr(out)) != 0:
            raise ValueError("grad_x needs a neural SDB")
        return out

    def grad_theta_point(self, p) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(3)
        out = np.zeros(self.nparam, np.float64)
        lib().or_grad_theta_point(self.h, _ptr(p), _ptr(out), self.nparam)
        return out

    def adjoint(self, verts, dldv) -> np.ndarray:
        v = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3)
        g = np.ascontiguousarray(dldv, dtype=np.float64).reshape(-1, 3)
        if self.kind == "csg":
            out = np.zeros((self.nprim, PRIM_STRIDE), np.float64)
            if lib().or_csg_adjoint(self.h, v.shape[0], _ptr(v), _ptr(g), _ptr(out)) != 0:
                raise ValueError("csg adjoint failed")
            return out
        out = np.zeros(self.nparam, np.float64)
        if lib().or_adjoint(self.h, v.shape[0], _ptr(v), _ptr(g), _ptr(out), self.nparam) != 0:
            raise ValueError("adjoint needs a neural SDB")
        return out


def csg(prims) -> SDB:
    """prims: [n, 17] float64 rows (type, op, centre[3], params[3], rot[9])."""
    a = np.ascontiguousarray(prims, dtype=np.float64).reshape(-1, PRIM_STRIDE)
    h = lib().or_csg_new(a.shape[0], _ptr(a))
    if not h:
        raise ValueError("empty CSG")
    sdb = SDB(h, "csg")
    sdb.nprim = a.shape[0]
    return sdb


def mlp_param_count(width: int, nmid: int) -> int:
    return 3 * width + width + nmid * (width * width + width) + width + 1


def mlp(width, nmid, params, r0=0.6, alpha=0.1, beta=1.1, lam=1.0, radial=True) -> SDB:
    """params: packed W0[W,3] b0[W] {W[W,W] b[W]}*nmid wout[W] bout (float64).
    radial=False drops the |p| term: f = (alpha g - r0) / beta / lam."""
    a = np.ascontiguousarray(params, dtype=np.float64).ravel()
    n = mlp_param_count(width, nmid)
    if a.size != n:
        raise ValueError("expected %d parameters, got %d" % (n, a.size))
    h = lib().or_mlp_new(width, nmid, _ptr(a), r0, alpha, beta, lam, 1.0 if radial else 0.0)
    sdb = SDB(h, "mlp", n)
    sdb.np_args = (a.copy(), int(width), int(nmid), dict(r0=r0, alpha=alpha, beta=beta, lam=lam, radial=radial))
    return sdb


def lattice(N, values, lo=-1.0, hi=1.0) -> SDB:
    """Trilinear interpolation of values[(N+1)^3] (index a + (N+1)(b + (N+1)c))
    given at the lattice points of an N-grid -- a device for driving Marching
    Cubes through arbitrary sign patterns; not an SDB in general."""
    lo3, h = _lo_h(N, lo, hi)
    v = np.ascontiguousarray(values, dtype=np.float64).ravel()
    if v.size != (N + 1) ** 3:
        raise ValueError("need (N+1)^3 values")
    return SDB(lib().or_lattice_new(int(N), _ptr(lo3), h, _ptr(v)), "lattice", keep=v)


class Result:
    def __init__(self, handle):
        if not handle:
            raise ValueError("oracle call rejected its arguments")
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_res_free(self.h)
            self.h = None

    def _get(self, slot, dtype, shape_tail=()):
        n = int(lib().or_res_count(self.h, slot))
        out = np.empty((n,) + tuple(shape_tail), dtype)
        if n:
            lib().or_res_copy(self.h, slot, _ptr(out))
        return out

    @property
    def cells(self):
        return self._get(R_CELL, np.int64)

    @property
    def cases(self):
        return self._get(R_CASE, np.int32)

    @property
    def tri_keys(self):
        return self._get(R_TKEY, np.int64, (3,))

    @property
    def tri_pos(self):
        return self._get(R_TPOS, np.float64, (3, 3))

    @property
    def tri_cell(self):
        return self._get(R_TCELL, np.int64)

    @property
    def col_evals(self):
        return self._get(R_COLEVAL, np.int64)

    @property
    def marks(self):
        return self._get(R_MARK, np.int64)

    @property
    def min_abs_f(self) -> float:
        return float(lib().or_res_minabs(self.h))


def _lo_h(N, lo, hi):
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (3,)))
    hi = np.broadcast_to(np.asarray(hi, np.float64), (3,))
    ext = hi - lo
    if not np.allclose(ext, ext[0], rtol=1e-12, atol=0):
        raise ValueError("the polygonization volume must be a cube")
    return lo, float(ext[0]) / N


def mc(sdb: SDB, N, cells, lo=-1.0, hi=1.0) -> Result:
    lo3, h = _lo_h(N, lo, hi)
    c = np.ascontiguousarray(cells, dtype=np.int64).ravel()
    return Result(lib().or_mc(sdb.h, N, _ptr(lo3), h, c.size, _ptr(c)))


def enum(sdb: SDB, N, lo=-1.0, hi=1.0, kmin=0, kmax=None) -> Result:
    lo3, h = _lo_h(N, lo, hi)
    return Result(lib().or_enum(sdb.h, N, _ptr(lo3), h, int(kmin), int(N if kmax is None else kmax)))


TAU_DIAGONAL, TAU_HALF_DIAGONAL = 0, 1


def tau_of(N, lo=-1.0, hi=1.0, tau_mode=TAU_DIAGONAL) -> float:
    _, h = _lo_h(N, lo, hi)
    return float(np.sqrt(3.0) * h * (1.0 if tau_mode == TAU_DIAGONAL else 0.5))


def hop(sdb: SDB, N, lo=-1.0, hi=1.0, tau_mode=TAU_DIAGONAL, eps=0.0, cols=None) -> Result:
    lo3, h = _lo_h(N, lo, hi)
    tau = tau_of(N, lo, hi, tau_mode)
    if cols is None:
        return Result(lib().or_hop(sdb.h, N, _ptr(lo3), h, tau, float(eps), 0, None))
    c = np.ascontiguousarray(cols, dtype=np.int64).ravel()
    return Result(lib().or_hop(sdb.h, N, _ptr(lo3), h, tau, float(eps), c.size, _ptr(c)))


def cont(sdb: SDB, N, seeds, lo=-1.0, hi=1.0) -> Result:
    """Continuation (Sec. 2): the surface crawled from seed points (cells of
    each seed's component, in visit order, with their triangles); col_evals
    holds each seed's cell id or -1."""
    lo3, h = _lo_h(N, lo, hi)
    sp = np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 3)
    return Result(lib().or_cont(sdb.h, N, _ptr(lo3), h, sp.shape[0], _ptr(sp)))


def polygonize(sdb: SDB, N, lo=-1.0, hi=1.0, tau_mode=TAU_DIAGONAL, cols=None):
    """Serial hopper followed by Marching Cubes on the marked cells."""
    hr = hop(sdb, N, lo, hi, tau_mode, cols=cols)
    return hr, mc(sdb, N, hr.marks, lo, hi)


def mc_table(maxt: int = 16):
    ntri = np.zeros(256, np.int32)
    edges = np.full((256, maxt, 3), -1, np.int32)
    mx = lib().or_mc_table(_ptr(ntri), _ptr(edges), maxt)
    return ntri, edges, int(mx)


# ---------------------------------------------------------------------------
# Batched FP64 evaluation of the neural SDB with numpy matrix products (the
# same definition as oracle.c's mlp_g / mlp_grads, written layer by layer;
# a matrix product per layer is the only library step).  Used where the C
# loops would be too slow: finite differences over ~10^5 mesh vertices.
# ---------------------------------------------------------------------------
def np_layers(params, width, nmid):
    p = np.asarray(params, np.float64).ravel()
    W = width
    shapes = [(W, 3)] + [(W, W)] * nmid + [(1, W)]
    out, o = [], 0
    for od, id_ in shapes:
        M = p[o:o + od * id_].reshape(od, id_)
        o += od * id_
        b = p[o:o + od]
        o += od
        out.append((M, b))
    assert o == p.size
    return out


def np_forward(layers, P):
    """Pre-activations z_0..z_L of the hidden layers and g."""
    P = np.asarray(P, np.float64).reshape(-1, 3)
    zs = []
    a = P
    for W, b in layers[:-1]:
        z = a @ W.T + b
        zs.append(z)
        a = np.maximum(z, 0.0)
    Wo, bo = layers[-1]
    g = (a @ Wo.T + bo)[:, 0]
    return zs, g


def np_eval(params, width, nmid, P, r0=0.6, alpha=0.1, beta=1.1, lam=1.0, radial=True):
    """f(p) = (|p| - r0 + alpha g(p)) / beta / lam at the rows of P (Sec. 5.2);
    radial=False drops |p|."""
    P = np.asarray(P, np.float64).reshape(-1, 3)
    _, g = np_forward(np_layers(params, width, nmid), P)
    rad = 1.0 if radial else 0.0
    return (rad * np.linalg.norm(P, axis=1) - r0 + alpha * g) / beta / lam


def np_grad_x(params, width, nmid, P, r0=0.6, alpha=0.1, beta=1.1, lam=1.0, radial=True):
    P = np.asarray(P, np.float64).reshape(-1, 3)
    layers = np_layers(params, width, nmid)
    zs, _ = np_forward(layers, P)
    d = layers[-1][0][0][None, :] * (zs[-1] > 0)  # dg/dz_L
    for l in range(len(zs) - 1, 0, -1):
        d = (d @ layers[l][0]) * (zs[l - 1] > 0)
    dgdp = d @ layers[0][0]
    r = np.linalg.norm(P, axis=1, keepdims=True)
    rad = 1.0 if radial else 0.0
    return (rad * P / np.where(r > 0, r, 1.0) + alpha * dgdp) / (beta * lam)


def np_adjoint(params, width, nmid, V, dLdv, r0=0.6, alpha=0.1, beta=1.1, lam=1.0, radial=True):
    """Implicit-surface adjoint sum_v s_v df/dtheta(v) with
    s_v = -(dL/dv . grad_x f)/|grad_x f|^2, packed like the parameters."""
    V = np.asarray(V, np.float64).reshape(-1, 3)
    G = np.asarray(dLdv, np.float64).reshape(-1, 3)
    layers = np_layers(params, width, nmid)
    zs, _ = np_forward(layers, V)
    ds = [None] * len(zs)
    d = layers[-1][0][0][None, :] * (zs[-1] > 0)
    ds[-1] = d
    for l in range(len(zs) - 1, 0, -1):
        d = (d @ layers[l][0]) * (zs[l - 1] > 0)
        ds[l - 1] = d
    dgdp = ds[0] @ layers[0][0]
    r = np.linalg.norm(V, axis=1, keepdims=True)
    rad = 1.0 if radial else 0.0
    gx = (rad * V / np.where(r > 0, r, 1.0) + alpha * dgdp) / (beta * lam)
    s = -(G * gx).sum(1) / (gx * gx).sum(1)
    c = alpha / (beta * lam)
    out = []
    acts = [V] + [np.maximum(z, 0.0) for z in zs]
    for l in range(len(zs)):
        sd = ds[l] * s[:, None]
        out.append((sd.T @ acts[l]).ravel())
        out.append(sd.sum(0))
    out.append((acts[-1] * s[:, None]).sum(0))
    out.append(np.array([s.sum()]))
    return c * np.concatenate(out)
